// The proximal map of alpha (R3 + delta_{>=0}) with all three terms of Eq.
// (reg-tv-l1-one): TV of every species, l1, and TV of every pulse image
// (S c)^n -- the lambda_3 term -- by Algorithm 2 on the stacked operator
//   L v = [ lam_tv D v_p (p < P) ;  lam_l1 v ;  lam_b D (S v)^n (n < N) ],
// with D the 3D forward differences (zero across the far faces) and
// (S v)^n[j] = sum_p S[m(n)][p][j] v_p[j], m(n) = n mod pulses_per_cycle.
// Dual u = [uc (P x 3 x L) ; ul (P x L) ; ub (N x 3 x L)] in the box
// |u| <= alpha (Eq. prox-dual, the lambdas inside L), dual step `step2` (at
// most 1/eig_max(L L^T)), u and the momentum iterate r start at zero:
//   w   = z - L^T r
//   u_i = clamp(r + step2 L w, -alpha, alpha)
//   r   = u_i + beta_i (u_i - u_{i-1})          (Beck-Teboulle beta_i)
// and x = max(z - L^T u, 0).  Every pulse keeps a dual of its own, as in the
// paper's sum over n, so the iterates are Algorithm 2's.
//
// Two voxel-parallel kernels per iteration (memory-bound stencils): L^T of
// the momentum iterate, then L of the result with the clamp and the momentum
// step fused.  Scratch (w, u, r) is taken from the stream-ordered allocator
// for the call.
#include <cmath>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kJointBlock = 256;
constexpr int kJointMaxSpecies = 8;

struct JointArgs {
    int P, N, Y, X, Z, ncyc;
    const float* Sm;  // [Q][P][Z] switching weights of the states
    float lam_tv, lam_l1, lam_b;
};

// (D^T g)[i] for one field g[3][Y][X][Z] (components y, x, z)
__device__ __forceinline__ float transpose_diff(const float* g, size_t L, size_t i, int y, int x, int j,
                                       int Y, int X, int Z)
{
    const size_t sy = (size_t)X * Z, sx = (size_t)Z;
    float acc = 0.f;
    if (y + 1 < Y) acc -= g[i];
    if (y > 0) acc += g[i - sy];
    if (x + 1 < X) acc -= g[L + i];
    if (x > 0) acc += g[L + i - sx];
    if (j + 1 < Z) acc -= g[2 * L + i];
    if (j > 0) acc += g[2 * L + i - 1];
    return acc;
}

// out = z - L^T r (clip: max(., 0)), one thread per voxel, all species
__global__ void joint_lt_kernel(const JointArgs a, const float* __restrict__ z,
                                const float* __restrict__ r, float* __restrict__ out, int clip)
{
    const size_t L = (size_t)a.Y * a.X * a.Z;
    const float* rc = r;
    const float* rl = r + (size_t)a.P * 3 * L;
    const float* rb = rl + (size_t)a.P * L;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % (size_t)a.Z);
        const int x = (int)((i / (size_t)a.Z) % (size_t)a.X);
        const int y = (int)(i / ((size_t)a.Z * a.X));
        float acc[kJointMaxSpecies];
#pragma unroll
        for (int p = 0; p < kJointMaxSpecies; ++p) {
            if (p >= a.P) break;
            acc[p] = a.lam_tv * transpose_diff(rc + (size_t)p * 3 * L, L, i, y, x, j, a.Y, a.X, a.Z) +
                     a.lam_l1 * rl[(size_t)p * L + i];
        }
        for (int n = 0; n < a.N; ++n) {
            const float d = a.lam_b * transpose_diff(rb + (size_t)n * 3 * L, L, i, y, x, j, a.Y, a.X, a.Z);
            const float* s = a.Sm + (size_t)(n % a.ncyc) * a.P * a.Z + j;
#pragma unroll
            for (int p = 0; p < kJointMaxSpecies; ++p) {
                if (p >= a.P) break;
                acc[p] = fmaf(s[(size_t)p * a.Z], d, acc[p]);
            }
        }
#pragma unroll
        for (int p = 0; p < kJointMaxSpecies; ++p) {
            if (p >= a.P) break;
            const float v = z[(size_t)p * L + i] - acc[p];
            out[(size_t)p * L + i] = clip ? fmaxf(v, 0.f) : v;
        }
    }
}

// u_new = clamp(r + step2 (L w)_e, -alpha, alpha); r = u_new + beta (u_new - u); u = u_new
__device__ __forceinline__ void dual_step(float* r, float* u, size_t e, float lw, float step2,
                                          float alpha, float beta)
{
    float v = fmaf(step2, lw, r[e]);
    v = fminf(fmaxf(v, -alpha), alpha);
    r[e] = fmaf(beta, v - u[e], v);
    u[e] = v;
}

// the dual update for every entry of voxel i, one thread per voxel
__global__ void joint_dual_kernel(const JointArgs a, const float* __restrict__ w,
                                  float* __restrict__ r, float* __restrict__ u, float step2,
                                  float alpha, float beta)
{
    const size_t L = (size_t)a.Y * a.X * a.Z;
    const size_t sy = (size_t)a.X * a.Z, sx = (size_t)a.Z;
    const size_t ol = (size_t)a.P * 3 * L, ob = ol + (size_t)a.P * L;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < L;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % (size_t)a.Z);
        const int x = (int)((i / (size_t)a.Z) % (size_t)a.X);
        const int y = (int)(i / ((size_t)a.Z * a.X));
        const bool hy = y + 1 < a.Y, hx = x + 1 < a.X, hz = j + 1 < a.Z;
        for (int p = 0; p < a.P; ++p) {
            const float* wp = w + (size_t)p * L;
            const float w0 = wp[i];
            const float g0 = hy ? wp[i + sy] - w0 : 0.f;
            const float g1 = hx ? wp[i + sx] - w0 : 0.f;
            const float g2 = hz ? wp[i + 1] - w0 : 0.f;
            const size_t e = (size_t)p * 3 * L + i;
            dual_step(r, u, e, a.lam_tv * g0, step2, alpha, beta);
            dual_step(r, u, e + L, a.lam_tv * g1, step2, alpha, beta);
            dual_step(r, u, e + 2 * L, a.lam_tv * g2, step2, alpha, beta);
            dual_step(r, u, ol + (size_t)p * L + i, a.lam_l1 * w0, step2, alpha, beta);
        }
        for (int n = 0; n < a.N; ++n) {
            const float* s = a.Sm + (size_t)(n % a.ncyc) * a.P * a.Z;
            float b0 = 0.f, by = 0.f, bx = 0.f, bz = 0.f;
            for (int p = 0; p < a.P; ++p) {
                const float* wp = w + (size_t)p * L;
                const float sj = s[(size_t)p * a.Z + j];
                b0 = fmaf(sj, wp[i], b0);
                if (hy) by = fmaf(sj, wp[i + sy], by);
                if (hx) bx = fmaf(sj, wp[i + sx], bx);
                if (hz) bz = fmaf(s[(size_t)p * a.Z + j + 1], wp[i + 1], bz);
            }
            const size_t e = ob + (size_t)n * 3 * L + i;
            dual_step(r, u, e, hy ? a.lam_b * (by - b0) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + L, hx ? a.lam_b * (bx - b0) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + 2 * L, hz ? a.lam_b * (bz - b0) : 0.f, step2, alpha, beta);
        }
    }
}

}  // namespace
}  // namespace swopt

using namespace swopt;

extern "C" {

swopt_status swopt_prox_joint(swopt_handle* h, const float* z_dev, float* x_dev, double alpha,
                              double lambda_tv, double lambda_l1, double lambda_b, int iters,
                              double step2, void* stream)
{
    clear_error();
    if (!h) {
        set_error("null handle");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!z_dev || !x_dev || !std::isfinite(alpha) || alpha < 0.0 || !std::isfinite(lambda_tv) ||
        lambda_tv < 0.0 || !std::isfinite(lambda_l1) || lambda_l1 < 0.0 ||
        !std::isfinite(lambda_b) || lambda_b < 0.0 || iters < 0 ||
        (iters > 0 && (!std::isfinite(step2) || !(step2 > 0.0)))) {
        set_error("invalid joint-prox arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (h->P > kJointMaxSpecies) {
        set_error("the joint prox supports at most %d species", kJointMaxSpecies);
        return SWOPT_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t L = (size_t)h->Y * h->X * h->Z;
    const size_t nc = (size_t)h->P * L;
    const size_t nu = (size_t)h->P * 4 * L + (size_t)h->N * 3 * L;
    float* ws = nullptr;
    SW_CUDA(cudaMallocAsync((void**)&ws, sizeof(float) * (nc + 2 * nu), st));
    float* w = ws;
    float* u = ws + nc;
    float* r = u + nu;
    JointArgs a;
    a.P = h->P;
    a.N = h->N;
    a.Y = h->Y;
    a.X = h->X;
    a.Z = h->Z;
    a.ncyc = h->ncyc;
    a.Sm = h->Sm;
    a.lam_tv = (float)lambda_tv;
    a.lam_l1 = (float)lambda_l1;
    a.lam_b = (float)lambda_b;
    const int grid = grid_for(L, kJointBlock) < 152 * 16 ? grid_for(L, kJointBlock) : 152 * 16;
    swopt_status s = SWOPT_OK;
    if (cudaMemsetAsync(u, 0, sizeof(float) * 2 * nu, st) != cudaSuccess) {
        set_error("cudaMemsetAsync failed");
        s = SWOPT_ERR_CUDA;
    }
    double t = 1.0;
    for (int it = 0; it < iters && s == SWOPT_OK; ++it) {
        const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const float beta = (float)((t - 1.0) / t1);
        t = t1;
        joint_lt_kernel<<<grid, kJointBlock, 0, st>>>(a, z_dev, r, w, 0);
        joint_dual_kernel<<<grid, kJointBlock, 0, st>>>(a, w, r, u, (float)step2, (float)alpha,
                                                        beta);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("joint-prox kernel launch failed");
            s = SWOPT_ERR_CUDA;
        }
        h->launches += 2;
    }
    if (s == SWOPT_OK) {
        joint_lt_kernel<<<grid, kJointBlock, 0, st>>>(a, z_dev, u, x_dev, 1);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("joint-prox kernel launch failed");
            s = SWOPT_ERR_CUDA;
        }
        h->launches += 1;
    }
    if (cudaFreeAsync(ws, st) != cudaSuccess && s == SWOPT_OK) {
        set_error("cudaFreeAsync failed");
        s = SWOPT_ERR_CUDA;
    }
    return s;
}

}  // extern "C"
