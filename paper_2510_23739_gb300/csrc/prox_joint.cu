// The proximal map of alpha (R3 + delta_{>=0}) with all three terms of Eq.
// (reg-tv-l1-one): TV of every species, l1, and TV of every pulse image
// (S c)^n -- the lambda_3 term -- by Algorithm 2 on the stacked operator
//   L v = [ lam_tv D v_p (p < P) ;  lam_l1 v ;  lam_b D (S v)^n (n < N) ],
// with D the 3D forward differences (zero across the far faces) and
// (S v)^n[j] = sum_p S[m(n)][p][j] v_p[j], m(n) = n mod pulses_per_cycle.
// The prox of Eq. (prox) includes the nonnegativity indicator, and Eq.
// (prox-dual) keeps the matching constraint z - L^T u >= 0, so the dual is
// min over |u| <= alpha of 1/2 ||max(z - L^T u, 0)||^2 and the projected
// primal point enters every step, from u = r = 0:
//   w   = max(z - L^T r, 0)
//   u_i = clamp(r + step2 L w, -alpha, alpha)
//   r   = u_i + beta_i (u_i - u_{i-1})          (Beck-Teboulle beta_i)
// and x = max(z - L^T u, 0).
//
// Pulses of one switching state m share the image S_m v, so their duals
// receive the same gradient from the same start and stay equal; one dual per
// state, entering L^T with the state's pulse count C_m, gives Algorithm 2's
// iterates with 3 Q instead of 3 N pulse-image components.
//
// Two voxel-parallel kernels per iteration (memory-bound stencils): L^T of
// the momentum iterate with the projection, then L of the result with the
// clamp and the momentum step fused.  Scratch (w, u, r) is the handle's.
#include <cmath>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kJointBlock = 256;
constexpr int kJointMaxSpecies = 8;

struct JointArgs {
    int P, Q, Y, X, Z;
    const float* Sm;   // [Q][P][Z] switching weights of the states
    const float* Cmf;  // [Q] pulses per state
    float lam_tv, lam_l1, lam_b;
};

// (D^T g)[i] for one field g[3][Y][X][Z] (components y, x, z)
__device__ __forceinline__ float transpose_diff(const float* g, size_t L, size_t i, int y, int x,
                                                int j, int Y, int X, int Z)
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

// out = max(z - L^T r, 0), one thread per voxel, all species.  z and out may
// be the same array: each thread reads z at its voxel before writing there.
__global__ void joint_lt_kernel(const JointArgs a, const float* z, const float* __restrict__ r,
                                float* out)
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
        for (int m = 0; m < a.Q; ++m) {
            const float d = a.Cmf[m] * a.lam_b *
                            transpose_diff(rb + (size_t)m * 3 * L, L, i, y, x, j, a.Y, a.X, a.Z);
            const float* s = a.Sm + (size_t)m * a.P * a.Z + j;
#pragma unroll
            for (int p = 0; p < kJointMaxSpecies; ++p) {
                if (p >= a.P) break;
                acc[p] = fmaf(s[(size_t)p * a.Z], d, acc[p]);
            }
        }
        float v[kJointMaxSpecies];
#pragma unroll
        for (int p = 0; p < kJointMaxSpecies; ++p) {
            if (p >= a.P) break;
            v[p] = fmaxf(z[(size_t)p * L + i] - acc[p], 0.f);
        }
#pragma unroll
        for (int p = 0; p < kJointMaxSpecies; ++p) {
            if (p >= a.P) break;
            out[(size_t)p * L + i] = v[p];
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
        // w at the voxel and its three forward neighbours (0 past the far faces)
        float w0[kJointMaxSpecies], wy[kJointMaxSpecies], wx[kJointMaxSpecies],
            wz[kJointMaxSpecies];
#pragma unroll
        for (int p = 0; p < kJointMaxSpecies; ++p) {
            if (p >= a.P) break;
            const float* wp = w + (size_t)p * L;
            w0[p] = wp[i];
            wy[p] = hy ? wp[i + sy] : 0.f;
            wx[p] = hx ? wp[i + sx] : 0.f;
            wz[p] = hz ? wp[i + 1] : 0.f;
            const size_t e = (size_t)p * 3 * L + i;
            dual_step(r, u, e, hy ? a.lam_tv * (wy[p] - w0[p]) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + L, hx ? a.lam_tv * (wx[p] - w0[p]) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + 2 * L, hz ? a.lam_tv * (wz[p] - w0[p]) : 0.f, step2, alpha,
                      beta);
            dual_step(r, u, ol + (size_t)p * L + i, a.lam_l1 * w0[p], step2, alpha, beta);
        }
        for (int m = 0; m < a.Q; ++m) {
            const float* s = a.Sm + (size_t)m * a.P * a.Z;
            float b0 = 0.f, by = 0.f, bx = 0.f, bz = 0.f;
#pragma unroll
            for (int p = 0; p < kJointMaxSpecies; ++p) {
                if (p >= a.P) break;
                const float sj = s[(size_t)p * a.Z + j];
                b0 = fmaf(sj, w0[p], b0);
                by = fmaf(sj, wy[p], by);
                bx = fmaf(sj, wx[p], bx);
                if (hz) bz = fmaf(s[(size_t)p * a.Z + j + 1], wz[p], bz);
            }
            const size_t e = ob + (size_t)m * 3 * L + i;
            dual_step(r, u, e, hy ? a.lam_b * (by - b0) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + L, hx ? a.lam_b * (bx - b0) : 0.f, step2, alpha, beta);
            dual_step(r, u, e + 2 * L, hz ? a.lam_b * (bz - b0) : 0.f, step2, alpha, beta);
        }
    }
}

}  // namespace

size_t joint_dual_floats(const swopt_handle* h)
{
    const size_t L = (size_t)h->Y * h->X * h->Z;
    return (size_t)h->P * 4 * L + (size_t)h->Q * 3 * L;
}

double joint_step_bound(const swopt_handle* h, double lambda_tv, double lambda_l1,
                        double lambda_b)
{
    // ||L||^2 <= 12 lam_tv^2 + lam_l1^2 + 12 lam_b^2 sum_n max_j sum_p S[n][p][j]^2
    // (||D||^2 <= 12 in 3D; |(S_n v)_voxel|^2 <= (sum_p S^2)(sum_p v_p^2) at every voxel)
    double s2 = 0.0;
    for (int m = 0; m < h->Q; ++m) {
        double mx = 0.0;  // max over depths of sum_p S_m[p][j]^2
        for (int j = 0; j < h->Z; ++j) {
            double a = 0.0;
            for (int p = 0; p < h->P; ++p) {
                const double v = h->Sm64[((size_t)m * h->P + p) * h->Z + j];
                a += v * v;
            }
            mx = a > mx ? a : mx;
        }
        s2 += h->Cm[m] * mx;
    }
    return 12.0 * lambda_tv * lambda_tv + lambda_l1 * lambda_l1 + 12.0 * lambda_b * lambda_b * s2;
}

// Algorithm 2 on the stacked L (see the file comment) with caller-given
// scratch: w [P L], u and r [(4 P + 3 Q) L] each.  Asynchronous on st.
swopt_status joint_prox_on(swopt_handle* h, const float* z, float* x, double alpha,
                           double lambda_tv, double lambda_l1, double lambda_b, int iters,
                           double step2, int momentum, float* w, float* u, float* r,
                           cudaStream_t st)
{
    if (h->P > kJointMaxSpecies) {
        set_error("the joint prox supports at most %d species", kJointMaxSpecies);
        return SWOPT_ERR_UNSUPPORTED;
    }
    const size_t L = (size_t)h->Y * h->X * h->Z;
    const size_t nu = joint_dual_floats(h);
    JointArgs a;
    a.P = h->P;
    a.Q = h->Q;
    a.Y = h->Y;
    a.X = h->X;
    a.Z = h->Z;
    a.Sm = h->Sm;
    a.Cmf = h->Cmf;
    a.lam_tv = (float)lambda_tv;
    a.lam_l1 = (float)lambda_l1;
    a.lam_b = (float)lambda_b;
    int sms = 0;
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = (int)std::min<size_t>((size_t)grid_for(L, kJointBlock), (size_t)sms * 16);
    SW_CUDA(cudaMemsetAsync(u, 0, sizeof(float) * nu, st));
    SW_CUDA(cudaMemsetAsync(r, 0, sizeof(float) * nu, st));
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const double b = momentum == SWOPT_MOMENTUM_BECK_TEBOULLE ? (t - 1.0) / t1
                         : momentum == SWOPT_MOMENTUM_PAPER_PRINTED ? (t - 1.0) / (t + 1.0)
                                                                    : 0.0;
        const float beta = (float)b;
        t = t1;
        joint_lt_kernel<<<grid, kJointBlock, 0, st>>>(a, z, r, w);
        SW_LAUNCHED(h);
        joint_dual_kernel<<<grid, kJointBlock, 0, st>>>(a, w, r, u, (float)step2, (float)alpha,
                                                        beta);
        SW_LAUNCHED(h);
    }
    joint_lt_kernel<<<grid, kJointBlock, 0, st>>>(a, z, u, x);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status ensure_joint_buffers(swopt_handle* h)
{
    const size_t nu = joint_dual_floats(h);
    if (!h->jw) SW_CUDA(cudaMalloc((void**)&h->jw, sizeof(float) * nc_of(h)));
    if (!h->ju) SW_CUDA(cudaMalloc((void**)&h->ju, sizeof(float) * nu));
    if (!h->jr) SW_CUDA(cudaMalloc((void**)&h->jr, sizeof(float) * nu));
    return SWOPT_OK;
}

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
    SW_TRY(ensure_joint_buffers(h));
    return joint_prox_on(h, z_dev, x_dev, alpha, lambda_tv, lambda_l1, lambda_b, iters, step2,
                         SWOPT_MOMENTUM_BECK_TEBOULLE, h->jw, h->ju, h->jr, (cudaStream_t)stream);
}

double swopt_prox_joint_step_bound(swopt_handle* h, double lambda_tv, double lambda_l1,
                                   double lambda_b)
{
    if (!h) return 0.0;
    return joint_step_bound(h, lambda_tv, lambda_l1, lambda_b);
}

}  // extern "C"
