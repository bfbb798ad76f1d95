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
// clamp and the momentum step fused, the second split over a grid dimension
// into the species entries and groups of kStateChunk switching states.  Per
// dual iteration they move (nd + 2 P) + (4 nd + P) volumes, nd = 4 P + 3 Q.
// Both are templated on P so that the per-species values stay in registers,
// and issue the loads of a group of states before their arithmetic (a thread
// keeps several loads in flight; measured on GB300 at 128 x 128 x 96, P = 3,
// Q = 10: 0.26 of the HBM copy rate one state at a time, 0.78 like this).
// The first iteration reads no dual (r = u = 0).  Scratch (w, u, r) is the
// handle's.
#include <cmath>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kJointBlock = 256;
constexpr int kJointMaxSpecies = 8;
constexpr int kStateChunk = 4;  // switching states whose loads are issued together

struct JointArgs {
    int P, Q, Y, X, Z;
    const float* Sm;   // [Q][P][Z] switching weights of the states
    const float* Cmf;  // [Q] pulses per state
    float lam_tv, lam_l1, lam_b;
};

// Voxel i = (y X + x) Z + j of a volume with fewer than 2^31 voxels.
struct Vox {
    int y, x, j;
    __device__ __forceinline__ Vox(unsigned i, const JointArgs& a)
    {
        const unsigned t = i / (unsigned)a.Z;
        j = (int)(i - t * (unsigned)a.Z);
        y = (int)(t / (unsigned)a.X);
        x = (int)(t - (unsigned)y * (unsigned)a.X);
    }
};

// The six terms of (D^T g)[i] for one field g[3][L] (components y, x, z),
// 0 where the difference does not exist; D^T g = v1 - v0 + v3 - v2 + v5 - v4.
__device__ __forceinline__ void load_dt(const float* g, size_t L, size_t i, size_t sy, size_t sx,
                                        const Vox& p, const JointArgs& a, float (&v)[6])
{
    v[0] = p.y + 1 < a.Y ? g[i] : 0.f;
    v[1] = p.y > 0 ? g[i - sy] : 0.f;
    v[2] = p.x + 1 < a.X ? g[L + i] : 0.f;
    v[3] = p.x > 0 ? g[L + i - sx] : 0.f;
    v[4] = p.j + 1 < a.Z ? g[2 * L + i] : 0.f;
    v[5] = p.j > 0 ? g[2 * L + i - 1] : 0.f;
}

__device__ __forceinline__ float dt_value(const float (&v)[6])
{
    return ((v[1] - v[0]) + (v[3] - v[2])) + (v[5] - v[4]);
}

// out = max(z - L^T r, 0), one thread per voxel, all NP species (r null:
// r = 0).  z and out may be the same array: each thread reads z at its voxel
// before writing there.  The loads of kStateChunk states are issued before
// their arithmetic, so that a thread keeps several of them in flight.
template <int NP>
__global__ void __launch_bounds__(kJointBlock, NP <= 4 ? 4 : 3)
    joint_lt_kernel(const JointArgs a, const float* z, const float* __restrict__ r, float* out)
{
    const unsigned L = (unsigned)a.Y * a.X * a.Z;
    const size_t Ls = L, sy = (size_t)a.X * a.Z, sx = (size_t)a.Z;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        const Vox q(i, a);
        float acc[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) acc[p] = 0.f;
        if (r) {
            const float* rl = r + (size_t)NP * 3 * Ls;
            const float* rb = rl + (size_t)NP * Ls;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float v[6];
                load_dt(r + (size_t)p * 3 * Ls, Ls, i, sy, sx, q, a, v);
                acc[p] = a.lam_tv * dt_value(v) + a.lam_l1 * rl[(size_t)p * Ls + i];
            }
            for (int m0 = 0; m0 < a.Q; m0 += kStateChunk) {
                float v[kStateChunk][6];
#pragma unroll
                for (int c = 0; c < kStateChunk; ++c) {
                    if (m0 + c < a.Q) {
                        load_dt(rb + (size_t)(m0 + c) * 3 * Ls, Ls, i, sy, sx, q, a, v[c]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 6; ++e) v[c][e] = 0.f;
                    }
                }
#pragma unroll
                for (int c = 0; c < kStateChunk; ++c) {
                    const int m = m0 + c;
                    if (m < a.Q) {
                        const float d = a.Cmf[m] * a.lam_b * dt_value(v[c]);
                        const float* s = a.Sm + (size_t)m * NP * a.Z + q.j;
#pragma unroll
                        for (int p = 0; p < NP; ++p) acc[p] = fmaf(s[(size_t)p * a.Z], d, acc[p]);
                    }
                }
            }
        }
        float v[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) v[p] = fmaxf(z[(size_t)p * Ls + i] - acc[p], 0.f);
#pragma unroll
        for (int p = 0; p < NP; ++p) out[(size_t)p * Ls + i] = v[p];
    }
}

// u_new = clamp(r + step2 lw, -alpha, alpha); r_new = u_new + beta (u_new - u)
__device__ __forceinline__ void dual_update(float& rv, float& uv, float lw, float step2,
                                            float alpha, float beta)
{
    float v = fmaf(step2, lw, rv);
    v = fminf(fmaxf(v, -alpha), alpha);
    rv = fmaf(beta, v - uv, v);
    uv = v;
}

// The dual update, one thread per voxel and entry group: blockIdx.y = 0 takes
// the species entries (3 TV components and the l1 entry of each species),
// blockIdx.y = g >= 1 the pulse-image TV entries of the switching states
// [(g - 1) kStateChunk, g kStateChunk).  first: the previous r and u are
// zero and are not read.
template <int NP>
__global__ void __launch_bounds__(kJointBlock, NP <= 4 ? 4 : 3)
    joint_dual_kernel(const JointArgs a, const float* __restrict__ w, float* __restrict__ r,
                      float* __restrict__ u, float step2, float alpha, float beta, int first)
{
    const unsigned L = (unsigned)a.Y * a.X * a.Z;
    const size_t Ls = L, sy = (size_t)a.X * a.Z, sx = (size_t)a.Z;
    const size_t ol = (size_t)NP * 3 * Ls, ob = ol + (size_t)NP * Ls;
    const int group = blockIdx.y;
    const int m0 = (group - 1) * kStateChunk;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        const Vox q(i, a);
        const bool hy = q.y + 1 < a.Y, hx = q.x + 1 < a.X, hz = q.j + 1 < a.Z;
        // w at the voxel and its three forward neighbours (0 past the far faces)
        float w0[NP], wy[NP], wx[NP], wz[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const float* wp = w + (size_t)p * Ls;
            w0[p] = wp[i];
            wy[p] = hy ? wp[i + sy] : 0.f;
            wx[p] = hx ? wp[i + sx] : 0.f;
            wz[p] = hz ? wp[i + 1] : 0.f;
        }
        if (group == 0) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const size_t e[4] = {(size_t)p * 3 * Ls + i, (size_t)p * 3 * Ls + Ls + i,
                                     (size_t)p * 3 * Ls + 2 * Ls + i, ol + (size_t)p * Ls + i};
                float rv[4], uv[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    rv[c] = first ? 0.f : r[e[c]];
                    uv[c] = first ? 0.f : u[e[c]];
                }
                const float lw[4] = {hy ? a.lam_tv * (wy[p] - w0[p]) : 0.f,
                                     hx ? a.lam_tv * (wx[p] - w0[p]) : 0.f,
                                     hz ? a.lam_tv * (wz[p] - w0[p]) : 0.f, a.lam_l1 * w0[p]};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    dual_update(rv[c], uv[c], lw[c], step2, alpha, beta);
                    r[e[c]] = rv[c];
                    u[e[c]] = uv[c];
                }
            }
            continue;
        }
        float rv[kStateChunk][3], uv[kStateChunk][3];
#pragma unroll
        for (int c = 0; c < kStateChunk; ++c) {
            const size_t e = ob + (size_t)(m0 + c) * 3 * Ls + i;
            const bool ld = !first && m0 + c < a.Q;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                rv[c][k] = ld ? r[e + k * Ls] : 0.f;
                uv[c][k] = ld ? u[e + k * Ls] : 0.f;
            }
        }
#pragma unroll
        for (int c = 0; c < kStateChunk; ++c) {
            const int m = m0 + c;
            if (m < a.Q) {
                const float* s = a.Sm + (size_t)m * NP * a.Z;
                float b0 = 0.f, by = 0.f, bx = 0.f, bz = 0.f;
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float sj = s[(size_t)p * a.Z + q.j];
                    b0 = fmaf(sj, w0[p], b0);
                    by = fmaf(sj, wy[p], by);
                    bx = fmaf(sj, wx[p], bx);
                    if (hz) bz = fmaf(s[(size_t)p * a.Z + q.j + 1], wz[p], bz);
                }
                const float lw[3] = {hy ? a.lam_b * (by - b0) : 0.f,
                                     hx ? a.lam_b * (bx - b0) : 0.f,
                                     hz ? a.lam_b * (bz - b0) : 0.f};
                const size_t e = ob + (size_t)m * 3 * Ls + i;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    dual_update(rv[c][k], uv[c][k], lw[k], step2, alpha, beta);
                    r[e + k * Ls] = rv[c][k];
                    u[e + k * Ls] = uv[c][k];
                }
            }
        }
    }
}

template <int NP>
swopt_status launch_joint_iteration(swopt_handle* h, const JointArgs& a, const float* z,
                                    const float* rin, float* out, float* w, float* r, float* u,
                                    float step2, float alpha, float beta, int first, bool dual,
                                    int grid, cudaStream_t st)
{
    joint_lt_kernel<NP><<<grid, kJointBlock, 0, st>>>(a, z, rin, dual ? w : out);
    SW_LAUNCHED(h);
    if (!dual) return SWOPT_OK;
    const dim3 g2(grid, 1 + (a.Q + kStateChunk - 1) / kStateChunk);
    joint_dual_kernel<NP><<<g2, kJointBlock, 0, st>>>(a, w, r, u, step2, alpha, beta, first);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

// One dual iteration (dual = true: L^T of rin into w, then the dual update)
// or the primal recovery (dual = false: out = max(z - L^T rin, 0)).
swopt_status joint_iteration(swopt_handle* h, const JointArgs& a, const float* z,
                             const float* rin, float* out, float* w, float* r, float* u,
                             float step2, float alpha, float beta, int first, bool dual, int grid,
                             cudaStream_t st)
{
    switch (a.P) {
#define SWOPT_JOINT_CASE(n)                                                                   \
    case n:                                                                                   \
        return launch_joint_iteration<n>(h, a, z, rin, out, w, r, u, step2, alpha, beta, first, \
                                         dual, grid, st);
        SWOPT_JOINT_CASE(1)
        SWOPT_JOINT_CASE(2)
        SWOPT_JOINT_CASE(3)
        SWOPT_JOINT_CASE(4)
        SWOPT_JOINT_CASE(5)
        SWOPT_JOINT_CASE(6)
        SWOPT_JOINT_CASE(7)
        SWOPT_JOINT_CASE(8)
#undef SWOPT_JOINT_CASE
    }
    set_error("the joint prox supports 1 to %d species", kJointMaxSpecies);
    return SWOPT_ERR_UNSUPPORTED;
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
    if (L >= (1ull << 31)) {
        set_error("the joint prox supports volumes below 2^31 voxels");
        return SWOPT_ERR_UNSUPPORTED;
    }
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
    // the first iteration starts from r = u = 0 without reading them
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        const double b = momentum == SWOPT_MOMENTUM_BECK_TEBOULLE ? (t - 1.0) / t1
                         : momentum == SWOPT_MOMENTUM_PAPER_PRINTED ? (t - 1.0) / (t + 1.0)
                                                                    : 0.0;
        t = t1;
        SW_TRY(joint_iteration(h, a, z, it == 0 ? nullptr : r, nullptr, w, r, u, (float)step2,
                               (float)alpha, (float)b, it == 0 ? 1 : 0, true, grid, st));
    }
    SW_TRY(joint_iteration(h, a, z, iters > 0 ? u : nullptr, x, w, r, u, 0.f, 0.f, 0.f, 0,
                           false, grid, st));
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
