// Reverse-mode derivative of the unrolled solve with respect to the
// switching parameters: for a cotangent w on the output c_K of K FISTA
// iterations (Algorithm 1, with Algorithm 2 as the TV prox), the gradient of
// <w, c_K> with respect to kappa_p and mu of Eq. (final-H), with the step
// alpha, the weights and the iteration counts held fixed.
//
// Forward, the momentum iterates xi_k are stored (K volumes); backward, each
// iteration is recomputed from xi_k (z_k = xi_k - alpha H^T (H xi_k - y),
// then Algorithm 2 with its clamp masks recorded) and its adjoint taken:
//   xi_{k+1} = (1 + b_k) c_{k+1} - b_k c_k : cbar_{k+1} += (1 + b_k) xibar_{k+1},
//                                           cbar_k = -b_k xibar_{k+1}
//   c_{k+1} = max(x_k - alpha lambda_l1, 0): xbar = [x_k - alpha lambda_l1 > 0] cbar_{k+1}
//   x_k = prox(z_k)                         : zbar = prox'(z_k)^T xbar (Algorithm 2 reversed)
//   z_k = xi_k - alpha H^T (H xi_k - y)     : xibar_k = zbar - alpha H^T H zbar,
//       theta_bar -= alpha d/dtheta [<r_k, H zbar> + <H zbar, H xi_k>] (r_k, H zbar held)
// Algorithm 2 (per species, dual q, its momentum iterate, clamp to [-tau, tau]):
//   w_i = z - D^T q_{i-1};  v_i = q_{i-1} + D w_i / 12;  u_i = clamp(v_i);
//   q_i = u_i + b_i (u_i - u_{i-1});  x = z - D^T u_K
// reversed with m_i = [|v_i| < tau]:
//   ubar_K = -D xbar, zbar = xbar, qbar_K = 0;  for i = K .. 1:
//     s = m_i (ubar_i + (1 + b_i) qbar_i);  ubar_{i-1} = -b_i qbar_i
//     wbar = D^T s / 12;  zbar += wbar;  qbar_{i-1} = s - D wbar
// The derivatives with respect to theta of <r, H(theta) v> come from the
// operator's parameter-weight reduction and the chain rule through Eq.
// (final-H) (the same as swopt_param_vjp).
#include <cmath>
#include <vector>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kUBlock = 256;

struct UVol {
    int Y, X, Z;
    size_t L;  // P Y X Z: component stride of the dual fields
};

struct UIdx {
    int y, x, j;
};

__device__ __forceinline__ UIdx uidx(const UVol& v, size_t i)
{
    UIdx q;
    q.j = (int)(i % (size_t)v.Z);
    const size_t t = i / (size_t)v.Z;
    q.x = (int)(t % (size_t)v.X);
    q.y = (int)((t / (size_t)v.X) % (size_t)v.Y);
    return q;
}

// (D^T g)[i], g with three components at stride L, in the order of the TV
// prox kernels
__device__ __forceinline__ float dt_at(const float* __restrict__ g, const UVol& v, size_t i,
                                       const UIdx& q)
{
    const size_t XZ = (size_t)v.X * v.Z;
    float acc = 0.f;
    if (q.y + 1 < v.Y) acc -= g[i];
    if (q.y > 0) acc += g[i - XZ];
    if (q.x + 1 < v.X) acc -= g[v.L + i];
    if (q.x > 0) acc += g[v.L + i - v.Z];
    if (q.j + 1 < v.Z) acc -= g[2 * v.L + i];
    if (q.j > 0) acc += g[2 * v.L + i - 1];
    return acc;
}

// (D f)[c][i]: forward difference along component c (0 past the far face)
__device__ __forceinline__ float d_at(const float* __restrict__ f, const UVol& v, size_t i,
                                      const UIdx& q, int c)
{
    const size_t XZ = (size_t)v.X * v.Z;
    if (c == 0) return q.y + 1 < v.Y ? f[i + XZ] - f[i] : 0.f;
    if (c == 1) return q.x + 1 < v.X ? f[i + v.Z] - f[i] : 0.f;
    return q.j + 1 < v.Z ? f[i + 1] - f[i] : 0.f;
}

#define U_FOR(i, n)                                                                            \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n);                    \
         i += (size_t)gridDim.x * blockDim.x)

// out = z - D^T q (q null: out = z)
__global__ void u_primal_kernel(const float* __restrict__ z, const float* __restrict__ q,
                                float* __restrict__ out, UVol v)
{
    U_FOR(i, v.L) out[i] = q ? z[i] - dt_at(q, v, i, uidx(v, i)) : z[i];
}

// One dual step of Algorithm 2 with its clamp mask:
//   v = q + D w / 12; u = clamp(v); q = u + b (u - uprev); uprev = u; mask = [|v| < tau]
__global__ void u_dual_kernel(const float* __restrict__ w, float* __restrict__ q,
                              float* __restrict__ uprev, uint8_t* __restrict__ mask, UVol v,
                              float tau, float beta)
{
    U_FOR(i, v.L) {
        const UIdx p = uidx(v, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const size_t e = (size_t)c * v.L + i;
            const float val = fmaf(d_at(w, v, i, p, c), 1.0f / 12.0f, q[e]);
            const float un = fminf(fmaxf(val, -tau), tau);
            mask[e] = fabsf(val) < tau ? 1 : 0;
            q[e] = fmaf(beta, un - uprev[e], un);
            uprev[e] = un;
        }
    }
}

// xbar = [x - theta > 0] cbar (the l1 and nonnegativity step reversed)
__global__ void u_l1_back_kernel(const float* __restrict__ x, const float* __restrict__ cbar,
                                 float* __restrict__ xbar, float theta, size_t n)
{
    U_FOR(i, n) xbar[i] = x[i] - theta > 0.f ? cbar[i] : 0.f;
}

// ubar = -D xbar; qbar = 0
__global__ void u_back_init_kernel(const float* __restrict__ xbar, float* __restrict__ ubar,
                                   float* __restrict__ qbar, UVol v)
{
    U_FOR(i, v.L) {
        const UIdx p = uidx(v, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ubar[(size_t)c * v.L + i] = -d_at(xbar, v, i, p, c);
            qbar[(size_t)c * v.L + i] = 0.f;
        }
    }
}

// s = m (ubar + (1 + b) qbar); ubar = -b qbar
__global__ void u_back_s_kernel(const uint8_t* __restrict__ mask, float* __restrict__ ubar,
                                const float* __restrict__ qbar, float* __restrict__ s, size_t n3,
                                float beta)
{
    U_FOR(e, n3) {
        const float qb = qbar[e];
        s[e] = mask[e] ? ubar[e] + (1.0f + beta) * qb : 0.f;
        ubar[e] = -beta * qb;
    }
}

// wbar = D^T s / 12; zbar += wbar
__global__ void u_back_w_kernel(const float* __restrict__ s, float* __restrict__ wbar,
                                float* __restrict__ zbar, UVol v)
{
    U_FOR(i, v.L) {
        const float wb = dt_at(s, v, i, uidx(v, i)) * (1.0f / 12.0f);
        wbar[i] = wb;
        zbar[i] += wb;
    }
}

// qbar = s - D wbar
__global__ void u_back_q_kernel(const float* __restrict__ s, const float* __restrict__ wbar,
                                float* __restrict__ qbar, UVol v)
{
    U_FOR(i, v.L) {
        const UIdx p = uidx(v, i);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            qbar[(size_t)c * v.L + i] = s[(size_t)c * v.L + i] - d_at(wbar, v, i, p, c);
    }
}

// y = a x + b y
__global__ void u_axpby_kernel(float a, const float* __restrict__ x, float b, float* __restrict__ y,
                               size_t n)
{
    U_FOR(i, n) y[i] = fmaf(a, x[i], b * y[i]);
}

int ugrid(size_t n)
{
    const size_t g = (n + kUBlock - 1) / kUBlock;
    return (int)(g < 152 * 32 ? g : 152 * 32);
}

double momentum_beta(int mode, double t, double t1)
{
    if (mode == SWOPT_MOMENTUM_BECK_TEBOULLE) return (t - 1.0) / t1;
    if (mode == SWOPT_MOMENTUM_PAPER_PRINTED) return (t - 1.0) / (t + 1.0);
    return 0.0;
}

double next_t(double t) { return 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t)); }

struct DevBuf {
    float* p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace

// the FISTA step of one iteration, the handle's helpers from api.cu
swopt_status fista_iterate_once(swopt_handle* h, cudaStream_t st);
swopt_status apply_forward_residual(swopt_handle* h, const float* v, const float* ytil,
                                    cudaStream_t st);
swopt_status apply_adjoint_folded(swopt_handle* h, cudaStream_t st);
void chain_rule(const swopt_handle* h, const std::vector<double>& W, double* dkappa,
                double* dmu);

}  // namespace swopt

using namespace swopt;

extern "C" swopt_status swopt_unrolled_vjp(swopt_handle* h, const float* y_dev,
                                           const swopt_solve_params* prm, const float* w_dev,
                                           float* c_dev, double* dkappa_host, double* dmu,
                                           void* stream)
{
    clear_error();
    if (!h) {
        set_error("null handle");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!y_dev || !prm || !w_dev || !dkappa_host || !dmu) {
        set_error("null argument");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!(prm->step > 0) || prm->max_iters < 1 || prm->refine_every != 0 || prm->lambda_3 != 0 ||
        prm->eps1 > 0 || prm->eps2 > 0) {
        set_error("the unrolled derivative needs an explicit step, max_iters >= 1, no "
                  "refinement, lambda_3 = 0 and no stopping tests");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int K = prm->max_iters;
    const size_t nc = nc_of(h), n3 = 3 * nc;
    const bool tv = prm->lambda_tv > 0 && prm->inner_iters > 0;
    const int inner = tv ? prm->inner_iters : 0;
    const float alpha = (float)prm->step;
    const float tau = (float)(prm->step * prm->lambda_tv);
    const float theta = (float)(prm->step * prm->lambda_l1);
    UVol v;
    v.Y = h->Y;
    v.X = h->X;
    v.Z = h->Z;
    v.L = nc;

    // storage: xi_k for every iteration, the adjoint vectors, Algorithm 2's state and masks
    DevBuf XI, work, masks;
    const size_t nwork = 8 * nc + 4 * n3;
    SW_CUDA(cudaMalloc((void**)&XI.p, sizeof(float) * (size_t)K * nc));
    SW_CUDA(cudaMalloc((void**)&work.p, sizeof(float) * nwork));
    if (inner > 0)
        SW_CUDA(cudaMalloc((void**)&masks.p, (size_t)inner * n3 + 16));
    uint8_t* mk = reinterpret_cast<uint8_t*>(masks.p);
    float* cbar = work.p;
    float* cnext = cbar + nc;
    float* xibar = cnext + nc;
    float* z = xibar + nc;
    float* x = z + nc;
    float* xbar = x + nc;
    float* zbar = xbar + nc;
    float* wbar = zbar + nc;
    float* q = wbar + nc;
    float* up = q + n3;
    float* ubar = up + n3;
    float* qbar = ubar + n3;
    DevBuf sbuf;
    SW_CUDA(cudaMalloc((void**)&sbuf.p, sizeof(float) * n3));
    float* s3 = sbuf.p;

    // forward: the solve, keeping xi_k
    SW_TRY(fista_init_impl(h, y_dev, prm, st));
    for (int k = 0; k < K; ++k) {
        SW_CUDA(cudaMemcpyAsync(XI.p + (size_t)k * nc, h->xi, sizeof(float) * nc,
                                cudaMemcpyDeviceToDevice, st));
        SW_TRY(fista_iterate_once(h, st));
    }
    if (c_dev)
        SW_CUDA(cudaMemcpyAsync(c_dev, h->c, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));

    // the outer and inner momentum coefficients
    std::vector<double> bo(K), bi(inner > 0 ? inner : 1);
    {
        double t = 1.0;
        for (int k = 0; k < K; ++k) {
            const double t1 = next_t(t);
            bo[k] = momentum_beta(prm->momentum, t, t1);
            t = t1;
        }
        t = 1.0;
        for (int i = 0; i < inner; ++i) {
            const double t1 = next_t(t);
            bi[i] = momentum_beta(prm->inner_momentum, t, t1);
            t = t1;
        }
    }

    const int g1 = ugrid(nc), g3 = ugrid(n3);
    SW_CUDA(cudaMemcpyAsync(cbar, w_dev, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));
    SW_CUDA(cudaMemsetAsync(xibar, 0, sizeof(float) * nc, st));
    std::vector<double> dk(h->P, 0.0);
    double dm_total = 0.0;
    const size_t nw = (size_t)h->Q * h->P * h->Z;
    std::vector<double> W1(nw), W2(nw);
    for (int k = K - 1; k >= 0; --k) {
        const float* xik = XI.p + (size_t)k * nc;
        const float b = (float)bo[k];
        // xi_{k+1} = (1 + b) c_{k+1} - b c_k
        u_axpby_kernel<<<g1, kUBlock, 0, st>>>(1.0f + b, xibar, 1.0f, cbar, nc);
        SW_LAUNCHED(h);
        SW_CUDA(cudaMemsetAsync(cnext, 0, sizeof(float) * nc, st));
        u_axpby_kernel<<<g1, kUBlock, 0, st>>>(-b, xibar, 1.0f, cnext, nc);
        SW_LAUNCHED(h);
        // z_k, with A^T of the folded residual r_k left in h->g
        SW_TRY(apply_forward_residual(h, xik, h->ytil, st));
        SW_TRY(apply_adjoint_folded(h, st));
        SW_TRY(launch_pt(h, h->g, xik, alpha, z, 1, st));
        // Algorithm 2 forward with its masks, x_k
        if (inner > 0) {
            SW_CUDA(cudaMemsetAsync(q, 0, sizeof(float) * n3, st));
            SW_CUDA(cudaMemsetAsync(up, 0, sizeof(float) * n3, st));
            for (int i = 0; i < inner; ++i) {
                u_primal_kernel<<<g1, kUBlock, 0, st>>>(z, i == 0 ? nullptr : q, x, v);
                SW_LAUNCHED(h);
                u_dual_kernel<<<g1, kUBlock, 0, st>>>(x, q, up, mk + (size_t)i * n3, v, tau,
                                                      (float)bi[i]);
                SW_LAUNCHED(h);
            }
            u_primal_kernel<<<g1, kUBlock, 0, st>>>(z, up, x, v);
            SW_LAUNCHED(h);
        } else {
            SW_CUDA(cudaMemcpyAsync(x, z, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));
        }
        // l1 and nonnegativity reversed, then Algorithm 2 reversed
        u_l1_back_kernel<<<g1, kUBlock, 0, st>>>(x, cbar, xbar, theta, nc);
        SW_LAUNCHED(h);
        SW_CUDA(cudaMemcpyAsync(zbar, xbar, sizeof(float) * nc, cudaMemcpyDeviceToDevice, st));
        if (inner > 0) {
            u_back_init_kernel<<<g1, kUBlock, 0, st>>>(xbar, ubar, qbar, v);
            SW_LAUNCHED(h);
            for (int i = inner - 1; i >= 0; --i) {
                u_back_s_kernel<<<g3, kUBlock, 0, st>>>(mk + (size_t)i * n3, ubar, qbar, s3, n3,
                                                        (float)bi[i]);
                SW_LAUNCHED(h);
                u_back_w_kernel<<<g1, kUBlock, 0, st>>>(s3, wbar, zbar, v);
                SW_LAUNCHED(h);
                u_back_q_kernel<<<g1, kUBlock, 0, st>>>(s3, wbar, qbar, v);
                SW_LAUNCHED(h);
            }
        }
        // theta: <r_k, H(theta) zbar>, with A^T r_k (folded) in h->g
        SW_TRY(param_weights(h, h->g, zbar, 0, st));
        SW_CUDA(cudaMemcpyAsync(W1.data(), h->red, nw * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
        SW_CUDA(cudaStreamSynchronize(st));
        // <H zbar, H(theta) xi_k>, and xibar_k = zbar - alpha H^T H zbar
        SW_TRY(apply_forward_residual(h, zbar, nullptr, st));
        SW_TRY(apply_adjoint_folded(h, st));
        SW_TRY(param_weights(h, h->g, xik, 0, st));
        SW_CUDA(cudaMemcpyAsync(W2.data(), h->red, nw * sizeof(double), cudaMemcpyDeviceToHost,
                                st));
        SW_TRY(launch_pt(h, h->g, zbar, alpha, xibar, 1, st));
        SW_CUDA(cudaStreamSynchronize(st));
        for (size_t i = 0; i < nw; ++i) W1[i] += W2[i];
        std::vector<double> dkk(h->P);
        double dmk = 0.0;
        chain_rule(h, W1, dkk.data(), &dmk);
        for (int p = 0; p < h->P; ++p) dk[p] -= prm->step * dkk[p];
        dm_total -= prm->step * dmk;
        std::swap(cbar, cnext);
    }
    SW_CUDA(cudaStreamSynchronize(st));
    for (int p = 0; p < h->P; ++p) dkappa_host[p] = dk[p];
    *dmu = dm_total;
    return SWOPT_OK;
}
