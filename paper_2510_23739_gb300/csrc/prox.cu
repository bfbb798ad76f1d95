// Memory-bound kernels of the FISTA iteration: the l1 and TV proximal maps
// (Eq. prox, Eq. prox-dual, Algorithm 2), the momentum update of Algorithm 1
// with its scalars kept on the device in FP64, and deterministic FP64
// reductions (fixed block count, fixed summation order).
//
// Layouts: volumes [P][Y][X][Z]; TV duals [3][P][Y][X][Z] with component 0
// along y, 1 along x, 2 along z (the entry of the last layer along an axis
// has no edge and stays zero).
#include <cmath>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

__device__ __forceinline__ float clampf(float v, float lo, float hi)
{
    return fminf(fmaxf(v, lo), hi);
}

__device__ __forceinline__ double block_sum(double v, double* sh)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

__global__ void prox_l1_kernel(float* __restrict__ x, size_t n, float th, int nonneg)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        float o;
        if (nonneg) o = fmaxf(v - th, 0.f);
        else o = v > th ? v - th : (v < -th ? v + th : 0.f);
        x[i] = o;
    }
}

struct Vol {
    int P, Y, X, Z;
    size_t L;  // P*Y*X*Z (component stride of the duals)
};

// (D^T q)[i] for the dual q (three components at stride L).
__device__ __forceinline__ float dtq(const float* __restrict__ q, const Vol& v, size_t i, int y,
                                     int x, int j)
{
    const size_t XZ = (size_t)v.X * v.Z;
    float acc = 0.f;
    if (y + 1 < v.Y) acc -= q[i];
    if (y > 0) acc += q[i - XZ];
    if (x + 1 < v.X) acc -= q[v.L + i];
    if (x > 0) acc += q[v.L + i - v.Z];
    if (j + 1 < v.Z) acc -= q[2 * v.L + i];
    if (j > 0) acc += q[2 * v.L + i - 1];
    return acc;
}

// Volume kernels use a 3D launch: threadIdx.x + 32 blockIdx.x runs along z,
// threadIdx.y + 8 blockIdx.y along x, blockIdx.z over (species, y).
struct VIdx {
    int j, x, y;
    size_t i;
    bool ok;
};

__device__ __forceinline__ VIdx vidx(const Vol& v)
{
    VIdx r;
    r.j = blockIdx.x * 32 + threadIdx.x;
    r.x = blockIdx.y * 8 + threadIdx.y;
    r.y = (int)(blockIdx.z % (unsigned)v.Y);
    const int p = (int)(blockIdx.z / (unsigned)v.Y);
    r.ok = r.j < v.Z && r.x < v.X;
    r.i = (((size_t)p * v.Y + r.y) * v.X + r.x) * v.Z + r.j;
    return r;
}

// One iteration of Algorithm 2 with L = D:
//   x   = z - D^T r_in          (recomputed at i and at its +y, +x, +z neighbours)
//   u_i = clamp(r_in + D x / 12, -tau, tau)
//   r_out = u_i + beta (u_i - u_{i-1})
// `first` means r_in = u_{i-1} = 0 (neither is read).
__global__ void __launch_bounds__(256) fgp_iter_kernel(const float* __restrict__ z,
                                                       const float* __restrict__ rin,
                                                       float* __restrict__ rout,
                                                       float* __restrict__ u, Vol v, float tau,
                                                       float beta, int first)
{
    const VIdx q = vidx(v);
    if (!q.ok) return;
    const size_t i = q.i, XZ = (size_t)v.X * v.Z;
    const int y = q.y, x = q.x, j = q.j;
    const bool has[3] = {y + 1 < v.Y, x + 1 < v.X, j + 1 < v.Z};
    const size_t step[3] = {XZ, (size_t)v.Z, 1};
    float xc, xn[3];
    if (first) {
        xc = z[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) xn[a] = has[a] ? z[i + step[a]] : 0.f;
    } else {
        xc = z[i] - dtq(rin, v, i, y, x, j);
        xn[0] = has[0] ? z[i + XZ] - dtq(rin, v, i + XZ, y + 1, x, j) : 0.f;
        xn[1] = has[1] ? z[i + v.Z] - dtq(rin, v, i + v.Z, y, x + 1, j) : 0.f;
        xn[2] = has[2] ? z[i + 1] - dtq(rin, v, i + 1, y, x, j + 1) : 0.f;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const size_t ia = (size_t)a * v.L + i;
        const float ra = first ? 0.f : rin[ia];
        const float ua_prev = first ? 0.f : u[ia];
        const float dx = has[a] ? xn[a] - xc : 0.f;
        const float un = clampf(fmaf(dx, 1.0f / 12.0f, ra), -tau, tau);
        u[ia] = un;
        rout[ia] = fmaf(beta, un - ua_prev, un);
    }
}

// x = z - D^T u
__global__ void __launch_bounds__(256) fgp_finish_kernel(const float* __restrict__ z,
                                                         const float* __restrict__ u,
                                                         float* __restrict__ xo, Vol v)
{
    const VIdx q = vidx(v);
    if (!q.ok) return;
    xo[q.i] = z[q.i] - dtq(u, v, q.i, q.y, q.x, q.j);
}

// End of one FISTA iteration (Algorithm 1):
//   x       = z - D^T u                 (TV prox output; x = z without TV)
//   c_{k+1} = max(x - theta, 0)        (l1 + nonnegativity)
//   xi      = c_{k+1} + beta_k (c_{k+1} - c_k),  beta_k from the device scalars
//   delta   = c_{k+1} - c_k                      (when delta is given)
__global__ void __launch_bounds__(256) fista_finish_kernel(const float* __restrict__ z,
                                                           const float* __restrict__ u,
                                                           float* __restrict__ c,
                                                           float* __restrict__ xi,
                                                           float* __restrict__ delta, Vol v,
                                                           float theta, int use_tv,
                                                           const double* __restrict__ scal)
{
    const VIdx q = vidx(v);
    if (!q.ok) return;
    const float beta = (float)scal[1];
    float xv = z[q.i];
    if (use_tv) xv -= dtq(u, v, q.i, q.y, q.x, q.j);
    const float cn = fmaxf(xv - theta, 0.f);
    const float d = cn - c[q.i];
    c[q.i] = cn;
    xi[q.i] = fmaf(beta, d, cn);
    if (delta) delta[q.i] = d;
}

// Momentum scalars of Algorithm 1 in FP64: scal[0] = t_k -> t_{k+1},
// scal[1] = beta_k.
__global__ void fista_scalars_kernel(double* scal, int mode)
{
    const double t = scal[0];
    const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    double beta = 0.0;
    if (mode == SWOPT_MOMENTUM_BECK_TEBOULLE) beta = (t - 1.0) / t1;
    else if (mode == SWOPT_MOMENTUM_PAPER_PRINTED) beta = (t - 1.0) / (t + 1.0);
    scal[1] = beta;
    scal[0] = t1;
}

__global__ void set_scalar_kernel(double* scal, int slot, double v) { scal[slot] = v; }

// ---- deterministic FP64 reductions (pass 1: fixed grid; pass 2: one block) ----
__global__ void red_sumsq_kernel(const float* __restrict__ x, size_t n, double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        s += v * v;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void red_dot_kernel(const float* __restrict__ x, const float* __restrict__ y, size_t n,
                               double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void red_abs_kernel(const float* __restrict__ x, size_t n, double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        s += fabs((double)x[i]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void red_tv_kernel(const float* __restrict__ x, Vol v, double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    const size_t XZ = (size_t)v.X * v.Z;
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < v.L;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % v.Z);
        const int xx = (int)((i / v.Z) % v.X);
        const int y = (int)((i / XZ) % v.Y);
        const double c = x[i];
        if (y + 1 < v.Y) s += fabs((double)x[i + XZ] - c);
        if (xx + 1 < v.X) s += fabs((double)x[i + v.Z] - c);
        if (j + 1 < v.Z) s += fabs((double)x[i + 1] - c);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) parts[blockIdx.x] = s;
}

__global__ void red_final_kernel(const double* parts, int count, double* out)
{
    __shared__ double sh[kRedThreads / 32];
    // fixed assignment of partials to threads, then a fixed tree: deterministic
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += parts[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

__global__ void scale_inv_sqrt_kernel(const float* __restrict__ in, float* __restrict__ out,
                                      size_t n, const double* __restrict__ s)
{
    const double inv = 1.0 / sqrt(*s);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)((double)in[i] * inv);
}

// splitmix64 (Steele, Lea, Flood 2014) of (seed + i), mapped to [-1, 1)
__global__ void counter_random_kernel(float* x, size_t n, uint64_t seed)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint64_t zz = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
        zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ull;
        zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBull;
        zz ^= zz >> 31;
        x[i] = (float)((double)(zz >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    }
}

// W[m][p][j] = sum_s g[m][s][j] c[p][s][j] in FP64 (one thread per (m, p, j),
// fixed order over s)
__global__ void param_weights_kernel(const float* __restrict__ g, const float* __restrict__ c,
                                     double* __restrict__ W, int Q, int P, int S, int Z)
{
    const int n = Q * P * Z;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = i % Z;
        const int p = (i / Z) % P;
        const int m = i / (Z * P);
        const float* gm = g + (size_t)m * S * Z + j;
        const float* cp = c + (size_t)p * S * Z + j;
        double s = 0.0;
        for (int q = 0; q < S; ++q) s += (double)gm[(size_t)q * Z] * (double)cp[(size_t)q * Z];
        W[i] = s;
    }
}

Vol vol_of(const swopt_handle* h)
{
    Vol v;
    v.P = h->P; v.Y = h->Y; v.X = h->X; v.Z = h->Z;
    v.L = nc_of(h);
    return v;
}

dim3 vol_grid(const Vol& v)
{
    return dim3((unsigned)((v.Z + 31) / 32), (unsigned)((v.X + 7) / 8), (unsigned)(v.P * v.Y));
}

const dim3 kVolBlock(32, 8);

int ew_grid(size_t n)
{
    int g = grid_for(n, 256);
    return g > 152 * 16 ? 152 * 16 : g;
}

}  // namespace

swopt_status prox_l1(swopt_handle* h, float* x, float thresh, int nonneg, cudaStream_t st)
{
    const size_t n = nc_of(h);
    prox_l1_kernel<<<ew_grid(n), 256, 0, st>>>(x, n, thresh, nonneg);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status prox_tv_iters(swopt_handle* h, const float* z, float tau, int iters,
                           const double* betas, cudaStream_t st)
{
    const Vol v = vol_of(h);
    float* rin = h->tvr0;
    float* rout = h->tvr1;
    for (int it = 0; it < iters; ++it) {
        fgp_iter_kernel<<<vol_grid(v), kVolBlock, 0, st>>>(z, rin, rout, h->tvu, v, tau,
                                                      (float)betas[it], it == 0 ? 1 : 0);
        SW_LAUNCHED(h);
        float* t = rin;
        rin = rout;
        rout = t;
    }
    return SWOPT_OK;
}

swopt_status prox_tv_finish(swopt_handle* h, const float* z, float* x, cudaStream_t st)
{
    const Vol v = vol_of(h);
    fgp_finish_kernel<<<vol_grid(v), kVolBlock, 0, st>>>(z, h->tvu, x, v);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status fista_finish(swopt_handle* h, const float* z, bool use_tv, float theta,
                          float* delta, cudaStream_t st)
{
    const Vol v = vol_of(h);
    fista_finish_kernel<<<vol_grid(v), kVolBlock, 0, st>>>(z, h->tvu, h->c, h->xi, delta, v,
                                                           theta, use_tv ? 1 : 0, h->scal);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status fista_scalars(swopt_handle* h, int momentum, cudaStream_t st)
{
    fista_scalars_kernel<<<1, 1, 0, st>>>(h->scal, momentum);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status fista_reset_scalars(swopt_handle* h, cudaStream_t st)
{
    set_scalar_kernel<<<1, 1, 0, st>>>(h->scal, 0, 1.0);
    SW_LAUNCHED(h);
    set_scalar_kernel<<<1, 1, 0, st>>>(h->scal, 1, 0.0);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

static swopt_status finish_reduction(swopt_handle* h, int count, int slot, cudaStream_t st)
{
    red_final_kernel<<<1, kRedThreads, 0, st>>>(h->red, count, h->scal + slot);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status reduce_sumsq(swopt_handle* h, const float* x, size_t n, int slot, cudaStream_t st)
{
    red_sumsq_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(x, n, h->red);
    SW_LAUNCHED(h);
    return finish_reduction(h, kRedBlocks, slot, st);
}

swopt_status reduce_dot(swopt_handle* h, const float* x, const float* y, size_t n, int slot,
                        cudaStream_t st)
{
    red_dot_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(x, y, n, h->red);
    SW_LAUNCHED(h);
    return finish_reduction(h, kRedBlocks, slot, st);
}

swopt_status reduce_abs(swopt_handle* h, const float* x, size_t n, int slot, cudaStream_t st)
{
    red_abs_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(x, n, h->red);
    SW_LAUNCHED(h);
    return finish_reduction(h, kRedBlocks, slot, st);
}

swopt_status reduce_tv(swopt_handle* h, const float* x, int slot, cudaStream_t st)
{
    red_tv_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(x, vol_of(h), h->red);
    SW_LAUNCHED(h);
    return finish_reduction(h, kRedBlocks, slot, st);
}

swopt_status reduce_partials(swopt_handle* h, const double* parts, int count, int slot,
                             cudaStream_t st)
{
    red_final_kernel<<<1, kRedThreads, 0, st>>>(parts, count, h->scal + slot);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status scale_by_inv_sqrt(swopt_handle* h, const float* in, float* out, size_t n, int slot,
                               cudaStream_t st)
{
    scale_inv_sqrt_kernel<<<ew_grid(n), 256, 0, st>>>(in, out, n, h->scal + slot);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status fill_counter_random(swopt_handle* h, float* x, size_t n, uint64_t seed,
                                 cudaStream_t st)
{
    counter_random_kernel<<<ew_grid(n), 256, 0, st>>>(x, n, seed);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status param_weights(swopt_handle* h, const float* g, const float* c, int slot0,
                           cudaStream_t st)
{
    const int n = h->Q * h->P * h->Z;
    param_weights_kernel<<<(n + 127) / 128, 128, 0, st>>>(g, c, h->red + slot0, h->Q, h->P, h->S,
                                                          h->Z);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

// Launchers on caller-given buffers, without a handle (used by the
// allocation-free entry point in noalloc.cu).
cudaError_t fgp_iter_on(const float* z, const float* rin, float* rout, float* u, int P, int Y,
                        int X, int Z, float tau, float beta, int first, cudaStream_t st)
{
    Vol v;
    v.P = P; v.Y = Y; v.X = X; v.Z = Z;
    v.L = (size_t)P * Y * X * Z;
    fgp_iter_kernel<<<vol_grid(v), kVolBlock, 0, st>>>(z, rin, rout, u, v, tau, beta, first);
    return cudaGetLastError();
}

cudaError_t fgp_finish_on(const float* z, const float* u, float* x, int P, int Y, int X, int Z,
                          cudaStream_t st)
{
    Vol v;
    v.P = P; v.Y = Y; v.X = X; v.Z = Z;
    v.L = (size_t)P * Y * X * Z;
    fgp_finish_kernel<<<vol_grid(v), kVolBlock, 0, st>>>(z, u, x, v);
    return cudaGetLastError();
}

}  // namespace swopt
