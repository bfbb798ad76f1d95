// Memory-bound kernels of the FISTA iteration: the l1 and TV proximal maps
// (Eq. prox, Eq. prox-dual, Algorithm 2), the momentum update of Algorithm 1
// with its scalars kept on the device in FP64, and deterministic FP64
// reductions (fixed block count, fixed summation order).
//
// Layouts: volumes [P][Y][X][Z]; TV duals [3][P][Y][X][Z] with component 0
// along y, 1 along x, 2 along z (the entry of the last layer along an axis
// has no edge and stays zero).
#include <algorithm>
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

__device__ __forceinline__ float soft(float v, float th, int nonneg)
{
    if (nonneg) return fmaxf(v - th, 0.f);
    return v > th ? v - th : (v < -th ? v + th : 0.f);
}

// In place; 16-byte accesses over the first n4 = n / 4 groups when x is
// 16-byte aligned (n4 = 0 otherwise), then the remaining entries.
__global__ void prox_l1_kernel(float* __restrict__ x, size_t n, size_t n4, float th, int nonneg)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t first = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    float4* x4 = reinterpret_cast<float4*>(x);
    for (size_t i = first; i < n4; i += stride) {
        float4 v = x4[i];
        v.x = soft(v.x, th, nonneg);
        v.y = soft(v.y, th, nonneg);
        v.z = soft(v.z, th, nonneg);
        v.w = soft(v.w, th, nonneg);
        x4[i] = v;
    }
    for (size_t i = 4 * n4 + first; i < n; i += stride) x[i] = soft(x[i], th, nonneg);
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

// ---------------------------------------------------------------------------
// The whole TV prox in one cooperative launch: every block of a grid sized to
// be co-resident loops over the volume, one grid-wide barrier per inner
// iteration i of Algorithm 2.  The volume is cut into tiles of 8 x 8 columns
// x 32 depths; per tile a block
//   1. computes x = z - D^T r_{i-1} (x = z for i = 1, where r = 0) on the
//      tile and on the points its forward differences reach (its +y and +x
//      faces and its +z cap), into shared memory, keeping the tile's r_{i-1};
//   2. takes u_i = clamp(r_{i-1} + D x / 12, -tau, tau) and
//      r_i = u_i + beta_i (u_i - u_{i-1}) on the tile (r ping-pongs between
//      two arrays, u is updated in place).
// After the last iteration: x = z - D^T u_K written out (mode 0), or the end
// of the FISTA iteration with the momentum scalars updated here (mode 1, as
// fista_finish_kernel).  The inner coefficients beta_i follow Algorithm 2's
// t recursion in FP64.  HBM traffic per entry and iteration is the 52
// algorithmic bytes (read z, r and the previous u, three components each;
// write u and r) plus the halo columns' share of z and r, which mostly hit L2
// because neighbouring tiles run at the same time.  Each warp loads
// kStBatch work units (32 points each) before it uses any of them.  On a
// GB300 this runs the 2 x 1024 x 512 x 256 sweep volume at 4.51 TB/s of
// algorithmic traffic and the 3 x 128 x 128 x 96 volume at 4.15 TB/s.  The
// same arithmetic in two phases per iteration (x through memory, 72 B moved,
// two barriers) ran at 4.35 / 3.56 TB/s.  One unit per warp at a time was
// latency-bound at 1.13 TB/s, and five blocks per SM with three units each
// ran at 4.09 TB/s.
// ---------------------------------------------------------------------------
constexpr int kCoopThreads = 256;
// Tiles of the single-barrier iteration: kStTY x kStTX columns x kStZC depths.
// x is computed on the tile and on the points its forward differences reach
// (the +y and +x faces, kStBoxCols columns with the tile's own, and the +z
// cap, kStTY * kStTX points in whole warps).
constexpr int kStTY = 8, kStTX = 8, kStZC = 32;
constexpr int kStBoxCols = kStTY * kStTX + kStTY + kStTX;
constexpr int kStUnits = kStBoxCols + (kStTY * kStTX + 31) / 32;
constexpr int kStBatch = 4;  // units a warp loads before it computes
constexpr uint32_t kBarrierPolls = 1u << 25;  // x 32 ns back-off: about a second

// Grid barrier over all blocks of a cooperative launch.  bar[0] counts
// arrivals, bar[1] is the generation, bar[2] an error word: a block that polls
// kBarrierPolls times without seeing the generation advance sets it, and from
// then on every barrier returns at once (the results are then invalid and the
// host reports a timeout).  bar[4] and bar[5] are a failure-detection test
// hook (swopt_debug_barrier): blocks the barrier waits for beyond the launch's
// own, and a poll limit replacing kBarrierPolls (0: the default).
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The arrival is an acquire-release atomic and the generation bump a release
// reduction, so the block's writes before the barrier are visible to every
// block that has observed the new generation with an acquire load; the CTA
// barriers extend that to all threads of the block.
__device__ __forceinline__ void grid_sync(unsigned* bar, unsigned nblocks)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vb = bar;
        if (vb[2] == 0u) {
            const unsigned expected = nblocks + vb[4];
            uint32_t limit = kBarrierPolls;
            if (vb[5] != 0u) limit = vb[5];
            const unsigned gen = ld_acquire(bar + 1);
            unsigned arrived;
            asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;"
                         : "=r"(arrived) : "l"(bar) : "memory");
            if (arrived == expected - 1) {
                atomicExch(&bar[0], 0u);
                asm volatile("red.release.gpu.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
            } else {
                uint32_t polls = 0;
                while (ld_acquire(bar + 1) == gen && vb[2] == 0u) {
                    if (++polls > limit) {
                        atomicExch(&bar[2], 1u);
                        break;
                    }
                    if (polls > 256) __nanosleep(32);
                }
            }
        }
    }
    __syncthreads();
}

// 4-byte asynchronous global -> shared copy (completed by cp_async_wait).
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// 16-byte asynchronous copy through L2 only (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(float* dst, const float* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// One column of Z floats, global -> shared, asynchronously by one warp:
// 16-byte copies when `vec` (Z a multiple of 4 and every source array 16-byte
// aligned, so that each column starts on a 16-byte boundary in both spaces),
// else 4-byte copies.
__device__ __forceinline__ void copy_column(float* dst, const float* src, int Z, int lane,
                                            bool vec)
{
    if (vec) {
        for (int j = 4 * lane; j < Z; j += 128) cp_async16(dst + j, src + j);
    } else {
        for (int j = lane; j < Z; j += 32) cp_async4(dst + j, src + j);
    }
}

__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

struct FgpCoop {
    const float* z;  // prox input
    float* u;        // dual iterate [3][L]
    float* r0;       // extrapolated duals (ping-pong) [3][L]
    float* r1;
    Vol v;
    float tau;
    int iters;       // >= 1
    int inner_momentum;
    int mode;        // 0: out = z - D^T u;  1: FISTA finish
    float* out;
    float* c;
    float* xi;
    float* delta;    // optional (mode 1)
    double* scal;    // FISTA t_k, beta_k (mode 1)
    int momentum;
    float theta;
    unsigned* bar;
    int TY, TX;      // shared-memory variant: tile of TY x TX columns of all z
    int tilesY, tilesX;
    bool vec;        // 16-byte column copies allowed (see copy_column)
};

__device__ __forceinline__ double momentum_coef(double t, double t1, int mode)
{
    if (mode == SWOPT_MOMENTUM_BECK_TEBOULLE) return (t - 1.0) / t1;
    if (mode == SWOPT_MOMENTUM_PAPER_PRINTED) return (t - 1.0) / (t + 1.0);
    return 0.0;
}

// Work split of the cooperative kernel: warp w of the grid takes the rows
// (p, y, x) = w, w + warps, ...; its lanes run along z (coalesced).  `body`
// is called with the row's coordinates and the linear index of its z = 0.
template <typename F>
__device__ __forceinline__ void for_rows(const Vol& v, F body)
{
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const unsigned w0 = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned rows = (unsigned)v.P * v.Y * v.X;
    for (unsigned row = w0; row < rows; row += warps) {
        const int x = (int)(row % (unsigned)v.X);
        const int y = (int)((row / (unsigned)v.X) % (unsigned)v.Y);
        body(y, x, (size_t)row * v.Z);
    }
}

__global__ void __launch_bounds__(kCoopThreads, 4) fgp_coop_kernel(const FgpCoop a)
{
    const Vol v = a.v;
    const size_t L = v.L, XZ = (size_t)v.X * v.Z;
    const int lane = threadIdx.x & 31;
    const unsigned nb = gridDim.x;
    if (a.mode == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        // Algorithm 1's t_k -> t_{k+1} and beta_k, read after the barriers below
        const double t = a.scal[0];
        const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        a.scal[1] = momentum_coef(t, t1, a.momentum);
        a.scal[0] = t1;
    }
    const float* rin = a.r0;
    float* rout = a.r1;
    // Algorithm 2's t recursion runs in FP64 in one thread per block (FP64
    // arithmetic is scarce on this GPU) and reaches the block through shared
    // memory
    __shared__ float s_beta;
    __shared__ float xs[kStTY + 1][kStTX + 1][kStZC + 1];
    __shared__ float rs[3][kStTY * kStTX][kStZC];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int tY = (v.Y + kStTY - 1) / kStTY, tX = (v.X + kStTX - 1) / kStTX;
    const int tZ = (v.Z + kStZC - 1) / kStZC;
    const long long ntiles = (long long)v.P * tY * tX * tZ;
    double t = 1.0;
    for (int it = 0; it < a.iters; ++it) {
        if (threadIdx.x == 0) {
            const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            s_beta = (float)momentum_coef(t, t1, a.inner_momentum);
            t = t1;
        }
        __syncthreads();
        const float beta = s_beta;
        for (long long tile = blockIdx.x; tile < ntiles; tile += nb) {
            long long q = tile;
            const int z0 = (int)(q % tZ) * kStZC;
            q /= tZ;
            const int x0 = (int)(q % tX) * kStTX;
            q /= tX;
            const int y0 = (int)(q % tY) * kStTY;
            const size_t pbase = (size_t)(q / tY) * v.Y * XZ;
            // x = z - D^T r_{i-1} on the tile, on its +y and +x faces and on
            // its +z cap (the points the forward differences reach), into
            // shared memory; the tile's r_{i-1} is kept there too
            // (kStBatch units per warp at a time, every load issued before any use)
            for (int u0 = warp; u0 < kStUnits; u0 += nwarps * kStBatch) {
                float zv[kStBatch], c0[kStBatch], c1[kStBatch], c2[kStBatch];
                float b0[kStBatch], b1[kStBatch], b2[kStBatch];
                int pos[kStBatch];  // yy | xx << 8 | zz << 16, or -1
#pragma unroll
                for (int k = 0; k < kStBatch; ++k) {
                    const int unit = u0 + k * nwarps;
                    int yy = 0, xx = 0, zz = lane;
                    bool ok = unit < kStUnits;
                    if (unit < kStTY * kStTX) {
                        yy = unit / kStTX;
                        xx = unit % kStTX;
                    } else if (unit < kStTY * kStTX + kStTX) {
                        yy = kStTY;
                        xx = unit - kStTY * kStTX;
                    } else if (unit < kStBoxCols) {
                        yy = unit - kStTY * kStTX - kStTX;
                        xx = kStTX;
                    } else {
                        const int col = (unit - kStBoxCols) * 32 + lane;
                        ok = ok && col < kStTY * kStTX;
                        yy = col / kStTX;
                        xx = col % kStTX;
                        zz = kStZC;
                    }
                    const int y = y0 + yy, x = x0 + xx, j = z0 + zz;
                    ok = ok && y < v.Y && x < v.X && j < v.Z;
                    pos[k] = ok ? (yy | xx << 8 | zz << 16) : -1;
                    zv[k] = c0[k] = c1[k] = c2[k] = b0[k] = b1[k] = b2[k] = 0.f;
                    if (!ok) continue;
                    const size_t e = pbase + ((size_t)y * v.X + x) * v.Z + j;
                    zv[k] = a.z[e];
                    if (it > 0) {
                        c0[k] = rin[e];
                        c1[k] = rin[L + e];
                        c2[k] = rin[2 * L + e];
                        if (y > 0) b0[k] = rin[e - XZ];
                        if (x > 0) b1[k] = rin[L + e - v.Z];
                        if (j > 0) b2[k] = rin[2 * L + e - 1];
                    }
                }
#pragma unroll
                for (int k = 0; k < kStBatch; ++k) {
                    if (pos[k] < 0) continue;
                    const int yy = pos[k] & 0xFF, xx = (pos[k] >> 8) & 0xFF, zz = pos[k] >> 16;
                    const int y = y0 + yy, x = x0 + xx, j = z0 + zz;
                    float xv = zv[k];
                    if (it > 0) {
                        // D^T r_{i-1}, in the order of dtq
                        float acc = 0.f;
                        if (y + 1 < v.Y) acc -= c0[k];
                        if (y > 0) acc += b0[k];
                        if (x + 1 < v.X) acc -= c1[k];
                        if (x > 0) acc += b1[k];
                        if (j + 1 < v.Z) acc -= c2[k];
                        if (j > 0) acc += b2[k];
                        xv -= acc;
                    }
                    if (yy < kStTY && xx < kStTX && zz < kStZC) {
                        const int col = yy * kStTX + xx;
                        rs[0][col][zz] = c0[k];
                        rs[1][col][zz] = c1[k];
                        rs[2][col][zz] = c2[k];
                    }
                    xs[yy][xx][zz] = xv;
                }
            }
            __syncthreads();
            // u_i = clamp(r_{i-1} + D x / 12), r_i = u_i + beta_i (u_i - u_{i-1})
            for (int k0 = warp; k0 < kStTY * kStTX; k0 += nwarps * kStBatch) {
                float up[kStBatch][3];
#pragma unroll
                for (int k = 0; k < kStBatch; ++k) {
                    const int col = k0 + k * nwarps;
                    const int y = y0 + col / kStTX, x = x0 + col % kStTX, j = z0 + lane;
                    const bool ok = col < kStTY * kStTX && y < v.Y && x < v.X && j < v.Z;
                    const size_t e = pbase + ((size_t)y * v.X + x) * v.Z + j;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        up[k][c] = ok && it > 0 ? a.u[(size_t)c * L + e] : 0.f;
                }
#pragma unroll
                for (int k = 0; k < kStBatch; ++k) {
                    const int col = k0 + k * nwarps;
                    const int yy = col / kStTX, xx = col % kStTX;
                    const int y = y0 + yy, x = x0 + xx, j = z0 + lane;
                    if (col >= kStTY * kStTX || y >= v.Y || x >= v.X || j >= v.Z) continue;
                    const size_t e = pbase + ((size_t)y * v.X + x) * v.Z + j;
                    const float xc = xs[yy][xx][lane];
                    const float d[3] = {y + 1 < v.Y ? xs[yy + 1][xx][lane] - xc : 0.f,
                                        x + 1 < v.X ? xs[yy][xx + 1][lane] - xc : 0.f,
                                        j + 1 < v.Z ? xs[yy][xx][lane + 1] - xc : 0.f};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const size_t ia = (size_t)c * L + e;
                        const float un =
                            clampf(fmaf(d[c], 1.0f / 12.0f, rs[c][col][lane]), -a.tau, a.tau);
                        a.u[ia] = un;
                        rout[ia] = fmaf(beta, un - up[k][c], un);
                    }
                }
            }
            __syncthreads();
        }
        grid_sync(a.bar, nb);  // also orders s_beta's next write after every read
        const float* tmp = rin;
        rin = rout;
        rout = const_cast<float*>(tmp);
    }
    const float fb = a.mode == 1 ? (float)a.scal[1] : 0.f;
    for_rows(v, [&](int y, int x, size_t base) {
        for (int j = lane; j < v.Z; j += 32) {
            const size_t e = base + j;
            const float xv = a.z[e] - dtq(a.u, v, e, y, x, j);
            if (a.mode == 0) {
                a.out[e] = xv;
            } else {
                const float cn = fmaxf(xv - a.theta, 0.f);
                const float dd = cn - a.c[e];
                a.c[e] = cn;
                a.xi[e] = fmaf(fb, dd, cn);
                if (a.delta) a.delta[e] = dd;
            }
        }
    });
}

// Shared-memory-resident variant of fgp_coop_kernel.  Block b owns the
// columns (p, y0 .. y0+TY-1, x0 .. x0+TX-1) over all z and keeps z, x, the
// duals u and r of its tile in shared memory for all inner iterations, with
// a ring of ghost columns around the tile (ghosted index (gy, gx) is the
// column (y0 + gy - 1, x0 + gx - 1)).  Only the tile's boundary columns of r
// go through global memory: after phase B each block publishes them (into
// r0 / r1 by iteration parity, so that a neighbour still reading the previous
// values is never overwritten), one grid barrier, then every block reads its
// ghost ring.  Phase A computes x on the tile and on the ghost row below and
// the ghost column to its right, which is where phase B's forward
// differences reach.  The arithmetic per entry is that of fgp_iter_kernel.
constexpr int kTileThreads = 1024;

// x = z - D^T q at ghosted shared index i of the column (y, x), depth j; q has
// three components at stride G; the terms are summed in dtq's order.
__device__ __forceinline__ float tile_x(const float* q, const float* sz, int i, int G, int GXZ,
                                        int Z, int j, bool ylo, bool yhi, bool xlo, bool xhi)
{
    float acc = 0.f;
    if (yhi) acc -= q[i];
    if (ylo) acc += q[i - GXZ];
    if (xhi) acc -= q[G + i];
    if (xlo) acc += q[G + i - Z];
    if (j + 1 < Z) acc -= q[2 * G + i];
    if (j > 0) acc += q[2 * G + i - 1];
    return sz[i] - acc;
}

__global__ void __launch_bounds__(kTileThreads) fgp_tile_kernel(const FgpCoop a)
{
    extern __shared__ __align__(16) float sm[];
    const Vol v = a.v;
    const int Z = v.Z;
    const size_t L = v.L;
    const int GY = a.TY + 2, GX = a.TX + 2;
    const int G = GY * GX * Z, GXZ = GX * Z;
    float* sz = sm;          // [GY][GX][Z]   z
    float* sx = sz + G;      // [GY][GX][Z]   x = z - D^T r
    float* sr = sx + G;      // [3][GY][GX][Z] r (then u with ghosts, for the output)
    float* su = sr + 3 * G;  // [3][TY][TX][Z] u
    const int T = a.TY * a.TX * Z;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned nb = gridDim.x;
    const int b = blockIdx.x;
    const int tx = b % a.tilesX, ty = (b / a.tilesX) % a.tilesY;
    const int p = b / (a.tilesX * a.tilesY);
    const int y0 = ty * a.TY, x0 = tx * a.TX;
    const int ny = min(a.TY, v.Y - y0), nx = min(a.TX, v.X - x0);
    auto gidx = [&](int gy, int gx) -> size_t {  // global index of column (gy, gx), z = 0
        return (((size_t)p * v.Y + (y0 + gy - 1)) * v.X + (x0 + gx - 1)) * Z;
    };
    auto sidx = [&](int gy, int gx) -> int { return (gy * GX + gx) * Z; };
    auto inside = [&](int gy, int gx) -> bool {
        const int y = y0 + gy - 1, x = x0 + gx - 1;
        return y >= 0 && y < v.Y && x >= 0 && x < v.X;
    };
    if (a.mode == 1 && b == 0 && threadIdx.x == 0) {
        const double t = a.scal[0];
        const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        a.scal[1] = momentum_coef(t, t1, a.momentum);
        a.scal[0] = t1;
    }
    // x on one column (gy, gx); lanes take the depths j and j + 32 together
    auto phase_a = [&](int gy, int gx) {
        const int y = y0 + gy - 1, x = x0 + gx - 1;
        const bool ylo = y > 0, yhi = y + 1 < v.Y, xlo = x > 0, xhi = x + 1 < v.X;
        const int s0 = sidx(gy, gx);
        for (int j = lane; j < Z; j += 64) {
            const int j2 = j + 32;
            const float v1 = tile_x(sr, sz, s0 + j, G, GXZ, Z, j, ylo, yhi, xlo, xhi);
            const float v2 = j2 < Z ? tile_x(sr, sz, s0 + j2, G, GXZ, Z, j2, ylo, yhi, xlo, xhi)
                                    : 0.f;
            sx[s0 + j] = v1;
            if (j2 < Z) sx[s0 + j2] = v2;
        }
    };
    // the ghost ring of r, asynchronously, from the published boundary columns
    auto load_ghosts = [&](const float* pub) {
        const int ring = 2 * (nx + 2) + 2 * ny;
        for (int k = warp; k < ring; k += nw) {
            int gy, gx;
            if (k < nx + 2) {
                gy = 0;
                gx = k;
            } else if (k < 2 * (nx + 2)) {
                gy = ny + 1;
                gx = k - (nx + 2);
            } else {
                const int q = k - 2 * (nx + 2);
                gy = 1 + (q >> 1);
                gx = (q & 1) ? nx + 1 : 0;
            }
            if (!inside(gy, gx)) continue;
            const size_t g0 = gidx(gy, gx);
            const int s0 = sidx(gy, gx);
            for (int c = 0; c < 3; ++c)
                copy_column(&sr[c * G + s0], &pub[(size_t)c * L + g0], Z, lane, a.vec);
        }
    };
    // r = u = 0; z on the tile, the ghost row below and the ghost column right
    for (int i = threadIdx.x; i < 3 * G; i += blockDim.x) sr[i] = 0.f;
    for (int i = threadIdx.x; i < 3 * T; i += blockDim.x) su[i] = 0.f;
    for (int cidx = warp; cidx < (ny + 1) * (nx + 1); cidx += nw) {
        const int gy = 1 + cidx / (nx + 1), gx = 1 + cidx % (nx + 1);
        if (!inside(gy, gx)) continue;
        copy_column(&sz[sidx(gy, gx)], &a.z[gidx(gy, gx)], Z, lane, a.vec);
    }
    cp_async_wait();
    __syncthreads();
    // Algorithm 2's t recursion: FP64 in one thread (FP64 arithmetic is scarce
    // on this GPU), published in shared memory before the barrier after phase A
    __shared__ float s_beta;
    double t = 1.0;
    for (int it = 0; it < a.iters; ++it) {
        if (threadIdx.x == 0) {
            const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            s_beta = (float)momentum_coef(t, t1, a.inner_momentum);
            t = t1;
        }
        const bool last = it + 1 == a.iters;
        // ghosts of the previous iteration in flight while the interior columns
        // (whose D^T r stays inside the tile) compute x
        if (it > 0) load_ghosts(((it - 1) & 1) ? a.r1 : a.r0);
        for (int cidx = warp; cidx < (ny - 1) * (nx - 1); cidx += nw)
            phase_a(2 + cidx / (nx - 1), 2 + cidx % (nx - 1));
        cp_async_wait();
        __syncthreads();
        // phase A on the remaining columns: the tile's first row and column, the
        // ghost row below and the ghost column right
        for (int cidx = warp; cidx < (ny + 1) * (nx + 1); cidx += nw) {
            const int gy = 1 + cidx / (nx + 1), gx = 1 + cidx % (nx + 1);
            const bool interior = gy >= 2 && gy <= ny && gx >= 2 && gx <= nx;
            if (interior || (gy == ny + 1 && gx == nx + 1) || !inside(gy, gx)) continue;
            phase_a(gy, gx);
        }
        __syncthreads();
        const float beta = s_beta;
        // phase B on the tile; boundary columns published
        float* pub = (it & 1) ? a.r1 : a.r0;
        for (int cidx = warp; cidx < ny * nx; cidx += nw) {
            const int gy = 1 + cidx / nx, gx = 1 + cidx % nx;
            const int y = y0 + gy - 1, x = x0 + gx - 1;
            const bool hy = y + 1 < v.Y, hx = x + 1 < v.X;
            const int s0 = sidx(gy, gx), u0 = ((gy - 1) * a.TX + (gx - 1)) * Z;
            const bool edge = gy == 1 || gy == ny || gx == 1 || gx == nx;
            const size_t g0 = gidx(gy, gx);
            for (int j = lane; j < Z; j += 32) {
                const int i = s0 + j;
                const float xc = sx[i];
                const float d[3] = {hy ? sx[i + GXZ] - xc : 0.f, hx ? sx[i + Z] - xc : 0.f,
                                    j + 1 < Z ? sx[i + 1] - xc : 0.f};
                float ra[3], up[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    ra[c] = sr[c * G + i];
                    up[c] = su[c * T + u0 + j];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float un = clampf(fmaf(d[c], 1.0f / 12.0f, ra[c]), -a.tau, a.tau);
                    const float rn = fmaf(beta, un - up[c], un);
                    su[c * T + u0 + j] = un;
                    sr[c * G + i] = rn;
                    if (edge) {
                        if (last) a.u[(size_t)c * L + g0 + j] = un;
                        else pub[(size_t)c * L + g0 + j] = rn;
                    }
                }
            }
        }
        grid_sync(a.bar, nb);
    }
    // u with the ghost row above and column left (all that D^T u reads)
    for (int cidx = warp; cidx < ny * nx; cidx += nw) {
        const int gy = 1 + cidx / nx, gx = 1 + cidx % nx;
        const int s0 = sidx(gy, gx), u0 = ((gy - 1) * a.TX + (gx - 1)) * Z;
        for (int c = 0; c < 3; ++c)
            for (int j = lane; j < Z; j += 32) sr[c * G + s0 + j] = su[c * T + u0 + j];
    }
    for (int k = warp; k < nx + ny; k += nw) {
        const int gy = k < nx ? 0 : 1 + (k - nx), gx = k < nx ? 1 + k : 0;
        if (!inside(gy, gx)) continue;
        const size_t g0 = gidx(gy, gx);
        const int s0 = sidx(gy, gx);
        for (int c = 0; c < 3; ++c)
            copy_column(&sr[c * G + s0], &a.u[(size_t)c * L + g0], Z, lane, a.vec);
    }
    cp_async_wait();
    __syncthreads();
    const float fb = a.mode == 1 ? (float)a.scal[1] : 0.f;
    for (int cidx = warp; cidx < ny * nx; cidx += nw) {
        const int gy = 1 + cidx / nx, gx = 1 + cidx % nx;
        const int y = y0 + gy - 1, x = x0 + gx - 1;
        const bool ylo = y > 0, yhi = y + 1 < v.Y, xlo = x > 0, xhi = x + 1 < v.X;
        const int s0 = sidx(gy, gx);
        const size_t g0 = gidx(gy, gx);
        for (int j = lane; j < Z; j += 32) {
            const float xv = tile_x(sr, sz, s0 + j, G, GXZ, Z, j, ylo, yhi, xlo, xhi);
            const size_t e = g0 + j;
            if (a.mode == 0) {
                a.out[e] = xv;
            } else {
                const float cn = fmaxf(xv - a.theta, 0.f);
                const float dd = cn - a.c[e];
                a.c[e] = cn;
                a.xi[e] = fmaf(fb, dd, cn);
                if (a.delta) a.delta[e] = dd;
            }
        }
    }
}

// Dynamic shared memory of fgp_tile_kernel for a TY x TX tile.
size_t tile_smem_bytes(int TY, int TX, int Z)
{
    return ((size_t)5 * (TY + 2) * (TX + 2) * Z + (size_t)3 * TY * TX * Z) * sizeof(float);
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

// sum over volumes m of w[m] TV(x_m), x = [v.P volumes][Y][X][Z]
__global__ void red_tv_weighted_kernel(const float* __restrict__ x, Vol v,
                                       const float* __restrict__ w, double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    const size_t XZ = (size_t)v.X * v.Z, V = XZ * v.Y;
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < v.L;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % v.Z);
        const int xx = (int)((i / v.Z) % v.X);
        const int y = (int)((i / XZ) % v.Y);
        const double c = x[i];
        double a = 0.0;
        if (y + 1 < v.Y) a += fabs((double)x[i + XZ] - c);
        if (xx + 1 < v.X) a += fabs((double)x[i + v.Z] - c);
        if (j + 1 < v.Z) a += fabs((double)x[i + 1] - c);
        s += (double)w[i / V] * a;
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

// parts[b] = this block's sum of d^2, parts[gridDim.x + b] = its sum of c^2
__global__ void red_pair_kernel(const float* __restrict__ d, const float* __restrict__ c,
                                size_t n, double* parts)
{
    __shared__ double sh[kRedThreads / 32];
    // a thread's few terms in FP32 (the ratio only steers the resync
    // schedule; FP64 arithmetic per element took 46 us on the large volume),
    // the block's sum in FP64
    float fd = 0.f, fc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float a = d[i], b = c[i];
        fd = fmaf(a, a, fd);
        fc = fmaf(b, b, fc);
    }
    double sd = fd, sc = fc;
    sd = block_sum(sd, sh);
    __syncthreads();  // sh is reused
    sc = block_sum(sc, sh);
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = sd;
        parts[gridDim.x + blockIdx.x] = sc;
    }
}

// The refined solve's device-side resync decision for the iteration just
// finished (sched[1] of them so far): rho = ||d|| / ||c|| joins the budget
// accumulator; the gate opens (sched[0] = 1) on every R-th iteration or once
// the accumulated rho exceeds the budget, and the accumulator restarts.
__global__ void refine_decide_kernel(const double* parts, int count, double* scal, int slot,
                                     int* sched, int* rlog, int R, double budget)
{
    __shared__ double sh[kRedThreads / 32];
    double sd = 0.0, sc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        sd += parts[i];
        sc += parts[count + i];
    }
    sd = block_sum(sd, sh);
    __syncthreads();
    sc = block_sum(sc, sh);
    if (threadIdx.x != 0) return;
    const int it = sched[1];
    const double rho = sc > 0.0 ? sqrt(sd / sc) : (sd > 0.0 ? 1e300 : 0.0);
    double acc = scal[slot] + rho;
    const int exact = ((R > 0 && (it + 1) % R == 0) || acc > budget) ? 1 : 0;
    if (exact) {
        acc = 0.0;
        sched[2] += 1;
    }
    scal[slot] = acc;
    sched[0] = exact;
    sched[1] = it + 1;
    rlog[it & (kRefineLog - 1)] = exact;
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
    const size_t n4 = ((uintptr_t)x & 15u) == 0 ? n / 4 : 0;
    prox_l1_kernel<<<ew_grid(n4 ? n4 : n), 256, 0, st>>>(x, n, n4, thresh, nonneg);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

// Barrier words and grid size of the cooperative TV prox: every SM, as many
// blocks as are co-resident, at most 4 per SM (synchronous; not while
// capturing).
swopt_status coop_prepare(swopt_handle* h)
{
    if (!h->coop_bar) {
        SW_CUDA(cudaMalloc((void**)&h->coop_bar, 8 * sizeof(unsigned)));
        SW_CUDA(cudaMemset(h->coop_bar, 0, 8 * sizeof(unsigned)));
    }
    if (h->tile_ty == 0) {
        // shared-memory tile: the fewest ghosted columns per SM with every tile
        // co-resident; else (tile_ty = -1) the global-memory kernel
        h->tile_ty = -1;
        int sms = 0;
        SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        const int dmax = max_dynamic_smem(h, (const void*)fgp_tile_kernel);
        double best = 1e300;
        for (int TY = 1; TY <= std::min(h->Y, 32); ++TY)
            for (int TX = 1; TX <= std::min(h->X, 32); ++TX) {
                const size_t sm = tile_smem_bytes(TY, TX, h->Z);
                if (dmax <= 0 || sm > (size_t)dmax) continue;
                const long tiles = (long)h->P * ((h->Y + TY - 1) / TY) * ((h->X + TX - 1) / TX);
                if (tiles > (long)sms * 8) continue;
                SW_CUDA(cudaFuncSetAttribute(fgp_tile_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, dmax));
                int per_sm = 0;
                SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fgp_tile_kernel,
                                                                      kTileThreads, sm));
                if (per_sm < 1 || tiles > (long)per_sm * sms) continue;
                const double cost = (double)((tiles + sms - 1) / sms) * (TY + 2) * (TX + 2) +
                                    1e-3 * (double)tiles;
                if (cost < best) {
                    best = cost;
                    h->tile_ty = TY;
                    h->tile_tx = TX;
                }
            }
    }
    if (h->coop_blocks == 0) {
        int per_sm = 0, sms = 0;
        SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fgp_coop_kernel,
                                                              kCoopThreads, 0));
        SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        if (per_sm < 1) {
            set_error("the TV prox kernel cannot be resident");
            return SWOPT_ERR_UNSUPPORTED;
        }
        h->coop_blocks = sms * std::min(per_sm, 8);
    }
    return SWOPT_OK;
}

static swopt_status launch_coop(swopt_handle* h, FgpCoop& a, cudaStream_t st)
{
    if (!h->coop_bar || h->coop_blocks == 0 || h->tile_ty == 0) {
        set_error("internal: the TV prox kernel was not prepared");
        return SWOPT_ERR_DEVICE_CHECK;
    }
    a.bar = h->coop_bar;
    if (h->tile_ty > 0) {
        auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
        a.vec = (h->Z % 4) == 0 && al16(a.z) && al16(a.u) && al16(a.r0) && al16(a.r1);
        a.TY = h->tile_ty;
        a.TX = h->tile_tx;
        a.tilesY = (h->Y + a.TY - 1) / a.TY;
        a.tilesX = (h->X + a.TX - 1) / a.TX;
        const int tiles = h->P * a.tilesY * a.tilesX;
        const int dmax = max_dynamic_smem(h, (const void*)fgp_tile_kernel);
        SW_CUDA(cudaFuncSetAttribute(fgp_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dmax));
        void* args[] = {&a};
        SW_CUDA(cudaLaunchCooperativeKernel((const void*)fgp_tile_kernel, dim3(tiles),
                                            dim3(kTileThreads), args,
                                            tile_smem_bytes(a.TY, a.TX, h->Z), st));
        SW_LAUNCHED(h);
        return SWOPT_OK;
    }
    void* args[] = {&a};
    SW_CUDA(cudaLaunchCooperativeKernel((const void*)fgp_coop_kernel, dim3(h->coop_blocks),
                                        dim3(kCoopThreads), args, 0, st));
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status prox_tv_coop(swopt_handle* h, const float* z, float tau, int iters,
                          int inner_momentum, float* out, cudaStream_t st)
{
    FgpCoop a{};
    a.z = z; a.u = h->tvu; a.r0 = h->tvr0; a.r1 = h->tvr1;
    a.v = vol_of(h); a.tau = tau; a.iters = iters; a.inner_momentum = inner_momentum;
    a.mode = 0; a.out = out;
    return launch_coop(h, a, st);
}

swopt_status fista_prox_finish(swopt_handle* h, const float* z, float tau, int iters,
                               int inner_momentum, float theta, float* delta, cudaStream_t st)
{
    FgpCoop a{};
    a.z = z; a.u = h->tvu; a.r0 = h->tvr0; a.r1 = h->tvr1;
    a.v = vol_of(h); a.tau = tau; a.iters = iters; a.inner_momentum = inner_momentum;
    a.mode = 1; a.c = h->c; a.xi = h->xi; a.delta = delta; a.scal = h->scal;
    a.momentum = h->prm.momentum; a.theta = theta;
    return launch_coop(h, a, st);
}

swopt_status coop_debug(swopt_handle* h, unsigned phantom, unsigned poll_limit)
{
    SW_TRY(coop_prepare(h));
    const unsigned w[2] = {phantom, poll_limit};
    SW_CUDA(cudaMemcpy(h->coop_bar + 4, w, sizeof(w), cudaMemcpyHostToDevice));
    return SWOPT_OK;
}

int coop_error_word(swopt_handle* h)
{
    if (!h->coop_bar) return 0;
    unsigned w[4] = {0, 0, 0, 0};
    if (cudaMemcpy(w, h->coop_bar, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (w[2] == 0) return 0;
    cudaMemset(h->coop_bar, 0, sizeof(w));
    return 1;
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

swopt_status reduce_tv_states(swopt_handle* h, const float* b, int slot, cudaStream_t st)
{
    Vol v = vol_of(h);
    v.P = h->Q;
    v.L = nb_of(h);
    red_tv_weighted_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(b, v, h->Cmf, h->red);
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

swopt_status refine_decide(swopt_handle* h, const float* d, const float* c, int slot, int R,
                           double budget, cudaStream_t st)
{
    red_pair_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(d, c, nc_of(h), h->red);
    SW_LAUNCHED(h);
    refine_decide_kernel<<<1, kRedThreads, 0, st>>>(h->red, kRedBlocks, h->scal, slot, h->sched,
                                                    h->rlog, R, budget);
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
