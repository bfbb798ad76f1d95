// FP32 operator kernels on the CUDA cores: the switching map P (Eq. final-H,
// Eq. Sij-detailed), the acoustic correlation A and its transpose (Sec. 2.3.3,
// Eq. acoustic-full-forward), and the layout kernels around them.
//
// Structure exploited (exact in real arithmetic):
//  * the switching weights depend on the pulse only through its position
//    m = n mod pulses_per_cycle inside the OFF-switching cycle, so H c has
//    only Q = min(N, pulses_per_cycle) distinct pulse images; A runs on the Q
//    state images and A^T on the measurements summed over equal states;
//  * every nonzero kernel sample lies in one time window [t0, t0 + tw), so
//    the contractions run on that window only (zero-padded to Twp, a
//    multiple of 32);
//  * inside the window the kernel is banded: for each (depth, tap) only a
//    few 8-sample sub-blocks are nonzero, and the kernels skip the rest
//    with warp-uniform branches (8-bit masks built at create time).
#include <algorithm>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kThreads = 128;

// ---------------------------------------------------------------------------
// A: u[m][y][x][w] = sum_j sum_{dy,dx} b[m][y+dy-r][x+dx-r][j] Kf[j][dy][dx][w]
// One CTA: one state m, a 16x16 tile of scan positions, a 32-sample chunk of
// the window.  Each thread owns two positions (rows ty and ty+8) x 32
// samples.  The b halo of a chunk of depths is staged in shared memory; the
// kernel rows are broadcast loads through L1.
// Epilogue: out = (scale ? Cm[m] : 1) * acc - (ytil ? ytil : 0); with
// partials != null each block also writes the FP64 sum of
// Cm*acc^2 - 2*acc*ytil (data-fit terms of the folded residual).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
fwd_simt_kernel(const float* __restrict__ b, const float* __restrict__ Kf,
                const uint8_t* __restrict__ fmask, const float* __restrict__ Cmf,
                const float* __restrict__ ytil, float* __restrict__ u,
                double* __restrict__ partials, int Y, int X, int Z, int k, int Twp,
                int nTc, int jc, int scale, const int* gate, int want)
{
    extern __shared__ float sm[];
    __shared__ double red[kThreads / 32];
    if (gated_off(gate, want)) return;
    const int r = k >> 1;
    const int HX = TILE + 2 * r, HY = TILE + 2 * r;
    const int tilesX = (X + TILE - 1) / TILE;
    const int x0 = (blockIdx.x % tilesX) * TILE, y0 = (blockIdx.x / tilesX) * TILE;
    const int m = blockIdx.y, tc = blockIdx.z;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float* bm = b + (size_t)m * Y * X * Z;

    float acc0[32], acc1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) { acc0[i] = 0.f; acc1[i] = 0.f; }

    for (int j0 = 0; j0 < Z; j0 += jc) {
        const int jn = min(jc, Z - j0);
        __syncthreads();
        const int tot = jn * HY * HX;
        for (int idx = tid; idx < tot; idx += kThreads) {
            const int jj = idx % jn;
            const int rest = idx / jn;
            const int hx = rest % HX, hy = rest / HX;
            const int gy = y0 - r + hy, gx = x0 - r + hx;
            float v = 0.f;
            if (gy >= 0 && gy < Y && gx >= 0 && gx < X)
                v = bm[((size_t)gy * X + gx) * Z + j0 + jj];
            sm[(jj * HY + hy) * HX + hx] = v;
        }
        __syncthreads();
        for (int jj = 0; jj < jn; ++jj) {
            const int j = j0 + jj;
            const float* srow = sm + jj * HY * HX;
            for (int dy = 0; dy < k; ++dy) {
                const float* s0 = srow + (ty + dy) * HX + tx;
                const float* s1 = s0 + 8 * HX;
                const size_t kd0 = ((size_t)j * k + dy) * k;
                for (int dx = 0; dx < k; ++dx) {
                    const unsigned msk = __ldg(fmask + (kd0 + dx) * nTc + tc);
                    if (msk == 0) continue;
                    const float b0 = s0[dx], b1 = s1[dx];
                    const float4* kp =
                        reinterpret_cast<const float4*>(Kf + (kd0 + dx) * Twp + tc * TCHUNK);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (msk & (1u << q)) {
                            const float4 ka = __ldg(kp + 2 * q), kb = __ldg(kp + 2 * q + 1);
                            acc0[8 * q + 0] = fmaf(b0, ka.x, acc0[8 * q + 0]);
                            acc0[8 * q + 1] = fmaf(b0, ka.y, acc0[8 * q + 1]);
                            acc0[8 * q + 2] = fmaf(b0, ka.z, acc0[8 * q + 2]);
                            acc0[8 * q + 3] = fmaf(b0, ka.w, acc0[8 * q + 3]);
                            acc0[8 * q + 4] = fmaf(b0, kb.x, acc0[8 * q + 4]);
                            acc0[8 * q + 5] = fmaf(b0, kb.y, acc0[8 * q + 5]);
                            acc0[8 * q + 6] = fmaf(b0, kb.z, acc0[8 * q + 6]);
                            acc0[8 * q + 7] = fmaf(b0, kb.w, acc0[8 * q + 7]);
                            acc1[8 * q + 0] = fmaf(b1, ka.x, acc1[8 * q + 0]);
                            acc1[8 * q + 1] = fmaf(b1, ka.y, acc1[8 * q + 1]);
                            acc1[8 * q + 2] = fmaf(b1, ka.z, acc1[8 * q + 2]);
                            acc1[8 * q + 3] = fmaf(b1, ka.w, acc1[8 * q + 3]);
                            acc1[8 * q + 4] = fmaf(b1, kb.x, acc1[8 * q + 4]);
                            acc1[8 * q + 5] = fmaf(b1, kb.y, acc1[8 * q + 5]);
                            acc1[8 * q + 6] = fmaf(b1, kb.z, acc1[8 * q + 6]);
                            acc1[8 * q + 7] = fmaf(b1, kb.w, acc1[8 * q + 7]);
                        }
                    }
                }
            }
        }
    }

    const float cm = scale ? Cmf[m] : 1.f;
    double part = 0.0;
    const int gx = x0 + tx;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int gy = y0 + ty + 8 * half;
        if (gy < Y && gx < X) {
            const size_t base = (((size_t)m * Y + gy) * X + gx) * Twp + tc * TCHUNK;
            float4* out = reinterpret_cast<float4*>(u + base);
            const float4* yt = ytil ? reinterpret_cast<const float4*>(ytil + base) : nullptr;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float4 v;
                v.x = half ? acc1[4 * q + 0] : acc0[4 * q + 0];
                v.y = half ? acc1[4 * q + 1] : acc0[4 * q + 1];
                v.z = half ? acc1[4 * q + 2] : acc0[4 * q + 2];
                v.w = half ? acc1[4 * q + 3] : acc0[4 * q + 3];
                float4 o;
                if (yt) {
                    const float4 w = yt[q];
                    o.x = cm * v.x - w.x; o.y = cm * v.y - w.y;
                    o.z = cm * v.z - w.z; o.w = cm * v.w - w.w;
                    if (partials) {
                        part += (double)cm * ((double)v.x * v.x + (double)v.y * v.y +
                                              (double)v.z * v.z + (double)v.w * v.w) -
                                2.0 * ((double)v.x * w.x + (double)v.y * w.y +
                                       (double)v.z * w.z + (double)v.w * w.w);
                    }
                } else {
                    o.x = cm * v.x; o.y = cm * v.y; o.z = cm * v.z; o.w = cm * v.w;
                }
                out[q] = o;
            }
        }
    }
    if (partials) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if ((tid & 31) == 0) red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) s += red[w];
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// A^T: g[m][y][x][j] = sum_{dy,dx} sum_w u[m][y-dy+r][x-dx+r][w] Ka[dy][dx][w][j]
// One CTA: one state, a 16x16 tile, a 32-depth chunk.  Each thread owns two
// positions x 32 depths.  The u halo of a chunk of window samples is staged
// in shared memory; the depth-contiguous kernel rows are broadcast loads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
adj_simt_kernel(const float* __restrict__ u, const float* __restrict__ Ka,
                const uint8_t* __restrict__ amask, float* __restrict__ g, int Y, int X,
                int Z, int k, int Twp, int Zp, int nJc, int tcs, const int* gate, int want)
{
    extern __shared__ float sm[];
    if (gated_off(gate, want)) return;
    const int r = k >> 1;
    const int HX = TILE + 2 * r, HY = TILE + 2 * r;
    const int tilesX = (X + TILE - 1) / TILE;
    const int x0 = (blockIdx.x % tilesX) * TILE, y0 = (blockIdx.x / tilesX) * TILE;
    const int m = blockIdx.y, jz = blockIdx.z;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float* um = u + (size_t)m * Y * X * Twp;

    float acc0[32], acc1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) { acc0[i] = 0.f; acc1[i] = 0.f; }

    for (int w0 = 0; w0 < Twp; w0 += tcs) {
        const int wn = min(tcs, Twp - w0);
        __syncthreads();
        const int tot = wn * HY * HX;
        for (int idx = tid; idx < tot; idx += kThreads) {
            const int ww = idx % wn;
            const int rest = idx / wn;
            const int hx = rest % HX, hy = rest / HX;
            const int gy = y0 - r + hy, gx = x0 - r + hx;
            float v = 0.f;
            if (gy >= 0 && gy < Y && gx >= 0 && gx < X)
                v = um[((size_t)gy * X + gx) * Twp + w0 + ww];
            sm[(ww * HY + hy) * HX + hx] = v;
        }
        __syncthreads();
        for (int ww = 0; ww < wn; ++ww) {
            const int w = w0 + ww;
            const float* srow = sm + ww * HY * HX;
            for (int dy = 0; dy < k; ++dy) {
                // source row y - (dy - r): halo row ty + 2r - dy
                const float* s0 = srow + (ty + 2 * r - dy) * HX + tx + 2 * r;
                const float* s1 = s0 + 8 * HX;
                for (int dx = 0; dx < k; ++dx) {
                    const size_t kw = ((size_t)(dy * k + dx) * Twp + w);
                    const unsigned msk = __ldg(amask + kw * nJc + jz);
                    if (msk == 0) continue;
                    const float a0 = s0[-dx], a1 = s1[-dx];
                    const float4* kp = reinterpret_cast<const float4*>(Ka + kw * Zp + jz * JCHUNK);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (msk & (1u << q)) {
                            const float4 ka = __ldg(kp + 2 * q), kb = __ldg(kp + 2 * q + 1);
                            acc0[8 * q + 0] = fmaf(a0, ka.x, acc0[8 * q + 0]);
                            acc0[8 * q + 1] = fmaf(a0, ka.y, acc0[8 * q + 1]);
                            acc0[8 * q + 2] = fmaf(a0, ka.z, acc0[8 * q + 2]);
                            acc0[8 * q + 3] = fmaf(a0, ka.w, acc0[8 * q + 3]);
                            acc0[8 * q + 4] = fmaf(a0, kb.x, acc0[8 * q + 4]);
                            acc0[8 * q + 5] = fmaf(a0, kb.y, acc0[8 * q + 5]);
                            acc0[8 * q + 6] = fmaf(a0, kb.z, acc0[8 * q + 6]);
                            acc0[8 * q + 7] = fmaf(a0, kb.w, acc0[8 * q + 7]);
                            acc1[8 * q + 0] = fmaf(a1, ka.x, acc1[8 * q + 0]);
                            acc1[8 * q + 1] = fmaf(a1, ka.y, acc1[8 * q + 1]);
                            acc1[8 * q + 2] = fmaf(a1, ka.z, acc1[8 * q + 2]);
                            acc1[8 * q + 3] = fmaf(a1, ka.w, acc1[8 * q + 3]);
                            acc1[8 * q + 4] = fmaf(a1, kb.x, acc1[8 * q + 4]);
                            acc1[8 * q + 5] = fmaf(a1, kb.y, acc1[8 * q + 5]);
                            acc1[8 * q + 6] = fmaf(a1, kb.z, acc1[8 * q + 6]);
                            acc1[8 * q + 7] = fmaf(a1, kb.w, acc1[8 * q + 7]);
                        }
                    }
                }
            }
        }
    }

    const int gx = x0 + tx;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int gy = y0 + ty + 8 * half;
        if (gy < Y && gx < X) {
            float* out = g + (((size_t)m * Y + gy) * X + gx) * Z + jz * JCHUNK;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (jz * JCHUNK + i < Z) out[i] = half ? acc1[i] : acc0[i];
        }
    }
}

// b[m][s][j] = sum_p Sm[m][p][j] c[p][s][j]
__global__ void states_kernel(const float* __restrict__ c, const float* __restrict__ Sm,
                              float* __restrict__ b, int Q, int P, int S, int Z,
                              const int* gate, int want)
{
    if (gated_off(gate, want)) return;
    const size_t n = (size_t)Q * S * Z;
    const size_t SZ = (size_t)S * Z;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % Z);
        const size_t sj = i % SZ;
        const int m = (int)(i / SZ);
        float acc = 0.f;
        for (int p = 0; p < P; ++p) acc = fmaf(Sm[(m * P + p) * Z + j], c[(size_t)p * SZ + sj], acc);
        b[i] = acc;
    }
}

// y[n][s][t] = u[n mod ncyc][s][t - t0] inside the window, 0 outside.
__global__ void expand_kernel(const float* __restrict__ u, float* __restrict__ y, int N, int S,
                              int T, int ncyc, int t0, int Twp)
{
    const size_t n = (size_t)N * S * T;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i % T);
        const size_t rest = i / T;
        const size_t s = rest % S;
        const int pn = (int)(rest / S);
        const int w = t - t0;
        float v = 0.f;
        if (w >= 0 && w < Twp) v = u[((size_t)(pn % ncyc) * S + s) * Twp + w];
        y[i] = v;
    }
}

// ytil[m][s][w] = sum_{n : n mod ncyc = m} y[n][s][t0 + w]  (0 beyond T)
__global__ void fold_kernel(const float* __restrict__ y, float* __restrict__ ytil, int N, int Q,
                            int S, int T, int ncyc, int t0, int Twp)
{
    const size_t n = (size_t)Q * S * Twp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int w = (int)(i % Twp);
        const size_t rest = i / Twp;
        const size_t s = rest % S;
        const int m = (int)(rest / S);
        const int t = t0 + w;
        float acc = 0.f;
        if (t < T)
            for (int pn = m; pn < N; pn += ncyc) acc += y[((size_t)pn * S + s) * T + t];
        ytil[i] = acc;
    }
}

// mode 0: out[p][s][j] = sum_m Sm[m][p][j] g[m][s][j]
// mode 1: out = xi - alpha * (that)
__global__ void pt_kernel(const float* __restrict__ g, const float* __restrict__ Sm,
                          const float* __restrict__ xi, float alpha, float* __restrict__ out,
                          int Q, int P, int S, int Z, int mode, const float* carry)
{
    const size_t SZ = (size_t)S * Z;
    const size_t n = (size_t)P * SZ;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % Z);
        const size_t sj = i % SZ;
        const int p = (int)(i / SZ);
        float acc = carry ? carry[i] : 0.f;
        for (int m = 0; m < Q; ++m) acc = fmaf(Sm[(m * P + p) * Z + j], g[(size_t)m * SZ + sj], acc);
        out[i] = mode ? fmaf(-alpha, acc, xi[i]) : acc;
    }
}

// Refined solve (gradient kept at c_k, updated by increments):
//   d  = sum_m Sm[m][p][j] g[m][s][j]       (P^T of the A^T output)
//   Gn = (add ? G : 0) + d                  (gradient at c_{k+1})
//   out = xi - alpha ((1 + beta) Gn - beta G)   (gradient step at the
//         momentum point xi_{k+1} = (1 + beta) c_{k+1} - beta c_k, by linearity)
//   G  = Gn
__global__ void pt_refine_kernel(const float* __restrict__ g, const float* __restrict__ Sm,
                                 const float* __restrict__ xi, float alpha, float* G,
                                 float* __restrict__ out, const double* __restrict__ scal,
                                 int Q, int P, int S, int Z, int add, const int* gate,
                                 int want)
{
    if (gated_off(gate, want)) return;
    const size_t SZ = (size_t)S * Z;
    const size_t n = (size_t)P * SZ;
    const float beta = (float)scal[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % Z);
        const size_t sj = i % SZ;
        const int p = (int)(i / SZ);
        float acc = 0.f;
        for (int m = 0; m < Q; ++m) acc = fmaf(Sm[(m * P + p) * Z + j], g[(size_t)m * SZ + sj], acc);
        const float go = G[i];
        const float gn = add ? go + acc : acc;
        out[i] = fmaf(-alpha, fmaf(beta, gn - go, gn), xi[i]);
        G[i] = gn;
    }
}

int fwd_jc(const swopt_handle* h)
{
    const int H = TILE + 2 * h->r;
    int jc = 40960 / (H * H * 4);
    if (jc > 16) jc = 16;
    if (jc < 1) jc = 1;
    return jc;
}

}  // namespace

int simt_forward_blocks(const swopt_handle* h)
{
    const int tiles = ((h->X + TILE - 1) / TILE) * ((h->Y + TILE - 1) / TILE);
    return tiles * h->Q * h->nTc;
}

swopt_status simt_forward(swopt_handle* h, const float* b, float* u, const float* ytil,
                          double* partials, int scale, cudaStream_t st)
{
    const int tiles = ((h->X + TILE - 1) / TILE) * ((h->Y + TILE - 1) / TILE);
    const int jc = fwd_jc(h);
    const int H = TILE + 2 * h->r;
    const size_t smem = (size_t)jc * H * H * sizeof(float);
    if (smem > 48 * 1024) {
        // a function attribute shared by all handles and captured launches:
        // raised to the device maximum, never lowered
        const int dmax = max_dynamic_smem(h, (const void*)fwd_simt_kernel);
        if (dmax <= 0 || smem > (size_t)dmax) {
            set_error("FP32 forward needs %zu bytes of shared memory (device limit %d)", smem,
                      dmax);
            return SWOPT_ERR_UNSUPPORTED;
        }
        SW_CUDA(cudaFuncSetAttribute(fwd_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dmax));
    }
    dim3 grid(tiles, h->Q, h->nTc);
    ProfileRec rec;
    prof_begin(h, 0, st, &rec);
    fwd_simt_kernel<<<grid, kThreads, smem, st>>>(b, h->Kf, h->fmask, h->Cmf, ytil, u, partials,
                                                  h->Y, h->X, h->Z, h->k, h->Twp, h->nTc, jc,
                                                  scale, h->gate, h->gate_want);
    SW_LAUNCHED(h);
    prof_end(h, &rec, st);
    return SWOPT_OK;
}

swopt_status simt_adjoint(swopt_handle* h, const float* u, float* g, cudaStream_t st)
{
    const int tiles = ((h->X + TILE - 1) / TILE) * ((h->Y + TILE - 1) / TILE);
    const int H = TILE + 2 * h->r;
    int tcs = 40960 / (H * H * 4);
    if (tcs > 16) tcs = 16;
    if (tcs < 1) tcs = 1;
    const size_t smem = (size_t)tcs * H * H * sizeof(float);
    dim3 grid(tiles, h->Q, h->nJc);
    ProfileRec rec;
    prof_begin(h, 1, st, &rec);
    adj_simt_kernel<<<grid, kThreads, smem, st>>>(u, h->Ka, h->amask, g, h->Y, h->X, h->Z, h->k,
                                                  h->Twp, h->Zp, h->nJc, tcs, h->gate,
                                                  h->gate_want);
    SW_LAUNCHED(h);
    prof_end(h, &rec, st);
    return SWOPT_OK;
}

swopt_status launch_states(swopt_handle* h, const float* c, float* b, cudaStream_t st)
{
    const size_t n = nb_of(h);
    states_kernel<<<std::min(grid_for(n, 256), 152 * 8), 256, 0, st>>>(c, h->Sm, b, h->Q, h->P,
                                                                        h->S, h->Z, h->gate,
                                                    h->gate_want);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status launch_expand(swopt_handle* h, const float* u, float* y, cudaStream_t st)
{
    const size_t n = (size_t)h->N * h->S * h->T;
    int grid = grid_for(n, 256);
    if (grid > 152 * 32) grid = 152 * 32;
    expand_kernel<<<grid, 256, 0, st>>>(u, y, h->N, h->S, h->T, h->ncyc, h->t0, h->Twp);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status launch_fold(swopt_handle* h, const float* y, float* ytil, cudaStream_t st)
{
    const size_t n = nu_of(h);
    int grid = grid_for(n, 256);
    if (grid > 152 * 32) grid = 152 * 32;
    fold_kernel<<<grid, 256, 0, st>>>(y, ytil, h->N, h->Q, h->S, h->T, h->ncyc, h->t0, h->Twp);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status launch_pt(swopt_handle* h, const float* g, const float* xi, float alpha, float* out,
                       int mode, cudaStream_t st)
{
    const size_t n = nc_of(h);
    pt_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, h->Sm, xi, alpha, out, h->Q, h->P, h->S, h->Z,
                                                 mode, nullptr);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status launch_pt_carry(swopt_handle* h, const float* g, const float* carry, float* out,
                             cudaStream_t st)
{
    const size_t n = nc_of(h);
    pt_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, h->Sm, nullptr, 0.f, out, h->Q, h->P, h->S,
                                                 h->Z, 0, carry);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

__global__ void grad_step_kernel(const float* __restrict__ g, const float* __restrict__ xi,
                                 float alpha, float* __restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = fmaf(-alpha, g[i], xi[i]);
}

swopt_status launch_grad_step(swopt_handle* h, const float* g, const float* xi, float alpha,
                              float* out, cudaStream_t st)
{
    const size_t n = nc_of(h);
    grad_step_kernel<<<grid_for(n, 256), 256, 0, st>>>(g, xi, alpha, out, n);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status launch_pt_refine(swopt_handle* h, const float* g, const float* xi, float alpha,
                              float* G, float* out, int add, cudaStream_t st)
{
    const size_t n = nc_of(h);
    // grid-stride: a launch behind a closed gate costs its blocks' start-up,
    // 40 us at one block per 256 elements of the large workload, 5 us like this
    const int grid = std::min(grid_for(n, 256), 152 * 8);
    pt_refine_kernel<<<grid, 256, 0, st>>>(g, h->Sm, xi, alpha, G, out, h->scal,
                                                        h->Q, h->P, h->S, h->Z, add, h->gate,
                                                        h->gate_want);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

}  // namespace swopt
