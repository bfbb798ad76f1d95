// Tensor-core (tcgen05, sm_103a) kernels for the acoustic correlation A and
// its transpose A^T (Sec. 2.3.3, Eq. acoustic-full-forward).
//
// Both are implicit GEMMs over a 16 x 8 tile of scan positions (M = 128, one
// TMEM lane per position):
//   A  : D[pos][t] += sum_j b[pos + d][j] K[j][d][t]     (K-dim: depth j)
//   A^T: D[pos][j] += sum_t r[pos - d][t] K[j][d][t]     (K-dim: window sample t)
// for every lateral tap d.  Operands live in shared memory in the
// no-swizzle K-major core-matrix layout: the A operand is a halo of the tile
// stored as [8-element slice][halo row][halo column][8 elements], so the
// operand of tap d is the same buffer at a byte offset (rows of 8 consecutive
// x are 16 B apart; 8-row groups are one halo row apart).  The B operand
// (the kernel) is pre-packed per tap in the same layout.  Each MMA covers
// K = 16 (two slices) and only the band of output columns where the kernel
// is nonzero (N = the band width rounded to 16, at a TMEM column offset), so
// the zero parts of the banded kernel cost nothing.
//
// Roles (192 threads): warp 0 stages operands with bulk asynchronous copies
// (the TMA engine) on mbarriers, one lane of warp 1 issues tcgen05.mma and
// commits, warps 2-5 zero the accumulator, then read it back with
// tcgen05.ld and write the epilogue.  Every wait is bounded: on a timeout the
// CTA records an error in a device word, drains its own copies, frees its
// TMEM and exits.
//
// Precisions: BF16 operands with FP32 accumulation, or a two-term BF16 split
// of both operands (v = hi + lo) with the three products hi*hi + hi*lo +
// lo*hi accumulated in FP32 (relative error ~2^-16 per product instead of
// ~2^-8).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "swopt_internal.cuh"

namespace swopt {

struct TcOperator {
    int split = 0;
    int tilesX = 0, tilesY = 0, Yp = 0, Xp = 0, HY = 0, HX = 0, npos = 0;
    int Zp16 = 0;
    // forward: slices of 8 depths
    int KSf = 0, GAf = 0, NGf = 0, NSf = 4;
    // adjoint: slices of 8 window samples
    int KSa = 0, GAa = 0, NGa = 0, NSa = 4;
    int colsF = 0, colsA = 0;
    size_t smemF = 0, smemA = 0;
    __nv_bfloat16 *bpad_hi = nullptr, *bpad_lo = nullptr;  // [Q][KSf][Yp][Xp][8]
    __nv_bfloat16 *rpad_hi = nullptr, *rpad_lo = nullptr;  // [Q][KSa][Yp][Xp][8]
    __nv_bfloat16 *Bf_hi = nullptr, *Bf_lo = nullptr;      // [NGf][kk][GAf][Twp][8]
    __nv_bfloat16 *Ba_hi = nullptr, *Ba_lo = nullptr;      // [NGa][kk][GAa][Zp16][8]
    uint32_t *band_f = nullptr, *band_a = nullptr;         // [NG][kk][GA/2] = lo | n << 16
    int* err = nullptr;
    double macs_f = 0, macs_a = 0;                         // issued MACs per launch
};

namespace {

constexpr int kTcThreads = 192;
constexpr int kMaxStages = 8;
constexpr uint32_t kWaitPolls = 1u << 22;  // x 256 ns back-off: about one second

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after about a second, or at once if the CTA aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag)
{
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (i > 32) __nanosleep(256);
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar)
                 : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (BF16 in, FP32 accumulate)
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start, leading-dimension byte
// offset (K direction), stride-dimension byte offset (M/N direction), all in
// 16-byte units; bits 46-48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9,
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__device__ __forceinline__ uint32_t make_idesc(uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_zero16(uint32_t taddr)
{
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// hi = bf16(v), lo = bf16(v - hi) for 8 values, packed as two uint4
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo)
{
    float h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const __nv_bfloat16 b = __float2bfloat16_rn(v[e]);
        h[e] = __bfloat162float(b);
        l[e] = v[e] - h[e];
    }
    hi = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                    pack_bf16x2(h[6], h[7]));
    lo = make_uint4(pack_bf16x2(l[0], l[1]), pack_bf16x2(l[2], l[3]), pack_bf16x2(l[4], l[5]),
                    pack_bf16x2(l[6], l[7]));
}

struct TcArgs {
    const __nv_bfloat16* a_hi;  // [Q][KS][Yp][Xp][8]
    const __nv_bfloat16* a_lo;
    const __nv_bfloat16* b_hi;  // [NG][kk][GA][NB][8]
    const __nv_bfloat16* b_lo;
    const uint32_t* band;       // [NG][kk][GA/2]
    float* out_f;               // forward mode 0: [Q][S][Twp]; adjoint: [Q][S][Z]
    __nv_bfloat16* out_hi;      // forward mode 1: [Q][KSo][Yp][Xp][8]
    __nv_bfloat16* out_lo;
    const float* ytil;          // [Q][S][Twp] or null
    const float* Cmf;           // [Q]
    double* partials;           // per block, or null
    int* err;
    int Y, X, Yp, Xp, Z, k, r, HY, HX, tilesX;
    int KS, GA, NG, NS, NB;
    int Twp, KSo;
    int adj, split, scale, mode;
    uint32_t tcols;
};

// ---------------------------------------------------------------------------
// The contraction kernel (forward or adjoint, see the file comment).
// grid = (tiles, Q); block = 192 threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1) tc_conv_kernel(const TcArgs a)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages];
    __shared__ __align__(8) uint64_t bar_empty[kMaxStages];
    __shared__ __align__(8) uint64_t bar_afull, bar_aempty, bar_acc;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ double s_red[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.y;
    const int x0 = (blockIdx.x % a.tilesX) * 8, y0 = (blockIdx.x / a.tilesX) * 16;
    const int kk = a.k * a.k;
    const uint32_t npos = (uint32_t)(a.HY * a.HX);
    const uint32_t a_slice = npos * 16u;                       // bytes of one A slice
    const uint32_t a_part = (uint32_t)a.GA * a_slice;          // hi (or lo) A bytes
    const uint32_t sA = smem_u32(smem);
    const uint32_t sA_lo = sA + a_part;
    const uint32_t sB = sA + a_part * (a.split ? 2u : 1u);
    const uint32_t b_part = (uint32_t)a.GA * (uint32_t)a.NB * 16u;  // hi (or lo) B bytes
    const uint32_t stage_bytes = b_part * (a.split ? 2u : 1u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < a.NS; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_afull), 1);
        mbar_init(smem_u32(&bar_aempty), 1);
        mbar_init(smem_u32(&bar_acc), 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(a.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    // zero the accumulator columns that the epilogue reads
    if (warp >= 2) {
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        for (int cb = 0; cb < a.NB / 16; ++cb) tmem_zero16(tmem + lanes + (uint32_t)cb * 16u);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        int stage = 0;
        uint32_t phase = 0;
        int fills[kMaxStages];
        for (int s = 0; s < kMaxStages; ++s) fills[s] = 0;
        int a_fills = 0;
        bool ok = true;
        for (int g = 0; g < a.NG && ok; ++g) {
            if (g > 0 && !mbar_wait(smem_u32(&bar_aempty), (uint32_t)(g - 1) & 1u, &s_abort)) {
                ok = false;
                break;
            }
            if (lane == 0) mbar_expect_tx(smem_u32(&bar_afull), a_part * (a.split ? 2u : 1u));
            ++a_fills;
            __syncwarp();
            const size_t img = (size_t)m * a.KS + (size_t)g * a.GA;
            for (int idx = lane; idx < a.GA * a.HY; idx += 32) {
                const int sl = idx / a.HY, hy = idx - sl * a.HY;
                const size_t goff = (((img + sl) * a.Yp + (size_t)(y0 + hy)) * a.Xp + x0) * 8;
                const uint32_t soff = (uint32_t)sl * a_slice + (uint32_t)(hy * a.HX) * 16u;
                bulk_g2s(sA + soff, a.a_hi + goff, (uint32_t)a.HX * 16u, smem_u32(&bar_afull));
                if (a.split)
                    bulk_g2s(sA_lo + soff, a.a_lo + goff, (uint32_t)a.HX * 16u,
                             smem_u32(&bar_afull));
            }
            for (int d = 0; d < kk; ++d) {
                if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &s_abort)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    const uint32_t bar = smem_u32(&bar_full[stage]);
                    mbar_expect_tx(bar, stage_bytes);
                    const size_t boff = ((size_t)g * kk + d) * (size_t)a.GA * a.NB * 8;
                    const uint32_t dst = sB + (uint32_t)stage * stage_bytes;
                    bulk_g2s(dst, a.b_hi + boff, b_part, bar);
                    if (a.split) bulk_g2s(dst + b_part, a.b_lo + boff, b_part, bar);
                }
                fills[stage]++;
                __syncwarp();
                if (++stage == a.NS) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
        }
        if (!ok && lane == 0) {
            s_abort = 1;
            atomicExch(a.err, 1);
        }
        // drain: every copy this warp issued has landed before the CTA exits
        if (lane == 0) {
            for (int s = 0; s < a.NS; ++s)
                if (fills[s] > 0) {
                    volatile int never = 0;
                    if (!mbar_wait(smem_u32(&bar_full[s]), (uint32_t)(fills[s] - 1) & 1u, &never))
                        atomicExch(a.err, 2);
                }
            if (a_fills > 0) {
                volatile int never = 0;
                if (!mbar_wait(smem_u32(&bar_afull), (uint32_t)(a_fills - 1) & 1u, &never))
                    atomicExch(a.err, 2);
            }
        }
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ----------------------------
        if (lane == 0) {
            const uint32_t lbo_a = a_slice, sbo_a = (uint32_t)a.HX * 16u;
            const uint32_t lbo_b = (uint32_t)a.NB * 16u, sbo_b = 128u;
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int g = 0; g < a.NG && ok; ++g) {
                if (!mbar_wait(smem_u32(&bar_afull), (uint32_t)g & 1u, &s_abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int d = 0; d < kk; ++d) {
                    if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int dy = d / a.k, dx = d - dy * a.k;
                    const uint32_t tap =
                        a.adj ? (uint32_t)((2 * a.r - dy) * a.HX + (2 * a.r - dx)) * 16u
                              : (uint32_t)(dy * a.HX + dx) * 16u;
                    const uint32_t* bandp = a.band + ((size_t)g * kk + d) * (size_t)(a.GA / 2);
                    const uint32_t bst = sB + (uint32_t)stage * stage_bytes;
                    for (int p = 0; p < a.GA / 2; ++p) {
                        const uint32_t e = __ldg(bandp + p);
                        const uint32_t n = e >> 16;
                        if (n == 0) continue;
                        const uint32_t lo = e & 0xFFFFu;
                        const uint32_t idesc = make_idesc(n);
                        const uint32_t aoff = 2u * (uint32_t)p * lbo_a + tap;
                        const uint32_t boff = 2u * (uint32_t)p * lbo_b + lo * 16u;
                        const uint64_t ad = make_desc(sA + aoff, lbo_a, sbo_a);
                        const uint64_t bd = make_desc(bst + boff, lbo_b, sbo_b);
                        const uint32_t dt = tmem + lo;
                        tc_mma(dt, ad, bd, idesc, 1u);
                        if (a.split) {
                            tc_mma(dt, ad, make_desc(bst + b_part + boff, lbo_b, sbo_b), idesc, 1u);
                            tc_mma(dt, make_desc(sA_lo + aoff, lbo_a, sbo_a), bd, idesc, 1u);
                        }
                    }
                    tc_commit(smem_u32(&bar_empty[stage]));
                    if (++stage == a.NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (ok) tc_commit(smem_u32(&bar_aempty));
            }
            // signals the epilogue; also covers every MMA issued above
            tc_commit(smem_u32(&bar_acc));
            if (!ok) {
                s_abort = 1;
                atomicExch(a.err, 1);
                volatile int never = 0;
                if (!mbar_wait(smem_u32(&bar_acc), 0u, &never)) atomicExch(a.err, 2);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------ epilogue ------------------------------
        const int q = warp & 3;
        const int i = q * 32 + lane;
        const int yl = i >> 3, xl = i & 7;
        const int y = y0 + yl, x = x0 + xl;
        const bool valid = (y < a.Y) && (x < a.X);
        bool ok = mbar_wait(smem_u32(&bar_acc), 0u, &s_abort);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        double part = 0.0;
        if (ok) {
            const uint32_t lanes = (uint32_t)(q * 32) << 16;
            const size_t pos = (size_t)y * a.X + x;
            const size_t S = (size_t)a.Y * a.X;
            const float cm = a.scale ? a.Cmf[m] : 1.f;
            for (int cb = 0; cb < a.NB / 16; ++cb) {
                float v[16];
                tmem_ld16(tmem + lanes + (uint32_t)cb * 16u, v);
                if (!valid) continue;
                if (a.adj) {
                    float* out = a.out_f + ((size_t)m * S + pos) * a.Z + cb * 16;
                    const int nz = min(16, a.Z - cb * 16);
                    if (nz == 16 && (a.Z & 3) == 0) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            *reinterpret_cast<float4*>(out + e) =
                                make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
                    } else {
                        for (int e = 0; e < nz; ++e) out[e] = v[e];
                    }
                } else {
                    const size_t ub = ((size_t)m * S + pos) * a.Twp + cb * 16;
                    float o[16];
                    if (a.ytil) {
                        const float4* yt = reinterpret_cast<const float4*>(a.ytil + ub);
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4) {
                            const float4 w = yt[e4];
                            const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const float acc = v[4 * e4 + c];
                                o[4 * e4 + c] = cm * acc - wv[c];
                                if (a.partials)
                                    part += (double)cm * (double)acc * acc -
                                            2.0 * (double)acc * wv[c];
                            }
                        }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) o[e] = cm * v[e];
                    }
                    if (a.mode == 0) {
                        float4* out = reinterpret_cast<float4*>(a.out_f + ub);
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4)
                            out[e4] = make_float4(o[4 * e4], o[4 * e4 + 1], o[4 * e4 + 2],
                                                  o[4 * e4 + 3]);
                    } else {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const size_t ro = ((((size_t)m * a.KSo + 2 * cb + h) * a.Yp +
                                                (y + a.r)) * a.Xp + (x + a.r)) * 8;
                            uint4 hi, lo;
                            split8(o + 8 * h, hi, lo);
                            *reinterpret_cast<uint4*>(a.out_hi + ro) = hi;
                            if (a.out_lo) *reinterpret_cast<uint4*>(a.out_lo + ro) = lo;
                        }
                    }
                }
            }
        }
        if (a.partials) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) s_red[q] = part;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (a.partials && threadIdx.x == 0)
        a.partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] =
            s_red[0] + s_red[1] + s_red[2] + s_red[3];
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tcols)
                     : "memory");
    }
}

// P into the padded BF16 state images: for each (m, slice, y, x) the 8
// depths j = 8 slice + e of b[m][y][x][j] = sum_p Sm[m][p][j] c[p][y][x][j].
__global__ void tc_states_kernel(const float* __restrict__ c, const float* __restrict__ Sm,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                 int Q, int P, int Y, int X, int Z, int slices, int KS, int Yp,
                                 int Xp, int r)
{
    const size_t n = (size_t)Q * slices * Y * X;
    const size_t SZ = (size_t)Y * X * Z;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % X);
        const int y = (int)((i / X) % Y);
        const int s8 = (int)((i / ((size_t)X * Y)) % slices);
        const int m = (int)(i / ((size_t)X * Y * slices));
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * s8 + e;
            float acc = 0.f;
            if (j < Z)
                for (int p = 0; p < P; ++p)
                    acc = fmaf(Sm[(m * P + p) * Z + j], c[p * SZ + ((size_t)y * X + x) * Z + j], acc);
            v[e] = acc;
        }
        uint4 h, l;
        split8(v, h, l);
        const size_t o = ((((size_t)m * KS + s8) * Yp + (y + r)) * Xp + (x + r)) * 8;
        *reinterpret_cast<uint4*>(hi + o) = h;
        if (lo) *reinterpret_cast<uint4*>(lo + o) = l;
    }
}

// FP32 u [Q][S][Twp] into the padded BF16 residual images
__global__ void tc_pack_kernel(const float* __restrict__ u, __nv_bfloat16* __restrict__ hi,
                               __nv_bfloat16* __restrict__ lo, int Q, int Y, int X, int Twp,
                               int KS, int Yp, int Xp, int r)
{
    const int slices = Twp / 8;
    const size_t n = (size_t)Q * slices * Y * X;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % X);
        const int y = (int)((i / X) % Y);
        const int s8 = (int)((i / ((size_t)X * Y)) % slices);
        const int m = (int)(i / ((size_t)X * Y * slices));
        const float4* src = reinterpret_cast<const float4*>(
            u + (((size_t)m * Y + y) * X + x) * Twp + 8 * s8);
        const float4 a0 = src[0], a1 = src[1];
        const float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        uint4 h, l;
        split8(v, h, l);
        const size_t o = ((((size_t)m * KS + s8) * Yp + (y + r)) * Xp + (x + r)) * 8;
        *reinterpret_cast<uint4*>(hi + o) = h;
        if (lo) *reinterpret_cast<uint4*>(lo + o) = l;
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
uint16_t f2bf(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
    const uint32_t rounding = 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
    return (uint16_t)((u + rounding) >> 16);
}

float bf2f(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

template <typename T>
swopt_status tc_alloc(T** p, size_t count)
{
    *p = nullptr;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SWOPT_ERR_OOM : SWOPT_ERR_CUDA;
    }
    return SWOPT_OK;
}

template <typename T>
swopt_status tc_upload(T** p, const std::vector<T>& v)
{
    SW_TRY(tc_alloc(p, v.size()));
    SW_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SWOPT_OK;
}

// Slices per group so that the operands of one CTA fit `budget` bytes.
bool pick_groups(int slices_min, int npos, int NB, int split, int NS, size_t budget, int* GA,
                 int* NG, size_t* smem)
{
    const size_t mult = split ? 2 : 1;
    for (int ng = 1; ng <= slices_min; ++ng) {
        int ga = (slices_min + ng - 1) / ng;
        ga += ga & 1;  // K = 16 per MMA: slices come in pairs
        const size_t bytes = mult * ((size_t)ga * npos * 16 + (size_t)NS * ga * NB * 16);
        if (bytes <= budget) {
            *GA = ga;
            *NG = (slices_min + ga - 1) / ga;
            *smem = bytes;
            return true;
        }
    }
    return false;
}

uint32_t pow2_cols(int n)
{
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

}  // namespace

void tc_release(swopt_handle* h)
{
    TcOperator* t = h->tc;
    if (!t) return;
    cudaFree(t->bpad_hi); cudaFree(t->bpad_lo); cudaFree(t->rpad_hi); cudaFree(t->rpad_lo);
    cudaFree(t->Bf_hi); cudaFree(t->Bf_lo); cudaFree(t->Ba_hi); cudaFree(t->Ba_lo);
    cudaFree(t->band_f); cudaFree(t->band_a); cudaFree(t->err);
    delete t;
    h->tc = nullptr;
}

swopt_status tc_prepare(swopt_handle* h)
{
    const int split = h->precision == SWOPT_PREC_BF16X3 ? 1 : 0;
    if (h->tc && h->tc->split == split) return SWOPT_OK;
    tc_release(h);
    const int kk = h->k * h->k;
    TcOperator* t = new TcOperator();
    t->split = split;
    t->tilesX = (h->X + 7) / 8;
    t->tilesY = (h->Y + 15) / 16;
    t->Xp = t->tilesX * 8 + 2 * h->r;
    t->Yp = t->tilesY * 16 + 2 * h->r;
    t->HX = 8 + 2 * h->r;
    t->HY = 16 + 2 * h->r;
    t->npos = t->HX * t->HY;
    t->Zp16 = ((h->Z + 15) / 16) * 16;
    if (h->Twp > 256 || t->Zp16 > 256) {
        delete t;
        set_error("tensor-core path supports a time window and a depth count up to 256 "
                  "(window %d, depths %d)", h->Twp, h->Z);
        return SWOPT_ERR_UNSUPPORTED;
    }
    // two CTAs per SM: operands within ~110 KB, accumulator within 256 TMEM columns
    const size_t budget = 110 * 1024;
    if (!pick_groups(t->Zp16 / 8, t->npos, h->Twp, split, t->NSf, budget, &t->GAf, &t->NGf,
                     &t->smemF) ||
        !pick_groups(h->Twp / 8, t->npos, t->Zp16, split, t->NSa, budget, &t->GAa, &t->NGa,
                     &t->smemA)) {
        delete t;
        set_error("lateral support k=%d too large for the tensor-core tile", h->k);
        return SWOPT_ERR_UNSUPPORTED;
    }
    t->KSf = t->NGf * t->GAf;
    t->KSa = t->NGa * t->GAa;
    t->colsF = (int)pow2_cols(h->Twp);
    t->colsA = (int)pow2_cols(t->Zp16);

    // FP32 values of the windowed kernel
    auto kval = [&](int j, int d, int w) -> float {
        const int tt = h->t0 + w;
        if (j >= h->Z || w >= h->Twp || tt >= h->T) return 0.f;
        return (float)h->K64[((size_t)j * kk + d) * h->T + tt];
    };
    // forward B blocks and bands
    std::vector<uint16_t> bfh((size_t)t->NGf * kk * t->GAf * h->Twp * 8, 0), bfl(bfh.size(), 0);
    std::vector<uint32_t> bandf((size_t)t->NGf * kk * (t->GAf / 2), 0);
    double macs_f = 0;
    for (int g = 0; g < t->NGf; ++g)
        for (int d = 0; d < kk; ++d) {
            for (int sl = 0; sl < t->GAf; ++sl)
                for (int w = 0; w < h->Twp; ++w)
                    for (int e = 0; e < 8; ++e) {
                        const float v = kval(8 * (g * t->GAf + sl) + e, d, w);
                        const uint16_t hb = f2bf(v);
                        const size_t o = ((((size_t)g * kk + d) * t->GAf + sl) * h->Twp + w) * 8 + e;
                        bfh[o] = hb;
                        bfl[o] = f2bf(v - bf2f(hb));
                    }
            for (int p = 0; p < t->GAf / 2; ++p) {
                int lo = -1, hi = -1;
                for (int e = 0; e < 16; ++e) {
                    const int j = 16 * (g * t->GAf / 2 + p) + e;
                    for (int w = 0; w < h->Twp; ++w)
                        if (kval(j, d, w) != 0.f) {
                            if (lo < 0 || w < lo) lo = w;
                            if (w > hi) hi = w;
                        }
                }
                uint32_t ent = 0;
                if (lo >= 0) {
                    const int l16 = lo & ~15;
                    const int n16 = ((hi + 1 - l16 + 15) / 16) * 16;
                    ent = (uint32_t)l16 | ((uint32_t)n16 << 16);
                    macs_f += 128.0 * n16 * 16 * (split ? 3 : 1);
                }
                bandf[((size_t)g * kk + d) * (t->GAf / 2) + p] = ent;
            }
        }
    // adjoint B blocks and bands
    std::vector<uint16_t> bah((size_t)t->NGa * kk * t->GAa * t->Zp16 * 8, 0), bal(bah.size(), 0);
    std::vector<uint32_t> banda((size_t)t->NGa * kk * (t->GAa / 2), 0);
    double macs_a = 0;
    for (int g = 0; g < t->NGa; ++g)
        for (int d = 0; d < kk; ++d) {
            for (int sl = 0; sl < t->GAa; ++sl)
                for (int j = 0; j < t->Zp16; ++j)
                    for (int e = 0; e < 8; ++e) {
                        const float v = kval(j, d, 8 * (g * t->GAa + sl) + e);
                        const uint16_t hb = f2bf(v);
                        const size_t o =
                            ((((size_t)g * kk + d) * t->GAa + sl) * t->Zp16 + j) * 8 + e;
                        bah[o] = hb;
                        bal[o] = f2bf(v - bf2f(hb));
                    }
            for (int p = 0; p < t->GAa / 2; ++p) {
                int lo = -1, hi = -1;
                for (int e = 0; e < 16; ++e) {
                    const int w = 16 * (g * t->GAa / 2 + p) + e;
                    for (int j = 0; j < t->Zp16; ++j)
                        if (kval(j, d, w) != 0.f) {
                            if (lo < 0 || j < lo) lo = j;
                            if (j > hi) hi = j;
                        }
                }
                uint32_t ent = 0;
                if (lo >= 0) {
                    const int l16 = lo & ~15;
                    const int n16 = ((hi + 1 - l16 + 15) / 16) * 16;
                    ent = (uint32_t)l16 | ((uint32_t)n16 << 16);
                    macs_a += 128.0 * n16 * 16 * (split ? 3 : 1);
                }
                banda[((size_t)g * kk + d) * (t->GAa / 2) + p] = ent;
            }
        }
    const double ctas = (double)t->tilesX * t->tilesY * h->Q;
    t->macs_f = macs_f * ctas;
    t->macs_a = macs_a * ctas;

    h->tc = t;
    const size_t nb = (size_t)h->Q * t->KSf * t->Yp * t->Xp * 8;
    const size_t nr = (size_t)h->Q * t->KSa * t->Yp * t->Xp * 8;
    swopt_status s = SWOPT_OK;
    auto step = [&](swopt_status v) { if (s == SWOPT_OK) s = v; };
    step(tc_alloc(&t->bpad_hi, nb));
    step(tc_alloc(&t->rpad_hi, nr));
    if (split) {
        step(tc_alloc(&t->bpad_lo, nb));
        step(tc_alloc(&t->rpad_lo, nr));
    }
    std::vector<__nv_bfloat16> tmp;
    auto up16 = [&](__nv_bfloat16** dst, const std::vector<uint16_t>& v) {
        if (s != SWOPT_OK) return;
        s = tc_alloc(dst, v.size());
        if (s != SWOPT_OK) return;
        if (cudaMemcpy(*dst, v.data(), v.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("cudaMemcpy of the tensor-core kernel failed");
            s = SWOPT_ERR_CUDA;
        }
    };
    up16(&t->Bf_hi, bfh);
    up16(&t->Ba_hi, bah);
    if (split) {
        up16(&t->Bf_lo, bfl);
        up16(&t->Ba_lo, bal);
    }
    if (s == SWOPT_OK) step(tc_upload(&t->band_f, bandf));
    if (s == SWOPT_OK) step(tc_upload(&t->band_a, banda));
    if (s == SWOPT_OK) step(tc_alloc(&t->err, 1));
    // zero borders and padded slices once; kernels only write the interior
    auto zero = [&](void* p, size_t bytes) {
        if (s == SWOPT_OK && p && cudaMemset(p, 0, bytes) != cudaSuccess) {
            set_error("cudaMemset failed");
            s = SWOPT_ERR_CUDA;
        }
    };
    zero(t->bpad_hi, nb * 2); zero(t->bpad_lo, nb * 2);
    zero(t->rpad_hi, nr * 2); zero(t->rpad_lo, nr * 2);
    zero(t->err, sizeof(int));
    // At most 512 / cols CTAs may share an SM's 512 TMEM columns: request
    // enough shared memory that no more can be resident (233472 B per SM).
    const size_t per_sm = 233472;
    t->smemF = std::max(t->smemF, per_sm / (512 / t->colsF) + 1024);
    t->smemA = std::max(t->smemA, per_sm / (512 / t->colsA) + 1024);
    if (s == SWOPT_OK) {
        const size_t mx = std::max(t->smemF, t->smemA);
        if (cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mx) != cudaSuccess) {
            set_error("cudaFuncSetAttribute failed for the tensor-core kernel");
            s = SWOPT_ERR_CUDA;
        }
    }
    if (s != SWOPT_OK) tc_release(h);
    return s;
}

int tc_forward_blocks(const swopt_handle* h)
{
    return ((h->X + 7) / 8) * ((h->Y + 15) / 16) * h->Q;
}

swopt_status tc_states(swopt_handle* h, const float* c, cudaStream_t st)
{
    TcOperator* t = h->tc;
    const int slices = (h->Z + 7) / 8;
    const size_t n = (size_t)h->Q * slices * h->Y * h->X;
    int grid = grid_for(n, 256);
    if (grid > 152 * 16) grid = 152 * 16;
    tc_states_kernel<<<grid, 256, 0, st>>>(c, h->Sm, t->bpad_hi, t->split ? t->bpad_lo : nullptr,
                                           h->Q, h->P, h->Y, h->X, h->Z, slices, t->KSf, t->Yp,
                                           t->Xp, h->r);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status tc_pack_u(swopt_handle* h, cudaStream_t st)
{
    TcOperator* t = h->tc;
    const size_t n = (size_t)h->Q * (h->Twp / 8) * h->Y * h->X;
    int grid = grid_for(n, 256);
    if (grid > 152 * 16) grid = 152 * 16;
    tc_pack_kernel<<<grid, 256, 0, st>>>(h->u, t->rpad_hi, t->split ? t->rpad_lo : nullptr, h->Q,
                                         h->Y, h->X, h->Twp, t->KSa, t->Yp, t->Xp, h->r);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

static TcArgs base_args(swopt_handle* h)
{
    TcOperator* t = h->tc;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Cmf = h->Cmf;
    a.err = t->err;
    a.Y = h->Y; a.X = h->X; a.Yp = t->Yp; a.Xp = t->Xp; a.Z = h->Z; a.k = h->k; a.r = h->r;
    a.HY = t->HY; a.HX = t->HX; a.tilesX = t->tilesX;
    a.Twp = h->Twp;
    a.KSo = t->KSa;
    a.split = t->split;
    return a;
}

swopt_status tc_forward(swopt_handle* h, bool to_r, const float* ytil, double* partials,
                        int scale, cudaStream_t st)
{
    TcOperator* t = h->tc;
    TcArgs a = base_args(h);
    a.a_hi = t->bpad_hi; a.a_lo = t->bpad_lo;
    a.b_hi = t->Bf_hi; a.b_lo = t->Bf_lo;
    a.band = t->band_f;
    a.KS = t->KSf; a.GA = t->GAf; a.NG = t->NGf; a.NS = t->NSf; a.NB = h->Twp;
    a.adj = 0;
    a.scale = scale;
    a.ytil = ytil;
    a.partials = partials;
    a.mode = to_r ? 1 : 0;
    a.out_f = to_r ? nullptr : h->u;
    a.out_hi = to_r ? t->rpad_hi : nullptr;
    a.out_lo = to_r ? t->rpad_lo : nullptr;
    a.tcols = (uint32_t)t->colsF;
    dim3 grid(t->tilesX * t->tilesY, h->Q);
    ProfileRec rec;
    prof_begin(h, 0, st, &rec);
    tc_conv_kernel<<<grid, kTcThreads, t->smemF, st>>>(a);
    SW_LAUNCHED(h);
    prof_end(h, &rec, st);
    return SWOPT_OK;
}

swopt_status tc_adjoint(swopt_handle* h, cudaStream_t st)
{
    TcOperator* t = h->tc;
    TcArgs a = base_args(h);
    a.a_hi = t->rpad_hi; a.a_lo = t->rpad_lo;
    a.b_hi = t->Ba_hi; a.b_lo = t->Ba_lo;
    a.band = t->band_a;
    a.KS = t->KSa; a.GA = t->GAa; a.NG = t->NGa; a.NS = t->NSa; a.NB = t->Zp16;
    a.adj = 1;
    a.out_f = h->g;
    a.tcols = (uint32_t)t->colsA;
    dim3 grid(t->tilesX * t->tilesY, h->Q);
    ProfileRec rec;
    prof_begin(h, 1, st, &rec);
    tc_conv_kernel<<<grid, kTcThreads, t->smemA, st>>>(a);
    SW_LAUNCHED(h);
    prof_end(h, &rec, st);
    return SWOPT_OK;
}

int tc_error_word(swopt_handle* h)
{
    if (!h->tc || !h->tc->err) return 0;
    int v = 0;
    if (cudaMemcpy(&v, h->tc->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (v) cudaMemset(h->tc->err, 0, sizeof(int));
    return v;
}

double tc_issued_macs(const swopt_handle* h, int kernel)
{
    if (!h->tc) return 0;
    return kernel == 0 ? h->tc->macs_f : h->tc->macs_a;
}

}  // namespace swopt
