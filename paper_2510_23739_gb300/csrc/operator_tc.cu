// Tensor-core (tcgen05, sm_103a) kernels for the acoustic correlation A and
// its transpose A^T (Sec. 2.3.3, Eq. acoustic-full-forward).
//
// Both are implicit GEMMs whose M dimension is the output channel and whose
// N dimension is a tile of 32 x 8 = 256 scan positions:
//   A  : D[t][pos] += sum_j K[j][d][t] b[pos + d][j]     (channel t, K-dim depth j)
//   A^T: D[j][pos] += sum_t K[j][d][t] r[pos - d][t]     (channel j, K-dim sample t)
// for every lateral tap d.  One MMA is M = 128 channels x N = 256 positions
// x K = 16 (one pair of 8-element slices of the contracted dimension).  The
// kernel block of a (tap, pair) is the A operand, streamed through a ring of
// shared-memory stages by bulk asynchronous copies; the image is the B
// operand: a halo of the CTA's tiles, staged once per group of slice pairs
// as [8-element slice][halo row][halo column][8 elements], so that the
// operand of tap d is the same buffer at a byte offset (8 consecutive x of
// a halo row form one 16 B x 8 core matrix; consecutive rows are one halo
// row apart).  MT tiles side by side share every staged kernel block.
//
// Measured on GB300 (one SM, operands in shared memory): an MMA of
// M = 128 x N x K = 16 takes max(N / 2, (128 + N) / 4) cycles, the larger
// term being the tensor core's shared-memory operand reads at 128 B per
// cycle; one issuing warp keeps the tensor core busy.  N = 256 makes the MMA
// compute-bound (128 cycles against 96 of operand reads), which leaves
// shared-memory bandwidth for the copies that feed the next MMAs.
//
// Measured too: the issue loop must stay simple.  With the MMAs of a stage
// issued from nested loops whose trip counts and branches depend on the
// configuration (pairs per group, channel blocks, tiles, which products),
// the issuing thread took about 230 cycles per MMA; the same stage issued
// from one loop over its taps with the products of a tap unrolled at
// compile time takes about 113 (the tensor core then sets the pace).  So
// each group holds one slice pair, and the products of a tap come from a
// loop specialised per (tiles, channel blocks, precision), chosen once per
// stage.
//
// Roles (192 threads) of a persistent CTA: warp 0 stages operands with bulk
// asynchronous copies (the TMA engine) on mbarriers; warp 1 issues
// tcgen05.mma and commits (its elected lane, in a converged warp); warps 2-5
// read the accumulators back with tcgen05.ld (lane = channel), run the
// epilogue and hand the accumulators back zeroed.  The CTAs share the runs of
// taps of all tile-states equally (the stream-K split), so a tile-state may be
// contracted in pieces by neighbouring CTAs and finished by the last of them
// to arrive.  Every wait is bounded: on a timeout the CTA records an error in
// a device word, drains its own copies and MMAs, frees its TMEM and exits.
//
// Precisions: BF16 operands with FP32 accumulation (1 term), or a split of
// both operands into 2 BF16 terms (v = v0 + v1, v1 the BF16 rounding of
// v - v0) with the 3 products v0 w0, v0 w1, v1 w0 (the dropped v1 w1 is
// below 2^-16 of |v w|) accumulated in FP32; the 2 correction products go to
// an accumulator of their own where TMEM holds it, so that the tensor core's
// FP32 accumulation rounds them on their own (2^-8 smaller) scale.  Or 3
// BF16 terms (v2 the BF16 rounding of v - v0 - v1) with the 6 products of
// total order up to 2 (v0 w0; v0 w1, v1 w0; v0 w2, v1 w1, v2 w0), the
// representation and the dropped products below about 2^-24 of |v w|, the
// 5 corrections in the correction accumulator.  Or FP8
// E4M3 operands (kind::f8f6f4, K = 32 per MMA in the same 32 bytes of a row)
// with FP32 accumulation and per-channel equilibration of the contracted
// dimension: the kernel is stored as K_j / s_j and the image as b_j s_j sigma,
// so every product is K_j b_j sigma exactly in real arithmetic; s_j (static,
// from the kernel) puts each depth's (A) or sample's (A^T) largest kernel
// entry at 256, and sigma (per launch, from the largest scaled image entry)
// does the same for the image; the epilogue divides by sigma.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "swopt_internal.cuh"

namespace swopt {

constexpr int kMaxTerms = 3;    // BF16 terms per operand of the split precisions
constexpr int kMaxSpecies = 8;  // the geometry's limit on P
constexpr int kRows = 128;      // MMA M: output channels per block
constexpr int kTileY = 32;      // scan rows of a position tile
constexpr int kTilePos = 256;   // MMA N: positions of a tile (32 rows x 8 columns)
constexpr int kBlockBytes = 2 * kRows * 16;  // one (tap, pair, channel block) kernel block

// Operator data of one direction (forward or adjoint).
struct TcDir {
    int GA = 0, NG = 0, KS = 0;   // image slices per group (even), groups, padded slices
    int MB = 1;                   // channel blocks of 128 rows
    int rows = 0;                 // valid channels (window samples for A, depths for A^T)
    int MT = 1;                   // position tiles per CTA, side by side along x
    int RA = 1;                   // accumulators per (block, tile): 2 keeps corrections apart
    int whole = 1;                // 1: CTAs take whole tile-states; 0: balanced runs (stream-K)
    int runs = 0;                 // runs of taps per tile-state (all groups)
    int NBUF = 1;                 // accumulator buffers in TMEM (2: epilogue overlaps the next unit)
    int grid = 0;                 // persistent CTAs launched
    int quantum = 1;              // runs per indivisible piece of work
    long long wq = 0;             // pieces of work in all: tile-states x runs / quantum
    int max_pieces = 1;           // most CTAs sharing one tile-state
    float* part = nullptr;        // max_pieces > 1: [tile-states][max_pieces][MB][MT][16][128][16]
    int* ticket = nullptr;        // max_pieces > 1: [tile-states] arrival counters (return to 0)
    int NS = 4;                   // stages of the kernel ring
    uint32_t stage_bytes = 0;     // bytes of one stage (hi part; lo is as large)
    int HX = 0, npos = 0;         // halo width and positions
    int cols = 0;                 // TMEM columns allocated
    size_t smem = 0;              // dynamic shared memory requested
    int groupsX = 0;              // CTAs along x
    __nv_bfloat16* Wt[kMaxTerms] = {};  // kernel per term,
                                  // [group][tap][pair][MB][2][128][8]
    uint32_t* tab = nullptr;      // per group: header + run table (see TcArgs)
    int tab_words = 0;
    double macs = 0;              // issued MACs per launch
};

struct TcOperator {
    int terms = 1;                // BF16 terms per operand (1, 2 or 3)
    bool fp8 = false;             // E4M3 operands (one term)
    int esl = 8;                  // contracted-dimension elements per 16-byte slice (8 or 16)
    int tilesX = 0, tilesY = 0, Yp = 0, Xp = 0, HY = 0;
    int Zp16 = 0;                 // depths padded to a whole slice pair (16 BF16 or 32 FP8)
    float* s_dep = nullptr;       // FP8: [Zp16] depth scales s_j of the forward
    float* s_tim = nullptr;       // FP8: [Twp] sample scales s_t of the adjoint
    unsigned* words = nullptr;    // FP8: [2] largest scaled image / residual entry (float bits)
    std::vector<double> s_dep_h, s_tim_h;  // FP8: host copies of the scales
    TcDir F, A;
    __nv_bfloat16* bpad[kMaxTerms] = {};  // [Q][F.KS][Yp][Xp][8] per term
    __nv_bfloat16* rpad[kMaxTerms] = {};  // [Q][A.KS][Yp][Xp][8] per term
    int* err = nullptr;
};

namespace {

constexpr int kTcThreads = 192;
constexpr int kMaxStages = 8;
constexpr int kMaxTapsPerStage = 8;  // taps per stage of the kernel ring (host-side cap)
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// Bounded wait by a whole converged warp: every lane gets the same answer.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity,
                                               volatile int* abort_flag)
{
    const bool ok = mbar_wait(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// One lane of a converged warp (the lowest) returns true.
__device__ __forceinline__ bool elect_one()
{
    uint32_t pred = 0;
    asm volatile(
        "{\n\t.reg .b32 rx;\n\t.reg .pred px;\n\t"
        "elect.sync rx|px, 0xffffffff;\n\t"
        "@px mov.s32 %0, 1;\n\t}"
        : "+r"(pred));
    return pred != 0;
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

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (BF16 in, FP32 accumulate).
// No memory clobber: the operands are read by the asynchronous proxy after
// the mbarrier waits (which are compiler barriers), so plain loads of the
// next items may be scheduled around the issue.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// D[tmem] (+)= A * B^T, kind::f8f6f4 with E4M3 A and B (K = 32), FP32 accumulate.
__device__ __forceinline__ void tc_mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
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

// The BF16 terms of 8 values: t0 = bf16(v), then t1 = bf16(v - t0) and
// t2 = bf16(v - t0 - t1) as `terms` asks, each packed as one uint4.
__device__ __forceinline__ void split_terms(const float* v, uint4* out, int terms)
{
    float r[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) r[e] = v[e];
    for (int tt = 0; tt < terms; ++tt) {
        float h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            h[e] = __bfloat162float(__float2bfloat16_rn(r[e]));
            r[e] -= h[e];
        }
        out[tt] = make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]),
                             pack_bf16x2(h[4], h[5]), pack_bf16x2(h[6], h[7]));
    }
}

struct TcArgs {
    const __nv_bfloat16* img[kMaxTerms];  // per term: padded images [Q][KS][Yp][Xp][8]
    const __nv_bfloat16* w[kMaxTerms];    // per term: kernel [group][tap][pair][MB][2][128][8]
    const uint4* tab;           // per group g: {base (16 B units), tap bytes, taps per
                                // run, pairs}, then per run of taps of a group (the
                                // same for every group) eight 16-bit halo offsets of
                                // its taps in 16-B units
    int tab_n;                  // uint4 entries in tab
    float* out_f;               // forward mode 0: [Q][S][Twp]; adjoint: [Q][S][Z]
    __nv_bfloat16* out_t[kMaxTerms];    // forward mode 1, per term: [Q][KSo][Yp][Xp][8]
    const float* ytil;          // [Q][S][Twp] or null
    const float* Cmf;           // [Q]
    double* partials;           // per block, or null
    int* err;
    int Y, X, Yp, Xp, Z, k, r, HY, HX, groupsX, MT, RA, MB, rows;
    float* part;                // partial sums of tile-states shared by several CTAs
    int* ticket;                // per tile-state arrival counters
    int KS, GA, NG, NS;
    uint32_t stage_bytes;
    int Twp, KSo;
    int adj, terms, scale, mode;
    uint32_t tcols;
    int NBUF;                   // accumulator buffers in TMEM (1, or 2: epilogue overlapped)
    int ntiles;                 // CTA tiles of the scan plane
    int runs;                   // runs of taps per tile-state
    int quantum;                // runs per indivisible piece of work
    long long wq;               // pieces of work in all: tile-states x runs / quantum
    int max_pieces;             // partial-sum slots per tile-state
    const int* gate;            // launch runs only if *gate == want (null: always)
    int want;
    int fp8;                    // E4M3 operands: kind::f8f6f4, output divided by sigma
    const unsigned* in_word;    // FP8: the largest scaled entry of the input images (sigma = 256 / it)
    unsigned* max_word;         // FP8 forward mode 0: atomic max of |out| s_t (the residual's scale)
    const float* s_out;         // FP8 forward: the adjoint's sample scales s_t
    const int* split_slot;      // shared launches: partial-sum slot of each split tile-state
                                // (null: the tile-state's own index)
};

// ---------------------------------------------------------------------------
// The contraction kernel (forward or adjoint, see the file comment).
// Persistent: grid = min(pieces of work, resident CTAs), block = 192 threads.
// The work is the runs of taps of every tile-state, in order (tile-state
// major); CTA b takes the b-th of gridDim.x equal shares of it, rounded to
// whole pieces of `quantum` runs (one run: the stream-K split, which leaves
// no wave tail; all runs of a tile-state: whole tile-states).  A CTA's share
// cut by tile-state boundaries gives its work units; every role walks the
// same unit sequence.  With NBUF = 2 the accumulators are double-buffered in
// TMEM, so that the epilogue of one unit overlaps the MMAs of the next.  A
// tile-state shared by several CTAs is finished by the last to arrive: each
// writes its summed accumulators to `part` and takes a ticket; the last adds
// the partial sums (two: a + b, the same bits whichever arrives last; more:
// in piece order) and runs the epilogue.  No CTA waits for another.
// ---------------------------------------------------------------------------
struct TcUnit {
    int p;               // problem (0 for a single-problem launch)
    int ts, r0, r1;      // tile-state (m * tiles + tile) and its runs [r0, r1)
    int m, x0, y0;
    int piece, pieces;   // this CTA's piece of the tile-state, of how many
};

// The CTA whose share holds run x of the whole work.
__device__ __forceinline__ int tc_owner(const TcArgs& a, long long x)
{
    const long long xq = x / a.quantum;
    return (int)(((xq + 1) * (long long)gridDim.x - 1) / a.wq);
}

// Unit k of this CTA; false past the end.
__device__ __forceinline__ bool tc_unit(const TcArgs& a, int k, TcUnit& u)
{
    const long long G = gridDim.x, R = a.runs;
    const long long b0 = (long long)a.quantum * ((long long)blockIdx.x * a.wq / G);
    const long long b1 = (long long)a.quantum * (((long long)blockIdx.x + 1) * a.wq / G);
    const long long ts = b0 / R + k;
    if (ts * R >= b1) return false;
    u.ts = (int)ts;
    u.r0 = (int)(b0 > ts * R ? b0 - ts * R : 0);
    u.r1 = (int)(b1 - ts * R < R ? b1 - ts * R : R);
    const int first = tc_owner(a, ts * R), last = tc_owner(a, ts * R + R - 1);
    u.pieces = last - first + 1;
    u.piece = (int)blockIdx.x - first;
    u.m = u.ts / a.ntiles;
    const int tile = u.ts - u.m * a.ntiles;
    u.x0 = (tile % a.groupsX) * 8 * a.MT;
    u.y0 = (tile / a.groupsX) * kTileY;
    return true;
}

// Constants of a launch's MMA products: the bytes between channel blocks of
// a kernel block, and the offsets (16-B descriptor units) of the second BF16
// terms of the halo and of the stage.
struct IssueCfg {
    uint32_t tap_bytes;     // the MB channel blocks of one tap (kBlockBytes apart)
    uint32_t halo_lo16;     // halo of the second term (the third follows at twice this)
    uint32_t stage_lo16;    // kernel blocks of the second term (likewise)
    uint32_t idesc;
};

// The products of every tap of a stage, specialised at compile time: MT
// tiles, MB channel blocks, and MODE 0 (one BF16 term), 1 (two terms, the
// corrections in accumulator set 1), 2 (two terms, one accumulator set), 3
// (one E4M3 term, kind::f8f6f4), 4 (three terms, the corrections in set 1)
// or 5 (three terms, one accumulator set).
// Accumulator of (set, block, tile): columns ((set MB + block) MT + tile) 256.
template <int MT, int MB, int MODE>
__device__ __forceinline__ void issue_taps(const IssueCfg& c, uint32_t tbuf, uint64_t a0,
                                           uint64_t b0, const uint32_t (&ow)[4], int nt)
{
    const uint64_t tap16 = (uint64_t)(c.tap_bytes >> 4);
    for (int t = 0; t < nt; ++t) {
        const uint32_t off = (ow[(t >> 1) & 3] >> (16 * (t & 1))) & 0xFFFFu;
        const uint64_t at = a0 + (uint64_t)t * tap16;
        const uint64_t bt = b0 + (uint64_t)off;
#pragma unroll
        for (int mb = 0; mb < MB; ++mb) {
            const uint64_t am = at + (uint64_t)(mb * (kBlockBytes >> 4));
#pragma unroll
            for (int i = 0; i < MT; ++i) {
                const uint64_t bi = bt + (uint64_t)(i * 8);  // the next tile: 8 positions x 16 B
                const uint32_t dm = tbuf + (uint32_t)((mb * MT + i) * kTilePos);
                if (MODE == 3) {
                    tc_mma_f8(dm, am, bi, c.idesc, 1u);
                    continue;
                }
                tc_mma(dm, am, bi, c.idesc, 1u);
                if (MODE != 0) {
                    const uint32_t dc = MODE == 1 || MODE == 4
                                            ? tbuf + (uint32_t)(((MB + mb) * MT + i) * kTilePos)
                                            : dm;
                    tc_mma(dc, am + c.stage_lo16, bi, c.idesc, 1u);
                    tc_mma(dc, am, bi + c.halo_lo16, c.idesc, 1u);
                    if (MODE >= 4) {
                        tc_mma(dc, am + 2 * (uint64_t)c.stage_lo16, bi, c.idesc, 1u);
                        tc_mma(dc, am + c.stage_lo16, bi + c.halo_lo16, c.idesc, 1u);
                        tc_mma(dc, am, bi + 2 * (uint64_t)c.halo_lo16, c.idesc, 1u);
                    }
                }
            }
        }
    }
}

__host__ __device__ __forceinline__ int issue_kind(int MT, int MB, int terms, int RA, int fp8)
{
    if (fp8) return 12 + (MT - 1) * 2 + (MB - 1);
    if (terms == 3) return 16 + ((MT - 1) * 2 + (MB - 1)) * 2 + (RA == 2 ? 0 : 1);
    const int mode = terms == 1 ? 0 : (RA == 2 ? 1 : 2);
    return ((MT - 1) * 2 + (MB - 1)) * 3 + mode;
}

__device__ __forceinline__ void issue_stage(int kind, const IssueCfg& c, uint32_t tbuf,
                                            uint64_t a0, uint64_t b0, const uint32_t (&ow)[4],
                                            int nt)
{
    switch (kind) {
    case 0: issue_taps<1, 1, 0>(c, tbuf, a0, b0, ow, nt); break;
    case 1: issue_taps<1, 1, 1>(c, tbuf, a0, b0, ow, nt); break;
    case 2: issue_taps<1, 1, 2>(c, tbuf, a0, b0, ow, nt); break;
    case 3: issue_taps<1, 2, 0>(c, tbuf, a0, b0, ow, nt); break;
    case 4: issue_taps<1, 2, 1>(c, tbuf, a0, b0, ow, nt); break;
    case 5: issue_taps<1, 2, 2>(c, tbuf, a0, b0, ow, nt); break;
    case 6: issue_taps<2, 1, 0>(c, tbuf, a0, b0, ow, nt); break;
    case 7: issue_taps<2, 1, 1>(c, tbuf, a0, b0, ow, nt); break;
    case 8: issue_taps<2, 1, 2>(c, tbuf, a0, b0, ow, nt); break;
    case 9: issue_taps<2, 2, 0>(c, tbuf, a0, b0, ow, nt); break;
    case 10: issue_taps<2, 2, 1>(c, tbuf, a0, b0, ow, nt); break;
    case 11: issue_taps<2, 2, 2>(c, tbuf, a0, b0, ow, nt); break;
    case 12: issue_taps<1, 1, 3>(c, tbuf, a0, b0, ow, nt); break;
    case 13: issue_taps<1, 2, 3>(c, tbuf, a0, b0, ow, nt); break;
    case 14: issue_taps<2, 1, 3>(c, tbuf, a0, b0, ow, nt); break;
    case 15: issue_taps<2, 2, 3>(c, tbuf, a0, b0, ow, nt); break;
    case 16: issue_taps<1, 1, 4>(c, tbuf, a0, b0, ow, nt); break;
    case 17: issue_taps<1, 1, 5>(c, tbuf, a0, b0, ow, nt); break;
    case 18: issue_taps<1, 2, 4>(c, tbuf, a0, b0, ow, nt); break;
    case 19: issue_taps<1, 2, 5>(c, tbuf, a0, b0, ow, nt); break;
    case 20: issue_taps<2, 1, 4>(c, tbuf, a0, b0, ow, nt); break;
    case 21: issue_taps<2, 1, 5>(c, tbuf, a0, b0, ow, nt); break;
    case 22: issue_taps<2, 2, 4>(c, tbuf, a0, b0, ow, nt); break;
    default: issue_taps<2, 2, 5>(c, tbuf, a0, b0, ow, nt); break;
    }
}

// A launch over several problems: the runs of every problem's tile-states, in
// problem order, shared out equally over the CTAs (TcMany::unit).  The stage ring, the halo region and
// the TMEM columns are sized for the largest problem.
struct TcBatchMeta {
    long long piece0;  // the problem's first run in the launch's work
    int tab_off;       // its run table's first entry among the staged tables
    int pad;
};

struct TcBatchArgs {
    const TcArgs* probs;      // [n] in device memory
    const TcBatchMeta* meta;  // [n]
    int n;
    long long W;              // runs of all problems
    int NS, NBUF;
    uint32_t halo_region;     // bytes of the largest halo (all terms)
    uint32_t stage_slot;      // bytes of the largest stage (all terms)
    uint32_t tcols;           // TMEM columns allocated
    uint32_t buf_stride;      // TMEM columns between the accumulator buffers
    const uint4* tab;         // the problems' group / run tables, concatenated
    int tab_n;
    int* err;
};

// The work and arguments of a launch over one problem ...
struct TcOne {
    const TcArgs& a;
    __device__ int NS() const { return a.NS; }
    __device__ int NBUF() const { return a.NBUF; }
    __device__ uint32_t halo_region() const
    {
        return (uint32_t)(a.GA * a.HY * a.HX) * 16u * (uint32_t)a.terms;
    }
    __device__ uint32_t stage_slot() const { return a.stage_bytes * (uint32_t)a.terms; }
    __device__ uint32_t tcols() const { return a.tcols; }
    __device__ uint32_t buf_stride() const { return (uint32_t)(a.RA * a.MB * a.MT * kTilePos); }
    __device__ const uint4* tab() const { return a.tab; }
    __device__ int tab_n() const { return a.tab_n; }
    __device__ int* err() const { return a.err; }
    __device__ double* partials() const { return a.partials; }
    __device__ unsigned* max_word() const { return a.max_word; }
    __device__ bool unit(int k, TcUnit& u) const
    {
        u.p = 0;
        return tc_unit(a, k, u);
    }
    __device__ const TcArgs& args(int) const { return a; }
    __device__ int tab_off(int) const { return 0; }
    __device__ bool skip(const TcArgs&) const { return false; }
};

// ... and over several (the gate of each problem is read per tile-state).
struct TcMany {
    const TcBatchArgs& B;
    __device__ int NS() const { return B.NS; }
    __device__ int NBUF() const { return B.NBUF; }
    __device__ uint32_t halo_region() const { return B.halo_region; }
    __device__ uint32_t stage_slot() const { return B.stage_slot; }
    __device__ uint32_t tcols() const { return B.tcols; }
    __device__ uint32_t buf_stride() const { return B.buf_stride; }
    __device__ const uint4* tab() const { return B.tab; }
    __device__ int tab_n() const { return B.tab_n; }
    __device__ int* err() const { return B.err; }
    __device__ double* partials() const { return nullptr; }
    __device__ unsigned* max_word() const { return nullptr; }
    // CTA b of G takes the b-th of G equal shares of the W runs of all
    // problems in order, [L, U) with b W <= x G < (b + 1) W, cut at tile-state
    // boundaries into units; a tile-state cut between CTAs is finished by the
    // last of them to arrive (the partial-sum path of the epilogue)
    __device__ static long long ceil_div(long long x, long long d)
    {
        return x >= 0 ? (x + d - 1) / d : -((-x) / d);
    }
    __device__ bool unit(int k, TcUnit& u) const
    {
        const long long G = gridDim.x;
        const long long L = ceil_div((long long)blockIdx.x * B.W, G);
        const long long U = ceil_div(((long long)blockIdx.x + 1) * B.W, G);
        for (int p = 0; p < B.n; ++p) {
            const TcArgs& a = B.probs[p];
            const long long R = a.runs, base = B.meta[p].piece0, end = base + a.wq * R;
            const long long lo = L > base ? L : base, hi = U < end ? U : end;
            if (lo >= hi) continue;
            const long long ts0 = (lo - base) / R, ts1 = (hi - 1 - base) / R;
            if (k <= ts1 - ts0) {
                const long long ts = ts0 + k, x0 = base + ts * R;
                u.p = p;
                u.ts = (int)ts;
                u.r0 = (int)(lo > x0 ? lo - x0 : 0);
                u.r1 = (int)(hi - x0 < R ? hi - x0 : R);
                const int first = (int)(x0 * G / B.W), last = (int)((x0 + R - 1) * G / B.W);
                u.pieces = last - first + 1;
                u.piece = (int)blockIdx.x - first;
                u.m = u.ts / a.ntiles;
                const int tile = u.ts - u.m * a.ntiles;
                u.x0 = (tile % a.groupsX) * 8 * a.MT;
                u.y0 = (tile / a.groupsX) * kTileY;
                return true;
            }
            k -= (int)(ts1 - ts0 + 1);
        }
        return false;
    }
    __device__ const TcArgs& args(int p) const { return B.probs[p]; }
    __device__ int tab_off(int p) const { return B.meta[p].tab_off; }
    __device__ bool skip(const TcArgs& a) const { return gated_off(a.gate, a.want); }
};

template <class Src>
__device__ __forceinline__ void tc_body(const Src& src)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_full[kMaxStages];
    __shared__ __align__(8) uint64_t bar_empty[kMaxStages];
    __shared__ __align__(8) uint64_t bar_afull, bar_aempty;
    __shared__ __align__(8) uint64_t bar_accfull[2], bar_accfree[2], bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;
    __shared__ double s_red[4];
    __shared__ int s_last;
    __shared__ int s_eok[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = src.NS(), NBUF = src.NBUF();
    int* const err = src.err();
    // shared memory: the halo region, the ring of NS stage slots, the tables
    const uint32_t sA = __shfl_sync(0xffffffffu, smem_u32(smem), 0);
    const uint32_t sW = sA + src.halo_region();
    const uint32_t stage_slot = src.stage_slot();
    const uint32_t tab_region = src.halo_region() + (uint32_t)NS * stage_slot;
    const uint4* s_tab = reinterpret_cast<const uint4*>(smem + tab_region);
    // TMEM columns between the accumulator buffers (a buffer: [set][block][tile][256 positions])
    const uint32_t buf_stride = src.buf_stride();

    // the group / run tables are small: stage them once
    for (int i = threadIdx.x; i < src.tab_n(); i += kTcThreads)
        reinterpret_cast<uint4*>(smem + tab_region)[i] = src.tab()[i];
    if (threadIdx.x == 0) {
        // the issuer commits to the stage-empty, halo-empty and
        // accumulator-full barriers; every epilogue thread arrives on
        // accumulator-free
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_afull), 1);
        mbar_init(smem_u32(&bar_aempty), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&bar_accfull[b]), 1);
            mbar_init(smem_u32(&bar_accfree[b]), 128u);
        }
        mbar_init(smem_u32(&bar_drain), 1u);
        s_abort = 0;
        s_red[0] = s_red[1] = s_red[2] = s_red[3] = 0.0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(src.tcols())
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // warp-uniform by construction (MMA operands must be uniform values)
    const uint32_t tmem = __shfl_sync(0xffffffffu, s_tmem, 0);

    // zero the accumulator columns of every buffer
    if (warp >= 2 && warp <= 5) {
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        for (uint32_t cb = 0; cb < (uint32_t)NBUF * buf_stride / 16u; ++cb)
            tmem_zero16(tmem + lanes + cb * 16u);
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
        TcUnit u;
        for (int k = 0; ok && src.unit(k, u); ++k) {
            const TcArgs& a = src.args(u.p);
            if (src.skip(a)) continue;
            const int kk = a.k * a.k;
            const uint32_t a_slice = (uint32_t)(a.HY * a.HX) * 16u;  // bytes of one image slice
            const uint32_t a_part = (uint32_t)a.GA * a_slice;        // hi (or lo) halo bytes
            const uint4* tb = s_tab + src.tab_off(u.p);
            int rb = 0;  // first run of group g
            for (int g = 0; g < a.NG && ok; ++g) {
                const uint4 hd = tb[g];  // {base16, tap bytes, taps per run, pairs}
                const int nr = (kk + (int)hd.z - 1) / (int)hd.z;
                const int lo = max(u.r0, rb), hi = min(u.r1, rb + nr);
                rb += nr;
                if (lo >= hi) continue;  // no run of this group in the unit
                if (a_fills > 0 &&
                    !mbar_wait_warp(smem_u32(&bar_aempty), (uint32_t)(a_fills - 1) & 1u,
                                    &s_abort)) {
                    ok = false;
                    break;
                }
                if (lane == 0) mbar_expect_tx(smem_u32(&bar_afull), a_part * (uint32_t)a.terms);
                ++a_fills;
                __syncwarp();
                const size_t img = (size_t)u.m * a.KS + (size_t)g * a.GA;
                for (int idx = lane; idx < a.GA * a.HY; idx += 32) {
                    const int sl = idx / a.HY, hy = idx - sl * a.HY;
                    const size_t goff =
                        (((img + sl) * a.Yp + (size_t)(u.y0 + hy)) * a.Xp + u.x0) * 8;
                    const uint32_t soff = (uint32_t)sl * a_slice + (uint32_t)(hy * a.HX) * 16u;
                    for (int tt = 0; tt < a.terms; ++tt)
                        bulk_g2s(sA + (uint32_t)tt * a_part + soff, a.img[tt] + goff,
                                 (uint32_t)a.HX * 16u, smem_u32(&bar_afull));
                }
                for (int run = lo; run < hi && ok; ++run) {
                    const int d0 = (run - (rb - nr)) * (int)hd.z;
                    const int nt = min((int)hd.z, kk - d0);
                    if (!mbar_wait_warp(smem_u32(&bar_empty[stage]), phase ^ 1u, &s_abort)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        const uint32_t bar = smem_u32(&bar_full[stage]);
                        const uint32_t dst = sW + (uint32_t)stage * stage_slot;
                        const uint32_t bytes = (uint32_t)nt * hd.y;
                        const size_t wsrc = ((size_t)hd.x * 16 + (size_t)d0 * hd.y) / 2;  // elements
                        mbar_expect_tx(bar, bytes * (uint32_t)a.terms);
                        for (int tt = 0; tt < a.terms; ++tt)
                            bulk_g2s(dst + (uint32_t)tt * a.stage_bytes, a.w[tt] + wsrc, bytes,
                                     bar);
                    }
                    fills[stage]++;
                    __syncwarp();
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            s_abort = 1;
            atomicExch(err, 1);
        }
        // drain: every copy this warp issued has landed before the CTA exits
        if (lane == 0) {
            volatile int never = 0;
            for (int s = 0; s < NS; ++s)
                if (fills[s] > 0 &&
                    !mbar_wait(smem_u32(&bar_full[s]), (uint32_t)(fills[s] - 1) & 1u, &never))
                    atomicExch(err, 2);
            if (a_fills > 0 &&
                !mbar_wait(smem_u32(&bar_afull), (uint32_t)(a_fills - 1) & 1u, &never))
                atomicExch(err, 2);
        }
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ----------------------------
        // The warp walks every unit, group and run as a converged warp (waits
        // and table reads are warp-wide, descriptors warp-uniform); its elected
        // lane issues the products of every tap of a stage, from the loop
        // specialised for this launch's tiles, channel blocks and precision.
        // The kernel block is the A operand (128 channel rows, K-major: the
        // two 8-element halves 2048 B apart, 8-row groups 128 B apart); the
        // halo is the B operand (256 position rows: the two slices one slice
        // apart, 8-position groups one halo row apart), offset by the tap.
        const bool leader = elect_one();
        const uint64_t adesc_c = ((uint64_t)(2048u >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) |
                                 ((uint64_t)1 << 46);
        int local = 0;  // this CTA's runs so far (ring position)
        int ag = 0;     // halo fills consumed
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        int done = 0;   // units taken (the accumulator buffers alternate over them)
        TcUnit u;
        for (int k = 0; ok && src.unit(k, u); ++k) {
            const TcArgs& a = src.args(u.p);
            if (src.skip(a)) continue;
            const int kb = done++;
            const int kk = a.k * a.k;
            const uint32_t a_slice = (uint32_t)(a.HY * a.HX) * 16u;
            const uint32_t a_part = (uint32_t)a.GA * a_slice;
            const uint64_t bdesc_c = ((uint64_t)(a_slice >> 4) << 16) | ((uint64_t)a.HX << 32) |
                                     ((uint64_t)1 << 46);
            // FP32 accumulator; BF16 (format 1) or E4M3 (format 0) A and B, K-major
            const uint32_t ab_fmt = a.fp8 ? 0u : ((1u << 7) | (1u << 10));
            const uint32_t idesc = (1u << 4) | ab_fmt | (((uint32_t)kTilePos >> 3) << 17) |
                                   (((uint32_t)kRows >> 4) << 24);
            const IssueCfg ic{(uint32_t)(a.MB * kBlockBytes), (uint32_t)(a_part >> 4),
                              (uint32_t)(a.stage_bytes >> 4), idesc};
            const int kind = issue_kind(a.MT, a.MB, a.terms, a.RA, a.fp8);
            const uint4* tb = s_tab + src.tab_off(u.p);
            const int buf = NBUF == 2 ? (kb & 1) : 0;
            if (kb >= NBUF) {  // the epilogue has drained this buffer
                if (!mbar_wait_warp(smem_u32(&bar_accfree[buf]), (uint32_t)(kb / NBUF - 1) & 1u,
                                    &s_abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
            }
            const uint32_t tbuf = tmem + (uint32_t)buf * buf_stride;
            int rb = 0;  // first run of group g
            for (int g = 0; g < a.NG && ok; ++g) {
                const uint4 hd = tb[g];
                const int tpr = __shfl_sync(0xffffffffu, (int)hd.z, 0);
                const int nr = (kk + tpr - 1) / tpr;
                const int lo = max(u.r0, rb), hi = min(u.r1, rb + nr);
                const int gb = rb;
                rb += nr;
                if (lo >= hi) continue;  // no run of this group in the unit
                if (ag > 0 && leader) tc_commit(smem_u32(&bar_aempty));
                __syncwarp();
                if (!mbar_wait_warp(smem_u32(&bar_afull), (uint32_t)ag & 1u, &s_abort)) {
                    ok = false;
                    break;
                }
                ++ag;
                tc_fence_after();
                for (int run = lo; run < hi; ++run, ++local) {
                    const int nt = min(tpr, kk - (run - gb) * tpr);
                    if (!mbar_wait_warp(smem_u32(&bar_full[stage]), phase, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // halo offsets of this stage's taps (16-B units), from the run table
                    const uint4 ro = tb[a.NG + (run - gb)];
                    const uint32_t ow[4] = {__shfl_sync(0xffffffffu, ro.x, 0),
                                            __shfl_sync(0xffffffffu, ro.y, 0),
                                            __shfl_sync(0xffffffffu, ro.z, 0),
                                            __shfl_sync(0xffffffffu, ro.w, 0)};
                    const uint32_t wst = sW + (uint32_t)stage * stage_slot;
                    if (leader) issue_stage(kind, ic, tbuf, adesc_c | (uint64_t)(wst >> 4),
                                            bdesc_c | (uint64_t)(sA >> 4), ow, nt);
                    __syncwarp();
                    if (leader) tc_commit(smem_u32(&bar_empty[stage]));
                    __syncwarp();
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) break;
            // the unit's accumulators are complete once every MMA issued so far is
            if (leader) tc_commit(smem_u32(&bar_accfull[buf]));
            __syncwarp();
        }
        if (!ok && leader) {
            s_abort = 1;
            atomicExch(err, 1);
        }
        // every MMA of this issuer has completed before TMEM is freed
        if (leader) tc_commit(smem_u32(&bar_drain));
        __syncwarp();
        volatile int never = 0;
        if (!mbar_wait_warp(smem_u32(&bar_drain), 0u, &never) && leader) atomicExch(err, 2);
    } else if (warp >= 2 && warp <= 5) {
        // ------------------------------ epilogue ------------------------------
        // Thread li (= 32 q + lane) owns TMEM lane li: channel mb * 128 + li of
        // every position column.
        const int q = warp & 3;
        const int li = q * 32 + lane;
        double part = 0.0;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        float rmax = 0.f;  // FP8 forward: largest |output| s_t of this thread
        int done = 0;
        TcUnit u;
        for (int k = 0; src.unit(k, u); ++k) {
            const TcArgs& a = src.args(u.p);
            if (src.skip(a)) continue;
            const int kb = done++;
            const size_t unit_floats = (size_t)a.MB * a.MT * kTilePos * kRows;
            const uint32_t buf_cols = (uint32_t)(a.RA * a.MB * a.MT * kTilePos);
            const size_t S = (size_t)a.Y * a.X;
            const float* __restrict__ ytil = a.ytil;
            // FP8: the accumulators hold sigma (sum of products); sigma = 256 / (largest
            // scaled input entry), so the output is the accumulator times that / 256
            const float inv_sigma = a.fp8 ? __uint_as_float(*a.in_word) * (1.0f / 256.0f) : 1.0f;
            const int buf = NBUF == 2 ? (kb & 1) : 0;
            const uint32_t tbuf = tmem + lanes + (uint32_t)buf * buf_stride;
            const bool w_ok =
                mbar_wait_warp(smem_u32(&bar_accfull[buf]), (uint32_t)(kb / NBUF) & 1u, &s_abort);
            tc_fence_after();
            if (lane == 0) s_eok[q] = w_ok ? 1 : 0;
            asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
            if (!(s_eok[0] && s_eok[1] && s_eok[2] && s_eok[3])) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicExch(err, 1);
                }
                break;  // the same decision in all four warps
            }
            // the summed accumulator sets of (block mb, tile ti), columns 16 cb .. 16 cb + 15
            auto acc16 = [&](int mb, int ti, int cb, float (&v)[16]) {
                tmem_ld16(tbuf + (uint32_t)((mb * a.MT + ti) * kTilePos + cb * 16), v);
                if (a.RA > 1) {
                    float w[16];
                    tmem_ld16(tbuf + (uint32_t)(((a.MB + mb) * a.MT + ti) * kTilePos + cb * 16), w);
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] += w[e];
                }
            };
            const size_t slot = a.split_slot ? (size_t)a.split_slot[u.ts] : (size_t)u.ts;
            auto part_at = [&](int piece, int mb, int ti, int cb) -> float* {
                return a.part + (slot * a.max_pieces + piece) * unit_floats +
                       ((((size_t)mb * a.MT + ti) * (kTilePos / 16) + cb) * kRows + li) * 16;
            };
            bool last = true;
            if (u.pieces > 1) {
                // publish this unit's partial sums, then the ticket decides who ends
                for (int mb = 0; mb < a.MB; ++mb)
                    for (int ti = 0; ti < a.MT; ++ti)
                        for (int cb = 0; cb < kTilePos / 16; ++cb) {
                            float v[16];
                            acc16(mb, ti, cb, v);
                            float4* dst = reinterpret_cast<float4*>(part_at(u.piece, mb, ti, cb));
#pragma unroll
                            for (int e4 = 0; e4 < 4; ++e4)
                                dst[e4] = make_float4(v[4 * e4], v[4 * e4 + 1], v[4 * e4 + 2],
                                                      v[4 * e4 + 3]);
                        }
                __threadfence();
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (warp == 2 && lane == 0) {
                    const int prev = atomicAdd(a.ticket + u.ts, 1);
                    s_last = prev == u.pieces - 1;
                    if (s_last) a.ticket[u.ts] = 0;  // ready for the next launch
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                last = s_last != 0;
                __threadfence();
            }
            if (last) {
                const float cm = a.scale ? a.Cmf[u.m] : 1.f;
                for (int mb = 0; mb < a.MB; ++mb) {
                    const int ch = mb * kRows + li;
                    const bool ch_ok = ch < a.rows;
                    for (int ti = 0; ti < a.MT; ++ti)
                        for (int cb = 0; cb < kTilePos / 16; ++cb) {
                            float v[16];
                            if (u.pieces <= 2) {
                                acc16(mb, ti, cb, v);
                                if (u.pieces == 2) {  // + the other piece's partial sums
                                    const float4* o4 = reinterpret_cast<const float4*>(
                                        part_at(1 - u.piece, mb, ti, cb));
#pragma unroll
                                    for (int e4 = 0; e4 < 4; ++e4) {
                                        const float4 w = __ldcg(o4 + e4);  // written by another SM
                                        v[4 * e4] += w.x;
                                        v[4 * e4 + 1] += w.y;
                                        v[4 * e4 + 2] += w.z;
                                        v[4 * e4 + 3] += w.w;
                                    }
                                }
                            } else {  // every piece's partial sums, in piece order
#pragma unroll
                                for (int e = 0; e < 16; ++e) v[e] = 0.f;
                                for (int pc = 0; pc < u.pieces; ++pc) {
                                    const float4* o4 =
                                        reinterpret_cast<const float4*>(part_at(pc, mb, ti, cb));
#pragma unroll
                                    for (int e4 = 0; e4 < 4; ++e4) {
                                        const float4 w = __ldcg(o4 + e4);
                                        v[4 * e4] += w.x;
                                        v[4 * e4 + 1] += w.y;
                                        v[4 * e4 + 2] += w.z;
                                        v[4 * e4 + 3] += w.w;
                                    }
                                }
                            }
                            if (a.fp8) {
#pragma unroll
                                for (int e = 0; e < 16; ++e) v[e] *= inv_sigma;
                            }
                            // column 16 cb + e is position (y0 + 2 cb + e / 8, x0 + 8 ti + e % 8);
                            // the chunk's measurements are loaded together first (the
                            // stores below would otherwise order every load behind them)
                            float yv[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const int y = u.y0 + 2 * cb + (e >> 3);
                                const int x = u.x0 + 8 * ti + (e & 7);
                                yv[e] = 0.f;
                                if (ytil && ch_ok && y < a.Y && x < a.X)
                                    yv[e] = __ldg(ytil + ((size_t)u.m * S + (size_t)y * a.X + x) *
                                                             a.Twp + ch);
                            }
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const int y = u.y0 + 2 * cb + (e >> 3);
                                const int x = u.x0 + 8 * ti + (e & 7);
                                const bool pos_ok = y < a.Y && x < a.X;  // warp-uniform
                                if (!pos_ok) continue;
                                const size_t pos = (size_t)y * a.X + x;
                                if (a.adj) {
                                    if (ch_ok) a.out_f[((size_t)u.m * S + pos) * a.Z + ch] = v[e];
                                    continue;
                                }
                                const size_t ub = ((size_t)u.m * S + pos) * a.Twp + ch;
                                float o = 0.f;
                                if (ch_ok) {
                                    if (ytil) {
                                        o = cm * v[e] - yv[e];
                                        if (a.partials)
                                            part += (double)cm * (double)v[e] * v[e] -
                                                    2.0 * (double)v[e] * yv[e];
                                    } else {
                                        o = cm * v[e];
                                    }
                                }
                                if (a.mode == 0) {
                                    if (ch_ok) {
                                        a.out_f[ub] = o;
                                        if (a.max_word) rmax = fmaxf(rmax, fabsf(o) * a.s_out[ch]);
                                    }
                                    continue;
                                }
                                // the BF16 terms of channels 8 g .. 8 g + 7 (lanes 8 g' ..
                                // 8 g' + 7 of the warp) gathered into lane 8 g' and written
                                // as one 16-byte row of the residual image
                                const __nv_bfloat16 h0 = __float2bfloat16_rn(o);
                                const float o1 = o - __bfloat162float(h0);
                                const __nv_bfloat16 h1 = __float2bfloat16_rn(o1);
                                const float o2 = o1 - __bfloat162float(h1);
                                uint32_t w0 = (uint32_t)__bfloat16_as_ushort(h0);
                                uint32_t w1 = (uint32_t)__bfloat16_as_ushort(h1);
                                w0 |= __shfl_down_sync(0xffffffffu, w0, 1) << 16;  // even lanes: pairs
                                w1 |= __shfl_down_sync(0xffffffffu, w1, 1) << 16;
                                uint4 q0, q1, q2 = make_uint4(0u, 0u, 0u, 0u);
                                q0.x = w0;
                                q0.y = __shfl_down_sync(0xffffffffu, w0, 2);
                                q0.z = __shfl_down_sync(0xffffffffu, w0, 4);
                                q0.w = __shfl_down_sync(0xffffffffu, w0, 6);
                                q1.x = w1;
                                q1.y = __shfl_down_sync(0xffffffffu, w1, 2);
                                q1.z = __shfl_down_sync(0xffffffffu, w1, 4);
                                q1.w = __shfl_down_sync(0xffffffffu, w1, 6);
                                if (a.terms > 2) {  // warp-uniform
                                    uint32_t w2 =
                                        (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(o2));
                                    w2 |= __shfl_down_sync(0xffffffffu, w2, 1) << 16;
                                    q2.x = w2;
                                    q2.y = __shfl_down_sync(0xffffffffu, w2, 2);
                                    q2.z = __shfl_down_sync(0xffffffffu, w2, 4);
                                    q2.w = __shfl_down_sync(0xffffffffu, w2, 6);
                                }
                                if ((lane & 7) == 0 && ch < a.Twp) {
                                    const size_t ro =
                                        ((((size_t)u.m * a.KSo + (ch >> 3)) * a.Yp + (y + a.r)) *
                                             a.Xp + (x + a.r)) * 8;
                                    *reinterpret_cast<uint4*>(a.out_t[0] + ro) = q0;
                                    if (a.terms > 1) *reinterpret_cast<uint4*>(a.out_t[1] + ro) = q1;
                                    if (a.terms > 2) *reinterpret_cast<uint4*>(a.out_t[2] + ro) = q2;
                                }
                            }
                        }
                }
            }
            // hand the buffer back zeroed for the unit after next
            for (uint32_t cb = 0; cb < buf_cols / 16u; ++cb) tmem_zero16(tbuf + cb * 16u);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(smem_u32(&bar_accfree[buf]));
            asm volatile("bar.sync 1, 128;" ::: "memory");  // s_eok and s_last are reused
        }
        if (src.partials()) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) s_red[q] = part;
        }
        if (src.max_word()) {
            // non-negative floats order as their bit patterns
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, off));
            if (lane == 0) atomicMax(src.max_word(), __float_as_uint(rmax));
        }
    }

    tc_fence_before();
    __syncthreads();
    if (src.partials() && threadIdx.x == 0)
        src.partials()[blockIdx.x] = s_red[0] + s_red[1] + s_red[2] + s_red[3];
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(src.tcols())
                     : "memory");
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_conv_kernel(const TcArgs a)
{
    // a closed gate: return before any barrier, TMEM or copy is set up
    if (gated_off(a.gate, a.want)) return;
    tc_body(TcOne{a});
}

// Several problems' tile-states in one persistent launch (no FP8, no data-fit
// partial sums).
__global__ void __launch_bounds__(kTcThreads, 1) tc_conv_many_kernel(const TcBatchArgs B)
{
    tc_body(TcMany{B});
}

// P into the padded BF16 state images: for each (m, slice, y, x) the 8
// depths j = 8 slice + e of b[m][y][x][j] = sum_p Sm[m][p][j] c[p][y][x][j].
struct TermPtrs {
    __nv_bfloat16* p[kMaxTerms];
};

__global__ void tc_states_kernel(const float* __restrict__ c, const float* __restrict__ Sm,
                                 TermPtrs out, int terms, int Q, int P, int Y, int X, int Z,
                                 int slices, int KS, int Yp, int Xp, int r, int vec,
                                 const int* gate, int want)
{
    if (gated_off(gate, want)) return;
    // one thread per (slice, y, x): the P x 8 values of c are read once and
    // every switching state m is written from them
    const unsigned n = (unsigned)slices * Y * X;
    const size_t SZ = (size_t)Y * X * Z;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x = (int)(i % (unsigned)X);
        const int y = (int)((i / (unsigned)X) % (unsigned)Y);
        const int s8 = (int)(i / ((unsigned)X * Y));
        const int j0 = 8 * s8;
        float cv[kMaxSpecies][8];  // static indices only: kept in registers
#pragma unroll
        for (int p = 0; p < kMaxSpecies; ++p) {
            if (p >= P) break;
            const float* src = c + p * SZ + ((size_t)y * X + x) * Z + j0;
            if (vec && j0 + 8 <= Z) {
                const float4 a = reinterpret_cast<const float4*>(src)[0];
                const float4 b = reinterpret_cast<const float4*>(src)[1];
                cv[p][0] = a.x; cv[p][1] = a.y; cv[p][2] = a.z; cv[p][3] = a.w;
                cv[p][4] = b.x; cv[p][5] = b.y; cv[p][6] = b.z; cv[p][7] = b.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) cv[p][e] = j0 + e < Z ? src[e] : 0.f;
            }
        }
        for (int m = 0; m < Q; ++m) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j0 + e;
                float acc = 0.f;
                if (j < Z) {
#pragma unroll
                    for (int p = 0; p < kMaxSpecies; ++p) {
                        if (p >= P) break;
                        acc = fmaf(Sm[(m * P + p) * Z + j], cv[p][e], acc);
                    }
                }
                v[e] = acc;
            }
            uint4 parts[kMaxTerms];
            split_terms(v, parts, terms);
            const size_t o = ((((size_t)m * KS + s8) * Yp + (y + r)) * Xp + (x + r)) * 8;
            for (int tt = 0; tt < terms; ++tt) *reinterpret_cast<uint4*>(out.p[tt] + o) = parts[tt];
        }
    }
}

// FP32 u [Q][S][Twp] into the padded BF16 residual images
__global__ void tc_pack_kernel(const float* __restrict__ u, TermPtrs out, int terms, int Q,
                               int Y, int X, int Twp, int KS, int Yp, int Xp, int r)
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
        uint4 parts[kMaxTerms];
        split_terms(v, parts, terms);
        const size_t o = ((((size_t)m * KS + s8) * Yp + (y + r)) * Xp + (x + r)) * 8;
        for (int tt = 0; tt < terms; ++tt) *reinterpret_cast<uint4*>(out.p[tt] + o) = parts[tt];
    }
}

// ---------------------------------------------------------------------------
// FP8 (E4M3) images.  Pass 0 of tc_states_f8_kernel finds the largest
// |b_j| s_j of the state images (atomic max of its float bits in *word; the
// caller zeroes it first); pass 1 writes b_j s_j sigma, sigma = 256 / *word,
// as E4M3, 16 depths per 16-byte slice row.  tc_pack_f8_kernel does the same
// for the residual u (FP32 [Q][S][Twp]) with the sample scales s_t;
// u_max_f8_kernel is its pass 0 when u did not come from the forward epilogue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    return (uint32_t)__nv_cvt_float_to_fp8(a, __NV_SATFINITE, __NV_E4M3) |
           ((uint32_t)__nv_cvt_float_to_fp8(b, __NV_SATFINITE, __NV_E4M3) << 8) |
           ((uint32_t)__nv_cvt_float_to_fp8(c, __NV_SATFINITE, __NV_E4M3) << 16) |
           ((uint32_t)__nv_cvt_float_to_fp8(d, __NV_SATFINITE, __NV_E4M3) << 24);
}

__device__ __forceinline__ uint4 pack_e4m3x16(const float (&v)[16], float scale)
{
    return make_uint4(pack_e4m3x4(v[0] * scale, v[1] * scale, v[2] * scale, v[3] * scale),
                      pack_e4m3x4(v[4] * scale, v[5] * scale, v[6] * scale, v[7] * scale),
                      pack_e4m3x4(v[8] * scale, v[9] * scale, v[10] * scale, v[11] * scale),
                      pack_e4m3x4(v[12] * scale, v[13] * scale, v[14] * scale, v[15] * scale));
}

__device__ __forceinline__ void warp_max_to(unsigned* word, float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) atomicMax(word, __float_as_uint(v));
}

__global__ void tc_states_f8_kernel(const float* __restrict__ c, const float* __restrict__ Sm,
                                    const float* __restrict__ s_dep, uint8_t* __restrict__ out,
                                    unsigned* word, int pass, int Q, int P, int Y, int X, int Z,
                                    int slices, int KS, int Yp, int Xp, int r, const int* gate,
                                    int want)
{
    if (gated_off(gate, want)) return;
    const unsigned n = (unsigned)slices * Y * X;
    const size_t SZ = (size_t)Y * X * Z;
    const float sigma = pass == 1 ? 256.0f / fmaxf(__uint_as_float(*word), 1e-30f) : 0.f;
    float lmax = 0.f;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ((n + 31u) & ~31u);
         i += gridDim.x * blockDim.x) {
        if (i < n) {
            const int x = (int)(i % (unsigned)X);
            const int y = (int)((i / (unsigned)X) % (unsigned)Y);
            const int s16 = (int)(i / ((unsigned)X * Y));
            const int j0 = 16 * s16;
            float cv[kMaxSpecies][16];
#pragma unroll
            for (int p = 0; p < kMaxSpecies; ++p) {
                if (p >= P) break;
                const float* src = c + p * SZ + ((size_t)y * X + x) * Z + j0;
#pragma unroll
                for (int e = 0; e < 16; ++e) cv[p][e] = j0 + e < Z ? src[e] : 0.f;
            }
            for (int m = 0; m < Q; ++m) {
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int j = j0 + e;
                    float acc = 0.f;
                    if (j < Z) {
#pragma unroll
                        for (int p = 0; p < kMaxSpecies; ++p) {
                            if (p >= P) break;
                            acc = fmaf(Sm[(m * P + p) * Z + j], cv[p][e], acc);
                        }
                        acc *= s_dep[j];
                    }
                    v[e] = acc;
                }
                if (pass == 0) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) lmax = fmaxf(lmax, fabsf(v[e]));
                } else {
                    const size_t o = ((((size_t)m * KS + s16) * Yp + (y + r)) * Xp + (x + r)) * 16;
                    *reinterpret_cast<uint4*>(out + o) = pack_e4m3x16(v, sigma);
                }
            }
        }
        if (pass == 0) warp_max_to(word, lmax);
        lmax = 0.f;
    }
}

__global__ void u_max_f8_kernel(const float* __restrict__ u, const float* __restrict__ s_tim,
                                unsigned* word, size_t n, int Twp, const int* gate, int want)
{
    if (gated_off(gate, want)) return;
    float lmax = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        lmax = fmaxf(lmax, fabsf(u[i]) * s_tim[i % (size_t)Twp]);
    warp_max_to(word, lmax);
}

__global__ void tc_pack_f8_kernel(const float* __restrict__ u, const float* __restrict__ s_tim,
                                  const unsigned* word, uint8_t* __restrict__ out, int Q, int Y,
                                  int X, int Twp, int KS, int Yp, int Xp, int r, const int* gate,
                                  int want)
{
    if (gated_off(gate, want)) return;
    const int slices = Twp / 16;
    const size_t n = (size_t)Q * slices * Y * X;
    const float sigma = 256.0f / fmaxf(__uint_as_float(*word), 1e-30f);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % X);
        const int y = (int)((i / X) % Y);
        const int s16 = (int)((i / ((size_t)X * Y)) % slices);
        const int m = (int)(i / ((size_t)X * Y * slices));
        const float4* src = reinterpret_cast<const float4*>(
            u + (((size_t)m * Y + y) * X + x) * Twp + 16 * s16);
        float v[16];
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            const float4 w = src[q4];
            v[4 * q4] = w.x * s_tim[16 * s16 + 4 * q4];
            v[4 * q4 + 1] = w.y * s_tim[16 * s16 + 4 * q4 + 1];
            v[4 * q4 + 2] = w.z * s_tim[16 * s16 + 4 * q4 + 2];
            v[4 * q4 + 3] = w.w * s_tim[16 * s16 + 4 * q4 + 3];
        }
        const size_t o = ((((size_t)m * KS + s16) * Yp + (y + r)) * Xp + (x + r)) * 16;
        *reinterpret_cast<uint4*>(out + o) = pack_e4m3x16(v, sigma);
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

// IEEE-style E4M3 (the OCP 8-bit format: 1 sign, 4 exponent bits with bias
// 7, 3 mantissa bits, subnormals below 2^-6, largest finite 448, no
// infinity): round to nearest even, saturating at +-448.
uint8_t f2e4m3(float f)
{
    const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
    const double a = std::fabs((double)f);
    if (!(a == a)) return 0x7F;                 // NaN
    if (a >= 448.0) return sign | 0x7E;         // saturate
    int e2 = 0;
    const double fr = std::frexp(a, &e2);       // a = fr 2^e2, fr in [0.5, 1)
    int e = e2 - 1;                             // a = (2 fr) 2^e
    if (a == 0.0 || e < -6) {
        // subnormal: a / 2^-9 rounded to an integer 0..8 (8 is the smallest normal)
        const double q = a * 512.0;
        double m = std::nearbyint(q);           // round half to even (default mode)
        return sign | (uint8_t)m;               // 8 encodes exponent 1, mantissa 0
    }
    double m = std::nearbyint((2.0 * fr - 1.0) * 8.0);  // 0..8
    if (m == 8.0) {
        m = 0.0;
        ++e;
    }
    if (e > 8 || (e == 8 && m > 6.0)) return sign | 0x7E;
    return sign | (uint8_t)(((e + 7) << 3) | (int)m);
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

uint32_t pow2_cols(int n)
{
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

}  // namespace

namespace {

void free_dir(TcDir& D)
{
    for (int tt = 0; tt < kMaxTerms; ++tt) {
        cudaFree(D.Wt[tt]);
        D.Wt[tt] = nullptr;
    }
    cudaFree(D.tab);
    D.tab = nullptr;
    cudaFree(D.part);
    D.part = nullptr;
    cudaFree(D.ticket);
    D.ticket = nullptr;
}

// Host image of one direction's configuration and tables (the kernel blocks
// are packed separately: their layout depends on the slice grouping only).
struct DirHost {
    TcDir cfg;
    std::vector<uint32_t> tab;              // group headers and run tables (uint4 entries)
    int npe = 0;                            // slice pairs holding a nonzero kernel entry
};

// Kernel value of direction `adj` at channel `row`, contraction index `kidx`, tap d.
float kernel_value(const swopt_handle* h, bool adj, int row, int kidx, int d)
{
    const int kk = h->k * h->k;
    const int j = adj ? row : kidx, w = adj ? kidx : row;
    const int tt = h->t0 + w;
    if (j >= h->Z || w >= h->Twp || tt >= h->T) return 0.f;
    return (float)h->K64[((size_t)j * kk + d) * h->T + tt];
}

// FP8 scale of contraction index kidx: the depth scale s_j for A, the sample
// scale s_t for A^T (1 for the BF16 precisions).
double fp8_scale(const swopt_handle* h, const std::vector<double>& s_dep,
                 const std::vector<double>& s_tim, bool adj, int kidx)
{
    (void)h;
    const std::vector<double>& sv = adj ? s_tim : s_dep;
    return kidx < (int)sv.size() ? sv[kidx] : 0.0;
}

// The kernel blocks [group][tap][pair][MB][2 halves][128 rows][16 bytes], per
// BF16 term (8 values a row), or for FP8 the E4M3 codes of K / s (16 values a
// row, two to a 16-bit slot), of a configuration's slice grouping.
void pack_dir(const swopt_handle* h, const TcOperator* t, bool adj, const TcDir& D, int npe,
              const std::vector<double>& s_dep, const std::vector<double>& s_tim,
              std::vector<uint16_t> (&w)[kMaxTerms])
{
    const int kk = h->k * h->k;
    const int gpairs = D.GA / 2;
    if (t->fp8) {
        for (int tt = 0; tt < kMaxTerms; ++tt) w[tt].clear();
        w[0].reserve((size_t)kk * npe * D.MB * kBlockBytes / 2);
        for (int g = 0; g < D.NG; ++g) {
            const int np = std::min(gpairs, npe - g * gpairs);
            for (int d = 0; d < kk; ++d)
                for (int p = 0; p < np; ++p) {
                    const int gp = g * gpairs + p;
                    for (int mb = 0; mb < D.MB; ++mb)
                        for (int half = 0; half < 2; ++half)
                            for (int row = 0; row < kRows; ++row)
                                for (int e = 0; e < 16; e += 2) {
                                    uint16_t pair = 0;
                                    for (int b = 0; b < 2; ++b) {
                                        const int kidx = 32 * gp + 16 * half + e + b;
                                        const double sc = fp8_scale(h, s_dep, s_tim, adj, kidx);
                                        const double v =
                                            sc > 0 ? kernel_value(h, adj, mb * kRows + row, kidx, d) / sc
                                                   : 0.0;
                                        pair |= (uint16_t)f2e4m3((float)v) << (8 * b);
                                    }
                                    w[0].push_back(pair);
                                }
                }
        }
        if (w[0].empty()) w[0].assign(8, 0);
        return;
    }
    for (int tt = 0; tt < kMaxTerms; ++tt) {
        w[tt].clear();
        w[tt].reserve((size_t)kk * npe * D.MB * kBlockBytes / 2);
    }
    for (int g = 0; g < D.NG; ++g) {
        const int np = std::min(gpairs, npe - g * gpairs);
        for (int d = 0; d < kk; ++d)
            for (int p = 0; p < np; ++p) {
                const int gp = g * gpairs + p;
                for (int mb = 0; mb < D.MB; ++mb)
                    for (int half = 0; half < 2; ++half)
                        for (int row = 0; row < kRows; ++row)
                            for (int e = 0; e < 8; ++e) {
                                float rv =
                                    kernel_value(h, adj, mb * kRows + row, 16 * gp + 8 * half + e, d);
                                for (int tt = 0; tt < kMaxTerms; ++tt) {
                                    const uint16_t hb = f2bf(rv);
                                    w[tt].push_back(hb);
                                    rv -= bf2f(hb);
                                }
                            }
            }
    }
    for (int tt = 0; tt < kMaxTerms; ++tt)
        if (w[tt].empty()) w[tt].assign(8, 0);
}

// Builds the kernel blocks of one direction for MT position tiles per CTA
// within a shared-memory budget.  Returns false if it does not fit.
bool plan_dir(const swopt_handle* h, const TcOperator* t, bool adj, int MT, int RA, int NBUF,
              int skip, int whole, size_t budget, DirHost* out)
{
    const int kk = h->k * h->k;
    const int terms = t->terms;
    TcDir D;
    D.MT = MT;
    D.RA = RA;
    D.whole = whole;
    D.NBUF = NBUF;
    D.rows = adj ? h->Z : h->Twp;
    D.MB = (D.rows + kRows - 1) / kRows;
    if (D.MB > 2) return false;
    // contracted slices (both even): 16-byte rows of 8 BF16 or 16 FP8 values
    const int ks_min = adj ? h->Twp / t->esl : t->Zp16 / t->esl;
    const int npairs = ks_min / 2;
    const int pair_elems = 2 * t->esl;
    D.HX = 8 * MT + 2 * h->r;
    D.npos = t->HY * D.HX;
    D.cols = (int)pow2_cols(NBUF * RA * D.MB * MT * kTilePos);
    if (D.cols > 512) return false;
    D.groupsX = (t->tilesX + MT - 1) / MT;

    // pairs with any nonzero kernel entry; trailing all-zero pairs are dropped
    int npe = 0;
    for (int gp = 0; gp < npairs; ++gp) {
        bool any = false;
        for (int d = 0; d < kk && !any; ++d)
            for (int row = 0; row < D.rows && !any; ++row)
                for (int e = 0; e < pair_elems; ++e)
                    if (kernel_value(h, adj, row, pair_elems * gp + e, d) != 0.f) {
                        any = true;
                        break;
                    }
        if (any) npe = gp + 1;
    }
    if (npe == 0) npe = 1;
    const size_t pair_b = (size_t)D.MB * kBlockBytes;
    // one slice pair per group (the issue loop has no loop over pairs); the
    // largest stage (whole taps, up to kMaxTapsPerStage, at least 3 stages)
    // that fits the budget with the halo, or with skip > 0 the next smaller
    const size_t mult = (size_t)terms;
    bool found = false;
    {
        const int GA = 2, NG = npe;
        const size_t tapb = pair_b;
        const size_t a_bytes = mult * (size_t)GA * D.npos * 16;
        for (int tps = kMaxTapsPerStage; tps >= 1 && !found; --tps) {
            const size_t stage = tapb * (size_t)std::min(tps, kk);
            const size_t tabr = ((size_t)NG + (size_t)((kk + tps - 1) / tps)) * 16;
            for (int ns = kMaxStages; ns >= 3; --ns) {
                const size_t total = a_bytes + (size_t)ns * stage * mult + tabr;
                if (total <= budget) {
                    if (skip > 0) {
                        --skip;
                        break;  // the next smaller stage
                    }
                    D.GA = GA;
                    D.NG = NG;
                    // slice stride of the image: at least every slice that the
                    // state / pack kernels and the forward epilogue write
                    D.KS = std::max(NG * GA, ks_min);
                    D.NS = ns;
                    D.stage_bytes = (uint32_t)stage;
                    D.smem = total;
                    found = true;
                    break;
                }
            }
        }
    }
    if (!found) return false;
    // At most 512 / cols CTAs may share an SM's 512 TMEM columns: request
    // enough shared memory that no more can be resident (233472 B per SM,
    // so more than 233472 / (512 / cols + 1) bytes per CTA).
    D.smem = std::max(D.smem, (size_t)233472 / (512 / D.cols + 1) + 1024);
    if (D.smem > 225 * 1024) return false;

    // group headers (kernel blocks at [group][tap][pair][MB][2][128][8]) and
    // run tables
    const int gpairs = D.GA / 2;
    out->tab.clear();
    std::vector<uint32_t> runtab;
    double macs = 0;
    size_t base_bytes = 0;
    // taps per run: what a stage holds of a full group's blocks (every group
    // uses the same runs, so that one run table serves them all)
    const uint32_t tpr = std::min<uint32_t>(
        kMaxTapsPerStage, std::max<uint32_t>(1, D.stage_bytes / (uint32_t)(gpairs * pair_b)));
    for (int g = 0; g < D.NG; ++g) {
        const int np = std::min(gpairs, npe - g * gpairs);
        const uint32_t tapb = (uint32_t)(np * pair_b);
        const uint32_t base16 = (uint32_t)(base_bytes / 16);
        base_bytes += (size_t)kk * tapb;
        out->tab.insert(out->tab.end(), {base16, tapb, tpr, (uint32_t)np});
        D.runs += (kk + (int)tpr - 1) / (int)tpr;
        macs += (double)kk * np * D.MB * kRows * kTilePos * pair_elems;
    }
    // runs of tpr taps: halo offsets (16-B units) of each tap of the run
    for (int d0 = 0; d0 < kk; d0 += (int)tpr) {
        uint32_t w[4] = {0, 0, 0, 0};
        for (int tt = 0; tt < (int)tpr && d0 + tt < kk; ++tt) {
            const int d = d0 + tt, dy = d / h->k, dx = d - dy * h->k;
            const int off = adj ? (2 * h->r - dy) * D.HX + (2 * h->r - dx) : dy * D.HX + dx;
            w[tt >> 1] |= (uint32_t)(off & 0xFFFF) << (16 * (tt & 1));
        }
        runtab.insert(runtab.end(), {w[0], w[1], w[2], w[3]});
    }
    if (base_bytes / 16 > 0xFFFFFFFFull) return false;
    out->tab.insert(out->tab.end(), runtab.begin(), runtab.end());
    out->npe = npe;
    D.tab_words = (int)out->tab.size();
    const double ctas = (double)D.groupsX * t->tilesY * h->Q;
    D.macs = macs * MT * (terms * (terms + 1) / 2) * ctas;
    out->cfg = D;
    return true;
}

// Packed kernel blocks on the device, one entry per slice grouping (GA).
struct WCache {
    int GA = 0;
    __nv_bfloat16* w[kMaxTerms] = {};
};

void free_wcache(std::vector<WCache>& c, const __nv_bfloat16* keep)
{
    for (auto& e : c)
        for (int tt = 0; tt < kMaxTerms; ++tt)
            if (e.w[tt] && e.w[0] != keep) cudaFree(e.w[tt]);
    c.clear();
}

// Device copies of a configuration: its tables, and its kernel blocks from
// the cache (packed and uploaded on the first use of its slice grouping).
// The kernel arrays stay owned by the cache until the caller keeps them.
swopt_status upload_dir(const swopt_handle* h, bool adj, const DirHost& H, int terms,
                        std::vector<WCache>& cache, TcDir* D)
{
    *D = H.cfg;
    for (int tt = 0; tt < kMaxTerms; ++tt) D->Wt[tt] = nullptr;
    D->tab = nullptr;
    D->part = nullptr;
    D->ticket = nullptr;
    WCache* e = nullptr;
    for (auto& c : cache)
        if (c.GA == D->GA) e = &c;
    if (!e) {
        std::vector<uint16_t> w[kMaxTerms];
        pack_dir(h, h->tc, adj, *D, H.npe, h->tc->s_dep_h, h->tc->s_tim_h, w);
        cache.push_back(WCache());
        e = &cache.back();
        e->GA = D->GA;
        for (int tt = 0; tt < terms; ++tt) {
            SW_TRY(tc_alloc(&e->w[tt], w[tt].size()));
            SW_CUDA(cudaMemcpy(e->w[tt], w[tt].data(), w[tt].size() * 2, cudaMemcpyHostToDevice));
        }
    }
    for (int tt = 0; tt < kMaxTerms; ++tt) D->Wt[tt] = e->w[tt];
    return tc_upload(&D->tab, H.tab);
}

// Frees a configuration's own device arrays (not its cached kernel blocks).
void free_dir_tables(TcDir& D)
{
    for (int tt = 0; tt < kMaxTerms; ++tt) D.Wt[tt] = nullptr;
    free_dir(D);
}

TcArgs dir_args(const swopt_handle* h, const TcOperator* t, const TcDir& D, bool adj)
{
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Cmf = h->Cmf;
    a.err = t->err;
    a.Y = h->Y; a.X = h->X; a.Yp = t->Yp; a.Xp = t->Xp; a.Z = h->Z; a.k = h->k; a.r = h->r;
    a.HY = t->HY; a.HX = D.HX; a.groupsX = D.groupsX; a.MT = D.MT; a.RA = D.RA;
    a.MB = D.MB; a.rows = D.rows;
    a.part = D.part;
    a.ticket = D.ticket;
    a.KS = D.KS; a.GA = D.GA; a.NG = D.NG; a.NS = D.NS;
    a.stage_bytes = D.stage_bytes;
    a.Twp = h->Twp;
    a.KSo = t->A.KS;
    a.terms = t->terms;
    a.adj = adj ? 1 : 0;
    for (int tt = 0; tt < kMaxTerms; ++tt) a.w[tt] = D.Wt[tt];
    a.tab = reinterpret_cast<const uint4*>(D.tab);
    a.tab_n = D.tab_words / 4;
    a.tcols = (uint32_t)D.cols;
    a.NBUF = D.NBUF;
    a.ntiles = D.groupsX * t->tilesY;
    a.runs = D.runs;
    a.quantum = D.quantum;
    a.wq = D.wq;
    a.max_pieces = D.max_pieces;
    for (int tt = 0; tt < kMaxTerms; ++tt) a.img[tt] = adj ? t->rpad[tt] : t->bpad[tt];
    a.gate = h->gate;
    a.want = h->gate_want;
    a.fp8 = t->fp8 ? 1 : 0;
    if (t->fp8) {
        a.in_word = adj ? t->words + 1 : t->words;
        a.s_out = t->s_tim;
    }
    return a;
}

swopt_status launch_conv(swopt_handle* h, const TcDir& D, const TcArgs& a, cudaStream_t st)
{
    // The dynamic shared-memory limit is an attribute of the function, shared
    // by every handle and by every launch already captured in a graph: it is
    // raised once to the device maximum and never lowered.
    const int dmax = max_dynamic_smem(h, (const void*)tc_conv_kernel);
    if (dmax <= 0 || D.smem > (size_t)dmax) {
        set_error("tensor-core kernel needs %zu bytes of shared memory (device limit %d)", D.smem,
                  dmax);
        return SWOPT_ERR_UNSUPPORTED;
    }
    SW_CUDA(cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dmax));
    if (D.grid <= 0) {
        set_error("internal: tensor-core configuration without a grid");
        return SWOPT_ERR_UNSUPPORTED;
    }
    tc_conv_kernel<<<D.grid, kTcThreads, D.smem, st>>>(a);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

// Persistent grid of a configuration: as many CTAs as can be resident at once
// (by shared memory, registers and TMEM columns), or one per piece of work if
// fewer; then the partial-sum slots and tickets of shared tile-states.
swopt_status set_grid(swopt_handle* h, TcDir* D)
{
    const int dmax = max_dynamic_smem(h, (const void*)tc_conv_kernel);
    if (dmax <= 0 || D->smem > (size_t)dmax) {
        set_error("tensor-core kernel needs %zu bytes of shared memory (device limit %d)", D->smem,
                  dmax);
        return SWOPT_ERR_UNSUPPORTED;
    }
    SW_CUDA(cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dmax));
    int nsm = 0, occ = 0;
    SW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
    SW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tc_conv_kernel, kTcThreads,
                                                          D->smem));
    occ = std::max(1, std::min(occ, 512 / D->cols));
    const long long units_ts = (long long)D->groupsX * h->tc->tilesY * h->Q;
    const long long R = std::max(D->runs, 1);
    D->quantum = D->whole ? (int)R : 1;
    D->wq = units_ts * R / D->quantum;
    const long long G = std::min<long long>(D->wq, (long long)std::max(nsm, 1) * occ);
    D->grid = (int)G;
    // CTAs sharing a tile-state: the owners of its first and last runs and
    // every CTA between (each share holds at least one piece of work)
    auto owner = [&](long long x) { return ((x / D->quantum + 1) * G - 1) / D->wq; };
    long long most = 1;
    for (long long ts = 0; ts < units_ts; ++ts)
        most = std::max(most, owner(ts * R + R - 1) - owner(ts * R) + 1);
    D->max_pieces = (int)most;
    if (most > 1) {
        const size_t unit_floats = (size_t)D->MB * D->MT * kTilePos * kRows;
        SW_TRY(tc_alloc(&D->part, (size_t)units_ts * most * unit_floats));
        SW_TRY(tc_alloc(&D->ticket, (size_t)units_ts));
        SW_CUDA(cudaMemset(D->ticket, 0, (size_t)units_ts * sizeof(int)));
    }
    return SWOPT_OK;
}

// Candidate configurations: position tiles per CTA and the shared-memory
// budget (two CTAs per SM, or one).
struct Cand {
    int MT;
    size_t budget;
};
const Cand kCands[] = {{1, 110 * 1024}, {1, 220 * 1024}, {2, 220 * 1024}};

}  // namespace

void tc_release(swopt_handle* h)
{
    TcOperator* t = h->tc;
    if (!t) return;
    free_dir(t->F);
    free_dir(t->A);
    for (int tt = 0; tt < kMaxTerms; ++tt) {
        cudaFree(t->bpad[tt]);
        cudaFree(t->rpad[tt]);
    }
    cudaFree(t->err);
    cudaFree(t->s_dep);
    cudaFree(t->s_tim);
    cudaFree(t->words);
    delete t;
    h->tc = nullptr;
}

// Chooses, for one direction, the fastest candidate configuration (timed
// with CUDA events on zeroed operands) among those the pins allow: `force_mt`
// tiles per CTA, `force_ctas` CTAs per SM, `force_ra` accumulators per tile,
// `force_split` (1: whole tile-states, 2: stream-K) and `force_nbuf`
// accumulator buffers, each 0 for free.  The padded images must already be
// sized for the largest slice count.
static swopt_status tune_dir(swopt_handle* h, bool adj, int force_mt, int force_ctas,
                             int force_ra, int force_split, int force_nbuf, TcDir* best)
{
    TcOperator* t = h->tc;
    std::vector<DirHost> plans;
    std::vector<WCache> cache;
    // The split precisions keep their correction products in an accumulator
    // of their own where TMEM holds it: they are about 2^-8 of the main sum,
    // so the FP32 rounding of each accumulation step into it is 2^-8 finer.
    const int ra_want = force_ra > 0 ? force_ra : (t->terms > 1 ? 2 : 1);
    for (int ra = ra_want; ra >= 1 && plans.empty(); --ra) {
        if (force_ra > 0 && ra != force_ra) break;
        for (const Cand& c : kCands) {
            if (force_mt > 0 && c.MT != force_mt) continue;
            if (force_ctas > 0 && (force_ctas == 2) != (c.budget < 200 * 1024)) continue;
            // the fewest slice groups that fit, and the next split (larger
            // stages); CTAs taking whole tile-states, or equal shares of all runs
            for (int skip = 0; skip < 2; ++skip)
                for (int whole = 1; whole >= 0; --whole) {
                    if (force_split > 0 && whole != (force_split == 1 ? 1 : 0)) continue;
                    // double-buffered accumulators (the epilogue overlaps the
                    // next unit's MMAs) where TMEM holds them, and single ones
                    for (int nbuf = 2; nbuf >= 1; --nbuf) {
                        if (force_nbuf > 0 && nbuf != force_nbuf) continue;
                        DirHost H;
                        if (plan_dir(h, t, adj, c.MT, ra, nbuf, skip, whole, c.budget, &H))
                            plans.push_back(std::move(H));
                    }
                }
        }
    }
    if (plans.empty()) {
        set_error("no tensor-core configuration fits this geometry (k=%d, window %d, depths %d)",
                  h->k, h->Twp, h->Z);
        return SWOPT_ERR_UNSUPPORTED;
    }
    int best_i = 0;
    if (plans.size() > 1) {
        cudaEvent_t e0, e1;
        SW_CUDA(cudaEventCreate(&e0));
        SW_CUDA(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        for (size_t i = 0; i < plans.size(); ++i) {
            TcDir D;
            if (swopt_status su = upload_dir(h, adj, plans[i], t->terms, cache, &D);
                su != SWOPT_OK) {
                free_dir_tables(D);
                free_wcache(cache, nullptr);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return su;
            }
            if (swopt_status sg = set_grid(h, &D); sg != SWOPT_OK) {
                free_dir_tables(D);
                free_wcache(cache, nullptr);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return sg;
            }
            TcArgs a = dir_args(h, t, D, adj);
            a.gate = nullptr;  // tuning launches always run
            if (adj) {
                a.out_f = h->g;
                a.mode = 0;
            } else if (t->fp8) {
                // as in the solve: FP32 output with the residual's scale taken
                a.out_f = h->u;
                a.mode = 0;
                a.max_word = t->words + 1;
            } else {
                // as in the solve: the scaled residual from measurements (h->u
                // stands in for them) into the residual images
                a.mode = 1;
                a.scale = 1;
                a.ytil = h->u;
                for (int tt = 0; tt < kMaxTerms; ++tt) a.out_t[tt] = t->rpad[tt];
            }
            swopt_status s = launch_conv(h, D, a, 0);  // warm-up
            float ms = 0.f;
            if (s == SWOPT_OK) {
                cudaEventRecord(e0, 0);
                for (int rep = 0; rep < 3 && s == SWOPT_OK; ++rep) s = launch_conv(h, D, a, 0);
                cudaEventRecord(e1, 0);
                if (cudaEventSynchronize(e1) != cudaSuccess) s = SWOPT_ERR_CUDA;
                cudaEventElapsedTime(&ms, e0, e1);
            }
            free_dir_tables(D);
            if (s != SWOPT_OK) {
                free_wcache(cache, nullptr);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return s;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_i = (int)i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (tc_error_word(h) != 0) {
            free_wcache(cache, nullptr);
            set_error("a tensor-core kernel gave up a bounded wait while tuning");
            return SWOPT_ERR_TIMEOUT;
        }
    }
    swopt_status s = upload_dir(h, adj, plans[best_i], t->terms, cache, best);
    free_wcache(cache, s == SWOPT_OK ? best->Wt[0] : nullptr);  // the chosen blocks stay
    if (s != SWOPT_OK) {
        free_dir_tables(*best);
        return s;
    }
    if (swopt_status sg = set_grid(h, best); sg != SWOPT_OK) {
        free_dir(*best);
        return sg;
    }
    return SWOPT_OK;
}

swopt_status tc_prepare(swopt_handle* h)
{
    const int terms =
        h->precision == SWOPT_PREC_BF16X6 ? 3 : (h->precision == SWOPT_PREC_BF16X3 ? 2 : 1);
    const bool fp8 = h->precision == SWOPT_PREC_FP8;
    if (h->tc && h->tc->terms == terms && h->tc->fp8 == fp8) return SWOPT_OK;
    tc_release(h);
    TcOperator* t = new TcOperator();
    t->terms = terms;
    t->fp8 = fp8;
    t->esl = fp8 ? 16 : 8;
    t->tilesX = (h->X + 7) / 8;
    t->tilesY = (h->Y + kTileY - 1) / kTileY;
    t->Xp = ((t->tilesX + 1) / 2) * 16 + 2 * h->r;  // room for up to 2 tiles per CTA
    t->Yp = t->tilesY * kTileY + 2 * h->r;
    t->HY = kTileY + 2 * h->r;
    t->Zp16 = ((h->Z + 2 * t->esl - 1) / (2 * t->esl)) * (2 * t->esl);
    h->tc = t;
    if (h->Twp > 2 * kRows || t->Zp16 > 2 * kRows) {
        set_error("tensor-core path supports a time window and a depth count up to 256 "
                  "(window %d, depths %d)", h->Twp, h->Z);
        tc_release(h);
        return SWOPT_ERR_UNSUPPORTED;
    }
    // padded images sized for the largest slice count any candidate may use
    // (NG groups of 2 ceil(pairs / NG) slices never exceed twice the pairs' slices)
    const int ksf_max = 2 * (t->Zp16 / t->esl), ksa_max = 2 * (h->Twp / t->esl);
    const size_t plane = (size_t)t->Yp * t->Xp * 8;
    const size_t nb = (size_t)h->Q * ksf_max * plane, nr = (size_t)h->Q * ksa_max * plane;
    swopt_status s = SWOPT_OK;
    auto step = [&](swopt_status v) { if (s == SWOPT_OK) s = v; };
    for (int tt = 0; tt < terms; ++tt) {
        step(tc_alloc(&t->bpad[tt], nb));
        step(tc_alloc(&t->rpad[tt], nr));
    }
    step(tc_alloc(&t->err, 1));
    auto zero = [&](void* p, size_t bytes) {
        if (s == SWOPT_OK && p && cudaMemset(p, 0, bytes) != cudaSuccess) {
            set_error("cudaMemset failed");
            s = SWOPT_ERR_CUDA;
        }
    };
    // borders and padded slices stay zero; kernels only write the interior
    for (int tt = 0; tt < terms; ++tt) {
        zero(t->bpad[tt], nb * 2);
        zero(t->rpad[tt], nr * 2);
    }
    zero(t->err, sizeof(int));
    if (fp8 && s == SWOPT_OK) {
        // FP8 equilibration: per depth (A) and per window sample (A^T), the
        // largest kernel entry maps to 256; a channel whose kernel is zero
        // (padding) gets scale 0, so that it takes no part in the image's
        // largest scaled entry and its image values are 0
        const int kk = h->k * h->k;
        t->s_dep_h.assign(t->Zp16, 0.0);
        t->s_tim_h.assign(h->Twp, 0.0);
        std::vector<double> mt(h->Twp, 0.0);
        for (int j = 0; j < h->Z; ++j) {
            double mj = 0.0;
            for (int d = 0; d < kk; ++d)
                for (int w = 0; w < h->Twp && h->t0 + w < h->T; ++w) {
                    const double v = std::fabs(h->K64[((size_t)j * kk + d) * h->T + h->t0 + w]);
                    mj = std::max(mj, v);
                    mt[w] = std::max(mt[w], v);
                }
            if (mj > 0) t->s_dep_h[j] = mj / 256.0;
        }
        for (int w = 0; w < h->Twp; ++w)
            if (mt[w] > 0) t->s_tim_h[w] = mt[w] / 256.0;
        std::vector<float> sd(t->s_dep_h.begin(), t->s_dep_h.end());
        std::vector<float> st(t->s_tim_h.begin(), t->s_tim_h.end());
        step(tc_upload(&t->s_dep, sd));
        step(tc_upload(&t->s_tim, st));
        step(tc_alloc(&t->words, 4));
        zero(t->words, 4 * sizeof(unsigned));
    }
    // the adjoint's slice count fixes the layout the forward epilogue writes
    if (s == SWOPT_OK)
        s = tune_dir(h, true, h->tc_force_mt[1], h->tc_force_ctas[1], h->tc_force_ra[1],
                     h->tc_force_split[1], h->tc_force_nbuf[1], &t->A);
    if (s == SWOPT_OK)
        s = tune_dir(h, false, h->tc_force_mt[0], h->tc_force_ctas[0], h->tc_force_ra[0],
                     h->tc_force_split[0], h->tc_force_nbuf[0], &t->F);
    if (s == SWOPT_OK && (t->F.KS > ksf_max || t->A.KS > ksa_max)) {
        set_error("internal: padded slice count exceeds the allocation");
        s = SWOPT_ERR_DEVICE_CHECK;
    }
    if (s == SWOPT_OK) {
        // the tuning launches left data in the workspaces; clear the images
        for (int tt = 0; tt < terms; ++tt) {
            zero(t->bpad[tt], nb * 2);
            zero(t->rpad[tt], nr * 2);
        }
        if (s == SWOPT_OK && cudaDeviceSynchronize() != cudaSuccess) {
            set_error("synchronisation after tensor-core set-up failed");
            s = SWOPT_ERR_CUDA;
        }
    }
    if (s != SWOPT_OK) tc_release(h);
    return s;
}

int tc_forward_blocks(const swopt_handle* h)
{
    // upper bound on the persistent grid: at most the resident CTAs (two per
    // SM at most, on up to 1024 SMs)
    (void)h;
    return 2048;
}

swopt_status tc_states(swopt_handle* h, const float* c, cudaStream_t st)
{
    TcOperator* t = h->tc;
    if (t->fp8) {
        const int slices = (h->Z + 15) / 16;
        const size_t n = (size_t)slices * h->Y * h->X;
        if (h->P > kMaxSpecies || n > 0x7FFFFFFFull) {
            set_error("internal: state images beyond the kernel's limits");
            return SWOPT_ERR_UNSUPPORTED;
        }
        int sms = 0;
        SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
        const int grid = (int)std::min<size_t>((size_t)grid_for(n, 256), (size_t)sms * 16);
        uint8_t* out = reinterpret_cast<uint8_t*>(t->bpad[0]);
        SW_CUDA(cudaMemsetAsync(t->words, 0, sizeof(unsigned), st));
        for (int pass = 0; pass < 2; ++pass) {
            tc_states_f8_kernel<<<grid, 256, 0, st>>>(c, h->Sm, t->s_dep, out, t->words, pass, h->Q,
                                                      h->P, h->Y, h->X, h->Z, slices, t->F.KS,
                                                      t->Yp, t->Xp, h->r, h->gate, h->gate_want);
            SW_LAUNCHED(h);
        }
        return SWOPT_OK;
    }
    const int slices = (h->Z + 7) / 8;
    const size_t n = (size_t)slices * h->Y * h->X;
    if (h->P > kMaxSpecies || n > 0x7FFFFFFFull) {
        set_error("internal: state images beyond the kernel's limits");
        return SWOPT_ERR_UNSUPPORTED;
    }
    int sms = 0;
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = (int)std::min<size_t>((size_t)grid_for(n, 256), (size_t)sms * 16);
    TermPtrs out{{t->bpad[0], t->bpad[1], t->bpad[2]}};
    // 16-byte loads when every run of 8 depths starts on a 16-byte boundary
    const int vec = (h->Z % 4) == 0 && ((uintptr_t)c & 15u) == 0;
    tc_states_kernel<<<grid, 256, 0, st>>>(c, h->Sm, out, t->terms, h->Q, h->P, h->Y, h->X, h->Z,
                                           slices, t->F.KS, t->Yp, t->Xp, h->r, vec, h->gate,
                                           h->gate_want);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

// FP8: u (FP32 [Q][S][Twp]) into the E4M3 residual images with the scale in
// words[1] (taken by the forward epilogue, or first here when take_max).
static swopt_status pack_f8(swopt_handle* h, bool take_max, cudaStream_t st)
{
    TcOperator* t = h->tc;
    int sms = 0;
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    if (take_max) {
        SW_CUDA(cudaMemsetAsync(t->words + 1, 0, sizeof(unsigned), st));
        const size_t nu = nu_of(h);
        u_max_f8_kernel<<<(int)std::min<size_t>((size_t)grid_for(nu, 256), (size_t)sms * 8), 256, 0,
                          st>>>(h->u, t->s_tim, t->words + 1, nu, h->Twp, h->gate, h->gate_want);
        SW_LAUNCHED(h);
    }
    const size_t n = (size_t)h->Q * (h->Twp / 16) * h->Y * h->X;
    const int grid = (int)std::min<size_t>((size_t)grid_for(n, 256), (size_t)sms * 16);
    tc_pack_f8_kernel<<<grid, 256, 0, st>>>(h->u, t->s_tim, t->words + 1,
                                            reinterpret_cast<uint8_t*>(t->rpad[0]), h->Q, h->Y,
                                            h->X, h->Twp, t->A.KS, t->Yp, t->Xp, h->r, h->gate,
                                            h->gate_want);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status tc_pack_u(swopt_handle* h, cudaStream_t st)
{
    TcOperator* t = h->tc;
    if (t->fp8) return pack_f8(h, true, st);
    const size_t n = (size_t)h->Q * (h->Twp / 8) * h->Y * h->X;
    int sms = 0;
    SW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    const int grid = (int)std::min<size_t>((size_t)grid_for(n, 256), (size_t)sms * 16);
    TermPtrs out{{t->rpad[0], t->rpad[1], t->rpad[2]}};
    tc_pack_kernel<<<grid, 256, 0, st>>>(h->u, out, t->terms, h->Q, h->Y, h->X, h->Twp, t->A.KS,
                                         t->Yp, t->Xp, h->r);
    SW_LAUNCHED(h);
    return SWOPT_OK;
}

swopt_status tc_forward(swopt_handle* h, bool to_r, const float* ytil, double* partials,
                        int scale, cudaStream_t st)
{
    TcOperator* t = h->tc;
    TcArgs a = dir_args(h, t, t->F, false);
    a.scale = scale;
    a.ytil = ytil;
    a.partials = partials;
    // FP8: the residual goes through FP32 u, whose largest scaled entry the
    // epilogue takes, into the E4M3 images by a pack pass
    const bool direct = to_r && !t->fp8;
    a.mode = direct ? 1 : 0;
    a.out_f = direct ? nullptr : h->u;
    for (int tt = 0; tt < kMaxTerms; ++tt) a.out_t[tt] = direct ? t->rpad[tt] : nullptr;
    if (t->fp8 && to_r) {
        a.max_word = t->words + 1;
        SW_CUDA(cudaMemsetAsync(t->words + 1, 0, sizeof(unsigned), st));
    }
    ProfileRec rec;
    prof_begin(h, 0, st, &rec);
    SW_TRY(launch_conv(h, t->F, a, st));
    prof_end(h, &rec, st);
    if (t->fp8 && to_r) return pack_f8(h, false, st);
    return SWOPT_OK;
}

swopt_status tc_adjoint(swopt_handle* h, cudaStream_t st)
{
    TcOperator* t = h->tc;
    TcArgs a = dir_args(h, t, t->A, true);
    a.out_f = h->g;
    ProfileRec rec;
    prof_begin(h, 1, st, &rec);
    SW_TRY(launch_conv(h, t->A, a, st));
    prof_end(h, &rec, st);
    return SWOPT_OK;
}

// A prepared launch of the contraction over several handles: every
// problem's tile-states, whole, in persistent kernels over a work list.  The
// problems are packed greedily (largest halo first) into groups whose largest
// halo, a ring of at least two of their largest stages and their run tables
// fit one CTA's shared memory; each group is one launch (usually one or two).
struct TcMultiGroup {
    TcBatchArgs B{};
    TcArgs* probs = nullptr;
    TcBatchMeta* meta = nullptr;
    uint4* tab = nullptr;
    std::vector<void*> owned;     // partial sums, tickets and slot tables of split tile-states
    size_t smem = 0;
    int grid = 0;
};

struct TcMulti {
    std::vector<TcMultiGroup> groups;
    int dmax = 0;                 // the kernel's dynamic shared-memory limit
    int64_t* launches = nullptr;  // the first handle's launch counter
};

void tc_multi_destroy(TcMulti* m)
{
    if (!m) return;
    for (TcMultiGroup& g : m->groups) {
        if (g.probs) cudaFree(g.probs);
        if (g.meta) cudaFree(g.meta);
        if (g.tab) cudaFree(g.tab);
        for (void* q : g.owned) cudaFree(q);
    }
    delete m;
}

swopt_status tc_multi_create(swopt_handle* const* hs, int n, bool adj, bool use_ytil,
                             TcMulti** out)
{
    *out = nullptr;
    if (n < 1) {
        set_error("no problems for a shared launch");
        return SWOPT_ERR_INVALID_ARG;
    }
    std::vector<TcArgs> args(n);
    std::vector<std::vector<uint4>> tabs(n);
    std::vector<uint32_t> halo(n), slot(n), cols(n);
    for (int i = 0; i < n; ++i) {
        swopt_handle* h = hs[i];
        TcOperator* t = h->tc;
        if (!t || t->fp8) {
            set_error("a shared launch needs BF16 tensor-core operators on every problem");
            return SWOPT_ERR_UNSUPPORTED;
        }
        const TcDir& D = adj ? t->A : t->F;
        TcArgs a = dir_args(h, t, D, adj);
        if (adj) {
            a.out_f = h->g;
        } else {  // as tc_forward's residual mode: the padded BF16 residual images
            a.scale = 1;
            a.ytil = use_ytil ? h->ytil : nullptr;
            a.mode = 1;
            for (int tt = 0; tt < kMaxTerms; ++tt) a.out_t[tt] = t->rpad[tt];
        }
        // the launch's split decides the partial-sum slots (set per group)
        a.quantum = 1;
        a.wq = (long long)a.ntiles * h->Q;  // tile-states
        a.max_pieces = 1;
        a.part = nullptr;
        a.ticket = nullptr;
        a.split_slot = nullptr;
        args[i] = a;
        tabs[i].resize((size_t)a.tab_n);
        SW_CUDA(cudaMemcpy(tabs[i].data(), a.tab, tabs[i].size() * sizeof(uint4),
                           cudaMemcpyDeviceToHost));
        halo[i] = (uint32_t)(a.GA * a.HY * a.HX) * 16u * (uint32_t)a.terms;
        slot[i] = a.stage_bytes * (uint32_t)a.terms;
        cols[i] = (uint32_t)(a.RA * a.MB * a.MT * kTilePos);
    }
    const int dmax = max_dynamic_smem(hs[0], (const void*)tc_conv_many_kernel);
    int nsm = 0;
    SW_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, hs[0]->device));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return halo[x] > halo[y]; });
    auto need = [&](uint32_t hmax, uint32_t smax, size_t tabn) {
        return (size_t)hmax + 2 * (size_t)smax + tabn * sizeof(uint4);
    };
    TcMulti* m = new TcMulti();
    m->dmax = dmax;
    m->launches = &hs[0]->launches;
    size_t at = 0;
    while (at < order.size()) {
        // the group: problems order[at .. end)
        uint32_t hmax = 0, smax = 0, cmax = 0;
        size_t tabn = 0, end = at;
        while (end < order.size()) {
            const int i = order[end];
            const uint32_t h2 = std::max(hmax, halo[i]), s2 = std::max(smax, slot[i]);
            if (dmax <= 0 || need(h2, s2, tabn + tabs[i].size()) > (size_t)dmax) break;
            hmax = h2;
            smax = s2;
            cmax = std::max(cmax, cols[i]);
            tabn += tabs[i].size();
            ++end;
        }
        if (end == at) {
            tc_multi_destroy(m);
            set_error("a problem's halo, stages and tables exceed shared memory");
            return SWOPT_ERR_UNSUPPORTED;
        }
        TcMultiGroup g;
        TcBatchArgs& B = g.B;
        std::vector<TcArgs> ga;
        std::vector<TcBatchMeta> gm;
        std::vector<uint4> gt;
        long long W = 0;
        for (size_t q = at; q < end; ++q) {
            const int i = order[q];
            TcBatchMeta mt{};
            mt.piece0 = W;
            mt.tab_off = (int)gt.size();
            W += args[i].wq * args[i].runs;
            gt.insert(gt.end(), tabs[i].begin(), tabs[i].end());
            ga.push_back(args[i]);
            gm.push_back(mt);
        }
        const long long G = std::min<long long>(W, nsm);
        // tile-states cut between CTAs: their partial-sum slots, as the kernel
        // assigns the runs (CTA of run x: x G / W)
        swopt_status s = SWOPT_OK;
        for (size_t q = 0; q < ga.size() && s == SWOPT_OK; ++q) {
            TcArgs& a = ga[q];
            const long long R = a.runs, base = gm[q].piece0;
            std::vector<int> slot((size_t)a.wq, -1);
            int nsplit = 0, maxp = 1;
            for (long long ts = 0; ts < a.wq; ++ts) {
                const long long x0 = base + ts * R;
                const int pieces = (int)((x0 + R - 1) * G / W - x0 * G / W) + 1;
                if (pieces > 1) {
                    slot[(size_t)ts] = nsplit++;
                    maxp = std::max(maxp, pieces);
                }
            }
            if (!nsplit) continue;
            const size_t unit_floats = (size_t)a.MB * a.MT * kTilePos * kRows;
            float* part = nullptr;
            int* ticket = nullptr;
            int* sl = nullptr;
            s = tc_alloc(&part, (size_t)nsplit * maxp * unit_floats);
            if (s == SWOPT_OK) g.owned.push_back(part);
            if (s == SWOPT_OK) s = tc_alloc(&ticket, (size_t)a.wq);
            if (s == SWOPT_OK) {
                g.owned.push_back(ticket);
                if (cudaMemset(ticket, 0, sizeof(int) * (size_t)a.wq) != cudaSuccess) {
                    set_error("cudaMemset failed");
                    s = SWOPT_ERR_CUDA;
                }
            }
            if (s == SWOPT_OK) s = tc_upload(&sl, slot);
            if (s == SWOPT_OK) g.owned.push_back(sl);
            a.part = part;
            a.ticket = ticket;
            a.split_slot = sl;
            a.max_pieces = maxp;
        }
        if (s != SWOPT_OK) {
            for (void* q : g.owned) cudaFree(q);
            tc_multi_destroy(m);
            return s;
        }
        B.n = (int)ga.size();
        B.W = W;
        B.NBUF = 2 * cmax <= 512 ? 2 : 1;
        B.buf_stride = cmax;
        B.tcols = pow2_cols((int)(B.NBUF * cmax));
        B.halo_region = hmax;
        B.stage_slot = smax;
        B.tab_n = (int)gt.size();
        B.err = hs[0]->tc->err;
        const size_t fixed = (size_t)hmax + gt.size() * sizeof(uint4);
        B.NS = 2;
        for (int k = kMaxStages; k > 2; --k)
            if (fixed + (size_t)k * smax <= (size_t)dmax) {
                B.NS = k;
                break;
            }
        // at most 512 / tcols CTAs may share an SM's TMEM: ask for enough shared memory
        g.smem = std::max(fixed + (size_t)B.NS * smax,
                          std::min((size_t)dmax, (size_t)233472 / (512 / B.tcols + 1) + 1024));
        g.grid = (int)G;
        s = tc_upload(&g.probs, ga);
        if (s == SWOPT_OK) s = tc_upload(&g.meta, gm);
        if (s == SWOPT_OK) s = tc_upload(&g.tab, gt);
        B.probs = g.probs;
        B.meta = g.meta;
        B.tab = g.tab;
        m->groups.push_back(g);
        if (s != SWOPT_OK) {
            tc_multi_destroy(m);
            return s;
        }
        at = end;
    }
    *out = m;
    return SWOPT_OK;
}

int tc_multi_groups(const TcMulti* m) { return m ? (int)m->groups.size() : 0; }

swopt_status tc_multi_launch(TcMulti* m, cudaStream_t st)
{
    SW_CUDA(cudaFuncSetAttribute(tc_conv_many_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 m->dmax));
    for (const TcMultiGroup& g : m->groups) {
        tc_conv_many_kernel<<<g.grid, kTcThreads, g.smem, st>>>(g.B);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("shared contraction launch failed: %s", cudaGetErrorString(e));
            return SWOPT_ERR_CUDA;
        }
        ++*m->launches;
    }
    return SWOPT_OK;
}

int tc_error_word(swopt_handle* h)
{
    if (!h->tc || !h->tc->err) return 0;
    int v = 0;
    if (cudaMemcpy(&v, h->tc->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (v) {
        cudaMemset(h->tc->err, 0, sizeof(int));
        // a launch that gave up may have left split tickets counted: clear
        // them so that later launches pair their partial sums correctly
        for (TcDir* D : {&h->tc->F, &h->tc->A})
            if (D->ticket)
                cudaMemset(D->ticket, 0,
                           sizeof(int) * (size_t)D->groupsX * h->tc->tilesY * h->Q);
    }
    return v;
}

double tc_issued_macs(const swopt_handle* h, int kernel)
{
    if (!h->tc) return 0;
    return kernel == 0 ? h->tc->F.macs : h->tc->A.macs;
}

void tc_config(const swopt_handle* h, int kernel, int* mt, int* ctas_per_sm, int* stages,
               int* groups, int* accumulators)
{
    const TcDir& D = kernel == 0 ? h->tc->F : h->tc->A;
    *mt = D.MT;
    *accumulators = D.RA;
    *ctas_per_sm = (int)(233472 / (D.smem + 1024));
    if (*ctas_per_sm > 512 / D.cols) *ctas_per_sm = 512 / D.cols;
    *stages = D.NS;
    *groups = D.NG;
}

void tc_schedule_info(const swopt_handle* h, int kernel, int* split, int* buffers, int* grid,
                      int* max_pieces)
{
    const TcDir& D = kernel == 0 ? h->tc->F : h->tc->A;
    *split = D.whole ? 1 : 2;
    *buffers = D.NBUF;
    *grid = D.grid;
    *max_pieces = D.max_pieces;
}

}  // namespace swopt
