// Internal declarations shared by the swopt CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "swopt.h"

namespace swopt {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message of the last failed call).
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define SW_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::swopt::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                               __FILE__, __LINE__);                                \
            return e_ == cudaErrorMemoryAllocation ? SWOPT_ERR_OOM : SWOPT_ERR_CUDA; \
        }                                                                          \
    } while (0)

#define SW_LAUNCHED(h)                                                             \
    do {                                                                           \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) {                                                   \
            ::swopt::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                               __FILE__, __LINE__);                                \
            return SWOPT_ERR_CUDA;                                                 \
        }                                                                          \
        (h)->launches++;                                                           \
    } while (0)

#define SW_TRY(expr)                                                               \
    do {                                                                           \
        swopt_status s_ = (expr);                                                  \
        if (s_ != SWOPT_OK) return s_;                                             \
    } while (0)

// Entries of the refined solve's decision log (a ring).
constexpr int kRefineLog = 1 << 16;

// Time samples are processed in chunks of 32 (a warp's worth of outputs in
// the FP32 kernels, two 16-wide N tiles on the tensor cores).
constexpr int TCHUNK = 32;
// Depths are processed in chunks of 32 by the FP32 adjoint.
constexpr int JCHUNK = 32;
// Lateral tile of the FP32 contraction kernels: 16 x 16 scan positions.
constexpr int TILE = 16;

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Tensor-core operator data (built lazily on first BF16 use).
struct TcOperator;

struct ProfileRec {
    cudaEvent_t a, b;
    int kernel;
    int64_t iter = -1;  // FISTA iteration of a gated launch (see swopt_handle::gate), else -1
};

// A kernel launched behind a gate runs only when the device word *gate
// equals `want`; otherwise every thread returns at once.  Both branches of a
// device-side decision are launched (and captured) unconditionally, so that
// one CUDA graph serves every iteration.
__device__ __forceinline__ bool gated_off(const int* gate, int want)
{
    return gate != nullptr && *(volatile const int*)gate != want;
}

// An event-record node pair of the captured FISTA iteration that brackets
// one launch of the A (0) or A^T (1) kernel.
struct GraphProbe {
    cudaGraphNode_t begin = nullptr, end = nullptr;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;  // placeholders used at capture
    int kernel = 0;
    bool gated = false;  // the bracketed launch runs behind the refinement gate
};

// One captured FISTA iteration (kind 0: plain or incremental-gradient
// iteration; kind 1: the resync iteration of the refined solve; kind 2: the
// refined iteration whose resync is decided on the device, both branches
// behind the gate).
struct IterGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t kernels = 0;
    std::vector<GraphProbe> probes;
};

}  // namespace swopt

struct swopt_handle {
    // geometry
    int X, Y, Z, T, N, P, k, r, ncyc;
    double dz_mm, mu;
    std::vector<double> kappa, eps_bar, eps_off;
    int S;       // X * Y
    int Q;       // distinct switching states min(N, ncyc)
    int state_offset = 0;  // pulse n sits state_offset + (n mod ncyc) pulses into its cycle
    int t0;      // first sample of the time window
    int tw;      // nonzero extent of the window (t0 + tw - 1 = last nonzero sample)
    int Twp;     // padded window length, multiple of TCHUNK
    int nTc;     // Twp / TCHUNK
    int Zp;      // Z padded to a multiple of JCHUNK
    int nJc;     // Zp / JCHUNK
    int64_t nnz; // nonzero kernel entries
    std::vector<double> K64;      // host copy [Z][k][k][T]
    std::vector<double> phi;      // [Z]
    bool phi_fixed = false;       // phi given (swopt_set_fluence), not exp(-mu j dz)
    std::vector<double> Sm64;     // [Q][P][Z] switching weights of the states
    std::vector<int> Cm;          // [Q] pulses per state
    int precision = SWOPT_PREC_FP32;
    int device = 0;
    int smem_optin = 0;           // opt-in shared memory per block (0: not queried)

    // FP32 operator data
    float* Kf = nullptr;          // [Z][k][k][Twp] forward kernel, window-padded
    float* Ka = nullptr;          // [k*k][Twp][Zp] adjoint kernel (depth fastest)
    uint8_t* fmask = nullptr;     // [Z*k*k][nTc] 8-sample nonzero sub-block masks
    uint8_t* amask = nullptr;     // [k*k][Twp][nJc] 8-depth nonzero sub-block masks
    float* Sm = nullptr;          // [Q][P][Z]
    float* Cmf = nullptr;         // [Q]

    // operator workspaces
    float* b = nullptr;           // [Q][Y][X][Z] state images (input of A)
    float* u = nullptr;           // [Q][Y][X][Twp] A output / folded residual
    float* g = nullptr;           // [Q][Y][X][Z] A^T output (before P^T)
    float* ytil = nullptr;        // [Q][Y][X][Twp] pulse-folded measurements
    double* red = nullptr;        // reduction partials
    int red_cap = 0;              // capacity in doubles
    double* scal = nullptr;       // small FP64 device scalars
    double* scal_host = nullptr;  // pinned host mirror

    // FISTA state
    bool fista_ready = false;
    swopt_solve_params prm{};
    double step = 0.0;
    double y_sq = 0.0;            // ||y||^2 of the bound measurements
    double jstep2 = 0.0;          // lambda_3 > 0: dual step of the joint prox
    float* c = nullptr;           // [P][Y][X][Z] current c_k
    float* xi = nullptr;          // momentum iterate
    float* zin = nullptr;         // gradient-step output (prox input)
    float* tvu = nullptr;         // [3][P][Y][X][Z] dual iterate
    float* tvr0 = nullptr;        // [3][..] extrapolated dual (ping)
    float* tvr1 = nullptr;        // [3][..] (pong)
    unsigned* coop_bar = nullptr; // grid barrier of the cooperative TV prox: count, generation, error
    int coop_blocks = 0;          // its grid size (0: not yet sized)
    int tile_ty = 0, tile_tx = 0; // shared-memory TV prox tile (0: not chosen, -1: none fits)
    float* tmp = nullptr;         // [P][Y][X][Z] scratch (c_{k+1} - c_k in the refined solve)
    float* G = nullptr;           // [P][Y][X][Z] refined solve: gradient at c_k
    float* jw = nullptr;          // [P][Y][X][Z] joint prox (lambda_3): projected primal point
    float* ju = nullptr;          // [(4 P + 3 Q) Y X Z] joint prox dual iterate
    float* jr = nullptr;          // [(4 P + 3 Q) Y X Z] joint prox momentum iterate
    float* xprev = nullptr;       // [P][Y][X][Z] previous momentum iterate (eps2 test)
    int64_t iter = 0;             // FISTA iterations since swopt_fista_init
    int64_t resyncs = 0;          // exact gradients of the refined solve (host-scheduled)
    // Device-side resync decision of the refined solve (refine_budget > 0):
    // sched[0] gate (1: this iteration recomputes the gradient exactly),
    // sched[1] iterations decided, sched[2] resyncs; rlog[i % kRefineLog] the
    // decision of iteration i (read back for the profile).
    int* sched = nullptr;
    int* rlog = nullptr;
    const int* gate = nullptr;    // while launching one branch: the gate word, else null
    int gate_want = 0;            // and the value that lets it run

    // tensor-core path
    swopt::TcOperator* tc = nullptr;      // operator of `precision`
    swopt::TcOperator* tc_ref = nullptr;  // operator of the refined solve's resync precision
    int tc_force_mt[2] = {0, 0};     // tiles per CTA of A / A^T (0: tuned)
    int tc_force_ctas[2] = {0, 0};   // CTAs per SM of A / A^T (0: tuned)
    int tc_force_ra[2] = {0, 0};     // accumulators per tile of A / A^T (0: default)
    int tc_force_split[2] = {0, 0};  // work split of A / A^T (1 whole, 2 stream-K; 0: tuned)
    int tc_force_nbuf[2] = {0, 0};   // accumulator buffers of A / A^T (0: tuned)

    // CUDA graph of one FISTA iteration (rebuilt when the settings change)
    bool use_graph = true;
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;
    swopt::IterGraph graphs[3];
    uint64_t graph_gen = 0;       // bumped whenever captured work may have gone stale
    std::vector<std::pair<cudaEvent_t, int>> cap_events;

    // instrumentation
    bool profile = false;
    std::vector<swopt::ProfileRec> prof;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[4] = {0, 0, 0, 0};   // A, A^T, and the two at the resync precision
    int64_t prof_n[4] = {0, 0, 0, 0};
    bool in_ref = false;                // launching the refined solve's resync
    int64_t launches = 0;
};

namespace swopt {

// Largest dynamic shared memory a block may opt in to on the handle's device
// (queried once; <= 0 if the query failed).
inline int smem_optin_bytes(swopt_handle* h)
{
    if (h->smem_optin == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) !=
            cudaSuccess)
            v = -1;
        h->smem_optin = v;
    }
    return h->smem_optin;
}

// Dynamic shared memory that `func` may be given: the opt-in limit less the
// function's static shared memory (<= 0 if a query failed).
inline int max_dynamic_smem(swopt_handle* h, const void* func)
{
    const int optin = smem_optin_bytes(h);
    cudaFuncAttributes fa;
    if (optin <= 0 || cudaFuncGetAttributes(&fa, func) != cudaSuccess) return -1;
    return optin - (int)fa.sharedSizeBytes;
}

inline size_t nc_of(const swopt_handle* h) { return (size_t)h->P * h->S * h->Z; }
inline size_t nb_of(const swopt_handle* h) { return (size_t)h->Q * h->S * h->Z; }
inline size_t nu_of(const swopt_handle* h) { return (size_t)h->Q * h->S * h->Twp; }
inline int grid_for(size_t n, int block) {
    size_t g = (n + block - 1) / block;
    return (int)(g > 2147483647ull ? 2147483647ull : g);
}

// FP32 contraction kernels (operator_simt.cu).
// out = (scale ? Cm[m] : 1) * (A b)[m] - (ytil ? ytil[m] : 0); partials (optional):
// per-block FP64 sums of Cm*(Ab)^2 - 2*(Ab)*ytil.
swopt_status simt_forward(swopt_handle* h, const float* b, float* u, const float* ytil,
                          double* partials, int scale, cudaStream_t st);
swopt_status simt_adjoint(swopt_handle* h, const float* u, float* g, cudaStream_t st);
int simt_forward_blocks(const swopt_handle* h);

// Tensor-core contraction kernels (operator_tc.cu).
// tc_prepare builds the BF16 operator data for h->precision (idempotent).
swopt_status tc_prepare(swopt_handle* h);
void tc_release(swopt_handle* h);
// P: c [P][Y][X][Z] -> padded BF16 state images (hi, and lo for the split mode)
swopt_status tc_states(swopt_handle* h, const float* c, cudaStream_t st);
// A on the state images.  to_r: write the padded BF16 residual images that
// tc_adjoint reads; else write h->u (FP32 [Q][S][Twp]).  Value:
// (scale ? Cm : 1) * acc - (ytil ? ytil : 0); partials as in simt_forward.
swopt_status tc_forward(swopt_handle* h, bool to_r, const float* ytil, double* partials,
                        int scale, cudaStream_t st);
// h->u (FP32) -> padded BF16 residual images
swopt_status tc_pack_u(swopt_handle* h, cudaStream_t st);
// A of several handles (adj false: into the residual images, as tc_forward
// with to_r, scale 1 and ytil = the handle's folded measurements or none) or
// A^T, as persistent launches over a work list of their tile-states (whole,
// one CTA each), the problems packed into as few launches as shared memory
// allows (tc_multi_groups), each with the handle's current gate and
// tensor-core operator.  Prepared on the host (never while capturing);
// UNSUPPORTED for FP8 operators.
struct TcMulti;
swopt_status tc_multi_create(swopt_handle* const* hs, int n, bool adj, bool use_ytil,
                             TcMulti** out);
swopt_status tc_multi_launch(TcMulti* m, cudaStream_t st);
int tc_multi_groups(const TcMulti* m);
void tc_multi_destroy(TcMulti* m);
// A^T of the padded residual images into h->g (FP32 [Q][S][Z])
swopt_status tc_adjoint(swopt_handle* h, cudaStream_t st);
int tc_forward_blocks(const swopt_handle* h);
// Reads and clears the tensor-core kernels' device error word (0 = none).
int tc_error_word(swopt_handle* h);
// MMA multiply-adds issued by one launch of the forward (0) / adjoint (1)
double tc_issued_macs(const swopt_handle* h, int kernel);
// configuration chosen for the forward (0) / adjoint (1)
void tc_config(const swopt_handle* h, int kernel, int* mt, int* ctas_per_sm, int* stages,
               int* groups, int* accumulators);
void tc_schedule_info(const swopt_handle* h, int kernel, int* split, int* buffers, int* grid,
                      int* max_pieces);

// Elementwise / layout kernels (operator_simt.cu).
swopt_status launch_states(swopt_handle* h, const float* c, float* b, cudaStream_t st);
swopt_status launch_expand(swopt_handle* h, const float* u, float* y, cudaStream_t st);
swopt_status launch_fold(swopt_handle* h, const float* y, float* ytil, cudaStream_t st);
// out = sum_m Sm[m][p][j] g[m] (mode 0); out = xi - alpha * that (mode 1)
swopt_status launch_pt(swopt_handle* h, const float* g, const float* xi, float alpha,
                       float* out, int mode, cudaStream_t st);
// out = carry + sum_m Sm[m][p][j] g[m], the sum continued from carry (or 0) in
// the order of the states, one FMA per state
swopt_status launch_pt_carry(swopt_handle* h, const float* g, const float* carry, float* out,
                             cudaStream_t st);
// out = xi - alpha g
swopt_status launch_grad_step(swopt_handle* h, const float* g, const float* xi, float alpha,
                              float* out, cudaStream_t st);
// Refined solve: d = sum_m Sm[m][p][j] g[m]; Gn = (add ? G : 0) + d;
// out = xi - alpha ((1 + beta) Gn - beta G) with beta = scal[1]; G = Gn.
swopt_status launch_pt_refine(swopt_handle* h, const float* g, const float* xi, float alpha,
                              float* G, float* out, int add, cudaStream_t st);

// Proximal / FISTA / reduction kernels (prox.cu).
swopt_status prox_l1(swopt_handle* h, float* x, float thresh, int nonneg, cudaStream_t st);
// delta (optional): also write c_{k+1} - c_k there
swopt_status fista_finish(swopt_handle* h, const float* z, bool use_tv, float theta,
                          float* delta, cudaStream_t st);
swopt_status fista_scalars(swopt_handle* h, int momentum, cudaStream_t st);
// The TV prox of Algorithm 2 (iters >= 1 inner iterations) in one cooperative
// launch: out = z - D^T u (prox_tv_coop), or with the FISTA scalars and
// fista_finish fused after it (fista_prox_finish).  Needs ensure'd TV buffers.
swopt_status prox_tv_coop(swopt_handle* h, const float* z, float tau, int iters,
                          int inner_momentum, float* out, cudaStream_t st);
swopt_status fista_prox_finish(swopt_handle* h, const float* z, float tau, int iters,
                               int inner_momentum, float theta, float* delta, cudaStream_t st);
swopt_status coop_prepare(swopt_handle* h);
// Failure-detection test hook of the cooperative kernels' grid barrier.
swopt_status coop_debug(swopt_handle* h, unsigned phantom, unsigned poll_limit);
// Reads and clears the cooperative kernel's barrier error word (0 = none).
int coop_error_word(swopt_handle* h);
swopt_status fista_reset_scalars(swopt_handle* h, cudaStream_t st);
// FP64 reductions, result written to h->scal[slot]
swopt_status reduce_sumsq(swopt_handle* h, const float* x, size_t n, int slot, cudaStream_t st);
swopt_status reduce_dot(swopt_handle* h, const float* x, const float* y, size_t n, int slot,
                        cudaStream_t st);
swopt_status reduce_abs(swopt_handle* h, const float* x, size_t n, int slot, cudaStream_t st);
swopt_status reduce_tv(swopt_handle* h, const float* x, int slot, cudaStream_t st);
// sum_m Cm[m] TV(b_m) of the Q state images b [Q][Y][X][Z] (= sum_n TV((S c)^n))
swopt_status reduce_tv_states(swopt_handle* h, const float* b, int slot, cudaStream_t st);
swopt_status reduce_partials(swopt_handle* h, const double* parts, int count, int slot,
                             cudaStream_t st);
// Refined solve, device-side schedule: rho = ||d|| / ||c|| (FP64) is added
// to the budget accumulator scal[slot]; the gate h->sched[0] opens the exact
// resync when the iteration is a multiple of R or the accumulated sum
// exceeds `budget` (which then restarts from 0).
swopt_status refine_decide(swopt_handle* h, const float* d, const float* c, int slot, int R,
                           double budget, cudaStream_t st);
swopt_status scale_by_inv_sqrt(swopt_handle* h, const float* in, float* out, size_t n, int slot,
                               cudaStream_t st);
swopt_status fill_counter_random(swopt_handle* h, float* x, size_t n, uint64_t seed,
                                 cudaStream_t st);
swopt_status param_weights(swopt_handle* h, const float* g, const float* c, int slot0,
                           cudaStream_t st);

// FISTA set-up on measurements y (api.cu; swopt_fista_init after its checks).
swopt_status fista_init_impl(swopt_handle* h, const float* y, const swopt_solve_params* prm,
                             cudaStream_t st);

// The joint prox of R3 with its lambda_3 term (prox_joint.cu): Algorithm 2 on
// the stacked operator with one dual per switching state, z and x may alias;
// scratch w [P L], u and r [joint_dual_floats] (ensure_joint_buffers gives the
// handle's).  joint_step_bound: an upper bound of eig_max(L L^T).
size_t joint_dual_floats(const swopt_handle* h);
double joint_step_bound(const swopt_handle* h, double lambda_tv, double lambda_l1,
                        double lambda_b);
swopt_status ensure_joint_buffers(swopt_handle* h);
swopt_status joint_prox_on(swopt_handle* h, const float* z, float* x, double alpha,
                           double lambda_tv, double lambda_l1, double lambda_b, int iters,
                           double step2, int momentum, float* w, float* u, float* r,
                           cudaStream_t st);

// Handle-free launchers of one FGP iteration / the primal recovery on
// caller-given buffers (prox.cu); the duals u, rin, rout have 3 components.
cudaError_t fgp_iter_on(const float* z, const float* rin, float* rout, float* u, int P, int Y,
                        int X, int Z, float tau, float beta, int first, cudaStream_t st);
cudaError_t fgp_finish_on(const float* z, const float* u, float* x, int P, int Y, int X, int Z,
                          cudaStream_t st);

// Instrumentation
void prof_begin(swopt_handle* h, int kernel, cudaStream_t st, ProfileRec* rec);
void prof_end(swopt_handle* h, ProfileRec* rec, cudaStream_t st);

}  // namespace swopt
