// C-ABI entry points of swopt: argument validation, handle set-up (kernel
// window, band masks, switching states) and the orchestration of each call
// out of the kernels in operator_simt.cu, operator_tc.cu and prox.cu.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <algorithm>
#include <cstdio>
#include <memory>
#include <vector>

#include "swopt_internal.cuh"

namespace swopt {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

// Slots of the FP64 device scalars.
enum {
    SC_T = 0,      // FISTA t_k
    SC_BETA = 1,   // FISTA beta_k
    SC_A = 2,      // reduction results
    SC_B = 3,
    SC_C = 4,
    SC_D = 5,
    SC_YSQ = 6,    // ||y||^2 of the measurements bound by fista_init
    SC_BUDGET = 7, // refined solve: accumulated rho since the last exact gradient
    SC_COUNT = 16
};

// Two timing events from the handle's pool (created when the pool is empty).
bool take_events(swopt_handle* h, cudaEvent_t* a, cudaEvent_t* b)
{
    if (h->event_pool.size() >= 2) {
        *a = h->event_pool.back(); h->event_pool.pop_back();
        *b = h->event_pool.back(); h->event_pool.pop_back();
        return true;
    }
    if (cudaEventCreate(a) != cudaSuccess) return false;
    if (cudaEventCreate(b) != cudaSuccess) {
        cudaEventDestroy(*a);
        return false;
    }
    return true;
}

void prof_begin(swopt_handle* h, int kernel, cudaStream_t st, ProfileRec* rec)
{
    rec->kernel = -1;
    rec->iter = h->gate ? h->iter : -1;
    if (h->in_ref) kernel += 2;  // launches at the refined solve's resync precision
    if (h->capturing) {
        // an event-record node in the graph; its event is swapped per replay
        cudaEvent_t a;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventRecordWithFlags(a, st, cudaEventRecordExternal) != cudaSuccess) {
            cudaEventDestroy(a);
            return;
        }
        // a gated launch is marked by an offset of 16 in the captured kind
        h->cap_events.push_back({a, kernel + (h->gate ? 16 : 0)});
        rec->a = a;
        rec->kernel = kernel;
        return;
    }
    if (!h->profile) return;
    cudaEvent_t a, b;
    if (!take_events(h, &a, &b)) return;
    rec->a = a;
    rec->b = b;
    rec->kernel = kernel;
    cudaEventRecord(a, st);
}

void prof_end(swopt_handle* h, ProfileRec* rec, cudaStream_t st)
{
    if (rec->kernel < 0) return;
    if (h->capturing) {
        cudaEvent_t b;
        if (cudaEventCreate(&b) != cudaSuccess) return;
        if (cudaEventRecordWithFlags(b, st, cudaEventRecordExternal) != cudaSuccess) {
            cudaEventDestroy(b);
            return;
        }
        h->cap_events.push_back({b, -1 - (rec->kernel + (h->gate ? 16 : 0))});  // end marker
        return;
    }
    cudaEventRecord(rec->b, st);
    h->prof.push_back(*rec);
}

}  // namespace swopt

using namespace swopt;

namespace {

bool is_fin(double v) { return std::isfinite(v); }

swopt_status check_handle(swopt_handle* h)
{
    if (!h) {
        set_error("null handle");
        return SWOPT_ERR_INVALID_ARG;
    }
    return SWOPT_OK;
}

template <typename T>
swopt_status dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SWOPT_ERR_OOM : SWOPT_ERR_CUDA;
    }
    return SWOPT_OK;
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void release_graph(swopt_handle* h)
{
    for (IterGraph& g : h->graphs) {
        if (g.gexec) cudaGraphExecDestroy(g.gexec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = IterGraph();
    }
    for (auto& e : h->cap_events) cudaEventDestroy(e.first);
    h->cap_events.clear();
    ++h->graph_gen;
}

// Within its scope the handle computes at the refined solve's resync
// precision: h->precision and the tensor-core operator are swapped for those
// of the resync (a no-op when the two precisions agree).
struct RefScope {
    swopt_handle* h;
    int prec;
    TcOperator* tc;
    bool active;
    RefScope(swopt_handle* hh, int ref_precision)
        : h(hh), prec(hh->precision), tc(hh->tc), active(ref_precision != hh->precision)
    {
        h->in_ref = true;
        if (!active) return;
        h->precision = ref_precision;
        h->tc = h->tc_ref;
    }
    ~RefScope()
    {
        h->in_ref = false;
        if (!active) return;
        h->tc_ref = h->tc;
        h->tc = tc;
        h->precision = prec;
    }
};

void release_ref(swopt_handle* h)
{
    std::swap(h->tc, h->tc_ref);
    tc_release(h);
    std::swap(h->tc, h->tc_ref);
}

void release_all(swopt_handle* h)
{
    release_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    tc_release(h);
    release_ref(h);
    dfree(h->Kf); dfree(h->Ka); dfree(h->fmask); dfree(h->amask); dfree(h->Sm); dfree(h->Cmf);
    dfree(h->b); dfree(h->u); dfree(h->g); dfree(h->ytil); dfree(h->red); dfree(h->scal);
    dfree(h->c); dfree(h->xi); dfree(h->zin); dfree(h->tvu); dfree(h->tvr0); dfree(h->tvr1);
    dfree(h->coop_bar);
    dfree(h->tmp); dfree(h->G); dfree(h->xprev); dfree(h->jw); dfree(h->ju); dfree(h->jr); dfree(h->sched); dfree(h->rlog);
    if (h->scal_host) cudaFreeHost(h->scal_host);
    h->scal_host = nullptr;
    for (auto& r : h->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    h->prof.clear();
    for (auto e : h->event_pool) cudaEventDestroy(e);
    h->event_pool.clear();
}

swopt_status ensure_tv_buffers(swopt_handle* h)
{
    const size_t n = nc_of(h);
    if (!h->tvu) SW_TRY(dalloc(&h->tvu, 3 * n));
    if (!h->tvr0) SW_TRY(dalloc(&h->tvr0, 3 * n));
    if (!h->tvr1) SW_TRY(dalloc(&h->tvr1, 3 * n));
    SW_TRY(coop_prepare(h));
    return SWOPT_OK;
}

swopt_status ensure_vectors(swopt_handle* h)
{
    const size_t n = nc_of(h);
    if (!h->c) SW_TRY(dalloc(&h->c, n));
    if (!h->xi) SW_TRY(dalloc(&h->xi, n));
    if (!h->zin) SW_TRY(dalloc(&h->zin, n));
    if (!h->tmp) SW_TRY(dalloc(&h->tmp, n));
    return SWOPT_OK;
}

swopt_status ensure_ytil(swopt_handle* h)
{
    if (!h->ytil) SW_TRY(dalloc(&h->ytil, nu_of(h)));
    return SWOPT_OK;
}

// Device-side failures recorded by the kernels (a bounded wait that gave up).
swopt_status device_errors(swopt_handle* h)
{
    // every error word is read (and so cleared, with the state it guards) on
    // every check, so that one failure is reported once and leaves no residue
    int w = tc_error_word(h);
    std::swap(h->tc, h->tc_ref);
    const int w_ref = tc_error_word(h);
    std::swap(h->tc, h->tc_ref);
    const int c = coop_error_word(h);
    if (w == 0) w = w_ref;
    if (w == 0 && c > 0) {
        set_error("the TV prox kernel gave up a bounded grid barrier");
        return SWOPT_ERR_TIMEOUT;
    }
    if (w == 0 && c < 0) w = -1;
    if (w > 0) {
        set_error("a tensor-core kernel gave up a bounded wait (code %d)", w);
        return SWOPT_ERR_TIMEOUT;
    }
    if (w < 0) {
        set_error("reading the device error word failed");
        return SWOPT_ERR_CUDA;
    }
    return SWOPT_OK;
}

swopt_status read_scalars(swopt_handle* h, cudaStream_t st)
{
    SW_CUDA(cudaMemcpyAsync(h->scal_host, h->scal, SC_COUNT * sizeof(double),
                            cudaMemcpyDeviceToHost, st));
    SW_CUDA(cudaStreamSynchronize(st));
    return device_errors(h);
}

bool use_tc(const swopt_handle* h) { return h->precision != SWOPT_PREC_FP32; }

// P then A.  out = A_OUT_U writes h->u (FP32 [Q][S][Twp]); out = A_OUT_R writes
// the input format of apply_AT (h->u for the FP32 kernels, the padded BF16
// residual images for the tensor-core kernels).  The result is
// (scale ? Cm : 1) * (A P c) - ytil  (see simt_forward).
enum { A_OUT_U = 0, A_OUT_R = 1 };

swopt_status no_tc_operator()
{
    set_error("internal: no tensor-core operator for the selected precision");
    return SWOPT_ERR_DEVICE_CHECK;
}

swopt_status apply_A(swopt_handle* h, const float* c, int out, const float* ytil,
                     double* partials, int scale, cudaStream_t st)
{
    if (use_tc(h)) {
        if (!h->tc) return no_tc_operator();
        SW_TRY(tc_states(h, c, st));
        return tc_forward(h, out == A_OUT_R, ytil, partials, scale, st);
    }
    SW_TRY(launch_states(h, c, h->b, st));
    return simt_forward(h, h->b, h->u, ytil, partials, scale, st);
}

// A^T into h->g.  from_u: the input is h->u (FP32) rather than the output of
// apply_A(A_OUT_R).
swopt_status apply_AT(swopt_handle* h, bool from_u, cudaStream_t st)
{
    if (use_tc(h)) {
        if (!h->tc) return no_tc_operator();
        if (from_u) SW_TRY(tc_pack_u(h, st));
        return tc_adjoint(h, st);
    }
    return simt_adjoint(h, h->u, h->g, st);
}

// w = H^T H v
swopt_status normal_op(swopt_handle* h, const float* v, float* w, cudaStream_t st)
{
    SW_TRY(apply_A(h, v, A_OUT_R, nullptr, nullptr, 1, st));
    SW_TRY(apply_AT(h, false, st));
    return launch_pt(h, h->g, nullptr, 0.f, w, 0, st);
}

swopt_status lipschitz_impl(swopt_handle* h, const float* v0, int iters, double* L,
                            cudaStream_t st)
{
    SW_TRY(ensure_vectors(h));
    const size_t n = nc_of(h);
    float* v = h->tmp;
    float* w = h->zin;
    if (v0) SW_CUDA(cudaMemcpyAsync(v, v0, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else SW_TRY(fill_counter_random(h, v, n, 0x5eed5eedull, st));
    SW_TRY(reduce_sumsq(h, v, n, SC_A, st));
    SW_TRY(scale_by_inv_sqrt(h, v, v, n, SC_A, st));
    for (int it = 0; it < iters; ++it) {
        SW_TRY(normal_op(h, v, w, st));
        SW_TRY(reduce_dot(h, v, w, n, SC_B, st));   // Rayleigh quotient (||v|| = 1)
        SW_TRY(reduce_sumsq(h, w, n, SC_A, st));
        SW_TRY(scale_by_inv_sqrt(h, w, v, n, SC_A, st));
    }
    SW_TRY(read_scalars(h, st));
    *L = h->scal_host[SC_B];
    return SWOPT_OK;
}

// Switching weights of the Q states (Eq. final-H): Phi_j = exp(-mu j dz) and
// S[m][p][j] = Phi_j (eps_bar_p exp(-kappa_p Phi_j m) + eps_off_p).
void switching_states(swopt_handle* h)
{
    if (!h->phi_fixed) {
        h->phi.resize(h->Z);
        for (int j = 0; j < h->Z; ++j) h->phi[j] = std::exp(-h->mu * j * h->dz_mm);
    }
    h->Sm64.resize((size_t)h->Q * h->P * h->Z);
    for (int m = 0; m < h->Q; ++m)
        for (int p = 0; p < h->P; ++p)
            for (int j = 0; j < h->Z; ++j) {
                const double ph = h->phi[j];
                h->Sm64[((size_t)m * h->P + p) * h->Z + j] =
                    ph * (h->eps_bar[p] * std::exp(-h->kappa[p] * ph * (m + h->state_offset)) +
                          h->eps_off[p]);
            }
}

swopt_status check_switching(const swopt_switching* sw, int P)
{
    if (!sw || !sw->kappa_host || !sw->eps_bar_host || !sw->eps_off_host) {
        set_error("null switching pointer");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!is_fin(sw->mu_per_mm)) {
        set_error("invalid mu_per_mm");
        return SWOPT_ERR_INVALID_ARG;
    }
    for (int p = 0; p < P; ++p)
        if (!is_fin(sw->kappa_host[p]) || !is_fin(sw->eps_bar_host[p]) ||
            !is_fin(sw->eps_off_host[p])) {
            set_error("non-finite switching parameter for species %d", p);
            return SWOPT_ERR_INVALID_ARG;
        }
    return SWOPT_OK;
}

// Chain rule through Eq. (final-H): W[m][p][j] = <(A^T w)_m, c_p> per depth
// (FP64, from param_weights) -> d/dkappa_p and d/dmu of <w, H c>.
void switching_chain_rule(const swopt_handle* h, const std::vector<double>& W, double* dkappa,
                          double* dmu)
{
    double dm = 0.0;
    for (int p = 0; p < h->P; ++p) dkappa[p] = 0.0;
    for (int q = 0; q < h->Q; ++q)
        for (int p = 0; p < h->P; ++p)
            for (int j = 0; j < h->Z; ++j) {
                const double ph = h->phi[j];
                const int m = q + h->state_offset;  // pulses into the cycle
                const double e = std::exp(-h->kappa[p] * ph * m);
                const double w = W[((size_t)q * h->P + p) * h->Z + j];
                const double dS_dk = ph * h->eps_bar[p] * e * (-ph * m);
                const double dS_dphi =
                    h->eps_bar[p] * e + h->eps_off[p] + ph * h->eps_bar[p] * e * (-h->kappa[p] * m);
                const double dphi_dmu = h->phi_fixed ? 0.0 : -(double)j * h->dz_mm * ph;
                dkappa[p] += w * dS_dk;
                dm += w * dS_dphi * dphi_dmu;
            }
    *dmu = dm;
}

// W from the A^T output in h->g and c, then the chain rule (synchronises).
swopt_status switching_gradient(swopt_handle* h, const float* c, double* dkappa, double* dmu,
                                cudaStream_t st)
{
    SW_TRY(param_weights(h, h->g, c, 0, st));
    const size_t nw = (size_t)h->Q * h->P * h->Z;
    std::vector<double> W(nw);
    SW_CUDA(cudaMemcpyAsync(W.data(), h->red, nw * sizeof(double), cudaMemcpyDeviceToHost, st));
    SW_CUDA(cudaStreamSynchronize(st));
    SW_TRY(device_errors(h));
    switching_chain_rule(h, W, dkappa, dmu);
    return SWOPT_OK;
}

swopt_status validate_params(const swopt_solve_params* p)
{
    if (!p) {
        set_error("null solve parameters");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!is_fin(p->step) || !is_fin(p->lambda_l1) || !is_fin(p->lambda_tv) || !is_fin(p->eps1) ||
        !is_fin(p->eps2) || p->lambda_l1 < 0 || p->lambda_tv < 0 || p->inner_iters < 0 ||
        p->inner_iters > 100000 || p->max_iters < 0 || p->momentum < 0 || p->momentum > 2 ||
        p->inner_momentum < 0 || p->inner_momentum > 2 || p->refine_every < 0 ||
        p->refine_precision < SWOPT_PREC_FP32 || p->refine_precision > SWOPT_PREC_BF16X6 ||
        p->refine_precision == SWOPT_PREC_FP8 ||
        !is_fin(p->refine_budget) || p->refine_budget < 0 || !is_fin(p->lambda_3) ||
        p->lambda_3 < 0 || !is_fin(p->joint_step2) || (p->lambda_3 > 0 && p->inner_iters < 1) ||
        (p->step <= 0 && (p->power_iters < 1 || p->power_iters > 100000))) {
        set_error("invalid solve parameters");
        return SWOPT_ERR_INVALID_ARG;
    }
    return SWOPT_OK;
}

// Refined solve: the gradient G = P^T A^T (C A P c - ytil) at c = h->c,
// evaluated at the resync precision, replaces h->G; h->zin receives the
// gradient step at the momentum point (see launch_pt_refine).
swopt_status exact_gradient(swopt_handle* h, cudaStream_t st)
{
    RefScope sc(h, h->prm.refine_precision);
    SW_TRY(apply_A(h, h->c, A_OUT_R, h->ytil, nullptr, 1, st));
    SW_TRY(apply_AT(h, false, st));
    return launch_pt_refine(h, h->g, h->xi, (float)h->step, h->G, h->zin, 0, st);
}

// Builds the resync precision's tensor-core operator if the refined solve
// needs one (synchronises; never called while capturing).
swopt_status ensure_ref(swopt_handle* h)
{
    const int rp = h->prm.refine_precision;
    if (h->prm.refine_every <= 0 || rp == SWOPT_PREC_FP32 || rp == h->precision) return SWOPT_OK;
    RefScope sc(h, rp);
    return tc_prepare(h);
}

// Kind of FISTA iteration number h->iter: 1 when the refined solve
// recomputes its gradient exactly at the end of it, else 0.
int iteration_kind(const swopt_handle* h)
{
    const int R = h->prm.refine_every;
    if (R > 0 && h->prm.refine_budget > 0) return 2;  // decided on the device
    return (R > 0 && (h->iter + 1) % R == 0) ? 1 : 0;
}

// Within its scope, launches run behind the refined solve's gate and only
// when the device decision equals `want`.
struct GateScope {
    swopt_handle* h;
    GateScope(swopt_handle* hh, int want) : h(hh)
    {
        h->gate = h->sched;
        h->gate_want = want;
    }
    ~GateScope() { h->gate = nullptr; }
};

// One FISTA iteration on the bound measurements (all on `st`, no host sync).
//
// Plain (refine_every = 0): the gradient at xi_k is evaluated directly,
//   z = xi_k - alpha P^T A^T (C A P xi_k - ytil), then the prox and momentum.
// Refined (refine_every = R): the prox input z_k is already in h->zin, and the
//   gradient at c_k in h->G.  After the prox and momentum update, the gradient
//   at c_{k+1} is G + H^T H (c_{k+1} - c_k), the normal operator applied to
//   the increment at the handle's precision (kind 0), or is recomputed
//   from c_{k+1} at the resync precision (kind 1).  The gradient step at
//   xi_{k+1} then follows by linearity.  In exact arithmetic both variants
//   give the iterates of Algorithm 1.
// The prox of the prox input h->zin and the momentum step (Algorithm 1 after
// the gradient step); refined: c_{k+1} - c_k also goes to h->tmp.
swopt_status fista_prox_momentum(swopt_handle* h, bool refined, cudaStream_t st)
{
    const bool tv = h->prm.lambda_tv > 0 && h->prm.inner_iters > 0;
    const float theta = (float)(h->step * h->prm.lambda_l1);
    if (h->prm.lambda_3 > 0) {
        // the prox of all three terms of R3 with the constraint (in place on
        // the prox input), then the momentum scalars and step
        SW_TRY(joint_prox_on(h, h->zin, h->zin, h->step, h->prm.lambda_tv, h->prm.lambda_l1,
                             h->prm.lambda_3, h->prm.inner_iters, h->jstep2,
                             h->prm.inner_momentum, h->jw, h->ju, h->jr, st));
        SW_TRY(fista_scalars(h, h->prm.momentum, st));
        SW_TRY(fista_finish(h, h->zin, false, 0.f, refined ? h->tmp : nullptr, st));
    } else if (tv) {
        // TV prox, momentum scalars, l1 prox and momentum step: one launch
        SW_TRY(fista_prox_finish(h, h->zin, (float)(h->step * h->prm.lambda_tv),
                                 h->prm.inner_iters, h->prm.inner_momentum, theta,
                                 refined ? h->tmp : nullptr, st));
    } else {
        SW_TRY(fista_scalars(h, h->prm.momentum, st));
        SW_TRY(fista_finish(h, h->zin, false, theta, refined ? h->tmp : nullptr, st));
    }
    return SWOPT_OK;
}

swopt_status fista_iteration(swopt_handle* h, int kind, cudaStream_t st)
{
    const float alpha = (float)h->step;
    const bool refined = h->prm.refine_every > 0;
    if (!refined) {
        SW_TRY(apply_A(h, h->xi, A_OUT_R, h->ytil, nullptr, 1, st));     // P, A, folded residual
        SW_TRY(apply_AT(h, false, st));                                   // A^T
        SW_TRY(launch_pt(h, h->g, h->xi, alpha, h->zin, 1, st));          // P^T, gradient step
    }
    SW_TRY(fista_prox_momentum(h, refined, st));
    if (!refined) return SWOPT_OK;
    if (kind == 1) return exact_gradient(h, st);
    if (kind == 2) {
        // the device decides between the increment and the exact gradient;
        // both branches are launched behind the gate
        SW_TRY(refine_decide(h, h->tmp, h->c, SC_BUDGET, h->prm.refine_every,
                             h->prm.refine_budget, st));
        {
            GateScope g0(h, 0);
            SW_TRY(apply_A(h, h->tmp, A_OUT_R, nullptr, nullptr, 1, st));
            SW_TRY(apply_AT(h, false, st));
            SW_TRY(launch_pt_refine(h, h->g, h->xi, alpha, h->G, h->zin, 1, st));
        }
        GateScope g1(h, 1);
        return exact_gradient(h, st);
    }
    SW_TRY(apply_A(h, h->tmp, A_OUT_R, nullptr, nullptr, 1, st));        // C A P delta
    SW_TRY(apply_AT(h, false, st));
    return launch_pt_refine(h, h->g, h->xi, alpha, h->G, h->zin, 1, st);
}

// Captures one FISTA iteration into a CUDA graph on the handle's capture
// stream (the caller's stream may be the legacy default stream, which cannot
// capture); the graph is then launched on the caller's stream.
swopt_status build_graph(swopt_handle* h, int kind)
{
    IterGraph& G = h->graphs[kind];
    if (!h->cap_stream) SW_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const int64_t launches0 = h->launches;
    const size_t ev0 = h->cap_events.size();
    SW_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    swopt_status s = fista_iteration(h, kind, h->cap_stream);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (s != SWOPT_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        set_error("graph capture failed: %s", cudaGetErrorString(e));
        return SWOPT_ERR_CUDA;
    }
    G.graph = g;
    G.kernels = h->launches - launches0;
    h->launches = launches0;
    SW_CUDA(cudaGraphInstantiate(&G.gexec, g, 0));
    // locate the event-record nodes that bracket the A / A^T kernels
    size_t n = 0;
    SW_CUDA(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    SW_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
    std::vector<std::pair<cudaEvent_t, cudaGraphNode_t>> rec;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        SW_CUDA(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        SW_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
        rec.push_back({ev, nd});
    }
    auto node_of = [&](cudaEvent_t ev) -> cudaGraphNode_t {
        for (auto& r : rec)
            if (r.first == ev) return r.second;
        return nullptr;
    };
    for (size_t i = ev0; i + 1 < h->cap_events.size(); ++i) {
        const auto& b = h->cap_events[i];
        const auto& en = h->cap_events[i + 1];
        if (b.second >= 0 && en.second == -1 - b.second) {
            GraphProbe pr;
            pr.begin = node_of(b.first);
            pr.end = node_of(en.first);
            pr.ev_begin = b.first;
            pr.ev_end = en.first;
            pr.gated = b.second >= 16;
            pr.kernel = b.second & 15;
            if (pr.begin && pr.end) G.probes.push_back(pr);
            ++i;
        }
    }
    return SWOPT_OK;
}

// One replay of a captured iteration on `st` (with fresh events on the
// probe nodes when profiling).
swopt_status launch_graph(swopt_handle* h, int kind, cudaStream_t st)
{
    IterGraph& G = h->graphs[kind];
    if (h->profile) {
        for (auto& pr : G.probes) {
            ProfileRec rec;
            if (!take_events(h, &rec.a, &rec.b)) continue;
            rec.kernel = pr.kernel;
            rec.iter = pr.gated ? h->iter : -1;
            SW_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.gexec, pr.begin, rec.a));
            SW_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.gexec, pr.end, rec.b));
            h->prof.push_back(rec);
        }
    }
    SW_CUDA(cudaGraphLaunch(G.gexec, st));
    h->launches += G.kernels;
    return SWOPT_OK;
}

// The next FISTA iteration, replayed from its graph when graphs are on.
swopt_status run_iteration(swopt_handle* h, cudaStream_t st)
{
    SW_TRY(ensure_ref(h));
    const int kind = iteration_kind(h);
    if (h->use_graph) {
        if (!h->graphs[kind].gexec) SW_TRY(build_graph(h, kind));
        SW_TRY(launch_graph(h, kind, st));
    } else {
        SW_TRY(fista_iteration(h, kind, st));
    }
    if (kind == 1) ++h->resyncs;
    ++h->iter;
    return SWOPT_OK;
}

// F(c) and the data fit on measurements y (FP64; slots SC_A..SC_D).
swopt_status objective_impl(swopt_handle* h, const float* c, const float* y, double lam_l1,
                            double lam_tv, double lam_3, double* F, double* fit, cudaStream_t st)
{
    SW_TRY(apply_A(h, c, A_OUT_U, nullptr, nullptr, 0, st));
    SW_TRY(ensure_vectors(h));
    // expand H c into the y layout chunk by chunk is avoided: the data fit is
    // the sum over pulses of ||u[m(n)] - y[n]||^2 including the samples
    // outside the window, computed as ||y||^2 + sum_m Cm ||u_m||^2 - 2 <u, ytil>.
    float* yt = nullptr;
    SW_TRY(dalloc(&yt, nu_of(h)));
    swopt_status s = launch_fold(h, y, yt, st);
    if (s == SWOPT_OK) s = reduce_sumsq(h, y, (size_t)h->N * h->S * h->T, SC_A, st);
    if (s == SWOPT_OK) s = reduce_dot(h, h->u, yt, nu_of(h), SC_B, st);
    // sum_m Cm ||u_m||^2 : one reduction per state
    double cu = 0.0;
    if (s == SWOPT_OK) s = read_scalars(h, st);
    double ysq = h->scal_host[SC_A], uy = h->scal_host[SC_B];
    for (int m = 0; m < h->Q && s == SWOPT_OK; ++m) {
        s = reduce_sumsq(h, h->u + (size_t)m * h->S * h->Twp, (size_t)h->S * h->Twp, SC_C, st);
        if (s == SWOPT_OK) s = read_scalars(h, st);
        cu += h->Cm[m] * h->scal_host[SC_C];
    }
    if (s == SWOPT_OK) s = reduce_abs(h, c, nc_of(h), SC_C, st);
    if (s == SWOPT_OK) s = reduce_tv(h, c, SC_D, st);
    if (s == SWOPT_OK) s = read_scalars(h, st);
    const double l1 = h->scal_host[SC_C], tvc = h->scal_host[SC_D];
    double tvs = 0.0;  // sum_n TV((S c)^n) = sum_m Cm TV(S_m c)
    if (s == SWOPT_OK && lam_3 != 0.0) {
        s = launch_states(h, c, h->b, st);
        if (s == SWOPT_OK) s = reduce_tv_states(h, h->b, SC_D, st);
        if (s == SWOPT_OK) s = read_scalars(h, st);
        tvs = h->scal_host[SC_D];
    }
    cudaFree(yt);
    SW_TRY(s);
    const double df = 0.5 * (ysq + cu - 2.0 * uy);
    if (fit) *fit = df;
    if (F) *F = df + lam_l1 * l1 + lam_tv * tvc + lam_3 * tvs;
    return SWOPT_OK;
}

}  // namespace

extern "C" {

const char* swopt_last_error(void) { return g_err; }

const char* swopt_version(void) { return "0.1.0"; }

swopt_status swopt_create(const swopt_geometry* geom, const double* K_host,
                          const swopt_switching* sw, swopt_handle** out)
{
    clear_error();
    if (!out) {
        set_error("null output pointer");
        return SWOPT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!geom || !K_host) {
        set_error("null geometry or kernel pointer");
        return SWOPT_ERR_INVALID_ARG;
    }
    const swopt_geometry& g = *geom;
    if (g.X < 1 || g.X > 4096 || g.Y < 1 || g.Y > 4096 || g.Z < 1 || g.Z > 1024 || g.T < 1 ||
        g.T > 8192 || g.N < 1 || g.N > 4096 || g.P < 1 || g.P > 8 || g.k < 1 || g.k > 63 ||
        (g.k % 2) == 0 || g.pulses_per_cycle < 1) {
        set_error("geometry out of range (X=%d Y=%d Z=%d T=%d N=%d P=%d k=%d cycle=%d)", g.X, g.Y,
                  g.Z, g.T, g.N, g.P, g.k, g.pulses_per_cycle);
        return SWOPT_ERR_SHAPE;
    }
    if (!is_fin(g.dz_mm) || g.dz_mm <= 0) {
        set_error("invalid dz_mm");
        return SWOPT_ERR_INVALID_ARG;
    }
    SW_TRY(check_switching(sw, g.P));
    const size_t kn = (size_t)g.Z * g.k * g.k * g.T;
    int tmin = g.T, tmax = -1;
    int64_t nnz = 0;
    for (size_t i = 0; i < kn; ++i) {
        const double v = K_host[i];
        if (!is_fin(v)) {
            set_error("non-finite kernel entry at %zu", i);
            return SWOPT_ERR_INVALID_ARG;
        }
        if (v != 0.0) {
            const int t = (int)(i % g.T);
            tmin = std::min(tmin, t);
            tmax = std::max(tmax, t);
            ++nnz;
        }
    }
    if (nnz == 0) {
        set_error("the kernel is identically zero");
        return SWOPT_ERR_SHAPE;
    }

    swopt_handle* h = new swopt_handle();
    h->X = g.X; h->Y = g.Y; h->Z = g.Z; h->T = g.T; h->N = g.N; h->P = g.P; h->k = g.k;
    h->r = g.k / 2; h->ncyc = g.pulses_per_cycle; h->dz_mm = g.dz_mm; h->mu = sw->mu_per_mm;
    h->kappa.assign(sw->kappa_host, sw->kappa_host + g.P);
    h->eps_bar.assign(sw->eps_bar_host, sw->eps_bar_host + g.P);
    h->eps_off.assign(sw->eps_off_host, sw->eps_off_host + g.P);
    h->S = g.X * g.Y;
    h->Q = std::min(g.N, g.pulses_per_cycle);
    h->nnz = nnz;
    h->t0 = tmin & ~3;
    h->tw = tmax - h->t0 + 1;
    h->Twp = ((h->tw + TCHUNK - 1) / TCHUNK) * TCHUNK;
    h->nTc = h->Twp / TCHUNK;
    h->Zp = ((g.Z + JCHUNK - 1) / JCHUNK) * JCHUNK;
    h->nJc = h->Zp / JCHUNK;
    h->K64.assign(K_host, K_host + kn);
    cudaGetDevice(&h->device);

    switching_states(h);
    h->Cm.assign(h->Q, 0);
    for (int n = 0; n < g.N; ++n) h->Cm[n % h->ncyc]++;

    // FP32 kernel copies and band masks
    const int kk = g.k * g.k;
    std::vector<float> Kf((size_t)g.Z * kk * h->Twp, 0.f);
    for (int j = 0; j < g.Z; ++j)
        for (int d = 0; d < kk; ++d)
            for (int w = 0; w < h->Twp; ++w) {
                const int t = h->t0 + w;
                if (t < g.T)
                    Kf[((size_t)j * kk + d) * h->Twp + w] =
                        (float)K_host[((size_t)j * kk + d) * g.T + t];
            }
    std::vector<uint8_t> fm((size_t)g.Z * kk * h->nTc, 0);
    for (size_t jd = 0; jd < (size_t)g.Z * kk; ++jd)
        for (int tc = 0; tc < h->nTc; ++tc) {
            uint8_t msk = 0;
            for (int q = 0; q < 4; ++q)
                for (int i = 0; i < 8; ++i)
                    if (Kf[jd * h->Twp + tc * TCHUNK + 8 * q + i] != 0.f) msk |= (uint8_t)(1u << q);
            fm[jd * h->nTc + tc] = msk;
        }
    std::vector<float> Ka((size_t)kk * h->Twp * h->Zp, 0.f);
    for (int j = 0; j < g.Z; ++j)
        for (int d = 0; d < kk; ++d)
            for (int w = 0; w < h->Twp; ++w)
                Ka[((size_t)d * h->Twp + w) * h->Zp + j] = Kf[((size_t)j * kk + d) * h->Twp + w];
    std::vector<uint8_t> am((size_t)kk * h->Twp * h->nJc, 0);
    for (size_t dw = 0; dw < (size_t)kk * h->Twp; ++dw)
        for (int jz = 0; jz < h->nJc; ++jz) {
            uint8_t msk = 0;
            for (int q = 0; q < 4; ++q)
                for (int i = 0; i < 8; ++i)
                    if (Ka[dw * h->Zp + jz * JCHUNK + 8 * q + i] != 0.f) msk |= (uint8_t)(1u << q);
            am[dw * h->nJc + jz] = msk;
        }
    std::vector<float> Smf(h->Sm64.begin(), h->Sm64.end());
    std::vector<float> Cmf(h->Cm.begin(), h->Cm.end());

    swopt_status s = SWOPT_OK;
    auto step = [&](swopt_status v) { if (s == SWOPT_OK) s = v; };
    step(dalloc(&h->Kf, Kf.size()));
    step(dalloc(&h->Ka, Ka.size()));
    step(dalloc(&h->fmask, fm.size()));
    step(dalloc(&h->amask, am.size()));
    step(dalloc(&h->Sm, Smf.size()));
    step(dalloc(&h->Cmf, Cmf.size()));
    step(dalloc(&h->b, nb_of(h)));
    step(dalloc(&h->u, nu_of(h)));
    step(dalloc(&h->g, nb_of(h)));
    h->red_cap = std::max({4096, simt_forward_blocks(h) + 64, tc_forward_blocks(h) + 64,
                           h->Q * h->P * h->Z + 64});
    step(dalloc(&h->red, (size_t)h->red_cap));
    step(dalloc(&h->scal, (size_t)SC_COUNT));
    if (s == SWOPT_OK) {
        cudaError_t e = cudaMallocHost((void**)&h->scal_host, SC_COUNT * sizeof(double));
        if (e != cudaSuccess) {
            set_error("cudaMallocHost failed: %s", cudaGetErrorString(e));
            s = SWOPT_ERR_OOM;
        }
    }
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (s != SWOPT_OK) return;
        cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            set_error("cudaMemcpy failed: %s", cudaGetErrorString(e));
            s = SWOPT_ERR_CUDA;
        }
    };
    up(h->Kf, Kf.data(), Kf.size() * sizeof(float));
    up(h->Ka, Ka.data(), Ka.size() * sizeof(float));
    up(h->fmask, fm.data(), fm.size());
    up(h->amask, am.data(), am.size());
    up(h->Sm, Smf.data(), Smf.size() * sizeof(float));
    up(h->Cmf, Cmf.data(), Cmf.size() * sizeof(float));
    if (s == SWOPT_OK) {
        cudaError_t e = cudaMemset(h->scal, 0, SC_COUNT * sizeof(double));
        if (e != cudaSuccess) {
            set_error("cudaMemset failed: %s", cudaGetErrorString(e));
            s = SWOPT_ERR_CUDA;
        }
    }
    if (s != SWOPT_OK) {
        release_all(h);
        delete h;
        return s;
    }
    *out = h;
    return SWOPT_OK;
}

swopt_status swopt_destroy(swopt_handle* h)
{
    clear_error();
    if (!h) return SWOPT_OK;
    release_all(h);
    delete h;
    return SWOPT_OK;
}

swopt_status swopt_set_precision(swopt_handle* h, int precision)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (precision < SWOPT_PREC_FP32 || precision > SWOPT_PREC_BF16X6) {
        set_error("unknown precision %d", precision);
        return SWOPT_ERR_INVALID_ARG;
    }
    release_graph(h);
    release_ref(h);
    if (precision != SWOPT_PREC_FP32) {
        const int prev = h->precision;
        h->precision = precision;
        swopt_status s = tc_prepare(h);
        if (s != SWOPT_OK) {
            h->precision = prev;
            return s;
        }
    }
    h->precision = precision;
    return SWOPT_OK;
}

swopt_status swopt_forward(swopt_handle* h, const float* c_dev, float* y_dev, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !y_dev) {
        set_error("null c or y");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    SW_TRY(apply_A(h, c_dev, A_OUT_U, nullptr, nullptr, 0, st));
    return launch_expand(h, h->u, y_dev, st);
}

swopt_status swopt_adjoint(swopt_handle* h, const float* y_dev, float* c_dev, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !y_dev) {
        set_error("null c or y");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    SW_TRY(launch_fold(h, y_dev, h->u, st));
    SW_TRY(apply_AT(h, true, st));
    return launch_pt(h, h->g, nullptr, 0.f, c_dev, 0, st);
}

swopt_status swopt_prox_l1(swopt_handle* h, float* x_dev, float thresh, int nonneg, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!x_dev || !std::isfinite(thresh) || thresh < 0) {
        set_error("null x or invalid threshold");
        return SWOPT_ERR_INVALID_ARG;
    }
    return prox_l1(h, x_dev, thresh, nonneg, (cudaStream_t)stream);
}

swopt_status swopt_prox_tv(swopt_handle* h, const float* z_dev, float* x_dev, float tau,
                           int inner_iters, int momentum, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!z_dev || !x_dev || z_dev == x_dev || !std::isfinite(tau) || tau < 0 || inner_iters < 0 ||
        inner_iters > 1000000 || momentum < 0 || momentum > 2) {
        set_error("invalid prox_tv arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (inner_iters == 0) {
        SW_CUDA(cudaMemcpyAsync(x_dev, z_dev, nc_of(h) * sizeof(float), cudaMemcpyDeviceToDevice,
                                st));
        return SWOPT_OK;
    }
    SW_TRY(ensure_tv_buffers(h));
    return prox_tv_coop(h, z_dev, tau, inner_iters, momentum, x_dev, st);
}

swopt_status swopt_lipschitz(swopt_handle* h, const float* v0_dev, int iters, double* L_out,
                             void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!L_out || iters < 1 || iters > 1000000) {
        set_error("invalid lipschitz arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    return lipschitz_impl(h, v0_dev, iters, L_out, (cudaStream_t)stream);
}

swopt_status swopt_fista_init(swopt_handle* h, const float* y_dev, const swopt_solve_params* prm,
                              void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!y_dev) {
        set_error("null y");
        return SWOPT_ERR_INVALID_ARG;
    }
    return fista_init_impl(h, y_dev, prm, (cudaStream_t)stream);
}

}  // extern "C"

namespace swopt {

// Helpers of the unrolled derivative (unrolled.cu).
swopt_status fista_iterate_once(swopt_handle* h, cudaStream_t st) { return run_iteration(h, st); }

swopt_status apply_forward_residual(swopt_handle* h, const float* v, const float* ytil,
                                    cudaStream_t st)
{
    return apply_A(h, v, A_OUT_R, ytil, nullptr, 1, st);
}

swopt_status apply_adjoint_folded(swopt_handle* h, cudaStream_t st)
{
    return apply_AT(h, false, st);
}

void chain_rule(const swopt_handle* h, const std::vector<double>& W, double* dkappa, double* dmu)
{
    switching_chain_rule(h, W, dkappa, dmu);
}

swopt_status fista_init_impl(swopt_handle* h, const float* y_dev, const swopt_solve_params* prm,
                             cudaStream_t st)
{
    SW_TRY(validate_params(prm));
    h->fista_ready = false;
    release_graph(h);
    SW_TRY(ensure_vectors(h));
    SW_TRY(ensure_ytil(h));
    if (prm->lambda_3 > 0) {
        if (h->P > 8) {
            set_error("lambda_3 > 0 supports at most 8 species");
            return SWOPT_ERR_UNSUPPORTED;
        }
        SW_TRY(ensure_joint_buffers(h));
        const double bound = joint_step_bound(h, prm->lambda_tv, prm->lambda_l1, prm->lambda_3);
        h->jstep2 = prm->joint_step2 > 0 ? prm->joint_step2 : 1.0 / bound;
    } else if (prm->lambda_tv > 0 && prm->inner_iters > 0) {
        SW_TRY(ensure_tv_buffers(h));
    }
    h->prm = *prm;
    SW_TRY(launch_fold(h, y_dev, h->ytil, st));
    SW_TRY(reduce_sumsq(h, y_dev, (size_t)h->N * h->S * h->T, SC_YSQ, st));
    if (prm->step > 0) {
        h->step = prm->step;
    } else {
        double L = 0.0;
        SW_TRY(lipschitz_impl(h, nullptr, prm->power_iters, &L, st));
        if (!(L > 0) || !std::isfinite(L)) {
            set_error("power iteration gave a non-positive estimate %g", L);
            return SWOPT_ERR_DEVICE_CHECK;
        }
        h->step = 1.0 / L;
    }
    SW_CUDA(cudaMemsetAsync(h->c, 0, nc_of(h) * sizeof(float), st));
    SW_CUDA(cudaMemsetAsync(h->xi, 0, nc_of(h) * sizeof(float), st));
    SW_TRY(fista_reset_scalars(h, st));
    h->iter = 0;
    h->resyncs = prm->refine_every > 0 ? 1 : 0;
    if (prm->refine_every > 0 && prm->refine_budget > 0) {
        if (!h->sched) SW_TRY(dalloc(&h->sched, 4));
        if (!h->rlog) SW_TRY(dalloc(&h->rlog, (size_t)kRefineLog));
        SW_CUDA(cudaMemsetAsync(h->sched, 0, 4 * sizeof(int), st));
        SW_CUDA(cudaMemsetAsync(h->rlog, 0xff, (size_t)kRefineLog * sizeof(int), st));
        SW_CUDA(cudaMemsetAsync(h->scal + SC_BUDGET, 0, sizeof(double), st));
    }
    if (prm->refine_every > 0) {
        // gradient at c_0 = 0 and the first prox input, at the resync precision
        if (!h->G) SW_TRY(dalloc(&h->G, nc_of(h)));
        SW_CUDA(cudaMemsetAsync(h->G, 0, nc_of(h) * sizeof(float), st));
        SW_TRY(ensure_ref(h));
        SW_TRY(exact_gradient(h, st));
    }
    h->fista_ready = true;
    return SWOPT_OK;
}

}  // namespace swopt

extern "C" {

swopt_status swopt_fista_step(swopt_handle* h, int iters, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!h->fista_ready) {
        set_error("swopt_fista_init has not been called");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (iters < 0) {
        set_error("negative iteration count");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < iters; ++i) SW_TRY(run_iteration(h, st));
    return SWOPT_OK;
}

swopt_status swopt_fista_get(swopt_handle* h, float* c_dev, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !h->fista_ready) {
        set_error("null c or no FISTA state");
        return SWOPT_ERR_INVALID_ARG;
    }
    SW_CUDA(cudaMemcpyAsync(c_dev, h->c, nc_of(h) * sizeof(float), cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return SWOPT_OK;
}

swopt_status swopt_fista_gradient(swopt_handle* h, const float* carry_dev, float* g_dev,
                                  void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!g_dev || !h->fista_ready || h->prm.refine_every > 0) {
        set_error("null gradient output, no FISTA state, or a refined solve");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    SW_TRY(apply_A(h, h->xi, A_OUT_R, h->ytil, nullptr, 1, st));
    SW_TRY(apply_AT(h, false, st));
    return launch_pt_carry(h, h->g, carry_dev, g_dev, st);
}

swopt_status swopt_fista_step_external(swopt_handle* h, const float* g_dev, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!g_dev || !h->fista_ready || h->prm.refine_every > 0) {
        set_error("null gradient, no FISTA state, or a refined solve");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    SW_TRY(launch_grad_step(h, g_dev, h->xi, (float)h->step, h->zin, st));
    SW_TRY(fista_prox_momentum(h, false, st));
    ++h->iter;
    return SWOPT_OK;
}

swopt_status swopt_set_fluence(swopt_handle* h, const double* phi_host)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (phi_host)
        for (int j = 0; j < h->Z; ++j)
            if (!std::isfinite(phi_host[j]) || phi_host[j] < 0) {
                set_error("the fluence must be finite and >= 0");
                return SWOPT_ERR_INVALID_ARG;
            }
    SW_CUDA(cudaDeviceSynchronize());
    h->phi_fixed = phi_host != nullptr;
    if (phi_host) h->phi.assign(phi_host, phi_host + h->Z);
    switching_states(h);
    std::vector<float> Smf(h->Sm64.begin(), h->Sm64.end());
    SW_CUDA(cudaMemcpy(h->Sm, Smf.data(), Smf.size() * sizeof(float), cudaMemcpyHostToDevice));
    return SWOPT_OK;
}

swopt_status swopt_set_state_offset(swopt_handle* h, int offset)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (offset < 0) {
        set_error("negative state offset");
        return SWOPT_ERR_INVALID_ARG;
    }
    SW_CUDA(cudaDeviceSynchronize());
    h->state_offset = offset;
    switching_states(h);
    std::vector<float> Smf(h->Sm64.begin(), h->Sm64.end());
    SW_CUDA(cudaMemcpy(h->Sm, Smf.data(), Smf.size() * sizeof(float), cudaMemcpyHostToDevice));
    return SWOPT_OK;
}

swopt_status swopt_refine_stats(swopt_handle* h, int64_t* iterations, int64_t* resyncs,
                                void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!iterations || !resyncs || !h->fista_ready) {
        set_error("null output or no FISTA state");
        return SWOPT_ERR_INVALID_ARG;
    }
    *iterations = h->iter;
    *resyncs = h->resyncs;
    if (iteration_kind(h) == 2) {
        int sc[4] = {0, 0, 0, 0};
        cudaStream_t st = (cudaStream_t)stream;
        SW_CUDA(cudaMemcpyAsync(sc, h->sched, sizeof(sc), cudaMemcpyDeviceToHost, st));
        SW_CUDA(cudaStreamSynchronize(st));
        *resyncs = 1 + (int64_t)sc[2];  // the initial exact gradient and the device's
    }
    return SWOPT_OK;
}

namespace {

// Host image of the FISTA state (swopt_fista_save / swopt_fista_restore).
struct FistaStateHeader {
    uint64_t magic;
    int32_t version, P, Y, X, Z, N, refine_every, refined, gated;
    int32_t inner_iters, momentum, inner_momentum, refine_precision;
    double step, lambda_l1, lambda_tv, refine_budget, lambda_3, joint_step2;
    int64_t iter, resyncs;
};
constexpr uint64_t kStateMagic = 0x5357'4F50'5446'5354ull;  // "SWOPTFST"

size_t fista_state_size(const swopt_handle* h)
{
    const size_t n = nc_of(h);
    const bool refined = h->prm.refine_every > 0;
    return sizeof(FistaStateHeader) + (refined ? 4 : 3) * n * sizeof(float) +
           SC_COUNT * sizeof(double) + 4 * sizeof(int);
}

}  // namespace

swopt_status swopt_fista_state_bytes(swopt_handle* h, size_t* bytes)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!bytes || !h->fista_ready) {
        set_error("null output or no FISTA state");
        return SWOPT_ERR_INVALID_ARG;
    }
    *bytes = fista_state_size(h);
    return SWOPT_OK;
}

swopt_status swopt_fista_save(swopt_handle* h, void* host_buf, size_t bytes, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!host_buf || !h->fista_ready || bytes < fista_state_size(h)) {
        set_error("null buffer, no FISTA state, or a buffer below swopt_fista_state_bytes");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = nc_of(h);
    FistaStateHeader hd{};
    hd.magic = kStateMagic;
    hd.version = 2;
    hd.P = h->P; hd.Y = h->Y; hd.X = h->X; hd.Z = h->Z; hd.N = h->N;
    hd.refine_every = h->prm.refine_every;
    hd.refined = h->prm.refine_every > 0;
    hd.gated = iteration_kind(h) == 2;
    hd.inner_iters = h->prm.inner_iters;
    hd.momentum = h->prm.momentum;
    hd.inner_momentum = h->prm.inner_momentum;
    hd.refine_precision = h->prm.refine_precision;
    hd.step = h->step;
    hd.lambda_l1 = h->prm.lambda_l1;
    hd.lambda_tv = h->prm.lambda_tv;
    hd.refine_budget = h->prm.refine_budget;
    hd.lambda_3 = h->prm.lambda_3;
    hd.joint_step2 = h->prm.lambda_3 > 0 ? h->jstep2 : 0.0;
    hd.iter = h->iter;
    hd.resyncs = h->resyncs;
    uint8_t* p = static_cast<uint8_t*>(host_buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const float* vecs[4] = {h->c, h->xi, h->zin, h->G};
    for (int v = 0; v < (hd.refined ? 4 : 3); ++v) {
        SW_CUDA(cudaMemcpyAsync(p, vecs[v], n * sizeof(float), cudaMemcpyDeviceToHost, st));
        p += n * sizeof(float);
    }
    SW_CUDA(cudaMemcpyAsync(p, h->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    p += SC_COUNT * sizeof(double);
    if (hd.gated) SW_CUDA(cudaMemcpyAsync(p, h->sched, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    else std::memset(p, 0, 4 * sizeof(int));
    SW_CUDA(cudaStreamSynchronize(st));
    return device_errors(h);
}

swopt_status swopt_fista_restore(swopt_handle* h, const void* host_buf, size_t bytes,
                                 void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!host_buf || !h->fista_ready || bytes < fista_state_size(h)) {
        set_error("null buffer, no FISTA state (call swopt_fista_init first), or a buffer "
                  "below swopt_fista_state_bytes");
        return SWOPT_ERR_INVALID_ARG;
    }
    FistaStateHeader hd;
    std::memcpy(&hd, host_buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.version != 2 || hd.P != h->P || hd.Y != h->Y ||
        hd.X != h->X || hd.Z != h->Z || hd.N != h->N ||
        hd.refine_every != h->prm.refine_every || hd.gated != (iteration_kind(h) == 2) ||
        hd.inner_iters != h->prm.inner_iters || hd.momentum != h->prm.momentum ||
        hd.inner_momentum != h->prm.inner_momentum ||
        hd.refine_precision != h->prm.refine_precision || hd.lambda_l1 != h->prm.lambda_l1 ||
        hd.lambda_tv != h->prm.lambda_tv || hd.refine_budget != h->prm.refine_budget ||
        hd.lambda_3 != h->prm.lambda_3 ||
        hd.joint_step2 != (h->prm.lambda_3 > 0 ? h->jstep2 : 0.0) || !(hd.step > 0) ||
        hd.iter < 0) {
        set_error("the saved FISTA state belongs to another geometry or other settings");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = nc_of(h);
    if (hd.refined && !h->G) SW_TRY(dalloc(&h->G, n));
    const uint8_t* p = static_cast<const uint8_t*>(host_buf) + sizeof(hd);
    float* vecs[4] = {h->c, h->xi, h->zin, h->G};
    for (int v = 0; v < (hd.refined ? 4 : 3); ++v) {
        SW_CUDA(cudaMemcpyAsync(vecs[v], p, n * sizeof(float), cudaMemcpyHostToDevice, st));
        p += n * sizeof(float);
    }
    SW_CUDA(cudaMemcpyAsync(h->scal, p, SC_COUNT * sizeof(double), cudaMemcpyHostToDevice, st));
    p += SC_COUNT * sizeof(double);
    if (hd.gated) SW_CUDA(cudaMemcpyAsync(h->sched, p, 4 * sizeof(int), cudaMemcpyHostToDevice, st));
    SW_CUDA(cudaStreamSynchronize(st));
    // the step is baked into captured iterations: capture again
    release_graph(h);
    h->step = hd.step;
    h->iter = hd.iter;
    h->resyncs = hd.resyncs;
    return SWOPT_OK;
}

swopt_status swopt_debug_barrier(swopt_handle* h, int phantom_arrivals, unsigned poll_limit)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (phantom_arrivals < 0 || phantom_arrivals > 1024) {
        set_error("phantom_arrivals must be in [0, 1024]");
        return SWOPT_ERR_INVALID_ARG;
    }
    SW_TRY(coop_debug(h, (unsigned)phantom_arrivals, poll_limit));
    SW_CUDA(cudaDeviceSynchronize());
    return SWOPT_OK;
}

swopt_status swopt_solve(swopt_handle* h, const float* y_dev, float* c_dev,
                         const swopt_solve_params* prm, swopt_solve_stats* stats, void* stream)
{
    SW_TRY(swopt_fista_init(h, y_dev, prm, stream));
    cudaStream_t st = (cudaStream_t)stream;
    const bool tests = prm->eps1 > 0 || prm->eps2 > 0 || prm->history_host;
    int it = 0;
    double f_prev = INFINITY;
    for (; it < prm->max_iters; ++it) {
        if (tests && prm->eps2 > 0) {
            if (!h->xprev) SW_TRY(dalloc(&h->xprev, nc_of(h)));
            SW_CUDA(cudaMemcpyAsync(h->xprev, h->xi, nc_of(h) * sizeof(float),
                                    cudaMemcpyDeviceToDevice, st));
        }
        SW_TRY(run_iteration(h, st));
        if (!tests) continue;
        double F = 0.0;
        if (prm->eps1 > 0 || prm->history_host)
            SW_TRY(objective_impl(h, h->c, y_dev, prm->lambda_l1, prm->lambda_tv, prm->lambda_3,
                                  &F, nullptr, st));
        if (prm->history_host) prm->history_host[it] = F;
        bool stop = false;
        if (it >= 1 && prm->eps1 > 0 && std::fabs(F - f_prev) < prm->eps1 * std::fabs(f_prev))
            stop = true;
        if (it >= 1 && prm->eps2 > 0) {
            // ||xi_{k+1} - xi_k|| / ||xi_k||
            SW_TRY(reduce_sumsq(h, h->xprev, nc_of(h), SC_C, st));
            SW_TRY(reduce_sumsq(h, h->xi, nc_of(h), SC_D, st));
            SW_TRY(reduce_dot(h, h->xi, h->xprev, nc_of(h), SC_A, st));
            SW_TRY(read_scalars(h, st));
            const double a = h->scal_host[SC_D], b = h->scal_host[SC_C], ab = h->scal_host[SC_A];
            const double diff = std::sqrt(std::max(0.0, a + b - 2.0 * ab));
            if (b > 0 && diff < prm->eps2 * std::sqrt(b)) stop = true;
        }
        f_prev = F;
        if (stop) {
            ++it;
            break;
        }
    }
    SW_CUDA(cudaMemcpyAsync(c_dev, h->c, nc_of(h) * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (stats) {
        stats->iters = it;
        stats->step = h->step;
        SW_TRY(objective_impl(h, h->c, y_dev, prm->lambda_l1, prm->lambda_tv, prm->lambda_3,
                              &stats->objective,
                              &stats->data_fit, st));
    } else {
        SW_CUDA(cudaStreamSynchronize(st));
    }
    return SWOPT_OK;
}

// The two-step approach (the paper's "Two-Step Approach"): first the acoustic
// problem of Eq. (acoustic-inverse), which separates over the pulses because
// W_tot is block diagonal, solved pulse by pulse on one handle whose
// switching model is the identity (one species, no switching, no fluence
// decay), then the unmixing problem of Eq. (unmixing) on a handle whose
// acoustic kernel is the identity (k = 1, T = Z, K[j][0][0][t] = [t = j]), so
// that its forward operator is S itself.  Both solves run Algorithm 1 with
// the caller's parameters (R1 = lambda_tv TV, R2 = lambda_l1 l1 + lambda_tv TV).
swopt_status swopt_two_step(const swopt_geometry* geom, const double* K_host,
                            const swopt_switching* sw, const float* y_dev, float* b_dev,
                            float* c_dev, const swopt_solve_params* acoustic,
                            const swopt_solve_params* unmixing, void* stream)
{
    clear_error();
    if (!geom || !K_host || !sw || !y_dev || !b_dev || !c_dev || !acoustic || !unmixing) {
        set_error("null argument");
        return SWOPT_ERR_INVALID_ARG;
    }
    auto keep_error = [](swopt_status s, swopt_handle* h) {
        char msg[sizeof(g_err)];
        std::snprintf(msg, sizeof(msg), "%s", g_err);
        swopt_destroy(h);
        if (s != SWOPT_OK) set_error("%s", msg);
        return s;
    };
    // step 1: per pulse, H = W (one species with weight 1 at every depth)
    swopt_geometry g1 = *geom;
    g1.N = 1;
    g1.P = 1;
    g1.pulses_per_cycle = 1;
    const double zero = 0.0, one = 1.0;
    const swopt_switching s1 = {&zero, &zero, &one, 0.0};
    swopt_handle* h1 = nullptr;
    SW_TRY(swopt_create(&g1, K_host, &s1, &h1));
    const size_t yxt = (size_t)geom->Y * geom->X * geom->T;
    const size_t yxz = (size_t)geom->Y * geom->X * geom->Z;
    swopt_status s = SWOPT_OK;
    for (int n = 0; n < geom->N && s == SWOPT_OK; ++n)
        s = swopt_solve(h1, y_dev + (size_t)n * yxt, b_dev + (size_t)n * yxz, acoustic, nullptr,
                        stream);
    SW_TRY(keep_error(s, h1));
    // step 2: H = S (identity acoustic kernel; b is read as the data [N][Y][X][T = Z])
    swopt_geometry g2 = *geom;
    g2.T = geom->Z;
    g2.k = 1;
    std::vector<double> eye((size_t)geom->Z * geom->Z, 0.0);
    for (int j = 0; j < geom->Z; ++j) eye[(size_t)j * geom->Z + j] = 1.0;
    swopt_handle* h2 = nullptr;
    SW_TRY(swopt_create(&g2, eye.data(), sw, &h2));
    s = swopt_solve(h2, b_dev, c_dev, unmixing, nullptr, stream);
    return keep_error(s, h2);
}

swopt_status swopt_objective(swopt_handle* h, const float* c_dev, const float* y_dev,
                             double lambda_l1, double lambda_tv, double lambda_3, double* F,
                             double* fit, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !y_dev || !is_fin(lambda_l1) || !is_fin(lambda_tv) || !is_fin(lambda_3)) {
        set_error("invalid objective arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    return objective_impl(h, c_dev, y_dev, lambda_l1, lambda_tv, lambda_3, F, fit,
                          (cudaStream_t)stream);
}

swopt_status swopt_param_grad(swopt_handle* h, const float* c_dev, const float* y_dev,
                              double* dkappa_host, double* dmu, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !y_dev || !dkappa_host || !dmu) {
        set_error("null argument");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // residual folded over equal states: C_m (A P c)_m - sum_{n=m mod cycle} y_n
    float* yt = nullptr;
    SW_TRY(dalloc(&yt, nu_of(h)));
    swopt_status s = launch_fold(h, y_dev, yt, st);
    if (s == SWOPT_OK) s = apply_A(h, c_dev, A_OUT_R, yt, nullptr, 1, st);
    if (s == SWOPT_OK) s = apply_AT(h, false, st);
    if (s == SWOPT_OK) s = switching_gradient(h, c_dev, dkappa_host, dmu, st);
    cudaFree(yt);
    return s;
}

swopt_status swopt_param_vjp(swopt_handle* h, const float* c_dev, const float* w_dev,
                             double* dkappa_host, double* dmu, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!c_dev || !w_dev || !dkappa_host || !dmu) {
        set_error("null argument");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // <w, dH/dtheta c> = sum_m <A^T w~_m, dS_m/dtheta c>, w~ the cotangent
    // folded over pulses of equal state (H c vanishes outside the window)
    SW_TRY(launch_fold(h, w_dev, h->u, st));
    SW_TRY(apply_AT(h, true, st));
    return switching_gradient(h, c_dev, dkappa_host, dmu, st);
}

swopt_status swopt_set_switching(swopt_handle* h, const swopt_switching* sw)
{
    clear_error();
    SW_TRY(check_handle(h));
    SW_TRY(check_switching(sw, h->P));
    SW_CUDA(cudaDeviceSynchronize());
    h->mu = sw->mu_per_mm;
    h->kappa.assign(sw->kappa_host, sw->kappa_host + h->P);
    h->eps_bar.assign(sw->eps_bar_host, sw->eps_bar_host + h->P);
    h->eps_off.assign(sw->eps_off_host, sw->eps_off_host + h->P);
    switching_states(h);
    std::vector<float> Smf(h->Sm64.begin(), h->Sm64.end());
    SW_CUDA(cudaMemcpy(h->Sm, Smf.data(), Smf.size() * sizeof(float), cudaMemcpyHostToDevice));
    return SWOPT_OK;
}

swopt_status swopt_use_graphs(swopt_handle* h, int on)
{
    clear_error();
    SW_TRY(check_handle(h));
    h->use_graph = on != 0;
    release_graph(h);
    return SWOPT_OK;
}

swopt_status swopt_profile_enable(swopt_handle* h, int on)
{
    clear_error();
    SW_TRY(check_handle(h));
    h->profile = on != 0;
    return SWOPT_OK;
}

swopt_status swopt_profile_read(swopt_handle* h, int kernel_id, double* total_ms,
                                int64_t* launches, double* flops_per_launch)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (kernel_id < 0 || kernel_id > 3) {
        set_error("kernel_id must be 0 (A), 1 (A^T), 2 or 3 (A, A^T at the resync precision)");
        return SWOPT_ERR_INVALID_ARG;
    }
    // launches behind the refined solve's gate count only where the device
    // decided for their branch (ids 0/1: the increment, 2/3: the exact
    // gradient), read from the decision log
    std::vector<int> dlog;
    for (auto& r : h->prof) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) {
            set_error("cudaEventSynchronize failed: %s", cudaGetErrorString(e));
            return SWOPT_ERR_CUDA;
        }
        bool ran = true;
        if (r.iter >= 0) {
            if (dlog.empty()) {
                if (!h->rlog) {
                    set_error("internal: gated launch without a decision log");
                    return SWOPT_ERR_DEVICE_CHECK;
                }
                dlog.resize(kRefineLog);
                SW_CUDA(cudaMemcpy(dlog.data(), h->rlog, kRefineLog * sizeof(int),
                                   cudaMemcpyDeviceToHost));
            }
            const int d = dlog[(size_t)(r.iter & (kRefineLog - 1))];
            ran = d == (r.kernel >= 2 ? 1 : 0);
        }
        if (ran) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, r.a, r.b);
            h->prof_ms[r.kernel] += ms;
            h->prof_n[r.kernel] += 1;
        }
        h->event_pool.push_back(r.a);
        h->event_pool.push_back(r.b);
    }
    h->prof.clear();
    if (total_ms) *total_ms = h->prof_ms[kernel_id];
    if (launches) *launches = h->prof_n[kernel_id];
    if (flops_per_launch) *flops_per_launch = 2.0 * (double)h->Q * h->S * (double)h->nnz;
    h->prof_ms[kernel_id] = 0;
    h->prof_n[kernel_id] = 0;
    return SWOPT_OK;
}

swopt_status swopt_check_device(swopt_handle* h, void* stream)
{
    clear_error();
    SW_TRY(check_handle(h));
    SW_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return device_errors(h);
}

swopt_status swopt_issued_flops(swopt_handle* h, int kernel_id, double* flops)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!flops || kernel_id < 0 || kernel_id > 1) {
        set_error("invalid arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (use_tc(h)) {
        *flops = 2.0 * tc_issued_macs(h, kernel_id);
        return SWOPT_OK;
    }
    // FP32 kernels: every nonzero 8-sample (8-depth) sub-block is issued for
    // every position of every state
    std::vector<uint8_t> m(kernel_id == 0 ? (size_t)h->Z * h->k * h->k * h->nTc
                                          : (size_t)h->k * h->k * h->Twp * h->nJc);
    SW_CUDA(cudaMemcpy(m.data(), kernel_id == 0 ? h->fmask : h->amask, m.size(),
                       cudaMemcpyDeviceToHost));
    double blocks = 0;
    for (uint8_t v : m) blocks += __builtin_popcount(v);
    *flops = 2.0 * blocks * 8.0 * (double)h->S * h->Q;
    return SWOPT_OK;
}

swopt_status swopt_tc_configure(swopt_handle* h, int kernel_id, int tiles_per_cta,
                                int ctas_per_sm, int accumulators)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (kernel_id < 0 || kernel_id > 1 || tiles_per_cta < 0 || tiles_per_cta > 4 ||
        tiles_per_cta == 3 || ctas_per_sm < 0 || ctas_per_sm > 2 || accumulators < 0 ||
        accumulators > 2) {
        set_error("invalid tensor-core configuration");
        return SWOPT_ERR_INVALID_ARG;
    }
    release_graph(h);
    h->tc_force_mt[kernel_id] = tiles_per_cta;
    h->tc_force_ctas[kernel_id] = ctas_per_sm;
    h->tc_force_ra[kernel_id] = accumulators;
    release_ref(h);
    if (h->tc) {
        tc_release(h);
        if (use_tc(h)) return tc_prepare(h);
    }
    return SWOPT_OK;
}

swopt_status swopt_tc_config(swopt_handle* h, int kernel_id, int* tiles_per_cta,
                             int* ctas_per_sm, int* stages, int* groups, int* accumulators)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (kernel_id < 0 || kernel_id > 1 || !tiles_per_cta || !ctas_per_sm || !stages || !groups ||
        !accumulators) {
        set_error("invalid arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!h->tc) {
        set_error("no tensor-core precision selected");
        return SWOPT_ERR_INVALID_ARG;
    }
    tc_config(h, kernel_id, tiles_per_cta, ctas_per_sm, stages, groups, accumulators);
    return SWOPT_OK;
}

swopt_status swopt_tc_schedule(swopt_handle* h, int kernel_id, int split, int buffers)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (kernel_id < 0 || kernel_id > 1 || split < 0 || split > 2 || buffers < 0 || buffers > 2) {
        set_error("invalid tensor-core schedule");
        return SWOPT_ERR_INVALID_ARG;
    }
    release_graph(h);
    h->tc_force_split[kernel_id] = split;
    h->tc_force_nbuf[kernel_id] = buffers;
    release_ref(h);
    if (h->tc) {
        tc_release(h);
        if (use_tc(h)) return tc_prepare(h);
    }
    return SWOPT_OK;
}

swopt_status swopt_tc_schedule_info(swopt_handle* h, int kernel_id, int* split, int* buffers,
                                    int* grid, int* max_pieces)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (kernel_id < 0 || kernel_id > 1 || !split || !buffers || !grid || !max_pieces) {
        set_error("invalid arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (!h->tc) {
        set_error("no tensor-core precision selected");
        return SWOPT_ERR_INVALID_ARG;
    }
    tc_schedule_info(h, kernel_id, split, buffers, grid, max_pieces);
    return SWOPT_OK;
}

swopt_status swopt_launch_count(swopt_handle* h, int64_t* count)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (!count) {
        set_error("null count");
        return SWOPT_ERR_INVALID_ARG;
    }
    *count = h->launches;
    return SWOPT_OK;
}

swopt_status swopt_info(swopt_handle* h, int* t0, int* tw, int* states, int64_t* kernel_nnz)
{
    clear_error();
    SW_TRY(check_handle(h));
    if (t0) *t0 = h->t0;
    if (tw) *tw = h->tw;
    if (states) *states = h->Q;
    if (kernel_nnz) *kernel_nnz = h->nnz;
    return SWOPT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched problems: one CUDA graph per iteration kind holds one FISTA
// iteration of every handle, each on its own forked stream, so that problems
// of uneven size run concurrently.
// ---------------------------------------------------------------------------
struct swopt_batch {
    std::vector<swopt_handle*> hs;
    std::vector<cudaStream_t> streams;  // one per problem (capture only)
    std::vector<cudaEvent_t> events;    // fork / join
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
    std::vector<uint64_t> gen;          // handle graph generations at capture
    int64_t kernels[3] = {0, 0, 0};
    int64_t iter = 0;
    bool shared = false;                // contractions as shared launches over all problems
    bool shared_used[3] = {false, false, false};
    int contraction_launches[3] = {0, 0, 0};  // per iteration of a captured kind
    std::vector<swopt::TcMulti*> multi; // the shared launches of the captured graphs
};

namespace {

void batch_release_graphs(swopt_batch* b)
{
    for (auto& g : b->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    for (auto* m : b->multi) tc_multi_destroy(m);
    b->multi.clear();
}

// Prepares one shared launch of A (adj false) or A^T over the batch, with every
// handle inside a gate (want >= 0) and / or at its resync precision (ref).
swopt_status batch_multi(swopt_batch* b, bool adj, bool ytil, int want, bool ref, TcMulti** out)
{
    std::vector<std::unique_ptr<GateScope>> gs;
    std::vector<std::unique_ptr<RefScope>> rs;
    for (swopt_handle* h : b->hs) {
        if (want >= 0) gs.emplace_back(new GateScope(h, want));
        if (ref) rs.emplace_back(new RefScope(h, h->prm.refine_precision));
    }
    const swopt_status s = tc_multi_create(b->hs.data(), (int)b->hs.size(), adj, ytil, out);
    if (s == SWOPT_OK) b->multi.push_back(*out);
    return s;
}

// One FISTA iteration of every problem (kind as iteration_kind) with the
// contractions of all problems in shared persistent launches (one for A, one
// for A^T, per gradient path) and the other steps launched per problem, all on
// st; the same arithmetic as fista_iteration per handle.
swopt_status batch_iteration_shared(swopt_batch* b, int kind, TcMulti* const* m, cudaStream_t st)
{
    const bool refined = b->hs[0]->prm.refine_every > 0;
    if (!refined) {
        for (swopt_handle* h : b->hs) SW_TRY(tc_states(h, h->xi, st));
        SW_TRY(tc_multi_launch(m[0], st));
        SW_TRY(tc_multi_launch(m[1], st));
        for (swopt_handle* h : b->hs) SW_TRY(launch_pt(h, h->g, h->xi, (float)h->step, h->zin, 1, st));
        for (swopt_handle* h : b->hs) SW_TRY(fista_prox_momentum(h, false, st));
        return SWOPT_OK;
    }
    for (swopt_handle* h : b->hs) SW_TRY(fista_prox_momentum(h, true, st));
    if (kind == 2)
        for (swopt_handle* h : b->hs)
            SW_TRY(refine_decide(h, h->tmp, h->c, SC_BUDGET, h->prm.refine_every,
                                 h->prm.refine_budget, st));
    if (kind == 0 || kind == 2) {  // the increment
        const int want = kind == 2 ? 0 : -1;
        for (swopt_handle* h : b->hs) {
            std::unique_ptr<GateScope> g(want >= 0 ? new GateScope(h, want) : nullptr);
            SW_TRY(tc_states(h, h->tmp, st));
        }
        SW_TRY(tc_multi_launch(m[0], st));
        SW_TRY(tc_multi_launch(m[1], st));
        for (swopt_handle* h : b->hs) {
            std::unique_ptr<GateScope> g(want >= 0 ? new GateScope(h, want) : nullptr);
            SW_TRY(launch_pt_refine(h, h->g, h->xi, (float)h->step, h->G, h->zin, 1, st));
        }
    }
    if (kind == 1 || kind == 2) {  // the exact gradient at the resync precision
        const int want = kind == 2 ? 1 : -1;
        for (swopt_handle* h : b->hs) {
            std::unique_ptr<GateScope> g(want >= 0 ? new GateScope(h, want) : nullptr);
            RefScope r(h, h->prm.refine_precision);
            SW_TRY(tc_states(h, h->c, st));
        }
        SW_TRY(tc_multi_launch(m[2], st));
        SW_TRY(tc_multi_launch(m[3], st));
        for (swopt_handle* h : b->hs) {
            std::unique_ptr<GateScope> g(want >= 0 ? new GateScope(h, want) : nullptr);
            SW_TRY(launch_pt_refine(h, h->g, h->xi, (float)h->step, h->G, h->zin, 0, st));
        }
    }
    return SWOPT_OK;
}

// Captures kind `kind` with shared contraction launches; UNSUPPORTED (nothing
// captured) when the problems cannot share them.
swopt_status batch_capture_shared(swopt_batch* b, int kind)
{
    for (swopt_handle* h : b->hs)
        if (!use_tc(h) || !h->tc) {
            set_error("shared launches need tensor-core precisions");
            return SWOPT_ERR_UNSUPPORTED;
        }
    const bool refined = b->hs[0]->prm.refine_every > 0;
    TcMulti* m[4] = {nullptr, nullptr, nullptr, nullptr};
    const size_t keep = b->multi.size();
    auto undo = [&](swopt_status s) {
        while (b->multi.size() > keep) {
            tc_multi_destroy(b->multi.back());
            b->multi.pop_back();
        }
        return s;
    };
    swopt_status s = SWOPT_OK;
    if (!refined) {
        s = batch_multi(b, false, true, -1, false, &m[0]);
        if (s == SWOPT_OK) s = batch_multi(b, true, false, -1, false, &m[1]);
    } else {
        if (kind == 0 || kind == 2) {
            const int want = kind == 2 ? 0 : -1;
            s = batch_multi(b, false, false, want, false, &m[0]);
            if (s == SWOPT_OK) s = batch_multi(b, true, false, want, false, &m[1]);
        }
        if (s == SWOPT_OK && (kind == 1 || kind == 2)) {
            const int want = kind == 2 ? 1 : -1;
            s = batch_multi(b, false, true, want, true, &m[2]);
            if (s == SWOPT_OK) s = batch_multi(b, true, false, want, true, &m[3]);
        }
    }
    if (s != SWOPT_OK) return undo(s);
    const int n = (int)b->hs.size();
    std::vector<int64_t> l0(n);
    std::vector<bool> prof(n);
    for (int i = 0; i < n; ++i) {
        l0[i] = b->hs[i]->launches;
        prof[i] = b->hs[i]->profile;
        b->hs[i]->profile = false;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = batch_iteration_shared(b, kind, m, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
    }
    int64_t kernels = 0;
    for (int i = 0; i < n; ++i) {
        kernels += b->hs[i]->launches - l0[i];
        b->hs[i]->launches = l0[i];
        b->hs[i]->profile = prof[i];
    }
    if (s != SWOPT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (s == SWOPT_OK) {
            set_error("batch capture failed: %s", cudaGetErrorString(e));
            s = SWOPT_ERR_CUDA;
        }
        return undo(s == SWOPT_ERR_UNSUPPORTED ? SWOPT_ERR_CUDA : s);
    }
    e = cudaGraphInstantiate(&b->gexec[kind], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec[kind] = nullptr;
        set_error("batch graph instantiation failed: %s", cudaGetErrorString(e));
        return undo(SWOPT_ERR_CUDA);
    }
    b->kernels[kind] = kernels;
    b->shared_used[kind] = true;
    b->contraction_launches[kind] = 0;
    for (TcMulti* x : m)
        if (x) b->contraction_launches[kind] += tc_multi_groups(x);
    return SWOPT_OK;
}

swopt_status batch_capture(swopt_batch* b, int kind)
{
    const int n = (int)b->hs.size();
    std::vector<int64_t> l0(n);
    std::vector<bool> prof(n);
    for (int i = 0; i < n; ++i) {
        l0[i] = b->hs[i]->launches;
        prof[i] = b->hs[i]->profile;
        b->hs[i]->profile = false;  // no timing events inside the batch graph
    }
    swopt_status s = SWOPT_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < n && s == SWOPT_OK; ++i) {
            // fork: problem i's stream waits for the capture origin
            if (cudaEventRecord(b->events[2 * i], b->cap) != cudaSuccess ||
                cudaStreamWaitEvent(b->streams[i], b->events[2 * i], 0) != cudaSuccess) {
                set_error("batch capture: fork failed");
                s = SWOPT_ERR_CUDA;
                break;
            }
            s = fista_iteration(b->hs[i], kind, b->streams[i]);
            if (s == SWOPT_OK && (cudaEventRecord(b->events[2 * i + 1], b->streams[i]) !=
                                      cudaSuccess ||
                                  cudaStreamWaitEvent(b->cap, b->events[2 * i + 1], 0) !=
                                      cudaSuccess)) {
                set_error("batch capture: join failed");
                s = SWOPT_ERR_CUDA;
            }
        }
        e = cudaStreamEndCapture(b->cap, &g);
    }
    int64_t kernels = 0;
    for (int i = 0; i < n; ++i) {
        kernels += b->hs[i]->launches - l0[i];
        b->hs[i]->launches = l0[i];
        b->hs[i]->profile = prof[i];
    }
    if (s != SWOPT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (s == SWOPT_OK) {
            set_error("batch capture failed: %s", cudaGetErrorString(e));
            s = SWOPT_ERR_CUDA;
        }
        return s;
    }
    e = cudaGraphInstantiate(&b->gexec[kind], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->gexec[kind] = nullptr;
        set_error("batch graph instantiation failed: %s", cudaGetErrorString(e));
        return SWOPT_ERR_CUDA;
    }
    b->kernels[kind] = kernels;
    return SWOPT_OK;
}

}  // namespace

extern "C" {

swopt_status swopt_batch_create(swopt_handle* const* hs, int count, swopt_batch** out)
{
    clear_error();
    if (!out || !hs || count < 1 || count > 4096) {
        set_error("invalid batch arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        swopt_handle* h = hs[i];
        if (!h || !h->fista_ready) {
            set_error("batch handle %d is null or has no FISTA state (swopt_fista_init)", i);
            return SWOPT_ERR_INVALID_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (hs[j] == h) {
                set_error("batch handle %d repeats handle %d", i, j);
                return SWOPT_ERR_INVALID_ARG;
            }
        if (h->device != hs[0]->device || h->iter != hs[0]->iter ||
            h->prm.refine_every != hs[0]->prm.refine_every ||
            (h->prm.refine_budget > 0) != (hs[0]->prm.refine_budget > 0)) {
            set_error("batch handle %d differs from handle 0 in device, iteration count, "
                      "refine_every or the use of refine_budget", i);
            return SWOPT_ERR_INVALID_ARG;
        }
    }
    swopt_batch* b = new swopt_batch();
    b->hs.assign(hs, hs + count);
    b->iter = hs[0]->iter;
    swopt_status s = SWOPT_OK;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) s = SWOPT_ERR_CUDA;
    for (int i = 0; i < count && s == SWOPT_OK; ++i) {
        cudaStream_t st;
        cudaEvent_t e0, e1;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            s = SWOPT_ERR_CUDA;
            break;
        }
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
            s = SWOPT_ERR_CUDA;
            break;
        }
        b->events.push_back(e0);
        b->events.push_back(e1);
    }
    if (s != SWOPT_OK) {
        set_error("batch: stream or event creation failed");
        swopt_batch_destroy(b);
        return s;
    }
    *out = b;
    return SWOPT_OK;
}

swopt_status swopt_batch_step(swopt_batch* b, int iters, void* stream)
{
    clear_error();
    if (!b || iters < 0) {
        set_error("invalid batch arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int n = (int)b->hs.size();
    for (int i = 0; i < n; ++i)
        if (!b->hs[i]->fista_ready || b->hs[i]->iter != b->iter) {
            set_error("batch handle %d was re-initialised or stepped on its own; create a new "
                      "batch", i);
            return SWOPT_ERR_INVALID_ARG;
        }
    // captured work is stale if any handle's own graphs were discarded
    bool stale = b->gen.size() != (size_t)n;
    for (int i = 0; i < n && !stale; ++i) stale = b->gen[i] != b->hs[i]->graph_gen;
    if (stale) {
        batch_release_graphs(b);
        b->gen.resize(n);
        for (int i = 0; i < n; ++i) b->gen[i] = b->hs[i]->graph_gen;
    }
    for (int it = 0; it < iters; ++it) {
        for (int i = 0; i < n; ++i) SW_TRY(ensure_ref(b->hs[i]));
        const int kind = iteration_kind(b->hs[0]);
        if (!b->gexec[kind]) {
            swopt_status s = SWOPT_ERR_UNSUPPORTED;
            b->shared_used[kind] = false;
            if (b->shared) s = batch_capture_shared(b, kind);
            if (s == SWOPT_ERR_UNSUPPORTED) s = batch_capture(b, kind);
            SW_TRY(s);
        }
        SW_CUDA(cudaGraphLaunch(b->gexec[kind], st));
        for (int i = 0; i < n; ++i) {
            if (kind == 1) ++b->hs[i]->resyncs;
            ++b->hs[i]->iter;
        }
        b->hs[0]->launches += b->kernels[kind];  // counted once, on the first handle
        ++b->iter;
    }
    return SWOPT_OK;
}

swopt_status swopt_batch_configure(swopt_batch* b, int shared_launch)
{
    clear_error();
    if (!b) {
        set_error("null batch");
        return SWOPT_ERR_INVALID_ARG;
    }
    b->shared = shared_launch != 0;
    batch_release_graphs(b);
    return SWOPT_OK;
}

swopt_status swopt_batch_query(swopt_batch* b, int* shared_launch_in_use,
                               int* contraction_launches)
{
    clear_error();
    if (!b || !shared_launch_in_use) {
        set_error("null argument");
        return SWOPT_ERR_INVALID_ARG;
    }
    bool any = false, all = true;
    int most = 0;
    for (int k = 0; k < 3; ++k)
        if (b->gexec[k]) {
            any = true;
            all = all && b->shared_used[k];
            most = std::max(most, b->shared_used[k] ? b->contraction_launches[k]
                                                    : 2 * (int)b->hs.size());
        }
    *shared_launch_in_use = any && all ? 1 : 0;
    if (contraction_launches) *contraction_launches = most;
    return SWOPT_OK;
}

swopt_status swopt_batch_destroy(swopt_batch* b)
{
    clear_error();
    if (!b) return SWOPT_OK;
    batch_release_graphs(b);
    for (auto st : b->streams) cudaStreamDestroy(st);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return SWOPT_OK;
}

}  // extern "C"
