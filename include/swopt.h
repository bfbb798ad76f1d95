/*
 * swopt: GB300-native (sm_103a) hot path of the one-step reconstruction for
 * photo-switching optoacoustic mesoscopy (arXiv 2510.23739).
 *
 * The library applies the matrix-free forward operator H = A o P and its
 * adjoint H^T (Sec. 2.3, Eq. full-forward), the l1 and TV proximal maps
 * (Eq. prox, Eq. prox-dual, Algorithm 2) and the FISTA iteration of
 * Algorithm 1 that combines them, all as CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - Array arguments named *_dev are DEVICE pointers owned by the caller
 *    (for example PyTorch tensors), dense and row-major in the layouts
 *    below; arguments named *_host are host pointers.  The library never
 *    frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless they return
 *    host scalars, which synchronise the stream before returning.
 *  - Every call returns a swopt_status.  On failure the call leaves caller
 *    buffers in an unspecified state and swopt_last_error() returns a
 *    message (thread-local).  Arguments are validated on the host before any
 *    GPU work is queued.
 *  - A handle is not thread-safe: calls on one handle must not overlap in
 *    time (host side) and share its workspaces (device side), so work on
 *    one handle must be issued to one stream at a time.
 *
 * Layouts (C order), with S = Y*X scan positions:
 *   concentrations c  float [P][Y][X][Z]   species, scan row, scan column, depth
 *   measurements   y  float [N][Y][X][T]   pulse, scan row, scan column, time
 *   kernel         K  double[Z][k][k][T]   depth j, dy+r, dx+r, time (r = k/2)
 */
#ifndef SWOPT_H
#define SWOPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SWOPT_OK = 0,
    SWOPT_ERR_INVALID_ARG = 1,  /* null pointer, bad enum or non-finite scalar */
    SWOPT_ERR_SHAPE = 2,        /* geometry out of the supported range */
    SWOPT_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SWOPT_ERR_OOM = 4,          /* device allocation failed */
    SWOPT_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    SWOPT_ERR_DEVICE_CHECK = 6, /* a device-side consistency check failed */
    SWOPT_ERR_UNSUPPORTED = 7   /* valid request the current build cannot serve */
} swopt_status;

typedef struct swopt_handle swopt_handle;

/* Grid and pulse train.  Limits: 1 <= X, Y <= 4096; 1 <= Z <= 1024;
 * 1 <= T <= 8192; 1 <= N <= 4096; 1 <= P <= 8; k odd, 1 <= k <= 63;
 * 1 <= pulses_per_cycle.  dz_mm > 0 is the depth pitch used by the fluence
 * model Phi_j = exp(-mu * j * dz_mm). */
typedef struct {
    int X, Y, Z, T, N, P, k;
    int pulses_per_cycle;
    double dz_mm;
} swopt_geometry;

/* Photo-switching parameters of Eq. (final-H), host arrays of length P.
 * Pulse n of the train sits m = n mod pulses_per_cycle pulse intervals into
 * its OFF-switching cycle, and depth j receives the weight
 *   S[n][p][j] = Phi_j * (eps_bar[p] * exp(-kappa[p] * Phi_j * m) + eps_off[p]).
 * The background species has kappa = 0, eps_bar = 0 (Sec. 2.1). */
typedef struct {
    const double* kappa_host;
    const double* eps_bar_host;
    const double* eps_off_host;
    double mu_per_mm;
} swopt_switching;

/* Arithmetic of the A / A^T contractions.
 *  SWOPT_PREC_FP32 : FP32 FMA on the CUDA cores (the accuracy reference).
 *  SWOPT_PREC_BF16 : tcgen05 tensor cores, BF16 operands, FP32 accumulation.
 *  SWOPT_PREC_BF16X3: tcgen05 tensor cores on a two-term BF16 split of both
 *                    operands (v = v0 + v1; v0 w0 + v0 w1 + v1 w0), FP32
 *                    accumulation with the two correction products in an
 *                    accumulator of their own: measured relative error of
 *                    the operator 4e-6 (A) and 1e-5 (A^T) at 64^3 x 256 with
 *                    15 x 15 support, against 1e-6 for SWOPT_PREC_FP32.
 *  SWOPT_PREC_BF16X6: tcgen05 tensor cores on a three-term BF16 split of both
 *                    operands (v = v0 + v1 + v2) with the six products of
 *                    total order up to 2, the five corrections in an
 *                    accumulator of their own: each product is kept to about
 *                    2^-24, so the operator meets the FP32 bound; twice the
 *                    MMAs of SWOPT_PREC_BF16X3.
 *  SWOPT_PREC_FP8  : tcgen05 tensor cores on FP8 E4M3 operands (3 mantissa
 *                    bits), FP32 accumulation, with per-channel
 *                    equilibration: the kernel is stored as K_j / s_j and the
 *                    image as b_j s_j sigma (s_j per depth for A and per
 *                    window sample for A^T, from the kernel; sigma per call,
 *                    from the image's largest scaled entry), so that each
 *                    product equals K_j b_j sigma in real arithmetic and both
 *                    operands use the format's range; the output is divided
 *                    by sigma.  An experiment: its operator error (a few
 *                    percent) is reported against the FP64 reference.  Not
 *                    a resync precision of the refined solve. */
typedef enum {
    SWOPT_PREC_FP32 = 0,
    SWOPT_PREC_BF16 = 1,
    SWOPT_PREC_BF16X3 = 2,
    SWOPT_PREC_FP8 = 3,
    SWOPT_PREC_BF16X6 = 4
} swopt_precision;

/* Momentum of Algorithms 1 and 2: Beck-Teboulle (t_k - 1)/t_{k+1}, the
 * coefficient as printed in the paper (t_k - 1)/(t_k + 1), or none. */
typedef enum {
    SWOPT_MOMENTUM_BECK_TEBOULLE = 0,
    SWOPT_MOMENTUM_PAPER_PRINTED = 1,
    SWOPT_MOMENTUM_NONE = 2
} swopt_momentum;

/* Settings of Algorithm 1 (FISTA) on Eq. (one-step) with Eq. (reg-tv-l1-one):
 * w(c) = lambda_tv sum_p TV(c_p) + lambda_l1 ||c||_1 + lambda_3 sum_n TV((S c)^n)
 * + indicator(c >= 0). */
typedef struct {
    double step;        /* alpha_1; <= 0 means 1/L with L from swopt_lipschitz */
    double lambda_l1;   /* >= 0 */
    double lambda_tv;   /* >= 0 */
    int inner_iters;    /* K2 of Algorithm 2 (>= 0; 0 skips the TV prox) */
    int max_iters;      /* K1 of Algorithm 1 (>= 0) */
    double eps1;        /* relative objective change stop (<= 0: off) */
    double eps2;        /* relative momentum-iterate change stop (<= 0: off) */
    int momentum;       /* swopt_momentum of Algorithm 1 */
    int inner_momentum; /* swopt_momentum of Algorithm 2 */
    int power_iters;    /* power iterations when step <= 0 (>= 1) */
    /* Refined gradient (not in the paper; an iterative-refinement scheme for
     * the low-precision contractions).  0: every iteration evaluates the
     * gradient at the momentum point directly, at the handle's precision.
     * R >= 1: the gradient G_k = H^T (H c_k - y) is kept in FP32 and updated
     * with the normal operator applied to the increment,
     * G_{k+1} = G_k + H^T H (c_{k+1} - c_k), at the handle's precision; every
     * R-th iteration (and at the start) it is recomputed from c_{k+1} at
     * refine_precision.  The gradient at the momentum point follows by
     * linearity, (1 + beta_k) G_{k+1} - beta_k G_k.  In exact arithmetic the
     * iterates are those of Algorithm 1; the increment's rounding error
     * scales with ||c_{k+1} - c_k|| and so shrinks as the solve converges. */
    int refine_every;
    int refine_precision; /* swopt_precision of the initial and periodic exact gradients */
    double* history_host; /* optional [max_iters]: F(c_{k+1}) per iteration */
    /* Device-side resync test of the refined solve (refine_every >= 1):
     * > 0 also recomputes the gradient exactly at the end of iteration k when
     * the sum of rho_i = ||c_{i+1} - c_i|| / ||c_{i+1}|| (FP64) over the
     * iterations since the last exact gradient, this one included, exceeds
     * refine_budget.  The low-precision increments since a resync then add a
     * gradient error of about eps * refine_budget relative to the gradient
     * (eps the rounding of the increment's arithmetic), whatever the phase of
     * the solve: early iterations, whose steps are large, resync every time;
     * late ones rarely.  The decision is made on the GPU (no host
     * synchronisation): both branches are launched, and the one not taken
     * returns at once.  0: off (resync every refine_every iterations only). */
    double refine_budget;
    /* lambda_3 of Eq. (reg-tv-l1-one), >= 0: TV of every pulse image (S c)^n.
     * 0 keeps the composite prox of the other two terms (TV prox, then the
     * l1 prox).  > 0 takes the prox of all three terms with the nonnegativity
     * constraint by Algorithm 2 on the stacked operator (swopt_prox_joint),
     * inner_iters dual iterations with inner_momentum; joint_step2 is its
     * dual step (<= 0: 1 / the bound of eig_max(L L^T) that
     * swopt_prox_joint_step_bound returns). */
    double lambda_3;
    double joint_step2;
} swopt_solve_params;

typedef struct {
    int iters;          /* iterations run */
    double step;        /* alpha_1 used */
    double objective;   /* F(c) of the returned iterate (FP64) */
    double data_fit;    /* 1/2 ||H c - y||^2 of the returned iterate (FP64) */
} swopt_solve_stats;

/* Thread-local message of the last failed call on this thread ("" if none). */
const char* swopt_last_error(void);

/* Library version, "major.minor.patch". */
const char* swopt_version(void);

/* Create a handle on the current CUDA device.  K_host is the FP64 per-depth
 * kernel K[Z][k][k][T] (copied; the caller may free it on return); it plays
 * the part of the transducer response of Sec. 2.3 with the electrical
 * impulse response of Eq. (acoustic-temporal-conv) folded in along t.
 * Errors: INVALID_ARG (null pointers, non-finite values), SHAPE (limits
 * above, or an all-zero kernel), OOM, CUDA. */
swopt_status swopt_create(const swopt_geometry* geom, const double* K_host,
                          const swopt_switching* sw, swopt_handle** out);

/* Release a handle and all device memory it owns (NULL is a no-op). */
swopt_status swopt_destroy(swopt_handle* h);

/* Select the contraction arithmetic for later calls (swopt_precision). */
swopt_status swopt_set_precision(swopt_handle* h, int precision);

/* Forward operator, y = H c = W_tot S c (Eq. full-forward): for every pulse n
 * and scan position (y, x),
 *   y[n][y][x][t] = sum_j sum_{|dy|,|dx|<=r} b[n][y+dy][x+dx][j] K[j][dy+r][dx+r][t],
 *   b[n][y][x][j] = sum_p S[n][p][j] c[p][y][x][j]      (Eq. Sij-detailed),
 * with b = 0 outside the scan grid.  c_dev: [P][Y][X][Z]; y_dev: [N][Y][X][T]
 * (fully overwritten). */
swopt_status swopt_forward(swopt_handle* h, const float* c_dev, float* y_dev, void* stream);

/* Adjoint operator, c = H^T y (the exact transpose of swopt_forward):
 *   c[p][y][x][j] = sum_n S[n][p][j] sum_{dy,dx} sum_t y[n][y-dy][x-dx][t] K[j][dy+r][dx+r][t].
 * y_dev: [N][Y][X][T]; c_dev: [P][Y][X][Z] (fully overwritten). */
swopt_status swopt_adjoint(swopt_handle* h, const float* y_dev, float* c_dev, void* stream);

/* l1 proximal map, in place on x_dev [P][Y][X][Z]: x <- sign(x) max(|x| - thresh, 0),
 * or with nonneg != 0 (l1 plus the indicator of Eq. one-step) x <- max(x - thresh, 0).
 * thresh >= 0. */
swopt_status swopt_prox_l1(swopt_handle* h, float* x_dev, float thresh, int nonneg, void* stream);

/* Anisotropic 3D TV proximal map of one volume per species by Algorithm 2
 * with L = the forward differences along y, x and z (interior edges only),
 * dual radius tau >= 0, dual step 1/12, zero dual start and inner_iters
 * iterations with the given swopt_momentum; x = z - D^T u.
 * z_dev, x_dev: [P][Y][X][Z] (may not alias). */
swopt_status swopt_prox_tv(swopt_handle* h, const float* z_dev, float* x_dev, float tau,
                           int inner_iters, int momentum, void* stream);

/* Step-size estimate of Algorithm 1: L ~ eig_max(H^T H) by iters >= 1 power
 * iterations v <- H^T H v / ||H^T H v|| (FP64 norms), returning the Rayleigh
 * quotient in *L_out.  v0_dev ([P][Y][X][Z], optional): start vector; NULL
 * starts from a fixed counter-based pseudo-random vector.  Synchronises. */
swopt_status swopt_lipschitz(swopt_handle* h, const float* v0_dev, int iters, double* L_out,
                             void* stream);

/* Algorithm 1 in steps.  swopt_fista_init binds the measurements y_dev
 * ([N][Y][X][T], read during this call only), sets c_0 = xi_0 = 0, t_0 = 1
 * and fixes the settings (a step <= 0 runs swopt_lipschitz first, which
 * synchronises).  swopt_fista_step runs `iters` iterations
 *   c_{k+1} = prox_{alpha w}(xi_k - alpha H^T (H xi_k - y)),  t_{k+1}, xi_{k+1}
 * asynchronously (no host synchronisation; the momentum scalars stay on the
 * device in FP64; the eps1/eps2 tests and the history are not evaluated).
 * swopt_fista_get copies the current c_k into c_dev [P][Y][X][Z]. */
swopt_status swopt_fista_init(swopt_handle* h, const float* y_dev, const swopt_solve_params* prm,
                              void* stream);
swopt_status swopt_fista_step(swopt_handle* h, int iters, void* stream);
swopt_status swopt_fista_get(swopt_handle* h, float* c_dev, void* stream);

/* Progress of the refined solve since swopt_fista_init: *iterations run and
 * *resyncs, the exact gradients computed (the initial one included; with
 * refine_every = 0 both count iterations and resyncs is 0).  Synchronises
 * the stream when the schedule is decided on the device. */
swopt_status swopt_refine_stats(swopt_handle* h, int64_t* iterations, int64_t* resyncs,
                                void* stream);

/* Checkpoint of the FISTA state (Algorithm 1 between two iterations): the
 * iterates c_k and xi_k, the next prox input and the refined solve's
 * gradient, the momentum scalars t_k, beta_k (FP64), the refined schedule's
 * state and the iteration counters.  swopt_fista_state_bytes gives the size
 * of the host buffer; swopt_fista_save copies the state into host_buf
 * (synchronises); swopt_fista_restore loads it into a handle with the same
 * geometry whose swopt_fista_init bound the same measurements and settings
 * (the measurements are not part of the state), after which the iterations
 * continue exactly as they would have from the saved point: 10 iterations,
 * save, restore, 10 iterations equal 20 iterations bit for bit.  Errors:
 * INVALID_ARG (no FISTA state, a buffer too small, or a state of another
 * geometry or settings). */
swopt_status swopt_fista_state_bytes(swopt_handle* h, size_t* bytes);
swopt_status swopt_fista_save(swopt_handle* h, void* host_buf, size_t bytes, void* stream);
swopt_status swopt_fista_restore(swopt_handle* h, const void* host_buf, size_t bytes,
                                 void* stream);

/* Failure-detection test hook for the cooperative TV prox's software grid
 * barrier (not needed in normal use).  phantom_arrivals > 0 makes every
 * barrier wait for that many blocks more than the launch has, so that no
 * barrier completes; poll_limit > 0 replaces the barrier's default poll
 * limit (about a second).  A barrier that reaches the limit records an
 * error, every later barrier of the launch returns at once, and the next
 * synchronising call (swopt_check_device) reports SWOPT_ERR_TIMEOUT and
 * clears the error, after which the handle works normally.  0, 0 restores
 * the defaults.  Synchronises. */
swopt_status swopt_debug_barrier(swopt_handle* h, int phantom_arrivals, unsigned poll_limit);

/* Sharding over switching states (pulses of one state together: the
 * measurement operator is block diagonal over pulses, Eq.
 * (acoustic-full-forward), and Eq. (final-H) makes pulses of one state share
 * their images).  A shard is a handle whose pulses are those of the states
 * [m0, m1) of the whole train, in cycle-major order (pulses_per_cycle =
 * m1 - m0, N = their count), with swopt_set_state_offset(h, m0) so that its
 * local state q is pulse-in-cycle m0 + q.  Every shard keeps a replica of the
 * iterate; one FISTA iteration is
 *   g_r = swopt_fista_gradient(shard r)     (its states' part of H^T (H xi - y))
 *   g   = sum over shards of g_r            (the caller's collective)
 *   swopt_fista_step_external(shard r, g)   (gradient step, prox, momentum)
 * Plain solves only (refine_every = 0). */

/* Sets the first state of the handle's pulses (default 0): pulse n sits
 * offset + (n mod pulses_per_cycle) pulses into its cycle in Eq. (final-H).
 * Errors: INVALID_ARG for offset < 0.  Synchronises. */
swopt_status swopt_set_state_offset(swopt_handle* h, int offset);

/* The data-fit gradient H^T (H xi - y) at the FISTA state's momentum iterate
 * (after swopt_fista_init; refine_every must be 0), into g_dev [P][Y][X][Z]:
 * per element, the P^T sum over the handle's states continues from
 * carry_dev (a previous shard's output, or NULL for 0) with one FMA per state
 * in state order.  Shards taken one after another, each continuing from the
 * last, give the bits of the unsharded gradient whenever each state's A^T
 * output has the same bits in both (FP32 operators; tensor-core operators
 * with whole tile-states per CTA, swopt_tc_schedule split 1, and the same
 * configuration).  Asynchronous on the stream. */
swopt_status swopt_fista_gradient(swopt_handle* h, const float* carry_dev, float* g_dev,
                                  void* stream);

/* One FISTA iteration with the data-fit gradient at the momentum iterate
 * supplied (g_dev, e.g. summed over shards): z = xi - alpha g, the prox of
 * the solve's regulariser, then the momentum step, exactly as
 * swopt_fista_step's plain iteration.  Asynchronous on the stream. */
swopt_status swopt_fista_step_external(swopt_handle* h, const float* g_dev, void* stream);

/* Complete solve (Algorithm 1): init, up to max_iters iterations with the
 * eps1/eps2 stopping tests and the optional history, then c_dev <- c_K and
 * the statistics (stats may be NULL).  Synchronises. */
swopt_status swopt_solve(swopt_handle* h, const float* y_dev, float* c_dev,
                         const swopt_solve_params* prm, swopt_solve_stats* stats, void* stream);

/* Proximal map of alpha (R3 + delta_{>=0}) with all three terms of Eq.
 * (reg-tv-l1-one), including lambda_3 sum_n TV((S c)^n) (lambda_b here), by
 * Algorithm 2 on the dual of Eq. (prox-dual) for the stacked
 * L = [lambda_tv D per species; lambda_l1 I; lambda_b D S per pulse]: the
 * nonnegativity constraint of Eq. (prox) makes the dual
 * min over |u| <= alpha of 1/2 ||max(z - L^T u, 0)||^2, so every dual step
 * takes L of the projected point w = max(z - L^T r, 0).  Dual step step2 (at
 * most 1/eig_max(L L^T); swopt_prox_joint_step_bound gives a bound of that
 * eigenvalue), `iters` dual iterations (Beck-Teboulle momentum) from a zero
 * dual, output max(z - L^T u, 0).  S is the handle's switching model (pulse n
 * takes state n mod pulses_per_cycle); pulses of one state share one dual,
 * which gives the same iterates as one dual per pulse.  z_dev, x_dev: device
 * [P][Y][X][Z]; x may equal z.  Scratch ((8 P + 6 Q) volumes, Q the switching
 * states, plus P) is the handle's, allocated on the first call.  Errors:
 * INVALID_ARG (null pointers, negative or non-finite weights, iters < 0,
 * step2 <= 0 with iters > 0), UNSUPPORTED for P > 8, OOM, CUDA.
 * Asynchronous on the stream. */
swopt_status swopt_prox_joint(swopt_handle* h, const float* z_dev, float* x_dev, double alpha,
                              double lambda_tv, double lambda_l1, double lambda_b, int iters,
                              double step2, void* stream);

/* An upper bound of eig_max(L L^T) for swopt_prox_joint's stacked L:
 * 12 lambda_tv^2 + lambda_l1^2 + 12 lambda_b^2 sum_n max_j sum_p S[n][p][j]^2
 * (||D||^2 <= 12 in 3D; a pulse image's Cauchy-Schwarz bound per voxel).
 * 0 for a null handle. */
double swopt_prox_joint_step_bound(swopt_handle* h, double lambda_tv, double lambda_l1,
                                   double lambda_b);

/* The two-step approach (the paper's "Two-Step Approach", the comparison
 * method of the one-step reconstruction): first the acoustic problem of
 * Eq. (acoustic-inverse) with R1 = lambda_tv TV (+ lambda_l1 l1 if nonzero),
 * pulse by pulse (W_tot is block diagonal over pulses), for b[N][Y][X][Z];
 * then the unmixing problem of Eq. (unmixing), min 1/2||S c - b||^2 +
 * lambda_l1 ||c||_1 + lambda_tv TV(c) + delta_{>=0}(c), for c[P][Y][X][Z].
 * Both are solved with Algorithm 1 (swopt_solve semantics: a step <= 0 is
 * taken from power iteration) on internal handles created and released by
 * the call: the first with the caller's kernel and an identity switching
 * model, the second with the caller's switching model and an identity
 * acoustic kernel.  geom, K_host and sw as for swopt_create; y_dev: device
 * [N][Y][X][T] (the data p); b_dev: device [N][Y][X][Z], caller-owned,
 * receives the acoustic reconstruction; c_dev: device [P][Y][X][Z] receives
 * the unmixed concentrations.  Precision FP32.  Errors as for swopt_create
 * and swopt_solve (the message of the failing step is kept).  Synchronises. */
swopt_status swopt_two_step(const swopt_geometry* geom, const double* K_host,
                            const swopt_switching* sw, const float* y_dev, float* b_dev,
                            float* c_dev, const swopt_solve_params* acoustic,
                            const swopt_solve_params* unmixing, void* stream);

/* Objective of Eq. (one-step), in FP64: *F = 1/2||H c - y||^2 + lambda_tv sum_p TV(c_p)
 * + lambda_l1 ||c||_1 + lambda_3 sum_n TV((S c)^n), *fit = the data-fit term
 * (either may be NULL).  c is not checked for nonnegativity.  Synchronises. */
swopt_status swopt_objective(swopt_handle* h, const float* c_dev, const float* y_dev,
                             double lambda_l1, double lambda_tv, double lambda_3, double* F,
                             double* fit, void* stream);

/* Gradient of f = 1/2||H c - y||^2 with respect to the switching parameters
 * with c held fixed (Eq. final-H differentiated): dkappa_host[p] = df/dkappa_p
 * (length P) and *dmu = df/dmu.  FP64 accumulation.  Synchronises. */
swopt_status swopt_param_grad(swopt_handle* h, const float* c_dev, const float* y_dev,
                              double* dkappa_host, double* dmu, void* stream);

/* Vector-Jacobian product of (kappa, mu) -> H(kappa, mu) c at fixed c: for a
 * cotangent w_dev in the measurement layout [N][Y][X][T],
 * dkappa_host[p] = <w, dH/dkappa_p c> (length P) and *dmu = <w, dH/dmu c>
 * (Eq. final-H differentiated).  swopt_param_grad is this product with
 * w = H c - y.  Uses the handle's precision for A^T; FP64 accumulation.
 * Synchronises. */
swopt_status swopt_param_vjp(swopt_handle* h, const float* c_dev, const float* w_dev,
                             double* dkappa_host, double* dmu, void* stream);

/* Fluence from the diffusion equation, Eqs. (de), (bc) and
 * (diffusion-coefficient), on the GPU: cell-centred finite volumes on a
 * Y x X x Z voxel grid (lateral pitch dx_mm, depth pitch dz_mm, depth index 0
 * the illuminated top face), per voxel
 *   mu_a Phi + sum over faces (outward flux) / h = s,
 * inner faces D_f (Phi_i - Phi_k) / h with the harmonic mean D_f, boundary
 * faces 2 D Phi / (4 D + h) from Phi + 2 D dPhi/dn = 0 (n the outward
 * normal), D = 1 / (3 (mu_a + (1 - g) mu_s)).  Lateral faces are boundary
 * faces (lateral_robin = 1) or carry no flux (0: a laterally unbounded
 * sample).  The illumination src_top_host [Y][X] (power per area) enters the
 * top layer as s = src / dz_mm.  mu_a_host, mu_s_host [Y][X][Z] in 1/mm (>= 0,
 * mu_a + (1 - g) mu_s > 0), 0 <= g < 1.  Solved by conjugate gradients with a
 * diagonal preconditioner in FP64 to ||r|| <= tol ||b|| within max_iters
 * iterations; phi_host [Y][X][Z] receives the solution, iters_out and
 * rel_residual_out (either may be NULL) the count and the final relative
 * residual.  Errors: INVALID_ARG, OOM, CUDA, DEVICE_CHECK (not converged; the
 * last iterate is still written).  Synchronises. */
swopt_status swopt_diffusion_fluence(int Y, int X, int Z, double dx_mm, double dz_mm,
                                     const double* mu_a_host, const double* mu_s_host, double g,
                                     const double* src_top_host, int lateral_robin, double tol,
                                     int max_iters, double* phi_host, int* iters_out,
                                     double* rel_residual_out);

/* Replaces exp(-mu j dz) in Eq. (final-H) by the depth profile phi_host [Z]
 * (e.g. the lateral mean of swopt_diffusion_fluence's solution; finite, >= 0),
 * or restores it (phi_host NULL).  With a given profile the derivatives with
 * respect to mu are 0.  Synchronises. */
swopt_status swopt_set_fluence(swopt_handle* h, const double* phi_host);

/* Reverse-mode derivative of the unrolled solve: with y, prm and the handle's
 * precision as in swopt_solve (explicit step > 0, max_iters >= 1 FISTA
 * iterations, refine_every = 0, lambda_3 = 0, no stopping tests), the
 * gradient of <w, c_K> with respect to kappa_p (dkappa_host[P]) and mu
 * (*dmu) of Eq. (final-H), c_K the output of Algorithm 1 (Algorithm 2 as the
 * TV prox, clamp masks and the l1/nonnegativity clip taken as fixed where
 * they are, the step, weights and counts held fixed).  The forward pass
 * keeps the K momentum iterates on the device (K volumes); the backward pass
 * recomputes each iteration, records Algorithm 2's masks and applies the
 * transposed steps, with the parameter derivatives of H taken as in
 * swopt_param_vjp.  c_dev (optional) receives c_K.  w_dev: [P][Y][X][Z].
 * Errors: INVALID_ARG, OOM, CUDA.  Synchronises; leaves the handle's FISTA
 * state at c_K. */
swopt_status swopt_unrolled_vjp(swopt_handle* h, const float* y_dev,
                                const swopt_solve_params* prm, const float* w_dev, float* c_dev,
                                double* dkappa_host, double* dmu, void* stream);

/* Replaces the switching parameters of Eq. (final-H) (kappa, eps_bar, eps_off
 * per species and mu, validated as in swopt_create); the geometry, kernel and
 * precision stay.  Captured FISTA iterations keep working (they read the
 * switching weights from device memory), but a FISTA state that is in
 * progress continues with the new model.  Synchronises the device. */
swopt_status swopt_set_switching(swopt_handle* h, const swopt_switching* sw);

/* CUDA graphs (default on): swopt_fista_step captures one iteration into a
 * CUDA graph on first use after swopt_fista_init (on a stream the handle
 * owns) and replays it on the caller's stream; on = 0 launches the kernels
 * one by one instead.  Changing the precision or the tensor-core
 * configuration discards the graph. */
swopt_status swopt_use_graphs(swopt_handle* h, int on);

/* Instrumentation.  swopt_profile_enable(h, 1) records CUDA events around
 * every launch of the A and A^T contraction kernels on the launching stream
 * (inside a replayed FISTA graph, through its event-record nodes);
 * swopt_profile_read returns, for kernel_id 0 (A) or 1 (A^T), the
 * summed device time in milliseconds, the number of launches and the
 * algorithmic FLOPs of one launch (2 x multiply-adds of nonzero kernel taps);
 * kernel_id 2 and 3 report the launches of A and A^T that the refined solve
 * makes at its resync precision (the initial and periodic exact gradients).
 * Reading synchronises on the recorded events and clears them.
 * swopt_launch_count returns the number of kernels this handle launched. */
swopt_status swopt_profile_enable(swopt_handle* h, int on);
swopt_status swopt_profile_read(swopt_handle* h, int kernel_id, double* total_ms,
                                int64_t* launches, double* flops_per_launch);
swopt_status swopt_launch_count(swopt_handle* h, int64_t* count);

/* Synchronises `stream` and reports device-side failures of earlier calls on
 * this handle: SWOPT_ERR_TIMEOUT if a tensor-core kernel gave up one of its
 * bounded waits (the word is then cleared), else SWOPT_OK.  Calls that
 * synchronise anyway (lipschitz, solve, objective, param_grad) check it too. */
swopt_status swopt_check_device(swopt_handle* h, void* stream);

/* FLOPs issued by one launch of the A (kernel_id 0) or A^T (1) contraction in
 * the current precision: 2 x the multiply-adds the kernel executes,
 * including the zero-padded parts of the kernel band it does not skip (for
 * the split BF16 modes, all 3 or 6 products). */
swopt_status swopt_issued_flops(swopt_handle* h, int kernel_id, double* flops);

/* Tensor-core tile configuration (autotuner).  When a BF16 precision is
 * selected, the library times each candidate configuration of the A (0) and
 * A^T (1) kernels on the handle's geometry and keeps the fastest.  A
 * configuration is: 1, 2 or 4 tiles of 16 x 8 positions per CTA; one or two
 * CTAs per SM; one or two FP32 accumulators per tile.  With two, the
 * correction products of the split precisions (every product but hi x hi)
 * accumulate apart from the main products and the epilogue adds the two: the
 * corrections are about 2^-8 of the main sum, so each accumulation step into
 * their accumulator rounds 2^-8 finer.  The default is two for the split
 * precisions where TMEM holds them, else one; the choice is not timed.
 * swopt_tc_configure pins tiles_per_cta (1, 2, 4), ctas_per_sm (1, 2) and
 * accumulators (1, 2) instead, 0 leaving a field at its default, and
 * rebuilds the operator if one is active (synchronises).  swopt_tc_config
 * reports the configuration in use (INVALID_ARG if no BF16 precision is
 * selected). */
swopt_status swopt_tc_configure(swopt_handle* h, int kernel_id, int tiles_per_cta, int ctas_per_sm,
                                int accumulators);
swopt_status swopt_tc_config(swopt_handle* h, int kernel_id, int* tiles_per_cta, int* ctas_per_sm,
                             int* stages, int* groups, int* accumulators);

/* Work schedule of the tensor-core contraction (kernel_id 0: A, 1: A^T).
 * The kernel is persistent (at most one CTA per resident slot).  split
 * selects how the runs of taps of all (switching state, tile) pairs are
 * shared out: 1 = whole pairs per CTA, 2 = equal shares of all runs (a pair
 * cut between neighbouring CTAs is summed by the last to finish, in a fixed
 * order: the results do not depend on which finishes last).  buffers = 2
 * double-buffers the TMEM accumulators (the epilogue overlaps the next
 * unit's MMAs), 1 does not.  0 leaves a field to the timed choice.
 * swopt_tc_schedule pins them and rebuilds the operator if one is active
 * (synchronises); INVALID_ARG for values out of range, UNSUPPORTED at the
 * rebuild if no configuration satisfies the pins.  swopt_tc_schedule_info
 * reports the schedule in use: split (1 or 2), buffers, the CTAs launched
 * and the most CTAs that share one pair (INVALID_ARG if no BF16 precision is
 * selected). */
swopt_status swopt_tc_schedule(swopt_handle* h, int kernel_id, int split, int buffers);
swopt_status swopt_tc_schedule_info(swopt_handle* h, int kernel_id, int* split, int* buffers,
                                    int* grid, int* max_pieces);

/* The paper-literal acoustic kernel (Sec. 2.3.1 "Acoustic Model", Eqs.
 * q-above-final / q-below-final with the discrete semicircles of Eqs.
 * discrete-upper-circle / discrete-lower-circle), as the per-depth kernel
 * that swopt_create takes.  Host only: no GPU is used.
 *   K_out[j][dy][dx][t] = sum_s M[j][dy][dx][t - s] eir[s + J],
 *   M[j][dy][dx][t] = eta[j][dy][dx] if voxel (j, dy, dx) meets the upper
 *   (t < focal_sample) or lower (t > focal_sample) half sphere of radius
 *   |t - focal_sample| about the focus, else 0,
 * in depth pitches (the time grid matches the depth grid, c0 dt = dz; one
 * lateral pitch is lateral_ratio depth pitches; the focus is at depth index
 * focal_depth, which may be fractional).  A voxel meets a half sphere when
 * its closed box, clipped to the half space (z <= 0 above the focus, z >= 0
 * below), has its nearest point at most and its farthest point at least the
 * radius from the focus; at t = focal_sample the voxels whose box holds the
 * focus count.  dims = 3 uses the voxel box; dims = 2 the pixel box in the
 * (x, z) plane, with dy = 0 only (a 2D scan is Y = 1).
 * eta: host [Z][k][k] FP64 (the spatial response of the transducer about
 * its focus, caller-owned); eir: host [eir_len] FP64, eir_len odd, centred
 * (s = -J .. J); K_out: host [Z][k][k][T] FP64, written.
 * Errors: SHAPE for Z, k (odd), T out of the limits of swopt_geometry;
 * INVALID_ARG for null pointers, dims not 2 or 3, a non-positive or
 * non-finite lateral_ratio, a non-finite focal_depth, focal_sample outside
 * [0, T) or an even eir_len. */
swopt_status swopt_semicircle_kernel(int Z, int k, int T, int dims, double lateral_ratio,
                                     double focal_depth, int focal_sample, const double* eta,
                                     const double* eir, int eir_len, double* K_out);

/* Operator facts: the time window [t0, t0 + tw) that holds every nonzero
 * kernel sample, the number of distinct switching states Q = min(N,
 * pulses_per_cycle) and the number of nonzero kernel entries. */
swopt_status swopt_info(swopt_handle* h, int* t0, int* tw, int* states, int64_t* kernel_nnz);

/* ---------------------------------------------------------------------------
 * Allocation-free TV proximal map.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory themselves
 * or through the library -- for example a host framework whose caching
 * allocator owns all of the GPU's memory and forbids outside cudaMalloc, or
 * a real-time loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation after start-up.  It needs no handle.
 *
 * It computes the same map as swopt_prox_tv with the same arithmetic (one
 * launch of the per-iteration FGP kernel per inner iteration, then the
 * primal recovery), and takes the same arguments apart from the volume shape
 * P x Y x X x Z given directly: z_dev and x_dev are caller-owned device
 * arrays [P][Y][X][Z] that may not alias.  Its scratch (the three FGP dual
 * arrays, 9 floats per volume element) is a file-scope static device array
 * sized for SWOPT_PROX_TV_STATIC_MAX_ELEMS elements (18 MiB).  The array is
 * placed on a device when the library's module is first loaded there (with
 * lazy module loading, the CUDA default, that may be this call's first use
 * of the device, and placing it is the only memory the call ever causes to
 * be reserved); it stays until the process exits or the context is reset.
 * Volumes with P*Y*X*Z above the limit are rejected with SWOPT_ERR_SHAPE and
 * a message; the call never allocates (no cudaMalloc, cudaFree or
 * allocating library routine).
 *
 * Every call looks up the device address of the array (cudaGetSymbolAddress)
 * in the current device's context; make the first call on each device before
 * any stream capture, so that the module load does not happen inside one.
 * All calls in the process share the one array:
 * calls whose GPU work overlaps in time (different streams, or host threads
 * using the same device) race on it, so serialise them.  The array keeps
 * the last call's contents, but nothing in it needs clearing: each call
 * writes every scratch element before reading it.
 * ------------------------------------------------------------------------- */
#define SWOPT_PROX_TV_STATIC_MAX_ELEMS ((size_t)1 << 19)

swopt_status swopt_prox_tv_static(int P, int Y, int X, int Z, const float* z_dev, float* x_dev,
                                  float tau, int inner_iters, int momentum, void* stream);

/* Batched problems (independent solves of uneven size).  swopt_batch_create
 * takes handles whose FISTA state is set up (swopt_fista_init, the same
 * refine_every and iteration count on all); swopt_batch_step then runs `iters`
 * FISTA iterations of every problem, each iteration one CUDA-graph launch in
 * which every problem's kernels run on a stream of their own, so that the
 * problems overlap on the GPU.  The iterates are those of swopt_fista_step on
 * each handle.  Stepping a handle on its own or re-initialising it makes the
 * batch refuse to step (INVALID_ARG); discarding a handle's graphs (precision
 * or tiling changes) makes it recapture.  The handles must outlive the batch.
 * swopt_launch_count of the first handle counts the batch's kernels. */
typedef struct swopt_batch swopt_batch;
swopt_status swopt_batch_create(swopt_handle* const* handles, int count, swopt_batch** out);
swopt_status swopt_batch_step(swopt_batch* b, int iters, void* stream);
swopt_status swopt_batch_destroy(swopt_batch* b);

/* Shared launches (shared_launch = 1; default 0): the batch's graph runs the contractions
 * of all problems as persistent launches over a work list of every
 * problem's tile-states (for A, then for A^T, per gradient path), the
 * other steps per problem (problems whose halos and stage rings do not fit
 * one CTA's shared memory together go to separate launches); it falls back to
 * a stream per problem for FP32 or FP8 operators.  shared_launch = 0 takes a
 * stream per problem.  Measured on 16 uneven problems, the shared launches ran
 * at 0.55 of the stream-per-problem graph: a shared stage ring is sized for the
 * largest problem's stages, so problems with small stages keep fewer bytes in
 * flight than in their own launches.  The sums per problem are the same either way, but for
 * the order of FP32 addition in a tile-state that the problem's own launch
 * splits over CTAs (a shared launch takes tile-states whole).
 * Errors: INVALID_ARG for a null batch. */
swopt_status swopt_batch_configure(swopt_batch* b, int shared_launch);

/* *shared_launch_in_use = 1 when every iteration graph captured so far uses
 * shared launches (0 before the first step); *contraction_launches (may be
 * NULL): the most contraction kernels of one gradient path in a captured
 * iteration (shared launches: the groups of A plus those of A^T; a stream per
 * problem: two per problem). */
swopt_status swopt_batch_query(swopt_batch* b, int* shared_launch_in_use,
                               int* contraction_launches);

#ifdef __cplusplus
}
#endif

#endif /* SWOPT_H */
