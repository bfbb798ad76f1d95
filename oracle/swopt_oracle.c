/*
 * FP64 CPU oracle for the one-step photo-switching optoacoustic reconstruction.
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow, obviously-correct
 * reference against which the CUDA library is checked.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every function follows a passage of the paper (arXiv 2510.23739):
 *   switching matrix      Eq. (final-H) and Eq. (Sij-detailed), Sec. 2.3.1
 *   forward  H = W_tot S  Eq. (q-above-final)/(q-below-final) read as a
 *                         per-depth lateral correlation, Eq. (acoustic-full-
 *                         forward), Eq. (full-forward)
 *   adjoint  H^T          the exact transpose of the forward
 *   TV / l1 prox          Eq. (prox), Eq. (prox-dual), Algorithm 2
 *   FISTA                 Algorithm 1 with the objective of Eq. (one-step)
 *                         and Eq. (reg-tv-l1-one) (lambda_3 = 0)
 *   power iteration       the step size alpha_1 = 1/eig_max(A^T A) of
 *                         Algorithm 1
 *
 * Layouts (row-major, C order):
 *   c  [P][Y][X][Z]    concentrations
 *   y  [N][Y][X][T]    measurements
 *   K  [Z][k][k][T]    per-depth kernel, index [j][dy+r][dx+r][t]
 *   S  [N][P][Z]       switching weights (depend on depth only)
 *
 * Parity is pinned for every function by the oracle test-suite (conv2d
 * special case, point absorber, adjoint identity, closed forms, exact
 * convex solutions computed by an independent solver, finite differences).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX4(a, b, c, d, B, C, D) ((((size_t)(a) * (B) + (b)) * (C) + (c)) * (D) + (d))

/* ---------------------------------------------------------------------------
 * Switching model, Eq. (final-H): per depth j and pulse n,
 *   S[n][p][j] = Phi_j * (eps_bar_p * exp(-kappa_p * Phi_j * m) + eps_off_p),
 * m = n mod pulses_per_cycle (switching time in pulse intervals since the
 * start of the cycle) and Phi_j = exp(-mu * j * dz) (fluence from the top
 * layer).  The background species has kappa = 0, eps_bar = 0.
 * ------------------------------------------------------------------------- */
void oracle_fluence(int Z, double mu_per_mm, double dz_mm, double* phi)
{
    for (int j = 0; j < Z; ++j) phi[j] = exp(-mu_per_mm * (double)j * dz_mm);
}

void oracle_switch_matrix(int N, int P, int Z, int pulses_per_cycle,
                          const double* phi, const double* kappa,
                          const double* eps_bar, const double* eps_off,
                          double* S)
{
    for (int n = 0; n < N; ++n) {
        int m = n % pulses_per_cycle;
        for (int p = 0; p < P; ++p)
            for (int j = 0; j < Z; ++j)
                S[IDX4(0, n, p, j, N, P, Z)] =
                    phi[j] * (eps_bar[p] * exp(-kappa[p] * phi[j] * (double)m) + eps_off[p]);
    }
}

/* b[n][y][x][j] = sum_p S[n][p][j] c[p][y][x][j]   (Eq. Sij-detailed) */
static void apply_S(int N, int P, int Y, int X, int Z, const double* S,
                    const double* c, double* b)
{
    for (int n = 0; n < N; ++n)
        for (int yy = 0; yy < Y; ++yy)
            for (int xx = 0; xx < X; ++xx)
                for (int j = 0; j < Z; ++j) {
                    double acc = 0.0;
                    for (int p = 0; p < P; ++p)
                        acc += S[IDX4(0, n, p, j, N, P, Z)] * c[IDX4(p, yy, xx, j, Y, X, Z)];
                    b[IDX4(n, yy, xx, j, Y, X, Z)] = acc;
                }
}

/* ---------------------------------------------------------------------------
 * Forward, y = W_tot S c.  For every pulse n and scan position (y, x):
 *   y[n][y][x][t] = sum_j sum_{|dy|,|dx| <= r} b[n][y+dy][x+dx][j] K[j][dy][dx][t]
 * with b = 0 outside the scan grid.  This is the paper's "correlate the OA
 * image with the masked response and take the row at the focal plane"
 * (Sec. 2.3.3), stacked over depths, with the electrical impulse response
 * already folded into K along t; the same W is used for every pulse
 * (Eq. acoustic-full-forward).
 * ------------------------------------------------------------------------- */
void oracle_forward(int N, int P, int Y, int X, int Z, int T, int k,
                    const double* S, const double* K, const double* c, double* y)
{
    const int r = k / 2;
    double* b = (double*)malloc(sizeof(double) * (size_t)N * Y * X * Z);
    apply_S(N, P, Y, X, Z, S, c, b);
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int yy = 0; yy < Y; ++yy)
            for (int xx = 0; xx < X; ++xx) {
                double* out = y + IDX4(n, yy, xx, 0, Y, X, T);
                for (int t = 0; t < T; ++t) out[t] = 0.0;
                for (int dy = -r; dy <= r; ++dy) {
                    int sy = yy + dy;
                    if (sy < 0 || sy >= Y) continue;
                    for (int dx = -r; dx <= r; ++dx) {
                        int sx = xx + dx;
                        if (sx < 0 || sx >= X) continue;
                        for (int j = 0; j < Z; ++j) {
                            double bv = b[IDX4(n, sy, sx, j, Y, X, Z)];
                            const double* Kp = K + IDX4(j, dy + r, dx + r, 0, k, k, T);
                            for (int t = 0; t < T; ++t) out[t] += bv * Kp[t];
                        }
                    }
                }
            }
    free(b);
}

/* ---------------------------------------------------------------------------
 * Adjoint, c = S^T W_tot^T y.  The transpose of the correlation above:
 *   g[n][y][x][j] = sum_{dy,dx} sum_t y[n][y-dy][x-dx][t] K[j][dy][dx][t]
 * then c[p][y][x][j] = sum_n S[n][p][j] g[n][y][x][j].
 * ------------------------------------------------------------------------- */
void oracle_adjoint(int N, int P, int Y, int X, int Z, int T, int k,
                    const double* S, const double* K, const double* yv, double* c)
{
    const int r = k / 2;
    double* g = (double*)malloc(sizeof(double) * (size_t)N * Y * X * Z);
#pragma omp parallel for collapse(2) schedule(static)
    for (int n = 0; n < N; ++n)
        for (int yy = 0; yy < Y; ++yy)
            for (int xx = 0; xx < X; ++xx)
                for (int j = 0; j < Z; ++j) {
                    double acc = 0.0;
                    for (int dy = -r; dy <= r; ++dy) {
                        int ty = yy - dy;
                        if (ty < 0 || ty >= Y) continue;
                        for (int dx = -r; dx <= r; ++dx) {
                            int tx = xx - dx;
                            if (tx < 0 || tx >= X) continue;
                            const double* yp = yv + IDX4(n, ty, tx, 0, Y, X, T);
                            const double* Kp = K + IDX4(j, dy + r, dx + r, 0, k, k, T);
                            for (int t = 0; t < T; ++t) acc += yp[t] * Kp[t];
                        }
                    }
                    g[IDX4(n, yy, xx, j, Y, X, Z)] = acc;
                }
    for (int p = 0; p < P; ++p)
        for (int yy = 0; yy < Y; ++yy)
            for (int xx = 0; xx < X; ++xx)
                for (int j = 0; j < Z; ++j) {
                    double acc = 0.0;
                    for (int n = 0; n < N; ++n)
                        acc += S[IDX4(0, n, p, j, N, P, Z)] * g[IDX4(n, yy, xx, j, Y, X, Z)];
                    c[IDX4(p, yy, xx, j, Y, X, Z)] = acc;
                }
    free(g);
}

/* Forward at selected outputs: for each (n, y, x) triple, the T samples
 * y[n][y][x][:] of the forward above (same definition, evaluated alone). */
void oracle_forward_at(int N, int P, int Y, int X, int Z, int T, int k,
                       const double* S, const double* K, const double* c,
                       int count, const int* nyx, double* out)
{
    const int r = k / 2;
    (void)N;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < count; ++i) {
        int n = nyx[3 * i], yy = nyx[3 * i + 1], xx = nyx[3 * i + 2];
        double* o = out + (size_t)i * T;
        for (int t = 0; t < T; ++t) o[t] = 0.0;
        for (int dy = -r; dy <= r; ++dy) {
            int sy = yy + dy;
            if (sy < 0 || sy >= Y) continue;
            for (int dx = -r; dx <= r; ++dx) {
                int sx = xx + dx;
                if (sx < 0 || sx >= X) continue;
                for (int j = 0; j < Z; ++j) {
                    double bv = 0.0;
                    for (int p = 0; p < P; ++p)
                        bv += S[IDX4(0, n, p, j, N, P, Z)] * c[IDX4(p, sy, sx, j, Y, X, Z)];
                    const double* Kp = K + IDX4(j, dy + r, dx + r, 0, k, k, T);
                    for (int t = 0; t < T; ++t) o[t] += bv * Kp[t];
                }
            }
        }
    }
}

/* Adjoint at selected outputs: for each (p, y, x, j), c[p][y][x][j]. */
void oracle_adjoint_at(int N, int P, int Y, int X, int Z, int T, int k,
                       const double* S, const double* K, const double* yv,
                       int count, const int* pyxj, double* out)
{
    const int r = k / 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < count; ++i) {
        int p = pyxj[4 * i], yy = pyxj[4 * i + 1], xx = pyxj[4 * i + 2], j = pyxj[4 * i + 3];
        double acc_c = 0.0;
        for (int n = 0; n < N; ++n) {
            double acc = 0.0;
            for (int dy = -r; dy <= r; ++dy) {
                int ty = yy - dy;
                if (ty < 0 || ty >= Y) continue;
                for (int dx = -r; dx <= r; ++dx) {
                    int tx = xx - dx;
                    if (tx < 0 || tx >= X) continue;
                    const double* yp = yv + IDX4(n, ty, tx, 0, Y, X, T);
                    const double* Kp = K + IDX4(j, dy + r, dx + r, 0, k, k, T);
                    for (int t = 0; t < T; ++t) acc += yp[t] * Kp[t];
                }
            }
            acc_c += S[IDX4(0, n, p, j, N, P, Z)] * acc;
        }
        out[i] = acc_c;
    }
}

/* ---------------------------------------------------------------------------
 * Anisotropic TV (Sec. 2.4.1, extended to three axes): forward differences
 * along y, x and z over interior edges only.  For one species volume
 * v[Y][X][Z], the gradient g[3][Y][X][Z] has component a equal to
 * v[i + e_a] - v[i] where i + e_a is inside the grid and 0 otherwise.
 * ------------------------------------------------------------------------- */
static void grad3(int Y, int X, int Z, const double* v, double* g)
{
    size_t L = (size_t)Y * X * Z;
    for (int yy = 0; yy < Y; ++yy)
        for (int xx = 0; xx < X; ++xx)
            for (int j = 0; j < Z; ++j) {
                size_t i = IDX4(0, yy, xx, j, Y, X, Z);
                g[0 * L + i] = (yy + 1 < Y) ? v[IDX4(0, yy + 1, xx, j, Y, X, Z)] - v[i] : 0.0;
                g[1 * L + i] = (xx + 1 < X) ? v[IDX4(0, yy, xx + 1, j, Y, X, Z)] - v[i] : 0.0;
                g[2 * L + i] = (j + 1 < Z) ? v[IDX4(0, yy, xx, j + 1, Y, X, Z)] - v[i] : 0.0;
            }
}

/* The transpose of grad3: (D^T g)[i] = sum_a (g_a[i - e_a] - g_a[i]) with the
 * terms that involve edges outside the grid removed. */
static void grad3T(int Y, int X, int Z, const double* g, double* v)
{
    size_t L = (size_t)Y * X * Z;
    for (int yy = 0; yy < Y; ++yy)
        for (int xx = 0; xx < X; ++xx)
            for (int j = 0; j < Z; ++j) {
                size_t i = IDX4(0, yy, xx, j, Y, X, Z);
                double acc = 0.0;
                if (yy + 1 < Y) acc -= g[0 * L + i];
                if (yy > 0) acc += g[0 * L + IDX4(0, yy - 1, xx, j, Y, X, Z)];
                if (xx + 1 < X) acc -= g[1 * L + i];
                if (xx > 0) acc += g[1 * L + IDX4(0, yy, xx - 1, j, Y, X, Z)];
                if (j + 1 < Z) acc -= g[2 * L + i];
                if (j > 0) acc += g[2 * L + IDX4(0, yy, xx, j - 1, Y, X, Z)];
                v[i] = acc;
            }
}

void oracle_grad3(int Y, int X, int Z, const double* v, double* g) { grad3(Y, X, Z, v, g); }
void oracle_grad3T(int Y, int X, int Z, const double* g, double* v) { grad3T(Y, X, Z, g, v); }

double oracle_tv(int P, int Y, int X, int Z, const double* c)
{
    size_t L = (size_t)Y * X * Z;
    double* g = (double*)malloc(sizeof(double) * 3 * L);
    double s = 0.0;
    for (int p = 0; p < P; ++p) {
        grad3(Y, X, Z, c + p * L, g);
        for (size_t i = 0; i < 3 * L; ++i) s += fabs(g[i]);
    }
    free(g);
    return s;
}

/* l1 prox (closed form): sign(x) max(|x| - theta, 0); with the nonnegativity
 * constraint of Eq. (one-step) it becomes max(x - theta, 0). */
void oracle_prox_l1(size_t count, double* x, double theta, int nonneg)
{
    for (size_t i = 0; i < count; ++i) {
        double v = x[i];
        if (nonneg) x[i] = (v - theta > 0.0) ? v - theta : 0.0;
        else x[i] = (v > theta) ? v - theta : ((v < -theta) ? v + theta : 0.0);
    }
}

/* Momentum modes of Algorithms 1 and 2. */
enum { MOM_BECK_TEBOULLE = 0, MOM_PAPER_PRINTED = 1, MOM_NONE = 2 };

static double next_t(double t) { return 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)); }

static double momentum_coef(int mode, double t_k, double t_k1)
{
    if (mode == MOM_BECK_TEBOULLE) return (t_k - 1.0) / t_k1;
    if (mode == MOM_PAPER_PRINTED) return (t_k - 1.0) / (t_k + 1.0);
    return 0.0;
}

/* ---------------------------------------------------------------------------
 * TV prox by Algorithm 2 with L = D (the 3D forward differences) applied per
 * species: the dual u lives in the box |u| <= tau (tau = alpha * lambda_TV),
 * the dual step is 1/12 (an upper bound of eig_max(D D^T) in 3D), the dual
 * iterate starts at zero and the primal is recovered as z - D^T u.
 *   for i = 1..iters:
 *     x   = z - D^T r
 *     u_i = clamp(r + (1/12) D x, -tau, tau)
 *     t_{i+1} = (1 + sqrt(1 + 4 t_i^2)) / 2
 *     r   = u_i + beta_i (u_i - u_{i-1})
 *   x = z - D^T u_iters
 * ------------------------------------------------------------------------- */
void oracle_prox_tv(int P, int Y, int X, int Z, const double* z, double* x,
                    double tau, int iters, int momentum)
{
    size_t L = (size_t)Y * X * Z;
    double* u = (double*)calloc(3 * L, sizeof(double));
    double* u_prev = (double*)calloc(3 * L, sizeof(double));
    double* rr = (double*)calloc(3 * L, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * 3 * L);
    double* xv = (double*)malloc(sizeof(double) * L);
    double* dt = (double*)malloc(sizeof(double) * L);
    for (int p = 0; p < P; ++p) {
        const double* zp = z + p * L;
        memset(u, 0, sizeof(double) * 3 * L);
        memset(u_prev, 0, sizeof(double) * 3 * L);
        memset(rr, 0, sizeof(double) * 3 * L);
        double t = 1.0;
        for (int it = 0; it < iters; ++it) {
            grad3T(Y, X, Z, rr, dt);
            for (size_t i = 0; i < L; ++i) xv[i] = zp[i] - dt[i];
            grad3(Y, X, Z, xv, g);
            for (size_t i = 0; i < 3 * L; ++i) {
                double v = rr[i] + g[i] / 12.0;
                u[i] = v > tau ? tau : (v < -tau ? -tau : v);
            }
            double t1 = next_t(t);
            double beta = momentum_coef(momentum, t, t1);
            for (size_t i = 0; i < 3 * L; ++i) {
                rr[i] = u[i] + beta * (u[i] - u_prev[i]);
                u_prev[i] = u[i];
            }
            t = t1;
        }
        grad3T(Y, X, Z, u, dt);
        for (size_t i = 0; i < L; ++i) x[p * L + i] = zp[i] - dt[i];
    }
    free(u); free(u_prev); free(rr); free(g); free(xv); free(dt);
}

/* Full proximal map of w = lambda_TV TV + lambda_l1 ||.||_1 + indicator(>= 0)
 * at step alpha: max(prox_TV(z) - alpha lambda_l1, 0). */
void oracle_prox(int P, int Y, int X, int Z, const double* z, double* x,
                 double alpha, double lam_l1, double lam_tv, int inner, int momentum)
{
    size_t n = (size_t)P * Y * X * Z;
    if (lam_tv > 0.0 && inner > 0) {
        oracle_prox_tv(P, Y, X, Z, z, x, alpha * lam_tv, inner, momentum);
    } else {
        memcpy(x, z, sizeof(double) * n);
    }
    oracle_prox_l1(n, x, alpha * lam_l1, 1);
}

/* ---------------------------------------------------------------------------
 * The proximal map of alpha (R3 + delta_{>=0}) with all three terms of Eq.
 * (reg-tv-l1-one), by Algorithm 2 on the stacked operator
 *   L v = [ lam_tv D v_p  (p = 0..P-1) ;  lam_l1 v ;  lam_b D (S v)^n  (n = 0..N-1) ],
 * (S v)^n[j] = sum_p S[n][p][j] v_p[j] at every voxel, D the 3D forward
 * differences (one TV per species and one per pulse image, as R3 sums them).
 * Dual u = [uc (P x 3L) ; ul (P L) ; ub (N x 3L)] in the box |u| <= alpha
 * (Eq. prox-dual; the lambdas live in L), dual step `step2` (at most
 * 1/eig_max(L L^T)), u and its momentum iterate start at zero.  The prox of
 * Eq. (prox) includes the nonnegativity indicator, and Eq. (prox-dual) keeps
 * the matching constraint z - L^T u >= 0: the dual of the constrained problem
 * is min over |u| <= alpha of 1/2 ||max(z - L^T u, 0)||^2, whose gradient is
 * -L max(z - L^T u, 0).  So the projected primal point enters every step
 * (Algorithm 2 on this dual; the paper prints the clip on the output only):
 *   for i = 1..iters:
 *     w   = max(z - L^T r, 0)
 *     u_i = clamp(r + step2 L w, -alpha, alpha)
 *     t_{i+1} = (1 + sqrt(1 + 4 t_i^2)) / 2
 *     r   = u_i + beta_i (u_i - u_{i-1})
 *   x = max(z - L^T u_iters, 0)
 * u_out (optional) receives u_iters.  Sizes: S [N][P][Z], z and x [P][Y][X][Z].
 * ------------------------------------------------------------------------- */
static void joint_LT(int N, int P, int Y, int X, int Z, const double* S, double lam_tv,
                     double lam_l1, double lam_b, const double* u, double* out, double* tmp)
{
    const size_t L = (size_t)Y * X * Z;
    const double* uc = u;
    const double* ul = u + (size_t)P * 3 * L;
    const double* ub = ul + (size_t)P * L;
    for (int p = 0; p < P; ++p) {
        grad3T(Y, X, Z, uc + (size_t)p * 3 * L, out + (size_t)p * L);
        for (size_t i = 0; i < L; ++i)
            out[(size_t)p * L + i] = lam_tv * out[(size_t)p * L + i] + lam_l1 * ul[(size_t)p * L + i];
    }
    for (int n = 0; n < N; ++n) {
        grad3T(Y, X, Z, ub + (size_t)n * 3 * L, tmp);  /* D^T ub_n, a pulse image */
        for (int p = 0; p < P; ++p)
            for (size_t i = 0; i < L; ++i) {
                const int j = (int)(i % (size_t)Z);
                out[(size_t)p * L + i] += lam_b * S[((size_t)n * P + p) * Z + j] * tmp[i];
            }
    }
}

static void joint_L(int N, int P, int Y, int X, int Z, const double* S, double lam_tv,
                    double lam_l1, double lam_b, const double* v, double* out, double* tmp)
{
    const size_t L = (size_t)Y * X * Z;
    double* oc = out;
    double* ol = out + (size_t)P * 3 * L;
    double* ob = ol + (size_t)P * L;
    for (int p = 0; p < P; ++p) {
        grad3(Y, X, Z, v + (size_t)p * L, oc + (size_t)p * 3 * L);
        for (size_t i = 0; i < 3 * L; ++i) oc[(size_t)p * 3 * L + i] *= lam_tv;
        for (size_t i = 0; i < L; ++i) ol[(size_t)p * L + i] = lam_l1 * v[(size_t)p * L + i];
    }
    for (int n = 0; n < N; ++n) {
        for (size_t i = 0; i < L; ++i) {
            const int j = (int)(i % (size_t)Z);
            double b = 0.0;
            for (int p = 0; p < P; ++p) b += S[((size_t)n * P + p) * Z + j] * v[(size_t)p * L + i];
            tmp[i] = b;
        }
        grad3(Y, X, Z, tmp, ob + (size_t)n * 3 * L);
        for (size_t i = 0; i < 3 * L; ++i) ob[(size_t)n * 3 * L + i] *= lam_b;
    }
}

void oracle_prox_joint(int N, int P, int Y, int X, int Z, const double* S, const double* z,
                       double* x, double alpha, double lam_tv, double lam_l1, double lam_b,
                       int iters, double step2, int momentum, double* u_out)
{
    const size_t L = (size_t)Y * X * Z, nc = (size_t)P * L;
    const size_t nu = (size_t)P * 3 * L + (size_t)P * L + (size_t)N * 3 * L;
    double* u = (double*)calloc(nu, sizeof(double));
    double* u_prev = (double*)calloc(nu, sizeof(double));
    double* rr = (double*)calloc(nu, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * nu);
    double* w = (double*)malloc(sizeof(double) * nc);
    double* tmp = (double*)malloc(sizeof(double) * 3 * L);
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        joint_LT(N, P, Y, X, Z, S, lam_tv, lam_l1, lam_b, rr, w, tmp);
        for (size_t i = 0; i < nc; ++i) {
            const double v = z[i] - w[i];
            w[i] = v > 0.0 ? v : 0.0;
        }
        joint_L(N, P, Y, X, Z, S, lam_tv, lam_l1, lam_b, w, g, tmp);
        for (size_t i = 0; i < nu; ++i) {
            const double v = rr[i] + step2 * g[i];
            u[i] = v > alpha ? alpha : (v < -alpha ? -alpha : v);
        }
        const double t1 = next_t(t);
        const double beta = momentum_coef(momentum, t, t1);
        for (size_t i = 0; i < nu; ++i) {
            rr[i] = u[i] + beta * (u[i] - u_prev[i]);
            u_prev[i] = u[i];
        }
        t = t1;
    }
    joint_LT(N, P, Y, X, Z, S, lam_tv, lam_l1, lam_b, u, w, tmp);
    for (size_t i = 0; i < nc; ++i) {
        const double v = z[i] - w[i];
        x[i] = v > 0.0 ? v : 0.0;
    }
    if (u_out) memcpy(u_out, u, sizeof(double) * nu);
    free(u); free(u_prev); free(rr); free(g); free(w); free(tmp);
}

/* F(c) = 1/2 ||Hc - y||^2 + lambda_TV sum_p TV(c_p) + lambda_l1 ||c||_1 for c >= 0
 * (Eq. one-step with Eq. reg-tv-l1-one, lambda_3 = 0).  Returns also the
 * data-fit term in *fit. */
double oracle_objective(int N, int P, int Y, int X, int Z, int T, int k,
                        const double* S, const double* K, const double* c,
                        const double* yv, double lam_l1, double lam_tv, double* fit)
{
    size_t ny = (size_t)N * Y * X * T, nc = (size_t)P * Y * X * Z;
    double* hc = (double*)malloc(sizeof(double) * ny);
    oracle_forward(N, P, Y, X, Z, T, k, S, K, c, hc);
    double f = 0.0;
    for (size_t i = 0; i < ny; ++i) { double d = hc[i] - yv[i]; f += d * d; }
    f *= 0.5;
    double l1 = 0.0;
    for (size_t i = 0; i < nc; ++i) l1 += fabs(c[i]);
    double reg = lam_l1 * l1 + (lam_tv > 0.0 ? lam_tv * oracle_tv(P, Y, X, Z, c) : 0.0);
    free(hc);
    if (fit) *fit = f;
    return f + reg;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 (FISTA) with a fixed iteration count and a given step alpha:
 *   c_0 = xi_0 = 0, t_0 = 1
 *   for k = 0..iters-1:
 *     c_{k+1} = prox(xi_k - alpha H^T (H xi_k - y))
 *     t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
 *     xi_{k+1} = c_{k+1} + beta_k (c_{k+1} - c_k)
 * history (optional, length iters) receives F(c_{k+1}).
 * ------------------------------------------------------------------------- */
void oracle_fista(int N, int P, int Y, int X, int Z, int T, int k,
                  const double* S, const double* K, const double* yv,
                  double alpha, int iters, double lam_l1, double lam_tv,
                  int inner, int momentum, int inner_momentum,
                  double* c_out, double* history)
{
    size_t ny = (size_t)N * Y * X * T, nc = (size_t)P * Y * X * Z;
    double* c = (double*)calloc(nc, sizeof(double));
    double* c_new = (double*)malloc(sizeof(double) * nc);
    double* xi = (double*)calloc(nc, sizeof(double));
    double* zin = (double*)malloc(sizeof(double) * nc);
    double* grad = (double*)malloc(sizeof(double) * nc);
    double* res = (double*)malloc(sizeof(double) * ny);
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        oracle_forward(N, P, Y, X, Z, T, k, S, K, xi, res);
        for (size_t i = 0; i < ny; ++i) res[i] -= yv[i];
        oracle_adjoint(N, P, Y, X, Z, T, k, S, K, res, grad);
        for (size_t i = 0; i < nc; ++i) zin[i] = xi[i] - alpha * grad[i];
        if (lam_tv > 0.0 && inner > 0)
            oracle_prox_tv(P, Y, X, Z, zin, c_new, alpha * lam_tv, inner, inner_momentum);
        else
            memcpy(c_new, zin, sizeof(double) * nc);
        oracle_prox_l1(nc, c_new, alpha * lam_l1, 1);
        double t1 = next_t(t);
        double beta = momentum_coef(momentum, t, t1);
        for (size_t i = 0; i < nc; ++i) {
            xi[i] = c_new[i] + beta * (c_new[i] - c[i]);
            c[i] = c_new[i];
        }
        t = t1;
        if (history)
            history[it] = oracle_objective(N, P, Y, X, Z, T, k, S, K, c, yv, lam_l1, lam_tv, NULL);
    }
    memcpy(c_out, c, sizeof(double) * nc);
    free(c); free(c_new); free(xi); free(zin); free(grad); free(res);
}

/* sum_n TV((S c)^n): the lambda_3 term of Eq. (reg-tv-l1-one), TV of every
 * pulse image (S c)^n[j] = sum_p S[n][p][j] c_p[j]. */
double oracle_tv_pulses(int N, int P, int Y, int X, int Z, const double* S, const double* c)
{
    const size_t L = (size_t)Y * X * Z;
    double* b = (double*)malloc(sizeof(double) * L);
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
        for (size_t i = 0; i < L; ++i) {
            const int j = (int)(i % (size_t)Z);
            double v = 0.0;
            for (int p = 0; p < P; ++p) v += S[((size_t)n * P + p) * Z + j] * c[(size_t)p * L + i];
            b[i] = v;
        }
        s += oracle_tv(1, Y, X, Z, b);
    }
    free(b);
    return s;
}

/* Algorithm 1 with all three terms of Eq. (reg-tv-l1-one): as oracle_fista,
 * with the prox of alpha (R3 + delta_{>=0}) taken by oracle_prox_joint
 * (inner dual iterations with dual step step2 and inner_momentum).  history
 * (optional) receives F(c_{k+1}) including lam_3 sum_n TV((S c)^n). */
void oracle_fista_joint(int N, int P, int Y, int X, int Z, int T, int k,
                        const double* S, const double* K, const double* yv,
                        double alpha, int iters, double lam_l1, double lam_tv, double lam_3,
                        int inner, double step2, int momentum, int inner_momentum,
                        double* c_out, double* history)
{
    size_t ny = (size_t)N * Y * X * T, nc = (size_t)P * Y * X * Z;
    double* c = (double*)calloc(nc, sizeof(double));
    double* c_new = (double*)malloc(sizeof(double) * nc);
    double* xi = (double*)calloc(nc, sizeof(double));
    double* zin = (double*)malloc(sizeof(double) * nc);
    double* grad = (double*)malloc(sizeof(double) * nc);
    double* res = (double*)malloc(sizeof(double) * ny);
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        oracle_forward(N, P, Y, X, Z, T, k, S, K, xi, res);
        for (size_t i = 0; i < ny; ++i) res[i] -= yv[i];
        oracle_adjoint(N, P, Y, X, Z, T, k, S, K, res, grad);
        for (size_t i = 0; i < nc; ++i) zin[i] = xi[i] - alpha * grad[i];
        oracle_prox_joint(N, P, Y, X, Z, S, zin, c_new, alpha, lam_tv, lam_l1, lam_3, inner,
                          step2, inner_momentum, NULL);
        double t1 = next_t(t);
        double beta = momentum_coef(momentum, t, t1);
        for (size_t i = 0; i < nc; ++i) {
            xi[i] = c_new[i] + beta * (c_new[i] - c[i]);
            c[i] = c_new[i];
        }
        t = t1;
        if (history)
            history[it] = oracle_objective(N, P, Y, X, Z, T, k, S, K, c, yv, lam_l1, lam_tv, NULL) +
                          lam_3 * oracle_tv_pulses(N, P, Y, X, Z, S, c);
    }
    memcpy(c_out, c, sizeof(double) * nc);
    free(c); free(c_new); free(xi); free(zin); free(grad); free(res);
}

/* ---------------------------------------------------------------------------
 * Fluence from the diffusion equation, Eqs. (de), (bc) and
 * (diffusion-coefficient), by cell-centred finite volumes on the voxel grid
 * (lateral pitch dx, depth pitch dz, voxel i = (y, x, j), j = 0 the
 * illuminated top face).  Per voxel, divided by its volume:
 *   mu_a_i Phi_i + sum over its six faces of (outward flux through the face) / h_face = s_i
 * with D = 1 / (3 (mu_a + (1 - g) mu_s)) per voxel and, across a face of
 * normal pitch h,
 *   inner face to voxel k : D_f (Phi_i - Phi_k) / h,   D_f = 2 D_i D_k / (D_i + D_k)
 *   boundary face         : 2 D_i Phi_i / (4 D_i + h)
 * the last from the boundary condition taken as Phi + 2 D dPhi/dn = 0 with n
 * the outward normal (the boundary value Phi_b from D (Phi_i - Phi_b)/(h/2) =
 * Phi_b / 2, the outgoing flux Phi_b / 2).  Lateral faces are boundary faces
 * (lateral_robin = 1) or carry no flux (0: a laterally unbounded sample).
 * The source is the illumination entering the top face, src_top[y][x] (power
 * per area), in the top layer: s = src_top / dz for j = 0.
 * Output: the matrix as (row, col, value) triplets (at most 7 per row;
 * returns their count) and the right-hand side; Phi is [Y][X][Z].
 * ------------------------------------------------------------------------- */
int oracle_diffusion_system(int Y, int X, int Z, double dx, double dz, const double* mu_a,
                            const double* mu_s, double g, const double* src_top,
                            int lateral_robin, int* rows, int* cols, double* vals, double* rhs)
{
    const size_t n = (size_t)Y * X * Z;
    double* D = (double*)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) D[i] = 1.0 / (3.0 * (mu_a[i] + (1.0 - g) * mu_s[i]));
    int cnt = 0;
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x)
            for (int j = 0; j < Z; ++j) {
                const int i = (y * X + x) * Z + j;
                double diag = mu_a[i];
                /* the six faces: (axis pitch, neighbour exists, neighbour index, boundary kind) */
                const int ny[6] = {y - 1, y + 1, y, y, y, y};
                const int nx[6] = {x, x, x - 1, x + 1, x, x};
                const int nj[6] = {j, j, j, j, j - 1, j + 1};
                for (int f = 0; f < 6; ++f) {
                    const double h = f < 4 ? dx : dz;
                    const int inside = ny[f] >= 0 && ny[f] < Y && nx[f] >= 0 && nx[f] < X &&
                                       nj[f] >= 0 && nj[f] < Z;
                    if (inside) {
                        const int k = (ny[f] * X + nx[f]) * Z + nj[f];
                        const double Df = 2.0 * D[i] * D[k] / (D[i] + D[k]);
                        const double w = Df / (h * h);
                        diag += w;
                        rows[cnt] = i; cols[cnt] = k; vals[cnt] = -w; ++cnt;
                    } else if (f >= 4 || lateral_robin) {
                        diag += 2.0 * D[i] / (4.0 * D[i] + h) / h;
                    }
                }
                rows[cnt] = i; cols[cnt] = i; vals[cnt] = diag; ++cnt;
                rhs[i] = j == 0 ? src_top[y * X + x] / dz : 0.0;
            }
    free(D);
    return cnt;
}

/* Power iteration for eig_max(H^T H): v <- H^T H v / ||H^T H v|| from the
 * given start vector; returns the Rayleigh quotient v^T H^T H v / v^T v. */
double oracle_power(int N, int P, int Y, int X, int Z, int T, int k,
                    const double* S, const double* K, const double* v0, int iters)
{
    size_t ny = (size_t)N * Y * X * T, nc = (size_t)P * Y * X * Z;
    double* v = (double*)malloc(sizeof(double) * nc);
    double* w = (double*)malloc(sizeof(double) * nc);
    double* hv = (double*)malloc(sizeof(double) * ny);
    double nrm = 0.0;
    for (size_t i = 0; i < nc; ++i) nrm += v0[i] * v0[i];
    nrm = sqrt(nrm);
    for (size_t i = 0; i < nc; ++i) v[i] = v0[i] / nrm;
    double rq = 0.0;
    for (int it = 0; it < iters; ++it) {
        oracle_forward(N, P, Y, X, Z, T, k, S, K, v, hv);
        oracle_adjoint(N, P, Y, X, Z, T, k, S, K, hv, w);
        double vw = 0.0, ww = 0.0;
        for (size_t i = 0; i < nc; ++i) { vw += v[i] * w[i]; ww += w[i] * w[i]; }
        rq = vw; /* v has unit norm */
        ww = sqrt(ww);
        for (size_t i = 0; i < nc; ++i) v[i] = w[i] / ww;
    }
    free(v); free(w); free(hv);
    return rq;
}

/* ---------------------------------------------------------------------------
 * Gradient of f = 1/2 ||H c - y||^2 with respect to the kinetic constants
 * kappa_p and the fluence decay mu, with c held fixed.  Writing
 * b = S c and g = W_tot^T (H c - y):
 *   df/dtheta = sum_{n,y,x,j} g[n][y][x][j] * sum_p dS[n][p][j]/dtheta c[p][y][x][j]
 * where, from Eq. (final-H) with Phi_j = exp(-mu j dz) and e = exp(-kappa_p Phi_j m):
 *   dS/dkappa_p = Phi_j * eps_bar_p * e * (-Phi_j m)
 *   dS/dPhi     = eps_bar_p e + eps_off_p + Phi_j eps_bar_p e (-kappa_p m)
 *   dS/dmu      = dS/dPhi * (-j dz Phi_j)
 * ------------------------------------------------------------------------- */
void oracle_param_grad(int N, int P, int Y, int X, int Z, int T, int k,
                       int pulses_per_cycle, double mu_per_mm, double dz_mm,
                       const double* kappa, const double* eps_bar, const double* eps_off,
                       const double* K, const double* c, const double* yv,
                       double* dkappa, double* dmu)
{
    const int r = k / 2;
    size_t ny = (size_t)N * Y * X * T;
    double* phi = (double*)malloc(sizeof(double) * Z);
    double* S = (double*)malloc(sizeof(double) * (size_t)N * P * Z);
    double* res = (double*)malloc(sizeof(double) * ny);
    double* g = (double*)malloc(sizeof(double) * (size_t)N * Y * X * Z);
    oracle_fluence(Z, mu_per_mm, dz_mm, phi);
    oracle_switch_matrix(N, P, Z, pulses_per_cycle, phi, kappa, eps_bar, eps_off, S);
    oracle_forward(N, P, Y, X, Z, T, k, S, K, c, res);
    for (size_t i = 0; i < ny; ++i) res[i] -= yv[i];
    /* g = W_tot^T res (acoustic adjoint only) */
    for (int n = 0; n < N; ++n)
        for (int yy = 0; yy < Y; ++yy)
            for (int xx = 0; xx < X; ++xx)
                for (int j = 0; j < Z; ++j) {
                    double acc = 0.0;
                    for (int dy = -r; dy <= r; ++dy) {
                        int ty = yy - dy;
                        if (ty < 0 || ty >= Y) continue;
                        for (int dx = -r; dx <= r; ++dx) {
                            int tx = xx - dx;
                            if (tx < 0 || tx >= X) continue;
                            const double* yp = res + IDX4(n, ty, tx, 0, Y, X, T);
                            const double* Kp = K + IDX4(j, dy + r, dx + r, 0, k, k, T);
                            for (int t = 0; t < T; ++t) acc += yp[t] * Kp[t];
                        }
                    }
                    g[IDX4(n, yy, xx, j, Y, X, Z)] = acc;
                }
    for (int p = 0; p < P; ++p) dkappa[p] = 0.0;
    *dmu = 0.0;
    for (int n = 0; n < N; ++n) {
        double m = (double)(n % pulses_per_cycle);
        for (int j = 0; j < Z; ++j) {
            double ph = phi[j];
            double dphi_dmu = -(double)j * dz_mm * ph;
            for (int p = 0; p < P; ++p) {
                double e = exp(-kappa[p] * ph * m);
                double dS_dk = ph * eps_bar[p] * e * (-ph * m);
                double dS_dphi = eps_bar[p] * e + eps_off[p] + ph * eps_bar[p] * e * (-kappa[p] * m);
                double dS_dmu = dS_dphi * dphi_dmu;
                double acc = 0.0;
                for (int yy = 0; yy < Y; ++yy)
                    for (int xx = 0; xx < X; ++xx)
                        acc += g[IDX4(n, yy, xx, j, Y, X, Z)] * c[IDX4(p, yy, xx, j, Y, X, Z)];
                dkappa[p] += dS_dk * acc;
                *dmu += dS_dmu * acc;
            }
        }
    }
    free(phi); free(S); free(res); free(g);
}

/* The paper-literal per-depth kernel (Sec. 2.3.1 "Acoustic Model", Eqs.
 * q-above-final and q-below-final, discrete semicircles of Eqs.
 * discrete-upper-circle / discrete-lower-circle): the weight of depth j,
 * lateral offset (dy, dx) and time sample t is eta[j][dy][dx] if the voxel
 * meets the half sphere of radius |t - tf| about the focus (depth kf), on
 * the side of the focus that sample t sees (upper for t < tf, lower for
 * t > tf), else 0; then every column is convolved with the centred impulse
 * response eir.  Units: depth pitches (time grid matched to the depth grid;
 * one lateral pitch is rho depth pitches).  "Meets" is read as: the closed
 * voxel box, clipped to the half space, holds a point at distance exactly
 * the radius; as |p| is continuous on the (connected) box, that is: the
 * nearest point of the box is within the radius and some corner is not
 * inside it.  2D (dims 2): the (x, z) plane, dy = 0 only. */
void oracle_semicircle_kernel(int Z, int k, int T, int dims, double rho, double kf, int tf,
                              const double* eta, const double* eir, int eir_len, double* K)
{
    const int r = k / 2, J = eir_len / 2;
    double* col = (double*)malloc(sizeof(double) * (size_t)T);
    for (int j = 0; j < Z; ++j)
        for (int iy = 0; iy < k; ++iy)
            for (int ix = 0; ix < k; ++ix) {
                const int dy = iy - r, dx = ix - r;
                const double w = eta[((size_t)j * k + iy) * k + ix];
                for (int t = 0; t < T; ++t) {
                    col[t] = 0.0;
                    if (dims == 2 && dy != 0) continue;
                    double lo[3], hi[3];
                    lo[0] = (dx - 0.5) * rho; hi[0] = (dx + 0.5) * rho;
                    lo[1] = (dy - 0.5) * rho; hi[1] = (dy + 0.5) * rho;
                    if (dims == 2) lo[1] = hi[1] = 0.0;
                    lo[2] = (double)j - kf - 0.5; hi[2] = (double)j - kf + 0.5;
                    if (t < tf && hi[2] > 0.0) hi[2] = 0.0;
                    if (t > tf && lo[2] < 0.0) lo[2] = 0.0;
                    if (lo[2] > hi[2]) continue;
                    const double n2 = (double)(t - tf) * (double)(t - tf);
                    /* nearest point of the box: the focus clamped into it */
                    double near2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        double c = 0.0;
                        if (c < lo[a]) c = lo[a];
                        if (c > hi[a]) c = hi[a];
                        near2 += c * c;
                    }
                    /* farthest point: one of the eight corners */
                    double far2 = 0.0;
                    for (int corner = 0; corner < 8; ++corner) {
                        double d2 = 0.0;
                        for (int a = 0; a < 3; ++a) {
                            const double c = (corner >> a) & 1 ? hi[a] : lo[a];
                            d2 += c * c;
                        }
                        if (d2 > far2) far2 = d2;
                    }
                    if (near2 <= n2 && far2 >= n2) col[t] = w;
                }
                /* each source sample u spreads over t = u + s, s in [-J, J] */
                double* out = K + (((size_t)j * k + iy) * k + ix) * (size_t)T;
                for (int t = 0; t < T; ++t) out[t] = 0.0;
                for (int u = 0; u < T; ++u) {
                    if (col[u] == 0.0) continue;
                    for (int s = -J; s <= J; ++s)
                        if (u + s >= 0 && u + s < T) out[u + s] += col[u] * eir[s + J];
                }
            }
    free(col);
}

/* The two-step approach (the paper's "Two-Step Approach"): the acoustic
 * problem of Eq. (acoustic-inverse) and then the unmixing problem of Eq.
 * (unmixing), each by Algorithm 1 (oracle_fista, Beck-Teboulle momentum).
 * W_tot is block diagonal over the pulses, so the acoustic problem is solved
 * pulse by pulse with the switching matrix 1 (one species, weight 1 at
 * every depth); the unmixing operator is S alone, which is H with the
 * depth-to-time identity as its acoustic kernel (k = 1, T = Z).
 * S: [N][P][Z]; yv: [N][Y][X][T]; b_out: [N][Y][X][Z]; c_out: [P][Y][X][Z]. */
void oracle_two_step(int N, int P, int Y, int X, int Z, int T, int k,
                     const double* S, const double* K, const double* yv,
                     double alpha1, int iters1, double lam_l1_1, double lam_tv_1, int inner1,
                     double alpha2, int iters2, double lam_l1_2, double lam_tv_2, int inner2,
                     double* b_out, double* c_out)
{
    const size_t yxt = (size_t)Y * X * T, yxz = (size_t)Y * X * Z;
    double* S1 = (double*)malloc(sizeof(double) * (size_t)Z);
    for (int j = 0; j < Z; ++j) S1[j] = 1.0;
    for (int n = 0; n < N; ++n)
        oracle_fista(1, 1, Y, X, Z, T, k, S1, K, yv + (size_t)n * yxt, alpha1, iters1, lam_l1_1,
                     lam_tv_1, inner1, 0, 0, b_out + (size_t)n * yxz, NULL);
    double* eye = (double*)calloc((size_t)Z * Z, sizeof(double));
    for (int j = 0; j < Z; ++j) eye[(size_t)j * Z + j] = 1.0;
    oracle_fista(N, P, Y, X, Z, Z, 1, S, eye, b_out, alpha2, iters2, lam_l1_2, lam_tv_2, inner2,
                 0, 0, c_out, NULL);
    free(S1);
    free(eye);
}

/* ---------------------------------------------------------------------------
 * Derivative of the switching matrix of Eq. (final-H) with respect to one
 * parameter: which = p (0 <= p < P) for kappa_p, which = P for mu.
 *   S = Phi (eps_bar e^{-kappa Phi m} + eps_off),  Phi = e^{-mu j dz}
 *   dS/dkappa_p = -Phi^2 m eps_bar_p e^{-kappa_p Phi m}   (species p only)
 *   dS/dmu      = dS/dPhi * dPhi/dmu,  dPhi/dmu = -j dz Phi,
 *   dS/dPhi     = eps_bar e^{-kappa Phi m} + eps_off - Phi eps_bar kappa m e^{-kappa Phi m}
 * ------------------------------------------------------------------------- */
void oracle_switch_matrix_derivative(int N, int P, int Z, int pulses_per_cycle, double mu_per_mm,
                                     double dz_mm, const double* kappa, const double* eps_bar,
                                     const double* eps_off, int which, double* dS)
{
    for (int n = 0; n < N; ++n) {
        const double m = (double)(n % pulses_per_cycle);
        for (int p = 0; p < P; ++p)
            for (int j = 0; j < Z; ++j) {
                const double ph = exp(-mu_per_mm * (double)j * dz_mm);
                const double e = exp(-kappa[p] * ph * m);
                double d = 0.0;
                if (which == P) {
                    const double dS_dphi = eps_bar[p] * e + eps_off[p] - ph * eps_bar[p] * kappa[p] * m * e;
                    d = dS_dphi * (-(double)j * dz_mm * ph);
                } else if (which == p) {
                    d = -ph * ph * m * eps_bar[p] * e;
                }
                dS[IDX4(0, n, p, j, N, P, Z)] = d;
            }
    }
}

/* ---------------------------------------------------------------------------
 * Differentiating through the unrolled solve (forward mode): Algorithm 1
 * exactly as oracle_fista (step alpha, weights and counts held fixed), with
 * the tangent of every quantity carried along for a change of S by dS (the
 * derivative of S with respect to one switching parameter):
 *   r  = H xi - y,                     dr  = A(dS xi) + A(S dxi)
 *   g  = H^T r,                        dg  = dS^T A^T r + S^T A^T dr
 *   z  = xi - alpha g,                 dz  = dxi - alpha dg
 *   Algorithm 2 (per species): w = z - D^T q, v = q + D w / 12,
 *     u = clamp(v, -tau, tau),         du  = [|v| < tau] (dq + D dw / 12)
 *     q = u + beta (u - u_prev),       dq  = du + beta (du - du_prev)
 *   x = z - D^T u,  c = max(x - alpha lambda_l1, 0),
 *                                      dc  = [x - alpha lambda_l1 > 0] dx
 *   xi = c + beta (c - c_prev),        dxi = dc + beta (dc - dc_prev)
 * The map is piecewise linear in the data; the tangent is the derivative
 * wherever no clamp or clip sits exactly on its threshold.
 * c_out, dc_out: [P][Y][X][Z].
 * ------------------------------------------------------------------------- */
static void prox_tv_tangent(int Y, int X, int Z, const double* z, const double* dz, double* x,
                            double* dx, double tau, int iters, int momentum)
{
    const size_t L = (size_t)Y * X * Z;
    double* u = (double*)calloc(3 * L, sizeof(double));
    double* up = (double*)calloc(3 * L, sizeof(double));
    double* q = (double*)calloc(3 * L, sizeof(double));
    double* du = (double*)calloc(3 * L, sizeof(double));
    double* dup = (double*)calloc(3 * L, sizeof(double));
    double* dq = (double*)calloc(3 * L, sizeof(double));
    double* g = (double*)malloc(sizeof(double) * 3 * L);
    double* dg = (double*)malloc(sizeof(double) * 3 * L);
    double* w = (double*)malloc(sizeof(double) * L);
    double* dw = (double*)malloc(sizeof(double) * L);
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        grad3T(Y, X, Z, q, w);
        grad3T(Y, X, Z, dq, dw);
        for (size_t i = 0; i < L; ++i) {
            w[i] = z[i] - w[i];
            dw[i] = dz[i] - dw[i];
        }
        grad3(Y, X, Z, w, g);
        grad3(Y, X, Z, dw, dg);
        for (size_t i = 0; i < 3 * L; ++i) {
            const double v = q[i] + g[i] / 12.0;
            if (v > tau) {
                u[i] = tau;
                du[i] = 0.0;
            } else if (v < -tau) {
                u[i] = -tau;
                du[i] = 0.0;
            } else {
                u[i] = v;
                du[i] = dq[i] + dg[i] / 12.0;
            }
        }
        const double t1 = next_t(t);
        const double beta = momentum_coef(momentum, t, t1);
        for (size_t i = 0; i < 3 * L; ++i) {
            q[i] = u[i] + beta * (u[i] - up[i]);
            dq[i] = du[i] + beta * (du[i] - dup[i]);
            up[i] = u[i];
            dup[i] = du[i];
        }
        t = t1;
    }
    grad3T(Y, X, Z, u, w);
    grad3T(Y, X, Z, du, dw);
    for (size_t i = 0; i < L; ++i) {
        x[i] = z[i] - w[i];
        dx[i] = dz[i] - dw[i];
    }
    free(u); free(up); free(q); free(du); free(dup); free(dq); free(g); free(dg); free(w); free(dw);
}

void oracle_fista_tangent(int N, int P, int Y, int X, int Z, int T, int k, const double* S,
                          const double* dS, const double* K, const double* yv, double alpha,
                          int iters, double lam_l1, double lam_tv, int inner, int momentum,
                          int inner_momentum, double* c_out, double* dc_out)
{
    const size_t ny = (size_t)N * Y * X * T, nc = (size_t)P * Y * X * Z, L = (size_t)Y * X * Z;
    double* c = (double*)calloc(nc, sizeof(double));
    double* dc = (double*)calloc(nc, sizeof(double));
    double* xi = (double*)calloc(nc, sizeof(double));
    double* dxi = (double*)calloc(nc, sizeof(double));
    double* zin = (double*)malloc(sizeof(double) * nc);
    double* dzin = (double*)malloc(sizeof(double) * nc);
    double* xv = (double*)malloc(sizeof(double) * nc);
    double* dxv = (double*)malloc(sizeof(double) * nc);
    double* g = (double*)malloc(sizeof(double) * nc);
    double* tmpc = (double*)malloc(sizeof(double) * nc);
    double* res = (double*)malloc(sizeof(double) * ny);
    double* dres = (double*)malloc(sizeof(double) * ny);
    double* tmpy = (double*)malloc(sizeof(double) * ny);
    double t = 1.0;
    for (int it = 0; it < iters; ++it) {
        oracle_forward(N, P, Y, X, Z, T, k, S, K, xi, res);
        for (size_t i = 0; i < ny; ++i) res[i] -= yv[i];
        oracle_forward(N, P, Y, X, Z, T, k, dS, K, xi, dres);
        oracle_forward(N, P, Y, X, Z, T, k, S, K, dxi, tmpy);
        for (size_t i = 0; i < ny; ++i) dres[i] += tmpy[i];
        oracle_adjoint(N, P, Y, X, Z, T, k, S, K, res, g);
        for (size_t i = 0; i < nc; ++i) zin[i] = xi[i] - alpha * g[i];
        oracle_adjoint(N, P, Y, X, Z, T, k, dS, K, res, g);
        oracle_adjoint(N, P, Y, X, Z, T, k, S, K, dres, tmpc);
        for (size_t i = 0; i < nc; ++i) dzin[i] = dxi[i] - alpha * (g[i] + tmpc[i]);
        if (lam_tv > 0.0 && inner > 0) {
            for (int p = 0; p < P; ++p)
                prox_tv_tangent(Y, X, Z, zin + p * L, dzin + p * L, xv + p * L, dxv + p * L,
                                alpha * lam_tv, inner, inner_momentum);
        } else {
            memcpy(xv, zin, sizeof(double) * nc);
            memcpy(dxv, dzin, sizeof(double) * nc);
        }
        const double t1 = next_t(t);
        const double beta = momentum_coef(momentum, t, t1);
        const double th = alpha * lam_l1;
        for (size_t i = 0; i < nc; ++i) {
            const double v = xv[i] - th;
            const double cn = v > 0.0 ? v : 0.0;
            const double dcn = v > 0.0 ? dxv[i] : 0.0;
            xi[i] = cn + beta * (cn - c[i]);
            dxi[i] = dcn + beta * (dcn - dc[i]);
            c[i] = cn;
            dc[i] = dcn;
        }
        t = t1;
    }
    memcpy(c_out, c, sizeof(double) * nc);
    memcpy(dc_out, dc, sizeof(double) * nc);
    free(c); free(dc); free(xi); free(dxi); free(zin); free(dzin); free(xv); free(dxv);
    free(g); free(tmpc); free(res); free(dres); free(tmpy);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of later parallel regions (timing only; no effect on results). */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
