/*
 * tco.c -- CPU oracle for the Coulomb-charges-in-a-disk hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * single-thread FP64 statement of what the GPU library computes.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline arm may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Every sum over pairs uses Neumaier-compensated accumulation; 1/r is
 * 1.0 / sqrt(r^2) with IEEE correctly rounded sqrt and divide.  Build with
 * -ffp-contract=off so no fused multiply-add changes the rounding.
 *
 * Paper: Thomson problem in a disk, N = 100 000 (Lavrov & Nikonov).
 *   Eq. (hamiltonian) + Eq. (potential), Sec. II A: E = sum_{i<j} 1/|r_i - r_j|,
 *       wall term 0 for |r| <= R = 1, infinite outside.
 *   Sec. II C, step 1: local energy e_i = 1/2 sum_{j != i} 1/|r_i - r_j|.
 *   Sec. II D: subdomain objective E_sub = sum_{i in A} e_i with
 *       e_i = 1/2 sum_{j in A, j != i} 1/r_ij + sum_{j in F} 1/r_ij,
 *       optimised by a box-constrained quasi-Newton method with analytic
 *       gradients (Sec. II C step 4).
 *   Sec. II E: each subproblem's gradient is n_act rows against all N charges.
 *   Sec. II C, steps 2-4: defect threshold on the local energies, centre
 *       choice (defect charge or uniform point), the zone around the centre,
 *       and the optimisation cycle built from them.
 *   Sec. II C step 4 + Sec. II D: L-BFGS-B (Byrd, Lu, Nocedal & Zhu 1995) on
 *       the (t, u) variables with the box t in [0, pi/2], for a whole
 *       configuration or a subdomain against the fixed others, and the cycle
 *       with it as the zone optimiser.
 *
 * Parity status: every function here is pinned by tests against closed forms,
 * brute force in extended precision, invariants or the paper's asymptotic
 * expansion (Eq. asym); see tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TCO_OK 0
#define TCO_ERR_INVALID_ARG 1
#define TCO_ERR_NONFINITE 3
#define TCO_ERR_OUTSIDE_DISK 4
#define TCO_ERR_NO_MEMORY 7

/* A charge with |r| above this radius is outside the hard wall of Eq. (potential);
 * the slack admits positions a projection left one rounding above R = 1. */
#define TCO_WALL_SLACK 1e-12

#define TCO_PI 3.14159265358979323846

/* ---------------------------------------------------------------- sums --- */

typedef struct {
    double s; /* running sum */
    double c; /* running compensation */
} acc_t;

static void acc_add(acc_t* a, double v)
{
    /* Neumaier's improvement of Kahan summation */
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static double acc_get(const acc_t* a) { return a->s + a->c; }

static double inv_dist(double xi, double yi, double xj, double yj)
{
    double dx = xi - xj;
    double dy = yi - yj;
    double r2 = dx * dx + dy * dy;
    return 1.0 / sqrt(r2);
}

static int check_inside(const double* pos, int64_t n)
{
    double lim = 1.0 + TCO_WALL_SLACK;
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1];
        if (!(isfinite(x) && isfinite(y))) return TCO_ERR_NONFINITE;
        if (sqrt(x * x + y * y) > lim) return TCO_ERR_OUTSIDE_DISK;
    }
    return TCO_OK;
}

/* ------------------------------------------------------------ energies --- */

/* E = sum_{i<j} 1/|r_i - r_j| (Eq. hamiltonian; V = 0 inside the disk).
 * local_e (nullable, n): e_i = 1/2 sum_{j != i} 1/r_ij (Sec. II C step 1). */
int tco_energy(const double* pos, int64_t n, double* energy, double* local_e)
{
    if (n < 0 || (n > 0 && !pos) || !energy) return TCO_ERR_INVALID_ARG;
    int st = check_inside(pos, n);
    if (st) return st;
    acc_t E = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            acc_add(&E, inv_dist(pos[2 * i], pos[2 * i + 1], pos[2 * j], pos[2 * j + 1]));
    *energy = acc_get(&E);
    if (local_e) {
        for (int64_t i = 0; i < n; ++i) {
            acc_t e = {0.0, 0.0};
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                acc_add(&e, inv_dist(pos[2 * i], pos[2 * i + 1], pos[2 * j], pos[2 * j + 1]));
            }
            local_e[i] = 0.5 * acc_get(&e);
        }
    }
    return isfinite(*energy) ? TCO_OK : TCO_ERR_NONFINITE;
}

/* One gradient row: g = sum over sources j (j != skip) of -(r - r_j)/|r - r_j|^3,
 * and the row's sum of 1/|r - r_j| (both compensated). */
static void grad_row(double x, double y, const double* src, int64_t ns, int64_t skip,
                     const unsigned char* exclude, acc_t* gx, acc_t* gy, acc_t* e)
{
    for (int64_t j = 0; j < ns; ++j) {
        if (j == skip) continue;
        if (exclude && exclude[j]) continue;
        double dx = x - src[2 * j];
        double dy = y - src[2 * j + 1];
        double r2 = dx * dx + dy * dy;
        double inv = 1.0 / sqrt(r2);
        double inv3 = inv * inv * inv;
        acc_add(gx, -dx * inv3);
        acc_add(gy, -dy * inv3);
        if (e) acc_add(e, inv);
    }
}

/* g_i = dE/dr_i = sum_{j != i} -(r_i - r_j)/|r_i - r_j|^3 (analytic gradient of
 * Eq. hamiltonian; the force is -g).  grad: 2n doubles, interleaved. */
int tco_grad(const double* pos, int64_t n, double* grad)
{
    if (n < 0 || (n > 0 && (!pos || !grad))) return TCO_ERR_INVALID_ARG;
    int st = check_inside(pos, n);
    if (st) return st;
    int bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        acc_t gx = {0.0, 0.0}, gy = {0.0, 0.0};
        grad_row(pos[2 * i], pos[2 * i + 1], pos, n, i, NULL, &gx, &gy, NULL);
        grad[2 * i] = acc_get(&gx);
        grad[2 * i + 1] = acc_get(&gy);
        if (!isfinite(grad[2 * i]) || !isfinite(grad[2 * i + 1])) bad = 1;
    }
    return bad ? TCO_ERR_NONFINITE : TCO_OK;
}

/* Gradient rows of selected charges against all n (Sec. II E: n_act rows x N).
 * rows: m indices; grad_rows: 2m; e_rows (nullable, m): sum_{j != i} 1/r_ij. */
int tco_rows_grad(const double* pos, int64_t n, const int32_t* rows, int64_t m,
                  double* grad_rows, double* e_rows)
{
    if (n < 0 || m < 0 || (m > 0 && (!rows || !grad_rows || !pos))) return TCO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < m; ++k)
        if (rows[k] < 0 || rows[k] >= n) return TCO_ERR_INVALID_ARG;
    int bad = 0;
    /* Rows are independent; the OpenMP build (libtco_omp.so) splits them over
     * threads with identical per-row arithmetic, so both builds agree bit for bit. */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
#endif
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = rows[k];
        acc_t gx = {0.0, 0.0}, gy = {0.0, 0.0}, e = {0.0, 0.0};
        grad_row(pos[2 * i], pos[2 * i + 1], pos, n, i, NULL, &gx, &gy, &e);
        grad_rows[2 * k] = acc_get(&gx);
        grad_rows[2 * k + 1] = acc_get(&gy);
        if (e_rows) e_rows[k] = acc_get(&e);
        if (!isfinite(grad_rows[2 * k]) || !isfinite(grad_rows[2 * k + 1])) bad = 1;
    }
    return bad ? TCO_ERR_NONFINITE : TCO_OK;
}

/* Threads the rows_grad loop runs on: 1 in the plain build. */
int tco_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static unsigned char* membership(int64_t n, const int32_t* idx, int64_t m, int* st)
{
    unsigned char* in_a = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    *st = TCO_OK;
    if (!in_a) { *st = TCO_ERR_NO_MEMORY; return NULL; }
    for (int64_t k = 0; k < m; ++k) {
        if (idx[k] < 0 || idx[k] >= n || in_a[idx[k]]) {
            free(in_a);
            *st = TCO_ERR_INVALID_ARG;
            return NULL;
        }
        in_a[idx[k]] = 1;
    }
    return in_a;
}

/* Subdomain objective of Sec. II D for active set A (idx, m) whose charges sit
 * at act (2m) while every other charge j in F sits at snap[j]:
 *   e_k = 1/2 sum_{k' in A, k' != k} 1/|a_k - a_k'| + sum_{j in F} 1/|a_k - s_j|,
 *   E_sub = sum_k e_k,  grad_k = dE_sub/da_k
 *         = sum_{k' != k} -(a_k - a_k')/|.|^3 + sum_{j in F} -(a_k - s_j)/|.|^3.
 * (The A-A pair enters E_sub once via the two halves, and each half-term's
 * derivative appears in both rows, so the row gradient carries the full A-A
 * term.)  grad (2m), e (nullable, m), e_sub (nullable). */
int tco_subdomain_grad(const double* snap, int64_t n, const int32_t* idx, int64_t m,
                       const double* act, double* grad, double* e, double* e_sub)
{
    if (n < 0 || m < 0 || (m > 0 && (!idx || !act || !grad || !snap))) return TCO_ERR_INVALID_ARG;
    int st;
    unsigned char* in_a = membership(n, idx, m, &st);
    if (!in_a) return st;
    acc_t tot = {0.0, 0.0};
    int bad = 0;
    for (int64_t k = 0; k < m; ++k) {
        acc_t gx = {0.0, 0.0}, gy = {0.0, 0.0}, ef = {0.0, 0.0}, ea = {0.0, 0.0};
        double x = act[2 * k], y = act[2 * k + 1];
        grad_row(x, y, snap, n, -1, in_a, &gx, &gy, &ef);
        grad_row(x, y, act, m, k, NULL, &gx, &gy, &ea);
        grad[2 * k] = acc_get(&gx);
        grad[2 * k + 1] = acc_get(&gy);
        double ek = 0.5 * acc_get(&ea) + acc_get(&ef);
        if (e) e[k] = ek;
        acc_add(&tot, ek);
        if (!isfinite(grad[2 * k]) || !isfinite(grad[2 * k + 1]) || !isfinite(ek)) bad = 1;
    }
    if (e_sub) *e_sub = acc_get(&tot);
    free(in_a);
    return bad ? TCO_ERR_NONFINITE : TCO_OK;
}

/* Energy change of moving the charges of A (idx, m) from pos[idx] to new_act (2m),
 * summed directly as pair differences (never as a difference of totals):
 *   dE = sum_{i in A} sum_{j not in A} (1/|n_i - p_j| - 1/|p_i - p_j|)
 *      + sum_{i<k in A} (1/|n_i - n_k| - 1/|p_i - p_k|).
 * This equals E_sub(new) - E_sub(old) of Sec. II D and E(new) - E(old) of
 * Eq. hamiltonian. */
int tco_delta_energy(const double* pos, int64_t n, const int32_t* idx, int64_t m,
                     const double* new_act, double* delta)
{
    if (n < 0 || m < 0 || !delta || (m > 0 && (!idx || !new_act || !pos))) return TCO_ERR_INVALID_ARG;
    int st;
    unsigned char* in_a = membership(n, idx, m, &st);
    if (!in_a) return st;
    acc_t d = {0.0, 0.0};
    for (int64_t a = 0; a < m; ++a) {
        int64_t i = idx[a];
        double nx = new_act[2 * a], ny = new_act[2 * a + 1];
        double px = pos[2 * i], py = pos[2 * i + 1];
        for (int64_t j = 0; j < n; ++j) {
            if (in_a[j]) continue;
            double qx = pos[2 * j], qy = pos[2 * j + 1];
            acc_add(&d, inv_dist(nx, ny, qx, qy) - inv_dist(px, py, qx, qy));
        }
        for (int64_t b = a + 1; b < m; ++b) {
            int64_t k = idx[b];
            acc_add(&d, inv_dist(nx, ny, new_act[2 * b], new_act[2 * b + 1]) -
                            inv_dist(px, py, pos[2 * k], pos[2 * k + 1]));
        }
    }
    *delta = acc_get(&d);
    free(in_a);
    return isfinite(*delta) ? TCO_OK : TCO_ERR_NONFINITE;
}

/* ---------------------------------------------------------- constraint --- */

/* Hard wall of Eq. (potential) as a projection: r <- r * min(1, radius/|r|).
 * A charge with flags[i] != 0 is pinned to the unit circle (the boundary
 * population of Sec. II B): r <- r/|r| (left unchanged at the origin). */
int tco_project(double* pos, int64_t n, double radius, const unsigned char* flags)
{
    if (n < 0 || (n > 0 && !pos) || !(radius > 0.0)) return TCO_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1];
        double r = sqrt(x * x + y * y);
        if (flags && flags[i]) {
            if (r > 0.0) {
                pos[2 * i] = x / r;
                pos[2 * i + 1] = y / r;
            }
        } else if (r > radius) {
            double s = radius / r;
            pos[2 * i] = x * s;
            pos[2 * i + 1] = y * s;
        }
    }
    return TCO_OK;
}

/* Gradient with the components the wall blocks removed ("tangential" gradient):
 * pinned charges keep only the component along the circle; a free charge at the
 * wall (|r| >= radius (1 - 1e-12)) whose force -g points outward keeps only the
 * tangential part; every other charge keeps g.  Returns RMS and max of |pg_i|. */
int tco_projected_grad(const double* pos, const double* grad, int64_t n, double radius,
                       const unsigned char* flags, double* pg, double* rms, double* gmax)
{
    if (n < 0 || (n > 0 && (!pos || !grad || !pg))) return TCO_ERR_INVALID_ARG;
    acc_t ss = {0.0, 0.0};
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1];
        double gx = grad[2 * i], gy = grad[2 * i + 1];
        double r = sqrt(x * x + y * y);
        int pinned = flags && flags[i];
        if (r > 0.0 && (pinned || r >= radius * (1.0 - 1e-12))) {
            double ux = x / r, uy = y / r;
            double gr = gx * ux + gy * uy;
            if (pinned || gr < 0.0) {
                gx -= gr * ux;
                gy -= gr * uy;
            }
        }
        pg[2 * i] = gx;
        pg[2 * i + 1] = gy;
        double a2 = gx * gx + gy * gy;
        acc_add(&ss, a2);
        if (sqrt(a2) > mx) mx = sqrt(a2);
    }
    if (rms) *rms = n > 0 ? sqrt(acc_get(&ss) / (double)n) : 0.0;
    if (gmax) *gmax = mx;
    return TCO_OK;
}

/* -------------------------------------------------------------- descent --- */

/* Projected gradient descent x <- P(x - eta g(x)), `steps` times, over all n
 * charges.  trace (nullable, steps+1): E before each step and after the last. */
int tco_pgd(double* pos, int64_t n, double eta, int64_t steps, double radius,
            const unsigned char* flags, double* trace)
{
    if (n < 0 || steps < 0 || (n > 0 && !pos)) return TCO_ERR_INVALID_ARG;
    double* g = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    if (!g) return TCO_ERR_NO_MEMORY;
    int st = TCO_OK;
    for (int64_t k = 0; k <= steps; ++k) {
        if (trace) {
            st = tco_energy(pos, n, &trace[k], NULL);
            if (st) break;
        }
        if (k == steps) break;
        st = tco_grad(pos, n, g);
        if (st) break;
        for (int64_t i = 0; i < 2 * n; ++i) pos[i] = pos[i] - eta * g[i];
        tco_project(pos, n, radius, flags);
    }
    free(g);
    return st;
}

/* Dot product of two length-len vectors, compensated. */
static double dot(const double* a, const double* b, int64_t len)
{
    acc_t s = {0.0, 0.0};
    for (int64_t i = 0; i < len; ++i) acc_add(&s, a[i] * b[i]);
    return acc_get(&s);
}

/* Projected gradient descent on one subdomain with Barzilai-Borwein steps.
 * Charges of A (idx, m) start at snap[idx] and move; every other charge stays
 * at snap.  Step k: g_k = grad E_sub(x_k) (tco_subdomain_grad),
 *   alpha_0 = step0;  alpha_k = s^T y / y^T y (BB2, s = x_k - x_{k-1},
 *   y = g_k - g_{k-1}) when s^T y > 0, else alpha_max; clamped to
 *   [alpha_min, alpha_max];  x_{k+1} = P(x_k - alpha_k g_k), P the projection of
 *   tco_project (charges with flags[idx[k]] != 0 pinned to the unit circle;
 *   flags over all n, nullable).
 * act_out (2m): x after `steps` steps. */
int tco_subdomain_bb(const double* snap, int64_t n, const int32_t* idx, int64_t m,
                     double step0, double alpha_min, double alpha_max, int64_t steps,
                     double radius, const unsigned char* flags, double* act_out)
{
    if (n < 0 || m < 0 || steps < 0 || (m > 0 && (!snap || !idx || !act_out))) return TCO_ERR_INVALID_ARG;
    size_t sz = sizeof(double) * 2 * (size_t)(m > 0 ? m : 1);
    double *x = act_out, *g = (double*)malloc(sz), *xp = (double*)malloc(sz), *gp = (double*)malloc(sz);
    double *s = (double*)malloc(sz), *y = (double*)malloc(sz);
    unsigned char* fa = flags ? (unsigned char*)malloc((size_t)(m > 0 ? m : 1)) : NULL;
    if (!g || !xp || !gp || !s || !y || (flags && !fa)) {
        free(g); free(xp); free(gp); free(s); free(y); free(fa);
        return TCO_ERR_NO_MEMORY;
    }
    if (fa)
        for (int64_t k = 0; k < m; ++k) fa[k] = flags[idx[k]];
    for (int64_t k = 0; k < m; ++k) {
        x[2 * k] = snap[2 * idx[k]];
        x[2 * k + 1] = snap[2 * idx[k] + 1];
    }
    int st = TCO_OK;
    for (int64_t it = 0; it < steps; ++it) {
        st = tco_subdomain_grad(snap, n, idx, m, x, g, NULL, NULL);
        if (st) break;
        double alpha = step0;
        if (it > 0) {
            for (int64_t i = 0; i < 2 * m; ++i) { s[i] = x[i] - xp[i]; y[i] = g[i] - gp[i]; }
            double sy = dot(s, y, 2 * m), yy = dot(y, y, 2 * m);
            alpha = (sy > 0.0 && yy > 0.0) ? sy / yy : alpha_max;
            if (alpha < alpha_min) alpha = alpha_min;
            if (alpha > alpha_max) alpha = alpha_max;
        }
        memcpy(xp, x, sz);
        memcpy(gp, g, sz);
        for (int64_t i = 0; i < 2 * m; ++i) x[i] = x[i] - alpha * g[i];
        tco_project(x, m, radius, fa);
    }
    free(g); free(xp); free(gp); free(s); free(y); free(fa);
    return st;
}

/* Sequential FP64 accept/reject of relaxed subdomains against the current
 * configuration pos (in/out).  For s = 0 .. n_sub-1 in order: a subdomain that
 * shares a charge with an already accepted one is skipped (accepted = 2);
 * otherwise dE_s = tco_delta_energy(current pos, A_s -> new_act_s) and the move
 * is applied iff dE_s < 0 (accepted = 1, else 0).  delta (n_sub), accepted (n_sub). */
int tco_accept_sequential(double* pos, int64_t n, const int32_t* idx, const int64_t* offsets,
                          int64_t n_sub, const double* new_act, double* delta, unsigned char* accepted)
{
    if (n < 0 || n_sub < 0 || (n_sub > 0 && (!idx || !offsets || !new_act || !delta || !accepted)))
        return TCO_ERR_INVALID_ARG;
    unsigned char* taken = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!taken) return TCO_ERR_NO_MEMORY;
    int st = TCO_OK;
    for (int64_t s = 0; s < n_sub; ++s) {
        int64_t b = offsets[s], e = offsets[s + 1];
        int clash = 0;
        for (int64_t k = b; k < e; ++k) if (taken[idx[k]]) clash = 1;
        if (clash) { delta[s] = 0.0; accepted[s] = 2; continue; }
        st = tco_delta_energy(pos, n, idx + b, e - b, new_act + 2 * b, &delta[s]);
        if (st) break;
        if (delta[s] < 0.0) {
            accepted[s] = 1;
            for (int64_t k = b; k < e; ++k) {
                taken[idx[k]] = 1;
                pos[2 * idx[k]] = new_act[2 * k];
                pos[2 * idx[k] + 1] = new_act[2 * k + 1];
            }
        } else {
            accepted[s] = 0;
        }
    }
    free(taken);
    return st;
}

/* Smooth wall parameterisation used by the quasi-Newton solver.
 *
 * The paper writes interior charges as r = sigma sin^2 t (Sec. II D), which makes
 * the wall r = sigma a smooth maximum of r(t), so the wall needs no projection.
 * The map used here has the same property in Cartesian form and no polar
 * singularity at the centre: a free charge is z in R^2 with
 *     x = sigma sin(|z|) z/|z|     (x = sigma z in the limit z -> 0),
 * and a pinned charge (the boundary population of Sec. II B) is x = z/|z|.
 * Chain rule (cf. the paper's dE/dt, dE/du): with g = dE/dx, u = z/|z|,
 * g_r = g.u, g_t = g - g_r u,
 *     free:   dE/dz = sigma ( sin|z|/|z| g_t + cos|z| g_r u )   (sigma g at z = 0)
 *     pinned: dE/dz = g_t / |z|.                                           */
static void z_to_x(const double* z, int64_t n, double sigma, const unsigned char* flags, double* x)
{
    for (int64_t i = 0; i < n; ++i) {
        double zx = z[2 * i], zy = z[2 * i + 1];
        double rho = sqrt(zx * zx + zy * zy);
        if (flags && flags[i]) {
            x[2 * i] = zx / rho;
            x[2 * i + 1] = zy / rho;
        } else if (rho > 0.0) {
            double f = sigma * sin(rho) / rho;
            x[2 * i] = zx * f;
            x[2 * i + 1] = zy * f;
        } else {
            x[2 * i] = 0.0;
            x[2 * i + 1] = 0.0;
        }
    }
}

static void x_to_z(const double* x, int64_t n, double sigma, const unsigned char* flags, double* z)
{
    for (int64_t i = 0; i < n; ++i) {
        double px = x[2 * i], py = x[2 * i + 1];
        double r = sqrt(px * px + py * py);
        if (flags && flags[i]) {
            z[2 * i] = r > 0.0 ? px / r : 1.0;
            z[2 * i + 1] = r > 0.0 ? py / r : 0.0;
        } else if (r > 0.0) {
            double q = r / sigma;
            if (q > 1.0) q = 1.0;
            double f = asin(q) / r;
            z[2 * i] = px * f;
            z[2 * i + 1] = py * f;
        } else {
            z[2 * i] = 0.0;
            z[2 * i + 1] = 0.0;
        }
    }
}

static void grad_z(const double* z, const double* g, int64_t n, double sigma, const unsigned char* flags,
                   double* gz)
{
    for (int64_t i = 0; i < n; ++i) {
        double zx = z[2 * i], zy = z[2 * i + 1];
        double gx = g[2 * i], gy = g[2 * i + 1];
        double rho = sqrt(zx * zx + zy * zy);
        if (rho == 0.0) {
            gz[2 * i] = (flags && flags[i]) ? 0.0 : sigma * gx;
            gz[2 * i + 1] = (flags && flags[i]) ? 0.0 : sigma * gy;
            continue;
        }
        double ux = zx / rho, uy = zy / rho;
        double gr = gx * ux + gy * uy;
        double tx = gx - gr * ux, ty = gy - gr * uy;
        if (flags && flags[i]) {
            gz[2 * i] = tx / rho;
            gz[2 * i + 1] = ty / rho;
        } else {
            double a = sin(rho) / rho, c = cos(rho);
            gz[2 * i] = sigma * (a * tx + c * gr * ux);
            gz[2 * i + 1] = sigma * (a * ty + c * gr * uy);
        }
    }
}

/* The paper's parameterisation (Sec. II D): an interior charge is (t, u) with
 * r = sigma sin^2 t and x = r (cos u, sin u); a boundary (pinned) charge is
 * x = (cos u, sin u), stored as (u, 0).  Its gradients are the printed chain
 * rule: dE/dt = (E_x cos u + E_y sin u) sigma sin 2t,
 * dE/du = -E_x r sin u + E_y r cos u, and for a boundary charge
 * dE/du = -E_x sin u + E_y cos u. */
static void tu_to_x(const double* z, int64_t n, double sigma, const unsigned char* flags, double* x)
{
    for (int64_t i = 0; i < n; ++i) {
        double t = z[2 * i], u = z[2 * i + 1];
        if (flags && flags[i]) {
            x[2 * i] = cos(t);
            x[2 * i + 1] = sin(t);
        } else {
            double st = sin(t), r = sigma * st * st;
            x[2 * i] = r * cos(u);
            x[2 * i + 1] = r * sin(u);
        }
    }
}

static void x_to_tu(const double* x, int64_t n, double sigma, const unsigned char* flags, double* z)
{
    for (int64_t i = 0; i < n; ++i) {
        double px = x[2 * i], py = x[2 * i + 1];
        double r = sqrt(px * px + py * py);
        double u = r > 0.0 ? atan2(py, px) : 0.0;
        if (flags && flags[i]) {
            z[2 * i] = u;
            z[2 * i + 1] = 0.0;
        } else {
            double q = r / sigma;
            if (q > 1.0) q = 1.0;
            z[2 * i] = asin(sqrt(q));
            z[2 * i + 1] = u;
        }
    }
}

static void grad_tu(const double* z, const double* g, int64_t n, double sigma, const unsigned char* flags,
                    double* gz)
{
    for (int64_t i = 0; i < n; ++i) {
        double gx = g[2 * i], gy = g[2 * i + 1];
        if (flags && flags[i]) {
            double u = z[2 * i];
            gz[2 * i] = -gx * sin(u) + gy * cos(u);
            gz[2 * i + 1] = 0.0;
        } else {
            double t = z[2 * i], u = z[2 * i + 1];
            double st = sin(t), r = sigma * st * st;
            gz[2 * i] = (gx * cos(u) + gy * sin(u)) * sigma * sin(2.0 * t);
            gz[2 * i + 1] = -gx * r * sin(u) + gy * r * cos(u);
        }
    }
}

/* Limited-memory BFGS on the smooth wall parameterisation, with a maximum
 * displacement cap and no line search, over all n charges of one configuration.
 *
 * State z (2n), gradient gz = dE/dz.  Iteration, memory M pairs (s_j, y_j) with
 * rho_j = 1/(s_j^T y_j):
 *   stop when RMS_i |gz_i| < gtol;
 *   two-loop recursion (Nocedal & Wright, Alg. 7.4) on q = gz with H0 = gamma I,
 *   gamma = s^T y / y^T y of the newest pair (step0 without history): d = -H gz;
 *   if gz^T d >= 0 the history is cleared and d = -step0 gz;
 *   alpha = min(1, maxstep / max_i |d_i|) (each charge moves at most maxstep in z,
 *   hence at most sigma maxstep in x);  z <- z + alpha d;
 *   the pair s = z_new - z, y = gz_new - gz is kept iff s^T y > 1e-12 |s||y|
 *   (the oldest drops out beyond M).
 * pos (in/out, 2n): x of the final z.  Reports iterations and final RMS |gz|. */
int tco_lbfgs_ls(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                 double step0, double maxstep, double sigma, const unsigned char* flags,
                 int64_t max_halvings, int64_t tu, int64_t* iters_out, double* rms_out);

/* The iteration of tco_lbfgs_ls with its path recorded (nullable arrays, one
 * row of 2n per iteration): z_tr[k] and gz_tr[k] the variables and dE/dz at
 * iterate k (k = 0 .. iterations), d_tr[k] the search direction taken at
 * iterate k after the descent check and alpha_tr[k] its step scale
 * (k < iterations).  Rows are written as the iteration reaches them. */
static int lbfgs_core(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                      double step0, double maxstep, double sigma, const unsigned char* flags,
                      int64_t max_halvings, int64_t tu, int64_t* iters_out, double* rms_out,
                      double* z_tr, double* gz_tr, double* d_tr, double* alpha_tr);

/* Energy change E(xn) - E(x) of moving every charge from x to xn, summed as
 * pair differences (compensated), not as a difference of totals. */
static double instance_delta(const double* x, const double* xn, int64_t n)
{
    acc_t a = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            acc_add(&a, inv_dist(xn[2 * i], xn[2 * i + 1], xn[2 * j], xn[2 * j + 1]) -
                            inv_dist(x[2 * i], x[2 * i + 1], x[2 * j], x[2 * j + 1]));
    return acc_get(&a);
}

int tco_lbfgs(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
              double step0, double maxstep, double sigma, const unsigned char* flags,
              int64_t* iters_out, double* rms_out)
{
    return tco_lbfgs_ls(pos, n, memory, max_iter, gtol, step0, maxstep, sigma, flags, 0, 0, iters_out, rms_out);
}

/* tco_lbfgs with an Armijo backtracking line search (max_halvings > 0): the
 * trial z + alpha d (alpha from the max-step cap) is kept once
 *     E(x(z + alpha d)) - E(x(z)) <= 1e-4 alpha (dE/dz . d),
 * the energy change summed as pair differences; otherwise alpha is halved, at
 * most max_halvings times, and the last trial is taken.  max_halvings = 0 is
 * the plain iteration.  tu != 0 runs the iteration on the paper's (t, u)
 * variables instead of the smooth map. */
int tco_lbfgs_ls(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                 double step0, double maxstep, double sigma, const unsigned char* flags,
                 int64_t max_halvings, int64_t tu, int64_t* iters_out, double* rms_out)
{
    return lbfgs_core(pos, n, memory, max_iter, gtol, step0, maxstep, sigma, flags, max_halvings, tu, iters_out,
                      rms_out, NULL, NULL, NULL, NULL);
}

int tco_lbfgs_trace(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                    double step0, double maxstep, double sigma, const unsigned char* flags,
                    int64_t max_halvings, int64_t tu, int64_t* iters_out, double* rms_out,
                    double* z_tr, double* gz_tr, double* d_tr, double* alpha_tr)
{
    return lbfgs_core(pos, n, memory, max_iter, gtol, step0, maxstep, sigma, flags, max_halvings, tu, iters_out,
                      rms_out, z_tr, gz_tr, d_tr, alpha_tr);
}

static int lbfgs_core(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                      double step0, double maxstep, double sigma, const unsigned char* flags,
                      int64_t max_halvings, int64_t tu, int64_t* iters_out, double* rms_out,
                      double* z_tr, double* gz_tr, double* d_tr, double* alpha_tr)
{
    if (n < 0 || memory < 1 || max_iter < 0 || max_halvings < 0 || (n > 0 && !pos) || !(sigma > 0.0))
        return TCO_ERR_INVALID_ARG;
    int64_t L = 2 * n;
    size_t sz = sizeof(double) * (size_t)(L > 0 ? L : 1);
    double* xk = (double*)malloc(sz);
    double* z = (double*)malloc(sz);
    double* zn = (double*)malloc(sz);
    double* g = (double*)malloc(sz);
    double* gz = (double*)malloc(sz);
    double* gzn = (double*)malloc(sz);
    double* d = (double*)malloc(sz);
    double* S = (double*)malloc(sz * (size_t)memory);
    double* Y = (double*)malloc(sz * (size_t)memory);
    double* rho = (double*)malloc(sizeof(double) * (size_t)memory);
    double* al = (double*)malloc(sizeof(double) * (size_t)memory);
    if (!xk || !z || !zn || !g || !gz || !gzn || !d || !S || !Y || !rho || !al) {
        free(xk); free(z); free(zn); free(g); free(gz); free(gzn); free(d); free(S); free(Y); free(rho); free(al);
        return TCO_ERR_NO_MEMORY;
    }
    memset(z, 0, sz);
    int64_t hist = 0, head = 0; /* ring buffer: newest pair at (head - 1) mod M */
    int64_t it = 0;
    double rms = 0.0;
    if (tu) x_to_tu(pos, n, sigma, flags, z); else x_to_z(pos, n, sigma, flags, z);
    if (tu) tu_to_x(z, n, sigma, flags, pos); else z_to_x(z, n, sigma, flags, pos);
    int st = tco_grad(pos, n, g);
    if (!st) {
        if (tu) grad_tu(z, g, n, sigma, flags, gz); else grad_z(z, g, n, sigma, flags, gz);
        rms = n > 0 ? sqrt(dot(gz, gz, L) / (double)n) : 0.0;
        if (z_tr) memcpy(z_tr, z, sz);
        if (gz_tr) memcpy(gz_tr, gz, sz);
    }
    for (; !st && it < max_iter; ++it) {
        if (rms < gtol) break;
        for (int64_t i = 0; i < L; ++i) d[i] = gz[i];
        for (int64_t q = 0; q < hist; ++q) {
            int64_t j = ((head - 1 - q) % memory + memory) % memory;
            al[j] = rho[j] * dot(S + j * L, d, L);
            for (int64_t i = 0; i < L; ++i) d[i] -= al[j] * Y[j * L + i];
        }
        double gamma = step0;
        if (hist > 0) {
            int64_t j = ((head - 1) % memory + memory) % memory;
            gamma = dot(S + j * L, Y + j * L, L) / dot(Y + j * L, Y + j * L, L);
        }
        for (int64_t i = 0; i < L; ++i) d[i] *= gamma;
        for (int64_t q = hist - 1; q >= 0; --q) {
            int64_t j = ((head - 1 - q) % memory + memory) % memory;
            double b = rho[j] * dot(Y + j * L, d, L);
            for (int64_t i = 0; i < L; ++i) d[i] += S[j * L + i] * (al[j] - b);
        }
        for (int64_t i = 0; i < L; ++i) d[i] = -d[i];
        if (dot(gz, d, L) >= 0.0) {
            hist = 0;
            head = 0;
            for (int64_t i = 0; i < L; ++i) d[i] = -step0 * gz[i];
        }
        double dmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double a = sqrt(d[2 * i] * d[2 * i] + d[2 * i + 1] * d[2 * i + 1]);
            if (a > dmax) dmax = a;
        }
        double alpha = (dmax > maxstep) ? maxstep / dmax : 1.0;
        if (d_tr) memcpy(d_tr + it * L, d, sz);
        for (int64_t i = 0; i < L; ++i) zn[i] = z[i] + alpha * d[i];
        if (max_halvings > 0) {
            memcpy(xk, pos, sz);
            const double gd = dot(gz, d, L);
            for (int64_t h = 0;; ++h) {
                if (tu) tu_to_x(zn, n, sigma, flags, pos); else z_to_x(zn, n, sigma, flags, pos);
                if (instance_delta(xk, pos, n) <= 1e-4 * alpha * gd || h == max_halvings) break;
                alpha *= 0.5;
                for (int64_t i = 0; i < L; ++i) zn[i] = z[i] + alpha * d[i];
            }
        } else {
            if (tu) tu_to_x(zn, n, sigma, flags, pos); else z_to_x(zn, n, sigma, flags, pos);
        }
        st = tco_grad(pos, n, g);
        if (st) break;
        if (tu) grad_tu(zn, g, n, sigma, flags, gzn); else grad_z(zn, g, n, sigma, flags, gzn);
        rms = n > 0 ? sqrt(dot(gzn, gzn, L) / (double)n) : 0.0;
        if (alpha_tr) alpha_tr[it] = alpha;
        if (z_tr) memcpy(z_tr + (it + 1) * L, zn, sz);
        if (gz_tr) memcpy(gz_tr + (it + 1) * L, gzn, sz);
        /* the candidate pair is tested first and stored only if kept, so a
         * rejected pair never overwrites the oldest stored one */
        acc_t sy_a = {0.0, 0.0}, ss_a = {0.0, 0.0}, yy_a = {0.0, 0.0};
        for (int64_t i = 0; i < L; ++i) {
            double si = zn[i] - z[i], yi = gzn[i] - gz[i];
            acc_add(&sy_a, si * yi);
            acc_add(&ss_a, si * si);
            acc_add(&yy_a, yi * yi);
        }
        double sy = acc_get(&sy_a);
        if (sy > 1e-12 * sqrt(acc_get(&ss_a)) * sqrt(acc_get(&yy_a))) {
            double* Sj = S + head * L;
            double* Yj = Y + head * L;
            for (int64_t i = 0; i < L; ++i) { Sj[i] = zn[i] - z[i]; Yj[i] = gzn[i] - gz[i]; }
            rho[head] = 1.0 / sy;
            head = (head + 1) % memory;
            if (hist < memory) ++hist;
        }
        memcpy(z, zn, sz);
        memcpy(gz, gzn, sz);
    }
    if (iters_out) *iters_out = it;
    if (rms_out) *rms_out = rms;
    free(xk); free(z); free(zn); free(g); free(gz); free(gzn); free(d); free(S); free(Y); free(rho); free(al);
    return st;
}

/* ------------------------------------------------------------ L-BFGS-B --- */

/* Sec. II C step 4 optimises each subdomain with L-BFGS-B (Byrd, Lu, Nocedal &
 * Zhu 1995) on the variables of Sec. II D.  The pieces below follow that
 * method; the variables are nv = 2n numbers, the box is lo <= v <= hi
 * (+-INFINITY for an unbounded side), and h stored pairs (s_a, y_a), a = 0 the
 * oldest, are rows of S and Y (h x nv).
 *
 * Compact representation (Byrd, Nocedal & Schnabel 1994, Thm 2.3) of the BFGS
 * matrix built from theta I by the h updates:
 *     B = theta I - W M W^T,  W = [Y^T, theta S^T] (nv x 2h),
 *     M = K^{-1},  K = [[-D, L^T], [L, theta S S^T]],
 * D = diag(s_a . y_a), L_ab = s_a . y_b for a > b (else 0). */

static double tco_wrow(int64_t h, const double* S, const double* Y, int64_t nv, double theta, int64_t i, int64_t a)
{
    /* element (i, a) of W */
    return a < h ? Y[a * nv + i] : theta * S[(a - h) * nv + i];
}

/* M = K^{-1} by Gauss-Jordan elimination with partial pivoting on [K | I]. */
int tco_lbfgsb_middle(int64_t h, const double* S, const double* Y, int64_t nv, double theta, double* M)
{
    if (h < 0 || nv < 0 || (h > 0 && (!S || !Y || !M))) return TCO_ERR_INVALID_ARG;
    int64_t q = 2 * h;
    if (q == 0) return TCO_OK;
    double* A = (double*)calloc((size_t)(q * 2 * q), sizeof(double));
    if (!A) return TCO_ERR_NO_MEMORY;
    for (int64_t a = 0; a < h; ++a)
        for (int64_t b = 0; b < h; ++b) {
            double sy_ab = dot(S + a * nv, Y + b * nv, nv);
            double ss_ab = dot(S + a * nv, S + b * nv, nv);
            if (a == b) A[a * 2 * q + b] = -sy_ab;            /* -D */
            if (a > b) A[(h + a) * 2 * q + b] = sy_ab;         /* L */
            if (a > b) A[b * 2 * q + (h + a)] = sy_ab;         /* L^T */
            A[(h + a) * 2 * q + (h + b)] = theta * ss_ab;      /* theta S S^T */
        }
    for (int64_t a = 0; a < q; ++a) A[a * 2 * q + q + a] = 1.0;
    int st = TCO_OK;
    for (int64_t col = 0; col < q && st == TCO_OK; ++col) {
        int64_t piv = col;
        for (int64_t r = col + 1; r < q; ++r)
            if (fabs(A[r * 2 * q + col]) > fabs(A[piv * 2 * q + col])) piv = r;
        if (!(fabs(A[piv * 2 * q + col]) > 0.0)) { st = TCO_ERR_NONFINITE; break; }
        if (piv != col)
            for (int64_t k = 0; k < 2 * q; ++k) {
                double t = A[col * 2 * q + k];
                A[col * 2 * q + k] = A[piv * 2 * q + k];
                A[piv * 2 * q + k] = t;
            }
        double pv = A[col * 2 * q + col];
        for (int64_t k = 0; k < 2 * q; ++k) A[col * 2 * q + k] /= pv;
        for (int64_t r = 0; r < q; ++r) {
            if (r == col) continue;
            double f = A[r * 2 * q + col];
            if (f != 0.0)
                for (int64_t k = 0; k < 2 * q; ++k) A[r * 2 * q + k] -= f * A[col * 2 * q + k];
        }
    }
    if (st == TCO_OK)
        for (int64_t a = 0; a < q; ++a)
            for (int64_t b = 0; b < q; ++b) M[a * q + b] = A[a * 2 * q + q + b];
    free(A);
    return st;
}

/* y = M x for the 2h x 2h matrix M. */
static void tco_matvec(int64_t q, const double* M, const double* x, double* y)
{
    for (int64_t a = 0; a < q; ++a) {
        double s = 0.0;
        for (int64_t b = 0; b < q; ++b) s += M[a * q + b] * x[b];
        y[a] = s;
    }
}

typedef struct {
    double t;
    int64_t i;
} brk_t;

static int brk_cmp(const void* a, const void* b)
{
    const brk_t* p = (const brk_t*)a;
    const brk_t* r = (const brk_t*)b;
    if (p->t < r->t) return -1;
    if (p->t > r->t) return 1;
    return (p->i > r->i) - (p->i < r->i);
}

/* Generalized Cauchy point (Byrd et al. 1995, Sec. 4): the first local
 * minimiser of the quadratic model m(v) = g.(v - x) + (v - x).B(v - x)/2 along
 * the projected steepest-descent path v(t) = P(x - t g), t >= 0.
 *   Breakpoint of variable i: t_i = (x_i - hi_i)/g_i (g_i < 0), (x_i - lo_i)/g_i
 *   (g_i > 0), infinity otherwise; direction d_i = -g_i, or 0 where t_i = 0.
 *   On the segment starting at t_old the model is f' dt + f'' dt^2 / 2 + const,
 *   with f' = g.d + ... kept in closed form through p = W^T d and
 *   c = W^T (v(t_old) - x):  initially p = W^T d, c = 0, f' = -d.d,
 *   f'' = theta d.d - p.M p.  The breakpoints are visited in increasing
 *   (t_i, i); while the segment minimiser dt* = -f'/f'' lies beyond the next
 *   breakpoint b, variable b is fixed at its bound (z_b = bound - x_b) and
 *       c += dt p,
 *       f' += dt f'' + g_b^2 + theta g_b z_b - g_b w_b.M c,
 *       f'' += -theta g_b^2 - 2 g_b w_b.M p - g_b^2 w_b.M w_b,
 *       p += g_b w_b,  d_b = 0
 *   (w_b = row b of W).  f'' is kept at least 2^-52 times its first value, as a
 *   guard against rounding (B is positive definite, so f'' > 0 in exact
 *   arithmetic while d != 0).  At the end dt* = max(dt*, 0), every variable not
 *   fixed moves to x + (t_old + dt*) d, and c += dt* p.
 * Writes xc (nv), c (2h) and the number of breakpoints passed (nullable). */
int tco_lbfgsb_cauchy(int64_t nv, const double* x, const double* g, const double* lo, const double* hi, int64_t h,
                      const double* S, const double* Y, double theta, const double* M, double* xc, double* c,
                      int64_t* n_break)
{
    if (nv < 0 || h < 0 || !(theta > 0.0) || (nv > 0 && (!x || !g || !lo || !hi || !xc)) ||
        (h > 0 && (!S || !Y || !M || !c)))
        return TCO_ERR_INVALID_ARG;
    int64_t q = 2 * h;
    double* d = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    double* tb = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    unsigned char* fixed = (unsigned char*)calloc((size_t)(nv > 0 ? nv : 1), 1);
    brk_t* br = (brk_t*)malloc(sizeof(brk_t) * (size_t)(nv > 0 ? nv : 1));
    double p[64], wb[64], mv[64];
    if (!d || !tb || !fixed || !br || q > 64) {
        free(d); free(tb); free(fixed); free(br);
        return q > 64 ? TCO_ERR_INVALID_ARG : TCO_ERR_NO_MEMORY;
    }
    int64_t nb = 0, passed = 0;
    acc_t dd = {0.0, 0.0};
    for (int64_t i = 0; i < nv; ++i) {
        double t = INFINITY;
        if (g[i] < 0.0 && hi[i] < INFINITY) t = (x[i] - hi[i]) / g[i];
        else if (g[i] > 0.0 && lo[i] > -INFINITY) t = (x[i] - lo[i]) / g[i];
        tb[i] = t;
        d[i] = t == 0.0 ? 0.0 : -g[i];
        acc_add(&dd, d[i] * d[i]);
        if (t > 0.0 && t < INFINITY) { br[nb].t = t; br[nb].i = i; ++nb; }
    }
    for (int64_t a = 0; a < q; ++a) {
        acc_t s = {0.0, 0.0};
        for (int64_t i = 0; i < nv; ++i) acc_add(&s, tco_wrow(h, S, Y, nv, theta, i, a) * d[i]);
        p[a] = acc_get(&s);
        c[a] = 0.0;
    }
    double fp = -acc_get(&dd);
    tco_matvec(q, M, p, mv);
    double pmp = 0.0;
    for (int64_t a = 0; a < q; ++a) pmp += p[a] * mv[a];
    double fpp = -theta * fp - pmp;
    const double fpp0 = fpp;
    double told = 0.0, dtm = 0.0;
    if (fpp0 > 0.0) {
        dtm = -fp / fpp;
        qsort(br, (size_t)nb, sizeof(brk_t), brk_cmp);
        for (int64_t k = 0; k < nb; ++k) {
            int64_t b = br[k].i;
            double t = br[k].t, dt = t - told;
            if (dtm < dt) break;
            double xb = d[b] > 0.0 ? hi[b] : lo[b];
            double zb = xb - x[b], gb = g[b];
            for (int64_t a = 0; a < q; ++a) { c[a] += dt * p[a]; wb[a] = tco_wrow(h, S, Y, nv, theta, b, a); }
            double wMc = 0.0, wMp = 0.0, wMw = 0.0;
            tco_matvec(q, M, c, mv);
            for (int64_t a = 0; a < q; ++a) wMc += wb[a] * mv[a];
            tco_matvec(q, M, p, mv);
            for (int64_t a = 0; a < q; ++a) wMp += wb[a] * mv[a];
            tco_matvec(q, M, wb, mv);
            for (int64_t a = 0; a < q; ++a) wMw += wb[a] * mv[a];
            fp = fp + dt * fpp + gb * gb + theta * gb * zb - gb * wMc;
            fpp = fpp - theta * gb * gb - 2.0 * gb * wMp - gb * gb * wMw;
            if (fpp < 0x1p-52 * fpp0) fpp = 0x1p-52 * fpp0;
            for (int64_t a = 0; a < q; ++a) p[a] += gb * wb[a];
            d[b] = 0.0;
            fixed[b] = 1;
            xc[b] = xb;
            dtm = -fp / fpp;
            told = t;
            ++passed;
        }
        if (dtm < 0.0) dtm = 0.0;
        told += dtm;
        for (int64_t a = 0; a < q; ++a) c[a] += dtm * p[a];
    }
    for (int64_t i = 0; i < nv; ++i)
        if (!fixed[i]) xc[i] = fpp0 > 0.0 ? x[i] + told * d[i] : x[i];
    if (n_break) *n_break = passed;
    free(d); free(tb); free(fixed); free(br);
    return TCO_OK;
}

/* Subspace minimisation, direct primal method (Byrd et al. 1995, Sec. 5.1).
 * Free variables F = { i : lo_i < xc_i < hi_i }; with Z selecting them:
 *     r = Z^T (g + theta (xc - x) - W M c)          (reduced model gradient at xc)
 *     v = M (W_F^T r),   N = I - M (W_F^T W_F) / theta,   v <- N^{-1} v
 *     du = -r / theta - W_F v / theta^2              (= -(Z^T B Z)^{-1} r)
 *     a* = max { a <= 1 : lo_i <= xc_i + a du_i <= hi_i, i in F }
 *     xbar = xc + a* du on F, xc elsewhere.
 * N^{-1} v is a Gauss elimination with partial pivoting. */
int tco_lbfgsb_subspace(int64_t nv, const double* x, const double* g, const double* lo, const double* hi, int64_t h,
                        const double* S, const double* Y, double theta, const double* M, const double* xc,
                        const double* c, double* xbar)
{
    if (nv < 0 || h < 0 || !(theta > 0.0) || (nv > 0 && (!x || !g || !lo || !hi || !xc || !xbar)) ||
        (h > 0 && (!S || !Y || !M || !c)) || h > 32)
        return TCO_ERR_INVALID_ARG;
    int64_t q = 2 * h;
    double Mc[64], v[64], wi[64], A[64 * 64], N[64 * 65];
    double* r = (double*)malloc(sizeof(double) * (size_t)(nv > 0 ? nv : 1));
    if (!r) return TCO_ERR_NO_MEMORY;
    tco_matvec(q, M, c, Mc);
    acc_t va[64], Aa[64 * 64];
    for (int64_t a = 0; a < q; ++a) { va[a].s = va[a].c = 0.0; for (int64_t b = 0; b < q; ++b) Aa[a * q + b].s = Aa[a * q + b].c = 0.0; }
    for (int64_t i = 0; i < nv; ++i) {
        r[i] = 0.0;
        if (!(lo[i] < xc[i] && xc[i] < hi[i])) continue;
        double wMc = 0.0;
        for (int64_t a = 0; a < q; ++a) { wi[a] = tco_wrow(h, S, Y, nv, theta, i, a); wMc += wi[a] * Mc[a]; }
        r[i] = g[i] + theta * (xc[i] - x[i]) - wMc;
        for (int64_t a = 0; a < q; ++a) {
            acc_add(&va[a], wi[a] * r[i]);
            for (int64_t b = 0; b < q; ++b) acc_add(&Aa[a * q + b], wi[a] * wi[b]);
        }
    }
    double wv[64];
    for (int64_t a = 0; a < q; ++a) {
        wv[a] = acc_get(&va[a]);
        for (int64_t b = 0; b < q; ++b) A[a * q + b] = acc_get(&Aa[a * q + b]);
    }
    tco_matvec(q, M, wv, v);
    /* N = I - M A / theta, augmented with v */
    for (int64_t a = 0; a < q; ++a) {
        for (int64_t b = 0; b < q; ++b) {
            double s = 0.0;
            for (int64_t k = 0; k < q; ++k) s += M[a * q + k] * A[k * q + b];
            N[a * (q + 1) + b] = (a == b ? 1.0 : 0.0) - s / theta;
        }
        N[a * (q + 1) + q] = v[a];
    }
    int st = TCO_OK;
    for (int64_t col = 0; col < q; ++col) {
        int64_t piv = col;
        for (int64_t rr = col + 1; rr < q; ++rr)
            if (fabs(N[rr * (q + 1) + col]) > fabs(N[piv * (q + 1) + col])) piv = rr;
        if (!(fabs(N[piv * (q + 1) + col]) > 0.0)) { st = TCO_ERR_NONFINITE; break; }
        if (piv != col)
            for (int64_t k = 0; k <= q; ++k) {
                double t = N[col * (q + 1) + k];
                N[col * (q + 1) + k] = N[piv * (q + 1) + k];
                N[piv * (q + 1) + k] = t;
            }
        for (int64_t rr = col + 1; rr < q; ++rr) {
            double f = N[rr * (q + 1) + col] / N[col * (q + 1) + col];
            for (int64_t k = col; k <= q; ++k) N[rr * (q + 1) + k] -= f * N[col * (q + 1) + k];
        }
    }
    if (st == TCO_OK) {
        for (int64_t a = q - 1; a >= 0; --a) {
            double s = N[a * (q + 1) + q];
            for (int64_t k = a + 1; k < q; ++k) s -= N[a * (q + 1) + k] * v[k];
            v[a] = s / N[a * (q + 1) + a];
        }
        double astar = 1.0;
        for (int64_t i = 0; i < nv; ++i) {
            if (!(lo[i] < xc[i] && xc[i] < hi[i])) continue;
            double wv2 = 0.0;
            for (int64_t a = 0; a < q; ++a) wv2 += tco_wrow(h, S, Y, nv, theta, i, a) * v[a];
            double du = -r[i] / theta - wv2 / (theta * theta);
            r[i] = du;
            if (du > 0.0 && hi[i] < INFINITY && (hi[i] - xc[i]) / du < astar) astar = (hi[i] - xc[i]) / du;
            if (du < 0.0 && lo[i] > -INFINITY && (lo[i] - xc[i]) / du < astar) astar = (lo[i] - xc[i]) / du;
        }
        for (int64_t i = 0; i < nv; ++i)
            xbar[i] = (lo[i] < xc[i] && xc[i] < hi[i]) ? xc[i] + astar * r[i] : xc[i];
    }
    free(r);
    return st;
}

/* Box of the (t, u) variables: a free charge (t, u) has t in [0, pi/2] (the
 * range of Sec. II D, on which r = sigma sin^2 t covers [0, sigma] once) and u
 * unbounded; a pinned charge (u, 0) has u unbounded and its unused second
 * variable fixed at 0. */
static const double TCO_HALF_PI = 1.5707963267948966;

static void tu_box(int64_t n, const unsigned char* flags, double* lo, double* hi)
{
    for (int64_t i = 0; i < n; ++i) {
        if (flags && flags[i]) {
            lo[2 * i] = -INFINITY; hi[2 * i] = INFINITY;
            lo[2 * i + 1] = 0.0; hi[2 * i + 1] = 0.0;
        } else {
            lo[2 * i] = 0.0; hi[2 * i] = TCO_HALF_PI;
            lo[2 * i + 1] = -INFINITY; hi[2 * i + 1] = INFINITY;
        }
    }
}

static void box_clamp(double* v, const double* lo, const double* hi, int64_t nv)
{
    for (int64_t i = 0; i < nv; ++i) v[i] = v[i] < lo[i] ? lo[i] : (v[i] > hi[i] ? hi[i] : v[i]);
}

/* RMS over charges of the projected gradient P(v - g) - v. */
static double proj_rms(const double* v, const double* g, const double* lo, const double* hi, int64_t n)
{
    acc_t s = {0.0, 0.0};
    for (int64_t i = 0; i < 2 * n; ++i) {
        double w = v[i] - g[i];
        w = w < lo[i] ? lo[i] : (w > hi[i] ? hi[i] : w);
        acc_add(&s, (w - v[i]) * (w - v[i]));
    }
    return n > 0 ? sqrt(acc_get(&s) / (double)n) : 0.0;
}

/* What one L-BFGS-B run minimises: a whole configuration (snap NULL: E of
 * Eq. hamiltonian over the moving charges alone), or the subdomain objective
 * E_sub of Sec. II D, whose moving charges are A = idx[0 .. m) and whose other
 * charges stay at snap (n charges). */
typedef struct {
    const double* snap;
    int64_t n;
    const int32_t* idx;
    double* cur; /* subdomain: scratch copy of snap (2n) */
} tco_obj_t;

static int obj_grad(const tco_obj_t* o, const double* x, int64_t m, double* g)
{
    if (!o->snap) return tco_grad(x, m, g);
    return tco_subdomain_grad(o->snap, o->n, o->idx, m, x, g, NULL, NULL);
}

/* Energy change of moving the charges from xold to xnew, as pair differences. */
static int obj_delta(const tco_obj_t* o, const double* xold, const double* xnew, int64_t m, double* de)
{
    if (!o->snap) {
        *de = instance_delta(xold, xnew, m);
        return TCO_OK;
    }
    memcpy(o->cur, o->snap, sizeof(double) * 2 * (size_t)o->n);
    for (int64_t k = 0; k < m; ++k) {
        o->cur[2 * (int64_t)o->idx[k]] = xold[2 * k];
        o->cur[2 * (int64_t)o->idx[k] + 1] = xold[2 * k + 1];
    }
    return tco_delta_energy(o->cur, o->n, o->idx, m, xnew, de);
}

static int lbfgsb_run(const tco_obj_t* o, double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                      double step0, double maxstep, double sigma, const unsigned char* flags, int64_t max_halvings,
                      int64_t* iters_out, double* rms_out, int64_t* breaks_out);

/* L-BFGS-B on the (t, u) variables of Sec. II D over all n charges of one
 * configuration (tco_subdomain_lbfgsb: over a subdomain, as Sec. II C step 4).  Iteration with
 * at most `memory` pairs:
 *   stop when the projected-gradient RMS < gtol;
 *   theta = y.y / s.y of the newest pair (1 / step0 without pairs);
 *   xc = generalized Cauchy point, xbar = subspace minimiser (above);
 *   d = xbar - v; if g.d >= 0 the pairs are dropped and d = P(v - step0 g) - v;
 *   alpha = min(1, maxstep / max_i |d_i|) (|d_i| of charge i's two variables);
 *   v+ = P(v + alpha d), with the Armijo halving of tco_lbfgs_ls when
 *   max_halvings > 0 (energy change as pair differences);
 *   the pair (v+ - v, g+ - g) is kept iff s.y > 1e-12 |s||y|.
 * pos (in/out): x of the final variables.  Reports iterations, the final
 * projected-gradient RMS and the number of breakpoints the Cauchy searches
 * passed (each nullable). */
int tco_lbfgsb(double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol, double step0, double maxstep,
               double sigma, const unsigned char* flags, int64_t max_halvings, int64_t* iters_out, double* rms_out,
               int64_t* breaks_out)
{
    tco_obj_t o = {NULL, n, NULL, NULL};
    return lbfgsb_run(&o, pos, n, memory, max_iter, gtol, step0, maxstep, sigma, flags, max_halvings, iters_out,
                      rms_out, breaks_out);
}

/* L-BFGS-B on one subdomain (Sec. II C step 4): the charges of A = idx[0 .. m)
 * start at snap[idx] and move, on the (t, u) variables with interior radius
 * sigma (charges with flags[idx[k]] != 0 pinned to the unit circle; flags over
 * all n, nullable); every other charge stays at snap.  The objective is E_sub
 * of Sec. II D (tco_subdomain_grad), the line search's energy change
 * tco_delta_energy against snap.  Iteration as tco_lbfgsb with gtol = 0.
 * act_out (2m): the positions after `steps` iterations. */
int tco_subdomain_lbfgsb(const double* snap, int64_t n, const int32_t* idx, int64_t m, int64_t memory,
                         int64_t steps, double step0, double maxstep, double sigma, const unsigned char* flags,
                         int64_t max_halvings, double* act_out)
{
    if (n < 1 || m < 0 || !snap || (m > 0 && (!idx || !act_out))) return TCO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < m; ++k)
        if (idx[k] < 0 || idx[k] >= n) return TCO_ERR_INVALID_ARG;
    double* cur = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    unsigned char* fa = flags ? (unsigned char*)malloc((size_t)(m > 0 ? m : 1)) : NULL;
    if (!cur || (flags && !fa)) { free(cur); free(fa); return TCO_ERR_NO_MEMORY; }
    for (int64_t k = 0; k < m; ++k) {
        act_out[2 * k] = snap[2 * (int64_t)idx[k]];
        act_out[2 * k + 1] = snap[2 * (int64_t)idx[k] + 1];
        if (fa) fa[k] = flags[idx[k]];
    }
    tco_obj_t o = {snap, n, idx, cur};
    int st = lbfgsb_run(&o, act_out, m, memory, steps, 0.0, step0, maxstep, sigma, fa, max_halvings, NULL, NULL, NULL);
    free(cur);
    free(fa);
    return st;
}

static int lbfgsb_run(const tco_obj_t* o, double* pos, int64_t n, int64_t memory, int64_t max_iter, double gtol,
                      double step0, double maxstep, double sigma, const unsigned char* flags, int64_t max_halvings,
                      int64_t* iters_out, double* rms_out, int64_t* breaks_out)
{
    if (n < 0 || memory < 1 || memory > 32 || max_iter < 0 || max_halvings < 0 || (n > 0 && !pos) ||
        !(sigma > 0.0) || !(step0 > 0.0) || !(maxstep > 0.0))
        return TCO_ERR_INVALID_ARG;
    int64_t L = 2 * n;
    size_t sz = sizeof(double) * (size_t)(L > 0 ? L : 1);
    double *xk = malloc(sz), *v = malloc(sz), *vn = malloc(sz), *g = malloc(sz), *gv = malloc(sz),
           *gvn = malloc(sz), *d = malloc(sz), *lo = malloc(sz), *hi = malloc(sz), *xc = malloc(sz),
           *xbar = malloc(sz);
    double* S = malloc(sz * (size_t)memory);
    double* Y = malloc(sz * (size_t)memory);
    double* So = malloc(sz * (size_t)memory);
    double* Yo = malloc(sz * (size_t)memory);
    double M[64 * 64], c[64];
    int st = TCO_OK;
    if (!xk || !v || !vn || !g || !gv || !gvn || !d || !lo || !hi || !xc || !xbar || !S || !Y || !So || !Yo)
        st = TCO_ERR_NO_MEMORY;
    int64_t hist = 0, head = 0, it = 0, breaks = 0;
    double rms = 0.0, theta = 1.0 / step0;
    if (!st) {
        tu_box(n, flags, lo, hi);
        x_to_tu(pos, n, sigma, flags, v);
        box_clamp(v, lo, hi, L);
        tu_to_x(v, n, sigma, flags, pos);
        st = obj_grad(o, pos, n, g);
    }
    if (!st) {
        grad_tu(v, g, n, sigma, flags, gv);
        rms = proj_rms(v, gv, lo, hi, n);
    }
    for (; !st && it < max_iter; ++it) {
        if (rms < gtol) break;
        for (int64_t a = 0; a < hist; ++a) { /* oldest first */
            int64_t j = ((head - hist + a) % memory + memory) % memory;
            memcpy(So + a * L, S + j * L, sz);
            memcpy(Yo + a * L, Y + j * L, sz);
        }
        int64_t nbk = 0;
        st = tco_lbfgsb_middle(hist, So, Yo, L, theta, M);
        if (!st) st = tco_lbfgsb_cauchy(L, v, gv, lo, hi, hist, So, Yo, theta, M, xc, c, &nbk);
        if (!st) st = tco_lbfgsb_subspace(L, v, gv, lo, hi, hist, So, Yo, theta, M, xc, c, xbar);
        if (st) break;
        breaks += nbk;
        for (int64_t i = 0; i < L; ++i) d[i] = xbar[i] - v[i];
        if (dot(gv, d, L) >= 0.0) {
            hist = 0;
            head = 0;
            theta = 1.0 / step0;
            for (int64_t i = 0; i < L; ++i) {
                double w = v[i] - step0 * gv[i];
                w = w < lo[i] ? lo[i] : (w > hi[i] ? hi[i] : w);
                d[i] = w - v[i];
            }
        }
        double dmax = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double a = sqrt(d[2 * i] * d[2 * i] + d[2 * i + 1] * d[2 * i + 1]);
            if (a > dmax) dmax = a;
        }
        double alpha = (dmax > maxstep) ? maxstep / dmax : 1.0;
        for (int64_t i = 0; i < L; ++i) vn[i] = v[i] + alpha * d[i];
        box_clamp(vn, lo, hi, L);
        if (max_halvings > 0) {
            memcpy(xk, pos, sz);
            const double gd = dot(gv, d, L);
            for (int64_t hh = 0;; ++hh) {
                tu_to_x(vn, n, sigma, flags, pos);
                double de = 0.0;
                st = obj_delta(o, xk, pos, n, &de);
                if (st || de <= 1e-4 * alpha * gd || hh == max_halvings) break;
                alpha *= 0.5;
                for (int64_t i = 0; i < L; ++i) vn[i] = v[i] + alpha * d[i];
                box_clamp(vn, lo, hi, L);
            }
        } else {
            tu_to_x(vn, n, sigma, flags, pos);
        }
        if (!st) st = obj_grad(o, pos, n, g);
        if (st) break;
        grad_tu(vn, g, n, sigma, flags, gvn);
        rms = proj_rms(vn, gvn, lo, hi, n);
        acc_t sy_a = {0.0, 0.0}, ss_a = {0.0, 0.0}, yy_a = {0.0, 0.0};
        for (int64_t i = 0; i < L; ++i) {
            double si = vn[i] - v[i], yi = gvn[i] - gv[i];
            acc_add(&sy_a, si * yi);
            acc_add(&ss_a, si * si);
            acc_add(&yy_a, yi * yi);
        }
        double sy = acc_get(&sy_a);
        if (sy > 1e-12 * sqrt(acc_get(&ss_a)) * sqrt(acc_get(&yy_a))) {
            for (int64_t i = 0; i < L; ++i) { S[head * L + i] = vn[i] - v[i]; Y[head * L + i] = gvn[i] - gv[i]; }
            theta = acc_get(&yy_a) / sy;
            head = (head + 1) % memory;
            if (hist < memory) ++hist;
        }
        memcpy(v, vn, sz);
        memcpy(gv, gvn, sz);
    }
    if (iters_out) *iters_out = it;
    if (rms_out) *rms_out = rms;
    if (breaks_out) *breaks_out = breaks;
    free(xk); free(v); free(vn); free(g); free(gv); free(gvn); free(d); free(lo); free(hi); free(xc); free(xbar);
    free(S); free(Y); free(So); free(Yo);
    return st;
}

/* ------------------------------------------------ adaptive subdomains --- */

/* Active-set size at schedule position q.  Sec. II C lets the zone radius
 * r_zone oscillate periodically over a cycle of T subdomain optimisations
 * without giving the law; the zone is read here as "the m charges nearest to
 * the centre" and m follows a triangle wave of the given period:
 *     q' = q mod period,  m = m_min + floor(2 (m_max - m_min) min(q', period - q') / period),
 * so m = m_min at q' = 0 and m = m_max at q' = period/2; m is capped at n. */
int64_t tco_zone_size(int64_t q, int64_t m_min, int64_t m_max, int64_t period, int64_t n)
{
    int64_t qq = q % period;
    int64_t tri = qq < period - qq ? qq : period - qq;
    int64_t m = m_min + (2 * (m_max - m_min) * tri) / period;
    return m < n ? m : n;
}

typedef struct {
    double d2;
    int32_t i;
} near_t;

static int near_cmp(const void* a, const void* b)
{
    const near_t* p = (const near_t*)a;
    const near_t* q = (const near_t*)b;
    if (p->d2 < q->d2) return -1;
    if (p->d2 > q->d2) return 1;
    return (p->i > q->i) - (p->i < q->i);
}

static int int_cmp(const void* a, const void* b)
{
    int32_t p = *(const int32_t*)a, q = *(const int32_t*)b;
    return (p > q) - (p < q);
}

/* Steps 1-3 of the optimisation cycle of Sec. II C, and the zone of step 4,
 * for n_sub subdomains at schedule positions phase, phase+1, ...:
 *   local_e: e_i of step 1 (tco_energy with local_e);
 *   mu = mean of e_i, sigma_e = its population standard deviation, over all n;
 *   defects D = { i : e_i > mu + kappa sigma_e, |r_i| < radius - wall_tol and
 *     flags[i] == 0 } in ascending i (the paper's rule is kappa = -1; charges
 *     at the wall and pinned charges (flags nullable) are the boundary
 *     population that step 2 does not target);
 *   subdomain s draws u = uniforms[3s .. 3s+2] in [0,1):
 *     centre = r_{D[floor(u1 |D|)]} when u0 < p_defect and D is not empty,
 *     otherwise the area-uniform point sqrt(u1) radius (cos 2 pi u2, sin 2 pi u2);
 *     active set = the m_s = tco_zone_size(phase + s) charges with the smallest
 *     (d^2, i), d^2 = (x_i - c_x)^2 + (y_i - c_y)^2, listed in ascending i.
 * offsets (n_sub + 1) are written; idx holds offsets[n_sub] entries;
 * centres (2 n_sub), stats (3: mu, sigma_e, |D|) are nullable. */
int tco_zone_select(const double* pos, int64_t n, const double* local_e, const unsigned char* flags,
                    double kappa, double p_defect, double radius, double wall_tol, int64_t m_min, int64_t m_max,
                    int64_t period, int64_t phase, int64_t n_sub, const double* uniforms, int32_t* idx,
                    int64_t* offsets, double* centres, double* stats)
{
    if (n < 0 || n_sub < 0 || m_min < 0 || m_max < m_min || period < 1 || phase < 0 || !(radius > 0.0) ||
        (n_sub > 0 && (!uniforms || !offsets || n < 1 || !pos || !local_e || !idx)))
        return TCO_ERR_INVALID_ARG;
    if (n_sub == 0) {
        if (offsets) offsets[0] = 0;
        return TCO_OK;
    }
    /* step 2: statistics of the local-energy distribution */
    acc_t s1 = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) acc_add(&s1, local_e[i]);
    double mu = acc_get(&s1) / (double)n;
    acc_t s2 = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) acc_add(&s2, (local_e[i] - mu) * (local_e[i] - mu));
    double sigma = sqrt(acc_get(&s2) / (double)n);
    double thr = mu + kappa * sigma;
    double rin = radius - wall_tol;
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    near_t* nr = (near_t*)malloc(sizeof(near_t) * (size_t)n);
    if (!D || !nr) { free(D); free(nr); return TCO_ERR_NO_MEMORY; }
    int64_t nd = 0;
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1];
        if (local_e[i] > thr && x * x + y * y < rin * rin && !(flags && flags[i])) D[nd++] = (int32_t)i;
    }
    if (stats) { stats[0] = mu; stats[1] = sigma; stats[2] = (double)nd; }
    offsets[0] = 0;
    for (int64_t s = 0; s < n_sub; ++s) {
        /* step 3: the centre */
        double u0 = uniforms[3 * s], u1 = uniforms[3 * s + 1], u2 = uniforms[3 * s + 2];
        double cx, cy;
        if (u0 < p_defect && nd > 0) {
            int64_t k = (int64_t)(u1 * (double)nd);
            if (k > nd - 1) k = nd - 1;
            if (k < 0) k = 0;
            cx = pos[2 * D[k]];
            cy = pos[2 * D[k] + 1];
        } else {
            double r = sqrt(u1) * radius, t = 2.0 * TCO_PI * u2;
            cx = r * cos(t);
            cy = r * sin(t);
        }
        if (centres) { centres[2 * s] = cx; centres[2 * s + 1] = cy; }
        /* step 4's zone: the m_s nearest charges */
        int64_t m = tco_zone_size(phase + s, m_min, m_max, period, n);
        for (int64_t i = 0; i < n; ++i) {
            double dx = pos[2 * i] - cx, dy = pos[2 * i + 1] - cy;
            nr[i].d2 = dx * dx + dy * dy;
            nr[i].i = (int32_t)i;
        }
        qsort(nr, (size_t)n, sizeof(near_t), near_cmp);
        int32_t* out = idx + offsets[s];
        for (int64_t k = 0; k < m; ++k) out[k] = nr[k].i;
        qsort(out, (size_t)m, sizeof(int32_t), int_cmp);
        offsets[s + 1] = offsets[s] + m;
    }
    free(D);
    free(nr);
    return TCO_OK;
}

/* Interior radius of batch b of n_batches (Sec. II B, Eq. sigma: sigma rises
 * gradually from its initial value to 1; the law is not given, so it is read
 * as linear in the batch index): sigma0 + (sigma1 - sigma0) b / (n_batches - 1),
 * sigma1 for a single batch. */
double tco_sigma_ramp(double sigma0, double sigma1, int64_t b, int64_t n_batches)
{
    if (n_batches <= 1) return sigma1;
    return sigma0 + (sigma1 - sigma0) * (double)b / (double)(n_batches - 1);
}

/* Eq. Nb: the number of boundary charges, N_b = 2.84328 N^(2/3) -
 * 0.530196 N^(1/3) - 2.32866 rounded to the nearest integer, within [0, n]. */
int64_t tco_boundary_count(int64_t n)
{
    if (n <= 0) return 0;
    double c = cbrt((double)n);
    double nb = 2.84328 * c * c - 0.530196 * c - 2.32866;
    int64_t k = (int64_t)floor(nb + 0.5);
    return k < 0 ? 0 : (k > n ? n : k);
}

/* The border-interior split of Sec. II B: ordering the charges by (|r|^2, i)
 * ascending, the last n_b become boundary charges pinned to the unit circle
 * (flags = 1, r <- r/|r|) and the others interior charges confined to radius
 * sigma (flags = 0, r <- r min(1, sigma/|r|)).  pos in/out, flags out (n). */
int tco_border_split(double* pos, int64_t n, int64_t n_b, double sigma, unsigned char* flags)
{
    if (n < 0 || n_b < 0 || n_b > n || !(sigma > 0.0) || (n > 0 && (!pos || !flags))) return TCO_ERR_INVALID_ARG;
    near_t* nr = (near_t*)malloc(sizeof(near_t) * (size_t)(n > 0 ? n : 1));
    if (!nr) return TCO_ERR_NO_MEMORY;
    for (int64_t i = 0; i < n; ++i) {
        double x = pos[2 * i], y = pos[2 * i + 1];
        nr[i].d2 = x * x + y * y;
        nr[i].i = (int32_t)i;
    }
    qsort(nr, (size_t)n, sizeof(near_t), near_cmp);
    for (int64_t k = 0; k < n; ++k) flags[nr[k].i] = k >= n - n_b ? 1 : 0;
    free(nr);
    tco_project(pos, n, sigma, flags);
    return TCO_OK;
}

/* One optimisation cycle of Sec. II C over n_sub subdomains, taken in batches
 * of `batch` consecutive subdomains (batch = 1 is the paper's one-at-a-time
 * cycle).  For each batch b, with sigma_b = tco_sigma_ramp(sigma0, sigma1, b, .)
 * the interior radius (Sec. II B; flags, nullable, marks the pinned boundary
 * charges):
 *   E_b, e_i = tco_energy(pos)                       (step 1; trace[b] = E_b)
 *   zones    = tco_zone_select(pos, e, flags, ..., radius = sigma_b,
 *                              phase = b batch)      (steps 2-3)
 *   each zone relaxes against the batch-start snapshot with tco_subdomain_bb
 *   (step 4, projected gradient descent with BB steps, `steps` steps, free
 *   charges confined to sigma_b, pinned ones to the unit circle), or, in
 *   tco_cycle_opt with optimizer 1, with tco_subdomain_lbfgsb (the paper's
 *   L-BFGS-B on (t, u), interior radius sigma_b)
 *   tco_accept_sequential applies the relaxed zones in order (dE < 0, no clash).
 * trace (nullable, n_batches + 1): E before each batch and after the last.
 * delta, accepted (n_sub): per subdomain, as tco_accept_sequential. */
int tco_cycle_opt(double* pos, int64_t n, const unsigned char* flags, double kappa, double p_defect, double sigma0,
                  double sigma1, double wall_tol, int64_t m_min, int64_t m_max, int64_t period, int64_t n_sub,
                  int64_t batch, const double* uniforms, int64_t optimizer, double step0, double alpha_min,
                  double alpha_max, int64_t memory, double maxstep, int64_t max_halvings, int64_t steps,
                  double* trace, double* delta, unsigned char* accepted);

int tco_cycle(double* pos, int64_t n, const unsigned char* flags, double kappa, double p_defect, double sigma0,
              double sigma1, double wall_tol, int64_t m_min, int64_t m_max, int64_t period, int64_t n_sub,
              int64_t batch, const double* uniforms, double step0, double alpha_min, double alpha_max,
              int64_t steps, double* trace, double* delta, unsigned char* accepted)
{
    return tco_cycle_opt(pos, n, flags, kappa, p_defect, sigma0, sigma1, wall_tol, m_min, m_max, period, n_sub, batch,
                         uniforms, 0, step0, alpha_min, alpha_max, 1, 1.0, 0, steps, trace, delta, accepted);
}

int tco_cycle_run(double* pos, int64_t n, const unsigned char* flags, double kappa, double p_defect, double sigma0,
                  double sigma1, double wall_tol, int64_t m_min, int64_t m_max, int64_t period, int64_t n_sub,
                  int64_t batch, int64_t disjoint, const double* uniforms, int64_t optimizer, double step0,
                  double alpha_min, double alpha_max, int64_t memory, double maxstep, int64_t max_halvings,
                  int64_t steps, double* trace, double* delta, unsigned char* accepted, int64_t* n_batches_out);

/* tco_cycle with the zone optimiser chosen: 0 = projected BB (step0,
 * alpha_min, alpha_max), 1 = L-BFGS-B on (t, u) (memory, step0, maxstep,
 * at most max_halvings Armijo halvings per step). */
int tco_cycle_opt(double* pos, int64_t n, const unsigned char* flags, double kappa, double p_defect, double sigma0,
                  double sigma1, double wall_tol, int64_t m_min, int64_t m_max, int64_t period, int64_t n_sub,
                  int64_t batch, const double* uniforms, int64_t optimizer, double step0, double alpha_min,
                  double alpha_max, int64_t memory, double maxstep, int64_t max_halvings, int64_t steps,
                  double* trace, double* delta, unsigned char* accepted)
{
    return tco_cycle_run(pos, n, flags, kappa, p_defect, sigma0, sigma1, wall_tol, m_min, m_max, period, n_sub,
                         batch, 0, uniforms, optimizer, step0, alpha_min, alpha_max, memory, maxstep, max_halvings,
                         steps, trace, delta, accepted, NULL);
}

/* Whether zone s of a CSR list shares a charge with one of the zones 0 .. s-1
 * (mark: n bytes, the charges of zones 0 .. s-1 set; the zone is added when free). */
static int zone_clashes(const int32_t* idx, const int64_t* off, int64_t s, unsigned char* mark)
{
    for (int64_t k = off[s]; k < off[s + 1]; ++k)
        if (mark[idx[k]]) return 1;
    for (int64_t k = off[s]; k < off[s + 1]; ++k) mark[idx[k]] = 1;
    return 0;
}

/* The cycle, with two ways to form a batch from the subdomains not yet run:
 *   disjoint = 0: the next `batch` subdomains (a zone that shares a charge
 *     with a zone accepted earlier in the batch is skipped by the accept);
 *   disjoint = 1: the zones of the next `batch` subdomains are selected, and
 *     the batch is their longest prefix of pairwise disjoint zones (at least
 *     one); the zones after it are dropped and selected again, from the
 *     configuration and local energies after this batch, as the start of the
 *     next batch.  No zone is then skipped, every drawn centre is optimised,
 *     and batch = 1 is the paper's one-at-a-time cycle.  The interior radius
 *     of a batch whose first subdomain is b0 is
 *     sigma0 + (sigma1 - sigma0) b0 / (n_sub - 1) (sigma1 for n_sub = 1).
 * trace (nullable): n_sub + 1 entries in the disjoint form, n_batches + 1 used.
 * n_batches_out (nullable): the number of batches run. */
int tco_cycle_run(double* pos, int64_t n, const unsigned char* flags, double kappa, double p_defect, double sigma0,
                  double sigma1, double wall_tol, int64_t m_min, int64_t m_max, int64_t period, int64_t n_sub,
                  int64_t batch, int64_t disjoint, const double* uniforms, int64_t optimizer, double step0,
                  double alpha_min, double alpha_max, int64_t memory, double maxstep, int64_t max_halvings,
                  int64_t steps, double* trace, double* delta, unsigned char* accepted, int64_t* n_batches_out)
{
    if (optimizer < 0 || optimizer > 1 || disjoint < 0 || disjoint > 1) return TCO_ERR_INVALID_ARG;
    if (n < 1 || n_sub < 0 || batch < 1 || !pos || (n_sub > 0 && (!uniforms || !delta || !accepted)))
        return TCO_ERR_INVALID_ARG;
    int64_t n_batches = (n_sub + batch - 1) / batch;
    int64_t cap = (m_max < n ? m_max : n) * (batch < n_sub ? batch : (n_sub > 0 ? n_sub : 1));
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(batch + 1));
    double* act = (double*)malloc(sizeof(double) * 2 * (size_t)(cap > 0 ? cap : 1));
    unsigned char* mark = (unsigned char*)malloc((size_t)n);
    if (!e || !idx || !off || !act || !mark) {
        free(e); free(idx); free(off); free(act); free(mark);
        return TCO_ERR_NO_MEMORY;
    }
    int st = TCO_OK;
    int64_t nb = 0;
    for (int64_t b0 = 0, k = 0; b0 < n_sub && !st; b0 += k, ++nb) {
        k = n_sub - b0 < batch ? n_sub - b0 : batch;
        double radius = !disjoint ? tco_sigma_ramp(sigma0, sigma1, nb, n_batches)
                                  : tco_sigma_ramp(sigma0, sigma1, b0, n_sub);
        double E;
        st = tco_energy(pos, n, &E, e);
        if (st) break;
        if (trace) trace[nb] = E;
        st = tco_zone_select(pos, n, e, flags, kappa, p_defect, radius, wall_tol, m_min, m_max, period, b0, k,
                             uniforms + 3 * b0, idx, off, NULL, NULL);
        if (!st && disjoint) {
            memset(mark, 0, (size_t)n);
            int64_t kk = 0;
            while (kk < k && !zone_clashes(idx, off, kk, mark)) ++kk;
            k = kk;
        }
        for (int64_t s = 0; s < k && !st; ++s)
            st = optimizer == 0 ? tco_subdomain_bb(pos, n, idx + off[s], off[s + 1] - off[s], step0, alpha_min,
                                                   alpha_max, steps, radius, flags, act + 2 * off[s])
                                : tco_subdomain_lbfgsb(pos, n, idx + off[s], off[s + 1] - off[s], memory, steps,
                                                       step0, maxstep, radius, flags, max_halvings, act + 2 * off[s]);
        if (!st) st = tco_accept_sequential(pos, n, idx, off, k, act, delta + b0, accepted + b0);
    }
    if (!st && trace) st = tco_energy(pos, n, &trace[nb], NULL);
    if (n_batches_out) *n_batches_out = nb;
    free(e); free(idx); free(off); free(act); free(mark);
    return st;
}
