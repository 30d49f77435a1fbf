/*
 * Plain FP64 CPU oracle for microlensing critical curves, caustics, caustic-crossing
 * maps and distance-to-caustic maps (Weisenbach 2025, "A GPU Code for Finding
 * Microlensing Critical Curves and Caustics").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Conventions
 *   - theta_* = 1 (Einstein radius of a unit mass); stars (x_i, y_i, m_i).
 *   - Lens model: circular field with the compensating sheet extended to infinity
 *     (Appendix A), so alpha_s(z) = -kappa_* z everywhere and
 *       w(z)    = (1 - kappa_s) z + gamma conj(z) - sum_i m_i / conj(z - z_i)   (Sec. 3.1)
 *       F(z,phi)= gamma + sum_i m_i / (z - z_i)^2 - (1 - kappa_s) e^{-i phi}     (Eq. parametric cc)
 *     where kappa_s is the smooth convergence (kappa - kappa_*); or the rectangular field
 *     of Sec. 4.2 with the polynomial alpha_s of Appendix B (the orc_rect_* functions).
 *   - Complex arrays are interleaved (re, im) doubles == C99 double complex.
 *   - Built with -ffp-contract=off and without fast-math: every operation is an IEEE
 *     round-to-nearest FP64 operation in the order written.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* pi to double precision (same value as the POSIX M_PI). */
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------
 * Lens model (Sec. 3.1, Sec. 4.2 and Appendices A and B)
 *
 * Two smooth-matter models:
 *   disc      the circular field with its compensating sheet extended to infinity
 *             (Appendix A): alpha_s(z) = -kappa_* z, so dalpha_s/dz = -kappa_* and
 *             dalpha_s/dconj(z) = 0.
 *   rectangle the rectangular field of corner c = c1 + i c2 (Sec. 4.2) with the complex
 *             logarithms of alpha_s replaced by their Taylor series truncated at an odd
 *             order t and the sheet extended to infinity (Appendix B).  Then
 *             dalpha_s/dz = -kappa_* and dalpha_s/dconj(z) is a polynomial in conj(z).
 * In both, 1 - kappa - dalpha_s/dz = 1 - kappa_s (kappa = kappa_s + kappa_*).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    const double *x, *y, *m;
    int64_t n;
    double kappa_s, gamma;
    int rect;          /* 0: disc; 1: rectangle */
    double kappa_star; /* rectangle: convergence of the smooth sheet */
    cplx c;            /* rectangle: corner c1 + i c2 */
    int t;             /* rectangle: odd truncation order of the logarithm series */
    int64_t nr;        /* roots per row: 2n (disc), 2n + t - 1 (rectangle) */
} lens_t;

static lens_t disc_lens(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                        double gamma) {
    lens_t L;
    memset(&L, 0, sizeof L);
    L.x = x;
    L.y = y;
    L.m = m;
    L.n = n;
    L.kappa_s = kappa_s;
    L.gamma = gamma;
    L.nr = 2 * n;
    return L;
}

static lens_t rect_lens(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                        double gamma, double kappa_star, double c1, double c2, int t) {
    lens_t L = disc_lens(x, y, m, n, kappa_s, gamma);
    L.rect = 1;
    L.kappa_star = kappa_star;
    L.c = c1 + I * c2;
    L.t = t;
    L.nr = 2 * n + (t - 1);
    return L;
}

/* Rectangle: dalpha_s/dconj(z) as a function of zb = conj(z), the final form of
 * Appendix B:
 *   (-kappa_* i / pi) [ (zb/c)^t (1 + (-1)^t)(1 - e^{2 i Arg(c) t})
 *                       + sum_{j=1}^{t} (1/j) (zb/c)^j (1 + (-1)^j)(1 - e^{2 i Arg(c) j}) ]
 *   + kappa_* - 4 kappa_* Arg(c) / pi. */
static cplx rect_dalpha_dzb(const lens_t* L, cplx zb) {
    const double th = carg(L->c);
    const cplx u = zb / L->c;
    cplx s = 0.0, p = 1.0;
    for (int j = 1; j <= L->t; j++) {
        p *= u; /* (zb/c)^j */
        const double ev = (j % 2 == 0) ? 2.0 : 0.0; /* 1 + (-1)^j */
        s += (1.0 / j) * p * ev * (1.0 - cexp(I * 2.0 * th * j));
    }
    const double evt = (L->t % 2 == 0) ? 2.0 : 0.0;
    s += p * evt * (1.0 - cexp(I * 2.0 * th * L->t));
    return (-L->kappa_star * I / ORC_PI) * s + L->kappa_star - 4.0 * L->kappa_star * th / ORC_PI;
}

/* Rectangle: d^2 alpha_s / dconj(z)^2 (Appendix B), with (zb/c)^j / zb written as
 * zb^(j-1) / c^j so that zb = 0 needs no division:
 *   (-kappa_* i / pi) [ t zb^(t-1)/c^t (1 + (-1)^t)(1 - e^{2 i Arg(c) t})
 *                       + sum_{j=1}^{t} zb^(j-1)/c^j (1 + (-1)^j)(1 - e^{2 i Arg(c) j}) ]. */
static cplx rect_d2alpha_dzb2(const lens_t* L, cplx zb) {
    const double th = carg(L->c);
    cplx s = 0.0, p = 1.0 / L->c; /* zb^(j-1) / c^j at j = 1 */
    cplx last = p;
    for (int j = 1; j <= L->t; j++) {
        const double ev = (j % 2 == 0) ? 2.0 : 0.0;
        s += p * ev * (1.0 - cexp(I * 2.0 * th * j));
        last = p;
        p *= zb / L->c;
    }
    const double evt = (L->t % 2 == 0) ? 2.0 : 0.0;
    s += (double)L->t * last * evt * (1.0 - cexp(I * 2.0 * th * L->t));
    return (-L->kappa_star * I / ORC_PI) * s;
}

/* Rectangle: alpha_s(z) (Appendix B) with every log(a - zb), a in {c, conj c, -c, -conj c},
 * replaced by log(a) - sum_{j=1}^{t} (1/j) (zb/a)^j.  t < 0 evaluates the series' limit
 * log(a) + log(1 - zb/a): the logarithm continued from zb = 0 without crossing a branch cut
 * for |z| < |c| (the principal log(a - zb) jumps outside the rectangle, Appendix A); inside
 * the rectangle the two are equal.
 *   alpha_s = (-kappa_* i / pi) [ (c - zb) L(c) - (conj c - zb) L(conj c)
 *                                 + (-c - zb) L(-c) - (-conj c - zb) L(-conj c) ]
 *             - kappa_* (c + conj c + zb + z). */
static cplx rect_log_term(cplx a, cplx zb, int t) {
    if (t < 0) return clog(a) + clog(1.0 - zb / a);
    cplx s = clog(a), p = 1.0;
    for (int j = 1; j <= t; j++) {
        p *= zb / a;
        s -= p / (double)j;
    }
    return s;
}

static cplx rect_alpha(const lens_t* L, cplx z, int t) {
    const cplx zb = conj(z), c = L->c, cb = conj(L->c);
    const cplx A = (c - zb) * rect_log_term(c, zb, t) - (cb - zb) * rect_log_term(cb, zb, t) +
                   (-c - zb) * rect_log_term(-c, zb, t) - (-cb - zb) * rect_log_term(-cb, zb, t);
    return (-L->kappa_star * I / ORC_PI) * A - L->kappa_star * (c + cb + zb + z);
}

/* F(z, phi) of the parametric critical-curve equation (Sec. 3.1):
 *   F = gamma + sum_i m_i/(z - z_i)^2 - conj(dalpha_s/dconj z) - (1 - kappa_s) e^{-i phi}. */
static cplx lens_F(const lens_t* L, cplx e_mphi, cplx z) {
    cplx s = 0.0;
    for (int64_t i = 0; i < L->n; i++) {
        cplx d = z - (L->x[i] + I * L->y[i]);
        s += L->m[i] / (d * d);
    }
    cplx f = L->gamma + s - (1.0 - L->kappa_s) * e_mphi;
    if (L->rect) f -= conj(rect_dalpha_dzb(L, conj(z)));
    return f;
}

/* dF/dz = -2 sum_i m_i / (z - z_i)^3 - d/dz conj(dalpha_s/dconj z)
 * (derivative of F, needed by P'/P in Sec. 3.2); d/dz conj(g(conj z)) = conj(g'(conj z)). */
static cplx lens_dF(const lens_t* L, cplx z) {
    cplx s = 0.0;
    for (int64_t i = 0; i < L->n; i++) {
        cplx d = z - (L->x[i] + I * L->y[i]);
        s += L->m[i] / (d * d * d);
    }
    cplx f = -2.0 * s;
    if (L->rect) f -= conj(rect_d2alpha_dzb2(L, conj(z)));
    return f;
}

/* Complex lens equation (Sec. 3.1): w = (1 - kappa) z + gamma conj(z)
 *   - sum_i m_i / (conj(z) - conj(z_i)) - alpha_s(z), kappa = kappa_s + kappa_*;
 * for the disc alpha_s = -kappa_* z, which leaves (1 - kappa_s) z. */
static cplx lens_w(const lens_t* L, cplx z) {
    cplx s = 0.0;
    for (int64_t i = 0; i < L->n; i++) {
        cplx d = conj(z) - (L->x[i] - I * L->y[i]);
        s += L->m[i] / d;
    }
    if (!L->rect) return (1.0 - L->kappa_s) * z + L->gamma * conj(z) - s;
    return (1.0 - L->kappa_s - L->kappa_star) * z + L->gamma * conj(z) - s - rect_alpha(L, z, L->t);
}

double orc_F(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
             double gamma, double phi, const double* z, double* out) {
    lens_t L = disc_lens(x, y, m, n, kappa_s, gamma);
    cplx e = cos(phi) - I * sin(phi);
    cplx f = lens_F(&L, e, z[0] + I * z[1]);
    out[0] = creal(f);
    out[1] = cimag(f);
    return cabs(f);
}

double orc_dF(const double* x, const double* y, const double* m, int64_t n, const double* z,
              double* out) {
    lens_t L = disc_lens(x, y, m, n, 0.0, 0.0);
    cplx f = lens_dF(&L, z[0] + I * z[1]);
    out[0] = creal(f);
    out[1] = cimag(f);
    return cabs(f);
}

/* Inverse magnification 1/mu = det J = (1 - kappa_s)^2 - |gamma + sum m_i/conj(z - z_i)^2|^2
 * (Sec. 2.1; Appendix C, with the infinite sheet). */
double orc_inv_mu(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                  double gamma, const double* z) {
    cplx zz = z[0] + I * z[1];
    cplx s = 0.0;
    for (int64_t i = 0; i < n; i++) {
        cplx d = zz - (x[i] + I * y[i]);
        s += m[i] / (d * d);
    }
    double a = 1.0 - kappa_s;
    double g = cabs(gamma + s);
    return a * a - g * g;
}

/* Rectangle versions of F, F', alpha_s and w (Sec. 4.2, Appendix B).  t_alpha < 0 in
 * orc_rect_alpha evaluates the exact logarithms. */
double orc_rect_F(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                  double gamma, double kappa_star, double c1, double c2, int t, double phi,
                  const double* z, double* out) {
    lens_t L = rect_lens(x, y, m, n, kappa_s, gamma, kappa_star, c1, c2, t);
    cplx e = cos(phi) - I * sin(phi);
    cplx f = lens_F(&L, e, z[0] + I * z[1]);
    out[0] = creal(f);
    out[1] = cimag(f);
    return cabs(f);
}

double orc_rect_dF(const double* x, const double* y, const double* m, int64_t n, double kappa_star,
                   double c1, double c2, int t, const double* z, double* out) {
    lens_t L = rect_lens(x, y, m, n, 0.0, 0.0, kappa_star, c1, c2, t);
    cplx f = lens_dF(&L, z[0] + I * z[1]);
    out[0] = creal(f);
    out[1] = cimag(f);
    return cabs(f);
}

void orc_rect_alpha(double kappa_star, double c1, double c2, int t_alpha, const double* z, double* out) {
    lens_t L = rect_lens(NULL, NULL, NULL, 0, 0.0, 0.0, kappa_star, c1, c2, t_alpha < 0 ? 1 : t_alpha);
    cplx a = rect_alpha(&L, z[0] + I * z[1], t_alpha);
    out[0] = creal(a);
    out[1] = cimag(a);
}

void orc_rect_dalpha_dzb(double kappa_star, double c1, double c2, int t, const double* z, double* out) {
    lens_t L = rect_lens(NULL, NULL, NULL, 0, 0.0, 0.0, kappa_star, c1, c2, t);
    cplx a = rect_dalpha_dzb(&L, conj(z[0] + I * z[1]));
    out[0] = creal(a);
    out[1] = cimag(a);
}

/* Truncation order t for the rectangle (Appendix B): the smallest odd t >= 3 whose bound
 *   (kappa_* / pi) (4 / (t + 1)) s^-(t+1) |c| (s + 1)/(s - 1)
 * on the alpha_s error for |z| s < |c| is <= eps; then t grows by 2 while (t - 1) Arg(c)
 * lies within 10% of pi of a multiple of pi (where the leading coefficient vanishes or
 * nearly so). */
int orc_rect_choose_t(double kappa_star, double c1, double c2, double eps, double s) {
    const double ac = sqrt(c1 * c1 + c2 * c2), th = atan2(c2, c1);
    int t = 3;
    for (; t < 1000; t += 2) {
        double b = (kappa_star / ORC_PI) * (4.0 / (t + 1)) * pow(1.0 / s, t + 1) * ac * (s + 1.0) / (s - 1.0);
        if (b <= eps) break;
    }
    for (int guard = 0; guard < 1000; guard++) {
        double r = fmod((t - 1) * th, ORC_PI);
        if (r > 0.1 * ORC_PI && r < 0.9 * ORC_PI) break;
        t += 2;
    }
    return t;
}

/* ------------------------------------------------------------------------------------
 * Aberth-Ehrlich iteration on P(z) = F(z) prod (z - z_i)^2 (Sec. 3.2)
 * ------------------------------------------------------------------------------------ */

/* One root's Aberth correction (Sec. 3.2):
 *   P'/P = F'/F + 2 sum_i 1/(z_k - z_i)
 *   Delta = 1 / (P'/P - sum_{r != k} 1/(z_k - z_r)),   z_k <- z_k - Delta. */
static cplx aberth_delta(const lens_t* L, cplx e_mphi, const cplx* z, int64_t nr, int64_t k) {
    cplx zk = z[k];
    cplx F = lens_F(L, e_mphi, zk);
    if (F == 0.0) return 0.0; /* z_k is an exact root */
    cplx dF = lens_dF(L, zk);
    cplx s1 = 0.0;
    for (int64_t i = 0; i < L->n; i++) s1 += 1.0 / (zk - (L->x[i] + I * L->y[i]));
    cplx pp = dF / F + 2.0 * s1;
    cplx ab = 0.0;
    for (int64_t r = 0; r < nr; r++)
        if (r != k) ab += 1.0 / (zk - z[r]);
    return 1.0 / (pp - ab);
}

/* Jacobi Aberth over the n_r roots of one phi row (Sec. 3.2): every iteration updates
 * all unfrozen roots from the previous iterate; frozen roots still enter the root sum.
 * A root is frozen once |z^{a+1} - z^a| < tol (Sec. 3.2 footnote).
 * Returns the number of roots still unfrozen after max_iter iterations. */
static int64_t aberth_jacobi(const lens_t* L, double phi, cplx* z, int max_iter, double tol, int32_t* iters) {
    int64_t nr = L->nr;
    cplx e = cos(phi) - I * sin(phi);
    cplx* nxt = (cplx*)malloc(sizeof(cplx) * (size_t)nr);
    unsigned char* frozen = (unsigned char*)calloc((size_t)nr, 1);
    unsigned char* frozen_nxt = (unsigned char*)calloc((size_t)nr, 1);
    int64_t active = nr;
    if (iters)
        for (int64_t k = 0; k < nr; k++) iters[k] = 0;
    for (int a = 0; a < max_iter && active > 0; a++) {
        int64_t still = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : still)
        for (int64_t k = 0; k < nr; k++) {
            if (frozen[k]) {
                nxt[k] = z[k];
                frozen_nxt[k] = 1;
                continue;
            }
            cplx d = aberth_delta(L, e, z, nr, k);
            nxt[k] = z[k] - d;
            if (iters) iters[k] = a + 1;
            if (cabs(d) < tol) {
                frozen_nxt[k] = 1;
            } else {
                frozen_nxt[k] = 0;
                still++;
            }
        }
        memcpy(z, nxt, sizeof(cplx) * (size_t)nr);
        memcpy(frozen, frozen_nxt, (size_t)nr);
        active = still;
    }
    free(nxt);
    free(frozen);
    free(frozen_nxt);
    return active;
}

/* Newton refinement of each root on F alone, to |dz| < 1e-13 max(1,|z|) (at most 8
 * steps).  This takes the Aberth result (accurate to ~1e-9) to the FP64 limit, so the
 * oracle's roots stand for the exact roots of F(., phi). */
static void newton_polish(const lens_t* L, double phi, cplx* z) {
    cplx e = cos(phi) - I * sin(phi);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < L->nr; k++) {
        cplx zk = z[k];
        for (int s = 0; s < 8; s++) {
            cplx F = lens_F(L, e, zk);
            cplx dF = lens_dF(L, zk);
            if (F == 0.0 || dF == 0.0) break;
            cplx d = F / dF;
            zk -= d;
            double sc = cabs(zk) > 1.0 ? cabs(zk) : 1.0;
            if (cabs(d) < 1e-13 * sc) break;
        }
        z[k] = zk;
    }
}

/* Initial guesses z_i + 1 and z_i - 1 for every star (Sec. 3.2), stored as
 * [2i] = z_i + 1, [2i+1] = z_i - 1; for the rectangle, the t - 1 further roots start
 * evenly spread on the circle of radius |c| around the field (Sec. 3.2), at angles
 * 2 pi (k + 1/2) / (t - 1).  A guess that coincides (within 1e-12) with an earlier one is
 * moved by 1e-6 (1 + i) so that the Aberth root sum stays finite. */
static void initial_guesses(const lens_t* L, cplx* z) {
    int64_t nr = L->nr, n = L->n;
    for (int64_t i = 0; i < n; i++) {
        z[2 * i] = (L->x[i] + 1.0) + I * L->y[i];
        z[2 * i + 1] = (L->x[i] - 1.0) + I * L->y[i];
    }
    for (int64_t k = 2 * n; k < nr; k++) {
        double a = 2.0 * ORC_PI * ((double)(k - 2 * n) + 0.5) / (double)(nr - 2 * n);
        z[k] = cabs(L->c) * (cos(a) + I * sin(a));
    }
    for (int64_t b = 1; b < nr; b++) {
        int moved = 1;
        while (moved) {
            moved = 0;
            for (int64_t a = 0; a < b; a++) {
                if (cabs(z[b] - z[a]) < 1e-12) {
                    z[b] += 1e-6 * (1.0 + I);
                    moved = 1;
                }
            }
        }
    }
}

/* Solve one phi row from a given start (warm) or from the initial guesses (z_in == NULL),
 * then Newton-polish.  Output: z_out[n_r] complex.  Returns the unfrozen count.
 * A warm start assumes a small phase step (Sec. 3.2); when it does not converge within
 * max_iter (e.g. a phase step of pi for an isolated star, whose warm start then lies on a
 * line the iteration never leaves), the row is solved again from the initial guesses. */
static int64_t solve_row(const lens_t* L, double phi, const double* z_in, double* z_out, int max_iter, double tol,
                         int32_t* iters) {
    cplx* z = (cplx*)z_out;
    if (z_in)
        memcpy(z, z_in, sizeof(cplx) * (size_t)L->nr);
    else
        initial_guesses(L, z);
    int64_t left = aberth_jacobi(L, phi, z, max_iter, tol, iters);
    if (left > 0 && z_in) {
        initial_guesses(L, z);
        left = aberth_jacobi(L, phi, z, max_iter, tol, iters);
    }
    newton_polish(L, phi, z);
    return left;
}

int64_t orc_solve_row(const double* x, const double* y, const double* m, int64_t n,
                      double kappa_s, double gamma, double phi, const double* z_in,
                      double* z_out, int max_iter, double tol, int32_t* iters) {
    lens_t L = disc_lens(x, y, m, n, kappa_s, gamma);
    return solve_row(&L, phi, z_in, z_out, max_iter, tol, iters);
}

int64_t orc_rect_solve_row(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                           double gamma, double kappa_star, double c1, double c2, int t, double phi,
                           const double* z_in, double* z_out, int max_iter, double tol, int32_t* iters) {
    lens_t L = rect_lens(x, y, m, n, kappa_s, gamma, kappa_star, c1, c2, t);
    return solve_row(&L, phi, z_in, z_out, max_iter, tol, iters);
}

/* phi_j = 2 pi j / m for the (m+1)-row chain matrix (Sec. 4.3). */
double orc_phi(int64_t j, int64_t msteps) { return 2.0 * ORC_PI * (double)j / (double)msteps; }

/* Chain matrix of Sec. 4.3: rows j = 0..m (m even) hold the n_r roots at phi_j.  The
 * central row m/2 (phi = pi) starts from the initial guesses (cap max_iter_cold); the
 * matrix then grows toward rows 0 and m, each row warm-started from its neighbour
 * nearer the centre (Sec. 3.2 last paragraph), cap max_iter_warm.
 * z_out: (m+1) x n_r complex; iters_out (optional): (m+1) x n_r.
 * Returns the total number of unfrozen roots over all rows (0 = all converged). */
static int64_t critical_curves(const lens_t* L, int64_t msteps, double tol, int max_iter_cold, int max_iter_warm,
                               double* z_out, int32_t* iters_out) {
    int64_t nr = L->nr;
    int64_t c = msteps / 2;
    int64_t bad = 0;
    double* zr = z_out;
    bad += solve_row(L, orc_phi(c, msteps), NULL, zr + 2 * nr * c, max_iter_cold, tol,
                     iters_out ? iters_out + nr * c : NULL);
    for (int64_t j = c - 1; j >= 0; j--)
        bad += solve_row(L, orc_phi(j, msteps), zr + 2 * nr * (j + 1), zr + 2 * nr * j, max_iter_warm, tol,
                         iters_out ? iters_out + nr * j : NULL);
    for (int64_t j = c + 1; j <= msteps; j++)
        bad += solve_row(L, orc_phi(j, msteps), zr + 2 * nr * (j - 1), zr + 2 * nr * j, max_iter_warm, tol,
                         iters_out ? iters_out + nr * j : NULL);
    return bad;
}

int64_t orc_critical_curves(const double* x, const double* y, const double* m, int64_t n,
                            double kappa_s, double gamma, int64_t msteps, double tol,
                            int max_iter_cold, int max_iter_warm, double* z_out,
                            int32_t* iters_out) {
    lens_t L = disc_lens(x, y, m, n, kappa_s, gamma);
    return critical_curves(&L, msteps, tol, max_iter_cold, max_iter_warm, z_out, iters_out);
}

int64_t orc_rect_critical_curves(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                                 double gamma, double kappa_star, double c1, double c2, int t, int64_t msteps,
                                 double tol, int max_iter_cold, int max_iter_warm, double* z_out,
                                 int32_t* iters_out) {
    lens_t L = rect_lens(x, y, m, n, kappa_s, gamma, kappa_star, c1, c2, t);
    return critical_curves(&L, msteps, tol, max_iter_cold, max_iter_warm, z_out, iters_out);
}

/* Caustic mapping (Sec. 3.1, Sec. 5.1): w = lens map of each critical point. */
static void map_caustics(const lens_t* L, const double* z, int64_t count, double* w_out) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < count; p++) {
        cplx w = lens_w(L, z[2 * p] + I * z[2 * p + 1]);
        w_out[2 * p] = creal(w);
        w_out[2 * p + 1] = cimag(w);
    }
}

void orc_map_caustics(const double* x, const double* y, const double* m, int64_t n,
                      double kappa_s, double gamma, const double* z, int64_t count,
                      double* w_out) {
    lens_t L = disc_lens(x, y, m, n, kappa_s, gamma);
    map_caustics(&L, z, count, w_out);
}

void orc_rect_map_caustics(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                           double gamma, double kappa_star, double c1, double c2, int t, const double* z,
                           int64_t count, double* w_out) {
    lens_t L = rect_lens(x, y, m, n, kappa_s, gamma, kappa_star, c1, c2, t);
    map_caustics(&L, z, count, w_out);
}

/* Newton correction and caustic point of given points of a disc field (Sec. 3.1 for F and
 * w, Sec. 3.2 for the Newton correction inside Aberth's step).  Point p = r * nr + k lies on
 * row j = row0 + r, phi_j = 2 pi j / m (orc_phi).  step[p] = |F(z_p, phi_j)| / |F'(z_p)|,
 * the length of the Newton correction: for a simple zero of F it is the distance from z_p
 * to that zero up to a second-order term.  w_out[p] = w(z_p), the lens map.
 * One pass over the stars per point: with u = 1/(z - z_i) = conj(z - z_i)/|z - z_i|^2,
 *   F  = gamma + sum m_i u^2 - (1 - kappa_s) e^{-i phi},   F' = -2 sum m_i u^3,
 *   w  = (1 - kappa_s) z + gamma conj(z) - sum m_i conj(u). */
void orc_newton_check(const double* x, const double* y, const double* m, int64_t n, double kappa_s,
                      double gamma, int64_t msteps, int64_t row0, int64_t rows, int64_t nr, const double* z,
                      double* step, double* w_out) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < rows * nr; p++) {
        const int64_t j = row0 + p / nr;
        const double phi = orc_phi(j, msteps);
        const cplx e_mphi = cos(phi) - I * sin(phi);
        const cplx zz = z[2 * p] + I * z[2 * p + 1];
        cplx sF = 0.0, sdF = 0.0, sW = 0.0;
        for (int64_t i = 0; i < n; i++) {
            const double dx = creal(zz) - x[i], dy = cimag(zz) - y[i];
            const double r2 = dx * dx + dy * dy;
            const cplx u = dx / r2 - I * (dy / r2);
            const cplx u2 = u * u;
            sF += m[i] * u2;
            sdF += m[i] * (u2 * u);
            sW += m[i] * conj(u);
        }
        const cplx F = gamma + sF - (1.0 - kappa_s) * e_mphi;
        const cplx dF = -2.0 * sdF;
        const cplx w = (1.0 - kappa_s) * zz + gamma * conj(zz) - sW;
        step[p] = cabs(F) / cabs(dF);
        w_out[2 * p] = creal(w);
        w_out[2 * p + 1] = cimag(w);
    }
}

/* Smallest pairwise distance among the n_r roots of one row (distinctness check). */
double orc_min_separation(const double* z, int64_t nr) {
    double best = INFINITY;
    for (int64_t a = 0; a < nr; a++)
        for (int64_t b = a + 1; b < nr; b++) {
            double dx = z[2 * a] - z[2 * b], dy = z[2 * a + 1] - z[2 * b + 1];
            double d = sqrt(dx * dx + dy * dy);
            if (d < best) best = d;
        }
    return best;
}

/* ------------------------------------------------------------------------------------
 * Exact orientation predicate by exact expansion arithmetic.
 *
 * sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx): +1 if c lies strictly to the left of the
 * directed line a->b, -1 strictly right, 0 on it.  Every difference is split exactly
 * into two doubles (Knuth's two-sum), every product of two doubles exactly into two
 * doubles (fma), and the 16 resulting terms are summed exactly into a non-overlapping
 * expansion (Shewchuk 1997, grow-expansion); the sign of the largest component is the
 * sign of the sum.  No floating-point filter: every call takes the exact route.
 * Exact as long as nothing overflows or underflows.
 * ------------------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

static void two_prod(double a, double b, double* p, double* e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* h <- h + b exactly (h non-overlapping, increasing magnitude); returns new length. */
static int grow_expansion(double* h, int len, double b) {
    double q = b;
    for (int i = 0; i < len; i++) {
        double s, e;
        two_sum(q, h[i], &s, &e);
        h[i] = e;
        q = s;
    }
    h[len] = q;
    return len + 1;
}

int orc_orient2d(double ax, double ay, double bx, double by, double cx, double cy) {
    double acx[2], bcy[2], acy[2], bcx[2];
    two_sum(ax, -cx, &acx[0], &acx[1]);
    two_sum(by, -cy, &bcy[0], &bcy[1]);
    two_sum(ay, -cy, &acy[0], &acy[1]);
    two_sum(bx, -cx, &bcx[0], &bcx[1]);
    double h[40];
    int len = 0;
    for (int u = 0; u < 2; u++)
        for (int v = 0; v < 2; v++) {
            double p, e;
            two_prod(acx[u], bcy[v], &p, &e);
            len = grow_expansion(h, len, e);
            len = grow_expansion(h, len, p);
            two_prod(acy[u], bcx[v], &p, &e);
            len = grow_expansion(h, len, -e);
            len = grow_expansion(h, len, -p);
        }
    for (int i = len - 1; i >= 0; i--) {
        if (h[i] > 0.0) return 1;
        if (h[i] < 0.0) return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Caustic-crossing counts (Sec. 5.1): winding numbers of the discretised caustics.
 *
 * The caustic polygons are the columns of the (rows x n_r) vertex matrix: segment
 * (w[j][k], w[j+1][k]) for j = 0..rows-2.  Sunday's (2001) crossing rule: an upward
 * edge (a.y <= P.y < b.y) with P strictly left adds +1, a downward edge
 * (b.y <= P.y < a.y) with P strictly right adds -1.  Caustics are traced clockwise
 * (Sec. 5.1), so the number of caustic crossings is N_cc = -winding number.
 * ------------------------------------------------------------------------------------ */

/* Pixel centre of index i on [lo, hi] split into cnt pixels. */
double orc_pixel_center(double lo, double hi, int32_t cnt, int32_t i) {
    double step = (hi - lo) / (double)cnt;
    return lo + ((double)i + 0.5) * step;
}

static int sunday_edge(double ax, double ay, double bx, double by, double px, double py) {
    if (ay <= py) {
        if (by > py && orc_orient2d(ax, ay, bx, by, px, py) > 0) return 1;
    } else {
        if (by <= py && orc_orient2d(ax, ay, bx, by, px, py) < 0) return -1;
    }
    return 0;
}

/* Winding number of all caustic polygons around one point (definition, all segments). */
int64_t orc_winding_at(const double* w, int64_t rows, int64_t nr, double px, double py) {
    int64_t wn = 0;
    for (int64_t k = 0; k < nr; k++)
        for (int64_t j = 0; j + 1 < rows; j++) {
            const double* a = w + 2 * (j * nr + k);
            const double* b = w + 2 * ((j + 1) * nr + k);
            wn += sunday_edge(a[0], a[1], b[0], b[1], px, py);
        }
    return wn;
}

/* Pixel rows rlist[0..count) of the N_cc map of a W x H grid (row 0 = y0 side, column 0 =
 * x0 side) into ncc[t * W + i] for row rlist[t].  Same decisions as evaluating
 * orc_winding_at at every pixel centre: a segment can only change the count of pixel rows
 * whose centre satisfies min(a.y,b.y) <= y < max(a.y,b.y), so other rows are skipped for
 * that segment. */
static void crossing_rows(const double* w, int64_t rows, int64_t nr, double x0, double x1, double y0,
                          double y1, int32_t W, int32_t H, const int32_t* rlist, int32_t count, int32_t* ncc) {
    int64_t npx = (int64_t)W * count;
    int64_t* wn = (int64_t*)calloc((size_t)npx, sizeof(int64_t));
    double* pxc = (double*)malloc(sizeof(double) * (size_t)W);
    for (int32_t i = 0; i < W; i++) pxc[i] = orc_pixel_center(x0, x1, W, i);
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t t = 0; t < count; t++) {
        double py = orc_pixel_center(y0, y1, H, rlist[t]);
        for (int64_t k = 0; k < nr; k++)
            for (int64_t j = 0; j + 1 < rows; j++) {
                const double* a = w + 2 * (j * nr + k);
                const double* b = w + 2 * ((j + 1) * nr + k);
                double lo = a[1] < b[1] ? a[1] : b[1];
                double hi = a[1] < b[1] ? b[1] : a[1];
                if (!(lo <= py && py < hi)) continue;
                for (int32_t i = 0; i < W; i++)
                    wn[(int64_t)t * W + i] += sunday_edge(a[0], a[1], b[0], b[1], pxc[i], py);
            }
    }
    for (int64_t p = 0; p < npx; p++) ncc[p] = (int32_t)(-wn[p]);
    free(wn);
    free(pxc);
}

/* Full N_cc map (row 0 = y0 side, column 0 = x0 side). */
void orc_crossing_map(const double* w, int64_t rows, int64_t nr, double x0, double x1,
                      double y0, double y1, int32_t W, int32_t H, int32_t* ncc) {
    int32_t* rlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)H);
    for (int32_t r = 0; r < H; r++) rlist[r] = r;
    crossing_rows(w, rows, nr, x0, x1, y0, y1, W, H, rlist, H, ncc);
    free(rlist);
}

/* The listed pixel rows of the N_cc map of the W x H grid (rows of orc_crossing_map, same
 * pixel centres), into a count x W array. */
void orc_crossing_rows(const double* w, int64_t rows, int64_t nr, double x0, double x1, double y0,
                       double y1, int32_t W, int32_t H, const int32_t* rlist, int32_t count, int32_t* ncc) {
    crossing_rows(w, rows, nr, x0, x1, y0, y1, W, H, rlist, count, ncc);
}

/* ------------------------------------------------------------------------------------
 * Distance to the nearest caustic for an expanding source (Sec. 5.2): Euclidean
 * distance transform of the N_cc map.  A feature pixel is one with a 4-neighbour (inside
 * the map) of different N_cc; the map border itself is not a caustic.  Distances are
 * pixel * sqrt(squared integer index distance); +inf when the map has no feature.
 * ------------------------------------------------------------------------------------ */
static int is_feature(const int32_t* ncc, int32_t W, int32_t H, int32_t r, int32_t i) {
    int32_t v = ncc[(int64_t)r * W + i];
    if (i > 0 && ncc[(int64_t)r * W + i - 1] != v) return 1;
    if (i + 1 < W && ncc[(int64_t)r * W + i + 1] != v) return 1;
    if (r > 0 && ncc[(int64_t)(r - 1) * W + i] != v) return 1;
    if (r + 1 < H && ncc[(int64_t)(r + 1) * W + i] != v) return 1;
    return 0;
}

void orc_feature_mask(const int32_t* ncc, int32_t W, int32_t H, uint8_t* mask) {
    for (int32_t r = 0; r < H; r++)
        for (int32_t i = 0; i < W; i++) mask[(int64_t)r * W + i] = (uint8_t)is_feature(ncc, W, H, r, i);
}

/* Brute force: every pixel against every feature pixel. */
void orc_distance_map_brute(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                            double* d_out) {
    int64_t npx = (int64_t)W * H;
    int32_t* fr = (int32_t*)malloc(sizeof(int32_t) * (size_t)npx);
    int32_t* fi = (int32_t*)malloc(sizeof(int32_t) * (size_t)npx);
    int64_t nf = 0;
    for (int32_t r = 0; r < H; r++)
        for (int32_t i = 0; i < W; i++)
            if (is_feature(ncc, W, H, r, i)) {
                fr[nf] = r;
                fi[nf] = i;
                nf++;
            }
#pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < H; r++)
        for (int32_t i = 0; i < W; i++) {
            int64_t best = -1;
            for (int64_t f = 0; f < nf; f++) {
                int64_t dr = r - fr[f], di = i - fi[f];
                int64_t d2 = dr * dr + di * di;
                if (best < 0 || d2 < best) best = d2;
            }
            d_out[(int64_t)r * W + i] = best < 0 ? INFINITY : pixel * sqrt((double)best);
        }
    free(fr);
    free(fi);
}

/* Separable exact EDT (Felzenszwalb & Huttenlocher 2012): a column pass giving the
 * vertical distance to the nearest feature in the same column, then per row the lower
 * envelope of the parabolas (i - q)^2 + g(q)^2.  Parabola intersections are compared
 * exactly as fractions of 64-bit integers. */
void orc_distance_map_separable(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                                double* d_out) {
    const int64_t INF = (int64_t)1 << 40;
    int64_t npx = (int64_t)W * H;
    int64_t* g = (int64_t*)malloc(sizeof(int64_t) * (size_t)npx); /* vertical distance */
    for (int32_t i = 0; i < W; i++) {
        int64_t last = -1;
        for (int32_t r = 0; r < H; r++) {
            if (is_feature(ncc, W, H, r, i)) last = r;
            g[(int64_t)r * W + i] = last < 0 ? INF : r - last;
        }
        last = -1;
        for (int32_t r = H - 1; r >= 0; r--) {
            if (is_feature(ncc, W, H, r, i)) last = r;
            if (last >= 0 && last - r < g[(int64_t)r * W + i]) g[(int64_t)r * W + i] = last - r;
        }
    }
#pragma omp parallel
    {
        int64_t* v = (int64_t*)malloc(sizeof(int64_t) * (size_t)W);
        int64_t* zn = (int64_t*)malloc(sizeof(int64_t) * (size_t)(W + 1)); /* boundary numerators */
        int64_t* zd = (int64_t*)malloc(sizeof(int64_t) * (size_t)(W + 1)); /* denominators > 0 */
        int* zinf = (int*)malloc(sizeof(int) * (size_t)(W + 1));          /* -1: -inf, +1: +inf */
#pragma omp for schedule(static)
        for (int32_t r = 0; r < H; r++) {
            const int64_t* f = g + (int64_t)r * W;
            int64_t k = -1;
            for (int64_t q = 0; q < W; q++) {
                if (f[q] >= INF) continue;
                int64_t fq = f[q] * f[q] + q * q;
                if (k < 0) {
                    k = 0;
                    v[0] = q;
                    zinf[0] = -1;
                    zinf[1] = 1;
                    continue;
                }
                for (;;) {
                    int64_t p = v[k];
                    int64_t sn = fq - (f[p] * f[p] + p * p); /* s = sn / sd */
                    int64_t sd = 2 * (q - p);
                    /* s <= z[k] ? */
                    int le;
                    if (zinf[k] == -1) le = 0;
                    else le = sn * zd[k] <= zn[k] * sd;
                    if (le) {
                        k--;
                        continue;
                    }
                    k++;
                    v[k] = q;
                    zn[k] = sn;
                    zd[k] = sd;
                    zinf[k] = 0;
                    zinf[k + 1] = 1;
                    break;
                }
            }
            double* out = d_out + (int64_t)r * W;
            if (k < 0) {
                for (int64_t i = 0; i < W; i++) out[i] = -1.0; /* no feature in this row's columns */
                continue;
            }
            int64_t j = 0;
            for (int64_t i = 0; i < W; i++) {
                /* advance while z[j+1] < i */
                while (zinf[j + 1] == 0 && zn[j + 1] < i * zd[j + 1]) j++;
                int64_t p = v[j];
                int64_t d2 = (i - p) * (i - p) + f[p] * f[p];
                out[i] = pixel * sqrt((double)d2);
            }
        }
        free(v);
        free(zn);
        free(zd);
        free(zinf);
    }
    /* rows whose columns all lack features: no feature anywhere in the map if every row
     * is marked; otherwise impossible (a feature in any column reaches every row). */
    for (int64_t p = 0; p < npx; p++)
        if (d_out[p] < 0.0) d_out[p] = INFINITY;
    free(g);
}

/* ------------------------------------------------------------------------------------
 * Distance to the nearest caustic for a source moving along a direction (Sec. 5.2, bottom
 * of the distance-map figure): from each pixel centre, the ray in direction
 * (cos angle, sin angle) (angle from the +x axis) is followed pixel by pixel (grid
 * traversal in units of pixels); the result is the ray parameter at which it enters the
 * first caustic (feature) pixel, times the pixel size.  A start pixel that is itself a
 * caustic pixel gives 0; a ray that leaves the map first gives +inf (the border is not a
 * caustic).  The traversal is written with IEEE single-precision operations in a fixed
 * order: the crossing parameter of the next vertical (horizontal) grid line after k
 * steps is (0.5 + k) * (1 / |cos|) (resp. |sin|); the smaller one is taken, the
 * horizontal-line crossing on ties.
 * ------------------------------------------------------------------------------------ */
void orc_moving_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, double angle,
                             double* d_out) {
    const float c = (float)cos(angle), s = (float)sin(angle);
    const int sx = c > 0.0f ? 1 : (c < 0.0f ? -1 : 0);
    const int sy = s > 0.0f ? 1 : (s < 0.0f ? -1 : 0);
    const float tdx = sx ? 1.0f / fabsf(c) : 0.0f;
    const float tdy = sy ? 1.0f / fabsf(s) : 0.0f;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t r = 0; r < H; r++)
        for (int32_t i = 0; i < W; i++) {
            double d;
            if (is_feature(ncc, W, H, r, i)) {
                d = 0.0;
            } else {
                int32_t x = i, y = r;
                int64_t nx = 0, ny = 0;
                float t = 0.0f;
                for (;;) {
                    const float tx = sx ? (0.5f + (float)nx) * tdx : INFINITY;
                    const float ty = sy ? (0.5f + (float)ny) * tdy : INFINITY;
                    if (tx < ty) {
                        x += sx;
                        nx++;
                        t = tx;
                    } else {
                        y += sy;
                        ny++;
                        t = ty;
                    }
                    if (x < 0 || x >= W || y < 0 || y >= H) {
                        d = INFINITY;
                        break;
                    }
                    if (is_feature(ncc, W, H, y, x)) {
                        d = pixel * (double)t;
                        break;
                    }
                }
            }
            d_out[(int64_t)r * W + i] = d;
        }
}

/* Threads of the oracle's parallel loops from now on (timing runs; n >= 1). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
