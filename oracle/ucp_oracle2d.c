/*
 * ucp_oracle2d.c -- TEST INFRASTRUCTURE ONLY: the plain FP64 oracle of the
 * sweep on the 2-dimensional Witsenhausen counterexample (Section V-D).
 * Loaded only by tests/ and the CPU-baseline leg of bench.py; shares no code
 * with the CUDA library.  Notation and conventions: ucp_oracle2d.h.
 *
 * What it computes, and where the paper defines it:
 *   - the problem of Section V-D (Witsenhausen's counterexample with x, u
 *     and y in R^2, objective (1/2) E[k^2 |u0|^2 + |x2|^2]);
 *   - Corollary 1: u0 is improved pointwise by the first minimiser of its
 *     marginal cost g(u; x) = k^2 |u - x|^2 + S(u), S(u) = E_w |u -
 *     u1(u + w)|^2 (the factor p(x) / 2 dropped), over a candidate list that
 *     holds eq. (2)'s neighbouring samples (r per direction on each axis);
 *   - Jacobi over the grid (Section IV-A);
 *   - u1 = E[x1 | y1] (the exact minimiser of its quadratic marginal cost,
 *     the closed form of Section IV-C), per component.
 * Arithmetic: FP64, -ffp-contract=off; S and the weight normalisation by the
 * fixed summation order of the one-dimensional oracle (32-term chunks, then
 * pairwise by levels) over the taps in row-major order; the u1 sums and J in
 * index order.
 *
 * Parity status: pinned in tests/test_oracle2d.py (separable controllers
 * reduce every quantity to the pinned one-dimensional oracle; closed form
 * for affine controllers; numpy's bilinear interpolation; brute force over
 * the candidate list; the weighted mean).
 */
#include "ucp_oracle2d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

extern int orc_get_threads(void);

typedef struct {
    orc2_params p;
    int64_t hx, hw, hy, hr, n_x, n_w, n_y;
    int32_t shift;
    int64_t one, q, n_cand;
    double kk;
} geom2;

static int steps_of(double half, double delta, int64_t* out) {
    double r = half / delta, n = floor(r + 0.5);
    if (!(n >= 0.0) || fabs(r - n) > 1e-9 * (n > 1.0 ? n : 1.0)) return -1;
    *out = (int64_t)n;
    return 0;
}

static int make2(const orc2_params* p, geom2* g) {
    memset(g, 0, sizeof(*g));
    g->p = *p;
    if (!(p->k > 0.0) || !(p->sigma > 0.0) || !(p->delta > 0.0)) return -1;
    if (steps_of(p->x_half, p->delta, &g->hx) || steps_of(p->w_half, p->delta, &g->hw) ||
        steps_of(p->y_half, p->delta, &g->hy) || steps_of(p->cand_half, p->delta, &g->hr))
        return -1;
    if (p->n_coarse < 2 || p->n_levels < 0 || p->n_levels > 40 || p->n_nbr < 0) return -1;
    g->n_x = 2 * g->hx + 1;
    g->n_w = 2 * g->hw + 1;
    g->n_y = 2 * g->hy + 1;
    g->shift = p->n_levels;
    g->one = (int64_t)1 << g->shift;
    int64_t nc1 = p->n_coarse - 1, c = (g->hr + nc1 - 1) / nc1;
    g->q = 2 * (c < 1 ? 1 : c);
    int64_t r = p->n_nbr;
    g->n_cand = 1 + ((2 * r + 1) * (2 * r + 1) - 1) + (int64_t)p->n_coarse * p->n_coarse +
                8 * (int64_t)p->n_levels;
    g->kk = p->k * p->k;
    return 0;
}

static int64_t fdiv(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static double val(const geom2* g, int64_t nu) { return ldexp((double)nu * g->p.delta, -g->shift); }
static double grid(const geom2* g, int64_t a, int64_t h) { return (double)(a - h) * g->p.delta; }

/* Sum of t[0..n) in the fixed order of the one-dimensional oracle. */
static double fsum(const double* t, int64_t n) {
    if (n <= 0) return 0.0;
    int64_t m = (n + 31) / 32;
    double* c = (double*)malloc(sizeof(double) * (size_t)m);
    for (int64_t k = 0; k < m; ++k) {
        double a = 0.0;
        int64_t e = (k + 1) * 32 < n ? (k + 1) * 32 : n;
        for (int64_t j = k * 32; j < e; ++j) a = a + t[j];
        c[k] = a;
    }
    while (m > 1) {
        int64_t h = m / 2;
        for (int64_t k = 0; k < h; ++k) c[k] = c[2 * k] + c[2 * k + 1];
        if (m & 1) c[h] = c[m - 1];
        m = h + (m & 1);
    }
    double r = c[0];
    free(c);
    return r;
}

int orc2_sizes(const orc2_params* p, int64_t* n_x, int64_t* n_w, int64_t* n_y,
               int64_t* n_cand, int32_t* shift) {
    geom2 g;
    if (make2(p, &g)) return -1;
    if (n_x) *n_x = g.n_x;
    if (n_w) *n_w = g.n_w;
    if (n_y) *n_y = g.n_y;
    if (n_cand) *n_cand = g.n_cand;
    if (shift) *shift = g.shift;
    return 0;
}

/* phi2[c m + d] = phi_c phi_d with phi_c ~ exp(-w_c^2 / 2) normalised. */
static void noise_weights(const geom2* g, double* phi2) {
    double* p1 = (double*)malloc(sizeof(double) * (size_t)g->n_w);
    for (int64_t c = 0; c < g->n_w; ++c) {
        double w = grid(g, c, g->hw);
        p1[c] = exp(-(w * w) / 2.0);
    }
    double s = fsum(p1, g->n_w);
    for (int64_t c = 0; c < g->n_w; ++c) p1[c] = p1[c] / s;
    for (int64_t c = 0; c < g->n_w; ++c)
        for (int64_t d = 0; d < g->n_w; ++d) phi2[c * g->n_w + d] = p1[c] * p1[d];
    free(p1);
}

int orc2_weights(const orc2_params* p, double* px, double* phi) {
    geom2 g;
    if (make2(p, &g)) return -1;
    int64_t n = g.n_x * g.n_x;
    double s2 = p->sigma * p->sigma;
    double* pr = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t a = 0; a < g.n_x; ++a)
        for (int64_t b = 0; b < g.n_x; ++b) {
            double xa = grid(&g, a, g.hx), xb = grid(&g, b, g.hx);
            pr[a * g.n_x + b] = exp(-(xa * xa + xb * xb) / (2.0 * s2));
        }
    double s = fsum(pr, n);
    if (px)
        for (int64_t i = 0; i < n; ++i) px[i] = pr[i] / s;
    free(pr);
    if (phi) noise_weights(&g, phi);
    return 0;
}

int orc2_init(const orc2_params* p, int kind, const double* table, int64_t* nu_out) {
    geom2 g;
    if (make2(p, &g)) return -1;
    for (int64_t a = 0; a < g.n_x; ++a)
        for (int64_t b = 0; b < g.n_x; ++b) {
            int64_t i = a * g.n_x + b;
            if (kind == 0) {             /* identity: f(x) = x (Section III-D) */
                nu_out[2 * i] = (a - g.hx) * g.one;
                nu_out[2 * i + 1] = (b - g.hx) * g.one;
            } else if (kind == 2 && table) {
                for (int k = 0; k < 2; ++k) {
                    double v = table[2 * i + k] / p->delta * (double)g.one;
                    if (!(fabs(v) < 9.0e15)) return -1;
                    nu_out[2 * i + k] = (int64_t)llround(v);
                }
            } else {
                return -1;
            }
        }
    return 0;
}

/* Bilinear interpolation of table component k at y-cell (j1, j2) + (t1, t2)
 * (indices clamped, so the table is constant beyond its edges): along axis 2
 * on both rows, then along axis 1. */
static double bilerp(const geom2* g, const double* U, int k, int64_t j1, int64_t j2,
                     double t1, double t2) {
    int64_t n = g->n_y, top = n - 1;
    int64_t a0 = j1 < 0 ? 0 : (j1 > top ? top : j1);
    int64_t a1 = j1 + 1 < 0 ? 0 : (j1 + 1 > top ? top : j1 + 1);
    int64_t b0 = j2 < 0 ? 0 : (j2 > top ? top : j2);
    int64_t b1 = j2 + 1 < 0 ? 0 : (j2 + 1 > top ? top : j2 + 1);
    double u00 = U[2 * (a0 * n + b0) + k], u01 = U[2 * (a0 * n + b1) + k];
    double u10 = U[2 * (a1 * n + b0) + k], u11 = U[2 * (a1 * n + b1) + k];
    double r0 = u00 + t2 * (u01 - u00);
    double r1 = u10 + t2 * (u11 - u10);
    return r0 + t1 * (r1 - r0);
}

static double S2_of(const geom2* g, const double* phi2, const double* U, int64_t nu1,
                    int64_t nu2) {
    int64_t c1 = fdiv(nu1, g->one), c2 = fdiv(nu2, g->one);
    double t1 = ldexp((double)(nu1 - c1 * g->one), -g->shift);
    double t2 = ldexp((double)(nu2 - c2 * g->one), -g->shift);
    int64_t jb1 = c1 - g->hw + g->hy, jb2 = c2 - g->hw + g->hy;
    double u1 = val(g, nu1), u2 = val(g, nu2);
    int64_t m = g->n_w, nt = m * m;
    double* terms = (double*)malloc(sizeof(double) * (size_t)nt);
    for (int64_t c = 0; c < m; ++c)
        for (int64_t d = 0; d < m; ++d) {
            double e1 = u1 - bilerp(g, U, 0, jb1 + c, jb2 + d, t1, t2);
            double e2 = u2 - bilerp(g, U, 1, jb1 + c, jb2 + d, t1, t2);
            terms[c * m + d] = phi2[c * m + d] * (e1 * e1 + e2 * e2);
        }
    double s = fsum(terms, nt);
    free(terms);
    return s;
}

static double cost2(const geom2* g, const double* phi2, const double* U, int64_t i,
                    int64_t nu1, int64_t nu2) {
    double d1 = val(g, nu1) - grid(g, i / g->n_x, g->hx);
    double d2 = val(g, nu2) - grid(g, i % g->n_x, g->hx);
    return g->kk * (d1 * d1 + d2 * d2) + S2_of(g, phi2, U, nu1, nu2);
}

static double* phi2_new(const geom2* g) {
    double* phi2 = (double*)malloc(sizeof(double) * (size_t)(g->n_w * g->n_w));
    noise_weights(g, phi2);
    return phi2;
}

double orc2_S(const orc2_params* p, const double* U, int64_t nu1, int64_t nu2) {
    geom2 g;
    if (make2(p, &g)) return NAN;
    double* phi2 = phi2_new(&g);
    double s = S2_of(&g, phi2, U, nu1, nu2);
    free(phi2);
    return s;
}

double orc2_cost(const orc2_params* p, const double* U, int64_t i, int64_t nu1, int64_t nu2) {
    geom2 g;
    if (make2(p, &g)) return NAN;
    double* phi2 = phi2_new(&g);
    double c = cost2(&g, phi2, U, i, nu1, nu2);
    free(phi2);
    return c;
}

/* Walk the candidate list of point i in order; the first strict minimum
 * wins (list: ucp_oracle2d.h). */
static void search_one2(const geom2* g, const double* phi2, const int64_t* nu_pre,
                        const double* U, int64_t i, int64_t* out1, int64_t* out2,
                        int32_t* idx_out, int64_t* nu_list, double* g_list) {
    const orc2_params* p = &g->p;
    int64_t a = i / g->n_x, b = i % g->n_x, r = p->n_nbr;
    int64_t b1 = nu_pre[2 * i], b2 = nu_pre[2 * i + 1];
    double gb = cost2(g, phi2, U, i, b1, b2);
    int32_t pos = 0, bp = 0;
    if (nu_list) { nu_list[0] = b1; nu_list[1] = b2; g_list[0] = gb; }
#define ORC2_TRY(N1, N2)                                                       \
    do {                                                                       \
        int64_t n1_ = (N1), n2_ = (N2);                                        \
        double c_ = cost2(g, phi2, U, i, n1_, n2_);                            \
        ++pos;                                                                 \
        if (nu_list) { nu_list[2 * pos] = n1_; nu_list[2 * pos + 1] = n2_; g_list[pos] = c_; } \
        if (c_ < gb) { gb = c_; b1 = n1_; b2 = n2_; bp = pos; }                \
    } while (0)
    for (int64_t da = -r; da <= r; ++da)
        for (int64_t db = -r; db <= r; ++db) {
            if (da == 0 && db == 0) continue;
            int64_t aa = a + da, bb = b + db;
            int64_t j = (aa < 0 || aa >= g->n_x || bb < 0 || bb >= g->n_x) ? i
                                                                             : aa * g->n_x + bb;
            ORC2_TRY(nu_pre[2 * j], nu_pre[2 * j + 1]);
        }
    int64_t hq = g->q / 2, nc = p->n_coarse;
    for (int64_t j1 = 0; j1 < nc; ++j1)
        for (int64_t j2 = 0; j2 < nc; ++j2)
            ORC2_TRY((2 * j1 - (nc - 1)) * hq * g->one, (2 * j2 - (nc - 1)) * hq * g->one);
    for (int32_t lv = 1; lv <= p->n_levels; ++lv) {
        int64_t h = g->q << (p->n_levels - lv);
        int64_t c1 = b1, c2 = b2;
        for (int s = -1; s <= 1; ++s)
            for (int t = -1; t <= 1; ++t) {
                if (s == 0 && t == 0) continue;
                ORC2_TRY(c1 + s * h, c2 + t * h);
            }
    }
#undef ORC2_TRY
    *out1 = b1;
    *out2 = b2;
    *idx_out = bp;
}

void orc2_search(const orc2_params* p, const int64_t* nu_pre, const double* U,
                 int64_t* nu_out, int32_t* idx_out, int64_t i0, int64_t i1) {
    geom2 g;
    if (make2(p, &g)) return;
    double* phi2 = phi2_new(&g);
#pragma omp parallel for schedule(dynamic, 4) num_threads(orc_get_threads())
    for (int64_t i = i0; i < i1; ++i)
        search_one2(&g, phi2, nu_pre, U, i, &nu_out[2 * i], &nu_out[2 * i + 1], &idx_out[i],
                    NULL, NULL);
    free(phi2);
}

int orc2_candidates(const orc2_params* p, const int64_t* nu_pre, const double* U,
                    int64_t i, int64_t* nu_list, double* g_list) {
    geom2 g;
    if (make2(p, &g)) return -1;
    double* phi2 = phi2_new(&g);
    int64_t o1, o2;
    int32_t idx;
    search_one2(&g, phi2, nu_pre, U, i, &o1, &o2, &idx, nu_list, g_list);
    free(phi2);
    return idx;
}

/* U(y) = sum_i p_i phi(y - f_i) f_i / sum_i p_i phi(y - f_i) per component,
 * phi the continuous 2-D standard normal density; each weight exp(-E_i) with
 * E_i = |x_i|^2 / 2 sigma^2 + |y - f_i|^2 / 2 shifted by the smallest E_i
 * (the ratio is unchanged, the largest weight is exactly 1). */
void orc2_mmse(const orc2_params* p, const int64_t* nu, double* U, int64_t t0, int64_t t1) {
    geom2 g;
    if (make2(p, &g)) return;
    const double two_s2 = 2.0 * p->sigma * p->sigma;
    const int64_t n = g.n_x * g.n_x;
#pragma omp parallel for schedule(dynamic, 8) num_threads(orc_get_threads())
    for (int64_t t = t0; t < t1; ++t) {
        double y1 = grid(&g, t / g.n_y, g.hy), y2 = grid(&g, t % g.n_y, g.hy);
        double emin = INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double xa = grid(&g, i / g.n_x, g.hx), xb = grid(&g, i % g.n_x, g.hx);
            double d1 = y1 - val(&g, nu[2 * i]), d2 = y2 - val(&g, nu[2 * i + 1]);
            double e = (xa * xa + xb * xb) / two_s2 + (d1 * d1 + d2 * d2) / 2.0;
            if (e < emin) emin = e;
        }
        double n1 = 0.0, n2 = 0.0, den = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double xa = grid(&g, i / g.n_x, g.hx), xb = grid(&g, i % g.n_x, g.hx);
            double f1 = val(&g, nu[2 * i]), f2 = val(&g, nu[2 * i + 1]);
            double d1 = y1 - f1, d2 = y2 - f2;
            double e = (xa * xa + xb * xb) / two_s2 + (d1 * d1 + d2 * d2) / 2.0;
            double w = exp(-(e - emin));
            n1 = n1 + w * f1;
            n2 = n2 + w * f2;
            den = den + w;
        }
        U[2 * t] = n1 / den;
        U[2 * t + 1] = n2 / den;
    }
}

double orc2_J(const orc2_params* p, const int64_t* nu, const double* U) {
    geom2 g;
    if (make2(p, &g)) return NAN;
    const int64_t n = g.n_x * g.n_x;
    double* px = (double*)malloc(sizeof(double) * (size_t)n);
    double* terms = (double*)malloc(sizeof(double) * (size_t)n);
    orc2_weights(p, px, NULL);
    double* phi2 = phi2_new(&g);
#pragma omp parallel for schedule(dynamic, 8) num_threads(orc_get_threads())
    for (int64_t i = 0; i < n; ++i) terms[i] = cost2(&g, phi2, U, i, nu[2 * i], nu[2 * i + 1]);
    double J = 0.0;
    for (int64_t i = 0; i < n; ++i) J = J + px[i] * terms[i];
    free(px);
    free(terms);
    free(phi2);
    return 0.5 * J;
}
