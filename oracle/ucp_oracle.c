/*
 * ucp_oracle.c -- TEST INFRASTRUCTURE ONLY: a plain, slow, FP64 CPU oracle
 * for the coordinate-descent sweep of the generic UCP solver (Tseng, ACC 2020)
 * on Witsenhausen's counterexample.  It is loaded only by tests/, by the smoke
 * check and by the CPU-baseline leg of bench.py; the product library never
 * links or calls it, and the two share no code.
 *
 * What it computes, and where the paper defines it:
 *   - Problem (Section V-A): x1 = x0 + u0(x0), y1 = x1 + w,
 *     x2 = x1 - u1(y1), J = E[k^2 u0^2 + x2^2], x0 ~ N(0, sigma^2),
 *     w ~ N(0, 1).  The first controller is carried as f(x0) = x1.
 *   - Decomposition eq. (1) and Corollary 1 (Section III-A): J is minimised
 *     pointwise; for u0 the marginal cost at x0 = x_i is, up to the positive
 *     factor p(x_i),  g(u; x_i) = k^2 (u - x_i)^2 + S(u),
 *     S(u) = sum_l phi_l (u - U^(u + w_l))^2.
 *   - Partial exhaustion eq. (2) (Section III-B/D) with r = 2 points per
 *     direction: candidates include f at the two neighbours on each side.
 *   - Coarse-to-fine candidate search (64 coarse values, then L levels of 16
 *     around the best so far): not in the paper; the reading is documented
 *     with the build's design notes.
 *   - Jacobi over the grid (Section IV-A): every x_i reads the pre-sweep f.
 *   - u1 update: C_1(v, y) is quadratic in v, so the paper's Newton local
 *     update (Section III-D) lands on its minimiser in one step,
 *     U(y) = E[x1 | y1 = y], the closed form mentioned in Section IV-C.
 *   - Step-function controllers on linearly spaced samples, identity init
 *     (Section III-D, "Initialization"); u1 is linearly interpolated between
 *     samples and held constant beyond them.
 *
 * Arithmetic: FP64; compile with -ffp-contract=off so that no multiply-add
 * is fused.  The w quadrature S(u) and the normalising sums of the prior and
 * quadrature weights are fixed_sum(): serial within chunks of 32 consecutive
 * terms, then the chunk sums pairwise by levels (the paper does not fix a
 * summation order; this one is the same on any machine and parallelises).
 * The u1 sums and J run in index order.  The parallel loops over i and j
 * give results independent of the thread count.
 *
 * Second problem (Section V-B, zero-delay source-channel coding): the same
 * sweep with x1 = u0(x0) + w, w ~ U(-W, W), J = E[k^2 u0^2 + (u1(x1) - x0)^2];
 * f = u0, equal quadrature weights, and u1(y) = E[x0 | x1 = y], a
 * prior-weighted mean over the sources within W of y (see ucp_oracle.h).
 *
 * Algorithm 1 (Sections III-B to III-D): the local update of u0 (Newton's
 * step on the marginal cost where its second derivative is positive, else a
 * gradient step), the adaptive split of each round's N iterations between
 * local update and partial exhaustion, and the termination at precision p.
 *
 * Parity status: S, g, the search, the u1 update and J are pinned by the
 * tests in tests/test_oracle_pins.py (closed forms, library interpolation,
 * brute force, invariants).  The converged J printed in Section V-A is a
 * plausibility band only.
 */
#include "ucp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return g_threads; }

/* ---- derived integer geometry ------------------------------------------ */

typedef struct {
    orc_params p;
    int64_t hx, hw, hy, hr;  /* half widths in units of delta            */
    int64_t n_x, n_w, n_y;
    int32_t shift;           /* lattice: value = nu * delta * 2^-shift   */
    int64_t one;             /* 2^shift                                  */
    int64_t q;               /* coarse spacing in units of delta         */
    int64_t n_cand;          /* length of the candidate list             */
    double kk;               /* k^2                                      */
} geom;

static int half_steps(double half, double delta, int64_t* out) {
    double r = half / delta;
    double n = floor(r + 0.5);
    if (!(n >= 0.0) || fabs(r - n) > 1e-9 * (n > 1.0 ? n : 1.0)) return -1;
    *out = (int64_t)n;
    return 0;
}

static int make_geom(const orc_params* p, geom* g) {
    memset(g, 0, sizeof(*g));
    g->p = *p;
    if (!(p->k > 0.0) || !(p->sigma > 0.0) || !(p->delta > 0.0)) return -1;
    if (half_steps(p->x_half, p->delta, &g->hx)) return -1;
    if (half_steps(p->w_half, p->delta, &g->hw)) return -1;
    if (half_steps(p->y_half, p->delta, &g->hy)) return -1;
    if (half_steps(p->cand_half, p->delta, &g->hr)) return -1;
    if (p->n_coarse < 2 || p->n_refine < 2 || (p->n_refine & 1)) return -1;
    if (p->n_levels < 0 || p->n_nbr < 0) return -1;
    if (p->problem != 0 && p->problem != 1) return -1;
    int32_t half_ref = p->n_refine / 2, bits = 0;
    while ((1 << bits) < half_ref) ++bits;
    if ((1 << bits) != half_ref) return -1;     /* ratio must be 2^bits */
    g->shift = bits * p->n_levels;
    if (g->shift > 40) return -1;
    g->one = (int64_t)1 << g->shift;
    g->n_x = 2 * g->hx + 1;
    g->n_w = 2 * g->hw + 1;
    g->n_y = 2 * g->hy + 1;
    /* q = 2 * ceil(hr / (n_coarse - 1)), at least 2 */
    int64_t nc1 = p->n_coarse - 1;
    int64_t c = (g->hr + nc1 - 1) / nc1;
    if (c < 1) c = 1;
    g->q = 2 * c;
    g->n_cand = 1 + 2 * (int64_t)p->n_nbr + p->n_coarse +
                (int64_t)p->n_levels * p->n_refine;
    g->kk = p->k * p->k;
    return 0;
}

static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

static double value_of(const geom* g, int64_t nu) {
    return ldexp((double)nu * g->p.delta, -g->shift);
}

static double x_of(const geom* g, int64_t i) {
    return (double)(i - g->hx) * g->p.delta;
}

static double w_of(const geom* g, int64_t l) {
    return (double)(l - g->hw) * g->p.delta;
}

static double y_of(const geom* g, int64_t j) {
    return (double)(j - g->hy) * g->p.delta;
}

/* ---- public sizes / grids ---------------------------------------------- */

int orc_sizes(const orc_params* p, int64_t* n_x, int64_t* n_w, int64_t* n_y,
              int64_t* n_cand, int32_t* shift) {
    geom g;
    if (make_geom(p, &g)) return -1;
    if (n_x) *n_x = g.n_x;
    if (n_w) *n_w = g.n_w;
    if (n_y) *n_y = g.n_y;
    if (n_cand) *n_cand = g.n_cand;
    if (shift) *shift = g.shift;
    return 0;
}

/* phi_l proportional to exp(-w_l^2 / 2), summing to 1 (rectangle rule). */
/* Sum of t[0..n) in a fixed order: chunk k = t[32k] + ... + t[32k + 31]
 * added left to right, then level by level the neighbours (2m, 2m + 1) of
 * the previous level are added, an unpaired last entry moving up as it is. */
#define ORC_CHUNK 32
static double fixed_sum(const double* t, int64_t n) {
    if (n <= 0) return 0.0;
    int64_t m = (n + ORC_CHUNK - 1) / ORC_CHUNK;
    double stack_buf[256];
    double* c = m <= 256 ? stack_buf : (double*)malloc(sizeof(double) * (size_t)m);
    for (int64_t k = 0; k < m; ++k) {
        double a = 0.0;
        int64_t e = (k + 1) * ORC_CHUNK < n ? (k + 1) * ORC_CHUNK : n;
        for (int64_t j = k * ORC_CHUNK; j < e; ++j) a = a + t[j];
        c[k] = a;
    }
    while (m > 1) {
        int64_t h = m / 2;
        for (int64_t k = 0; k < h; ++k) c[k] = c[2 * k] + c[2 * k + 1];
        if (m & 1) c[h] = c[m - 1];
        m = h + (m & 1);
    }
    double r = c[0];
    if (c != stack_buf) free(c);
    return r;
}

static void phi_weights(const geom* g, double* phi) {
    for (int64_t l = 0; l < g->n_w; ++l) {
        double w = w_of(g, l);
        phi[l] = exp(-(w * w) / 2.0);
        if (g->p.problem == 1) phi[l] = 1.0;   /* w ~ U(-w_half, w_half) */
    }
    double sum = fixed_sum(phi, g->n_w);
    for (int64_t l = 0; l < g->n_w; ++l) phi[l] = phi[l] / sum;
}

int orc_grids(const orc_params* p, double* x, double* px, double* w,
              double* phi, double* y) {
    geom g;
    if (make_geom(p, &g)) return -1;
    double s2 = p->sigma * p->sigma;
    double* pr = (double*)malloc(sizeof(double) * (size_t)g.n_x);
    if (!pr) return -1;
    for (int64_t i = 0; i < g.n_x; ++i) {
        double xi = x_of(&g, i);
        if (x) x[i] = xi;
        pr[i] = exp(-(xi * xi) / (2.0 * s2));
    }
    double sum = fixed_sum(pr, g.n_x);
    if (px)
        for (int64_t i = 0; i < g.n_x; ++i) px[i] = pr[i] / sum;
    free(pr);
    for (int64_t l = 0; l < g.n_w; ++l)
        if (w) w[l] = w_of(&g, l);
    if (phi) phi_weights(&g, phi);
    for (int64_t j = 0; j < g.n_y; ++j)
        if (y) y[j] = y_of(&g, j);
    return 0;
}

double orc_value(const orc_params* p, int64_t nu) {
    geom g;
    if (make_geom(p, &g)) return NAN;
    return value_of(&g, nu);
}

/* ---- initial controller ------------------------------------------------ */

int orc_init(const orc_params* p, int kind, const double* table,
             int64_t* nu_out) {
    geom g;
    if (make_geom(p, &g)) return -1;
    if (kind == 0) {
        /* identity map u(y) = y (Section III-D): f(x_i) = x_i */
        for (int64_t i = 0; i < g.n_x; ++i) nu_out[i] = (i - g.hx) * g.one;
        return 0;
    }
    if (kind == 1) {
        /* odd 3-step staircase: f = 3.5 sgn(x) (2 min(floor(|x|/7), 2) + 1),
         * f(0) = 0; step width 7 and half level 3.5 in units of delta. */
        int64_t n7;
        if (half_steps(7.0, p->delta, &n7) || n7 < 1) return -1;
        for (int64_t i = 0; i < g.n_x; ++i) {
            int64_t a = i - g.hx, m;
            if (a == 0) { nu_out[i] = 0; continue; }
            m = (a < 0 ? -a : a) / n7;
            if (m > 2) m = 2;
            double v = 3.5 * (double)(2 * m + 1) / p->delta * (double)g.one;
            int64_t nu = (int64_t)llround(v);
            nu_out[i] = a < 0 ? -nu : nu;
        }
        return 0;
    }
    if (kind == 2) {
        if (!table) return -1;
        for (int64_t i = 0; i < g.n_x; ++i) {
            double v = table[i] / p->delta * (double)g.one;
            if (!(fabs(v) < 9.0e15)) return -1;
            nu_out[i] = (int64_t)llround(v);
        }
        return 0;
    }
    return -1;
}

/* ---- marginal cost ----------------------------------------------------- */

/* S(u) at u = value(nu): the w quadrature of (u - U^(u + w))^2 where U^ is
 * the linear interpolant of the table U on the y grid, held constant beyond
 * its ends.  The position of u + w_l on the y grid is jb + l + t with an
 * integer jb and a fraction t that are exact because u is on the lattice. */
static double S_of(const geom* g, const double* phi, const double* U,
                   int64_t nu) {
    int64_t cell = floor_div(nu, g->one);
    double t = ldexp((double)(nu - cell * g->one), -g->shift);
    int64_t jb = cell - g->hw + g->hy;
    double u = value_of(g, nu);
    double buf[4096];
    double* terms = g->n_w <= 4096 ? buf : (double*)malloc(sizeof(double) * (size_t)g->n_w);
    for (int64_t l = 0; l < g->n_w; ++l) {
        int64_t j = jb + l;
        int64_t jl = j < 0 ? 0 : (j > g->n_y - 1 ? g->n_y - 1 : j);
        int64_t jr = j + 1 < 0 ? 0 : (j + 1 > g->n_y - 1 ? g->n_y - 1 : j + 1);
        double uh = U[jl] + t * (U[jr] - U[jl]);
        double e = u - uh;
        terms[l] = phi[l] * (e * e);
    }
    double acc = fixed_sum(terms, g->n_w);
    if (terms != buf) free(terms);
    return acc;
}

/* Problem 1: k^2 u^2 + sum_l phi_l (U^(u + w_l) - x_i)^2 at u = value(nu),
 * the same positions and interpolation as S_of, the same summation order. */
static double cost_sc(const geom* g, const double* phi, const double* U,
                      int64_t i, int64_t nu) {
    int64_t cell = floor_div(nu, g->one);
    double t = ldexp((double)(nu - cell * g->one), -g->shift);
    int64_t jb = cell - g->hw + g->hy;
    double u = value_of(g, nu), x = x_of(g, i);
    double* terms = (double*)malloc(sizeof(double) * (size_t)g->n_w);
    for (int64_t l = 0; l < g->n_w; ++l) {
        int64_t j = jb + l;
        int64_t jl = j < 0 ? 0 : (j > g->n_y - 1 ? g->n_y - 1 : j);
        int64_t jr = j + 1 < 0 ? 0 : (j + 1 > g->n_y - 1 ? g->n_y - 1 : j + 1);
        double uh = U[jl] + t * (U[jr] - U[jl]);
        double d = uh - x;
        terms[l] = phi[l] * (d * d);
    }
    double acc = fixed_sum(terms, g->n_w);
    free(terms);
    return g->kk * (u * u) + acc;
}

static double cost_of(const geom* g, const double* phi, const double* U,
                      int64_t i, int64_t nu) {
    if (g->p.problem == 1) return cost_sc(g, phi, U, i, nu);
    double a = value_of(g, nu) - x_of(g, i);
    return g->kk * (a * a) + S_of(g, phi, U, nu);
}

double orc_S(const orc_params* p, const double* U, int64_t nu) {
    geom g;
    if (make_geom(p, &g) || p->problem != 0) return NAN;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
    double s = S_of(&g, phi, U, nu);
    free(phi);
    return s;
}

double orc_cost(const orc_params* p, const double* U, int64_t i, int64_t nu) {
    geom g;
    if (make_geom(p, &g)) return NAN;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
    double c = cost_of(&g, phi, U, i, nu);
    free(phi);
    return c;
}

/* ---- candidate search -------------------------------------------------- */

/* Walk the candidate list of x_i in order; the first strict minimum wins.
 * List: incumbent f_i; neighbours f_{i-r..i-1}, f_{i+1..i+r} (missing ones
 * replaced by the incumbent); n_coarse values symmetric about 0 with spacing
 * q*delta; then per level n_refine values best + m*h around the best so far,
 * m = -n_refine/2..-1, 1..n_refine/2, h shrinking by n_refine/2 per level. */
static void search_one(const geom* g, const double* phi, const int64_t* nu_pre,
                       const double* U, int64_t i, int64_t* nu_best_out,
                       int32_t* idx_out, int64_t* nu_list, double* g_list) {
    const orc_params* p = &g->p;
    int32_t pos = 0, best_pos = 0;
    int64_t nu_best = nu_pre[i];
    double g_best = cost_of(g, phi, U, i, nu_best);
    if (nu_list) { nu_list[0] = nu_best; g_list[0] = g_best; }
    pos = 1;

    for (int64_t d = -p->n_nbr; d <= p->n_nbr; ++d) {
        if (d == 0) continue;
        int64_t ii = i + d;
        int64_t nu = (ii < 0 || ii >= g->n_x) ? nu_pre[i] : nu_pre[ii];
        double c = cost_of(g, phi, U, i, nu);
        if (nu_list) { nu_list[pos] = nu; g_list[pos] = c; }
        if (c < g_best) { g_best = c; nu_best = nu; best_pos = pos; }
        ++pos;
    }

    int64_t half_q = g->q / 2;
    for (int64_t j = 0; j < p->n_coarse; ++j) {
        int64_t nu = (2 * j - (p->n_coarse - 1)) * half_q * g->one;
        double c = cost_of(g, phi, U, i, nu);
        if (nu_list) { nu_list[pos] = nu; g_list[pos] = c; }
        if (c < g_best) { g_best = c; nu_best = nu; best_pos = pos; }
        ++pos;
    }

    int32_t bits = 0;
    while ((1 << bits) < p->n_refine / 2) ++bits;
    for (int32_t lv = 1; lv <= p->n_levels; ++lv) {
        int64_t h = g->q * ((int64_t)1 << (bits * (p->n_levels - lv)));
        int64_t centre = nu_best;
        for (int32_t m = -p->n_refine / 2; m <= p->n_refine / 2; ++m) {
            if (m == 0) continue;
            int64_t nu = centre + (int64_t)m * h;
            double c = cost_of(g, phi, U, i, nu);
            if (nu_list) { nu_list[pos] = nu; g_list[pos] = c; }
            if (c < g_best) { g_best = c; nu_best = nu; best_pos = pos; }
            ++pos;
        }
    }
    *nu_best_out = nu_best;
    *idx_out = best_pos;
}

void orc_search(const orc_params* p, const int64_t* nu_pre, const double* U,
                int64_t* nu_out, int32_t* idx_out, int64_t i0, int64_t i1) {
    geom g;
    if (make_geom(p, &g)) return;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
    for (int64_t i = i0; i < i1; ++i)
        search_one(&g, phi, nu_pre, U, i, &nu_out[i], &idx_out[i], NULL, NULL);
    free(phi);
}

int orc_candidates(const orc_params* p, const int64_t* nu_pre, const double* U,
                   int64_t i, int64_t* nu_list, double* g_list) {
    geom g;
    if (make_geom(p, &g)) return -1;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
    int64_t nb;
    int32_t idx;
    search_one(&g, phi, nu_pre, U, i, &nb, &idx, nu_list, g_list);
    free(phi);
    return idx;
}

/* ---- u1 update: U_j = E[x1 | y1 = y_j] --------------------------------- */

/* Ratio of Gaussian sums over all x_i, weights p(x_i) phi(y_j - f_i) with the
 * continuous phi.  Writing each weight as exp(-E_ij), the minimum of E_ij
 * over i is subtracted first; this cancels in the ratio and keeps the
 * largest weight at exactly 1. */
/* Problem 1: the likelihood of x1 = y given x0 = x_i is constant for
 * |y - f_i| <= w_half and zero beyond, so U_j is the mean of those x_i
 * weighted by the prior alone (exponents shifted by their minimum, as in the
 * Gaussian case).  Where no source is that close, the sources nearest to y
 * take their place (the limit of a slightly wider window). */
static void mmse_uniform(const geom* g, const int64_t* nu, double* U, int64_t j0,
                         int64_t j1) {
    const double W = g->p.w_half;
    const double two_s2 = 2.0 * g->p.sigma * g->p.sigma;
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
    for (int64_t j = j0; j < j1; ++j) {
        double yj = y_of(g, j);
        double dmin = INFINITY;
        for (int64_t i = 0; i < g->n_x; ++i) {
            double d = fabs(yj - value_of(g, nu[i]));
            if (d < dmin) dmin = d;
        }
        double reach = dmin <= W ? W : dmin;
        double emin = INFINITY;
        for (int64_t i = 0; i < g->n_x; ++i) {
            double xi = x_of(g, i);
            if (fabs(yj - value_of(g, nu[i])) > reach) continue;
            double e = (xi * xi) / two_s2;
            if (e < emin) emin = e;
        }
        double num = 0.0, den = 0.0;
        for (int64_t i = 0; i < g->n_x; ++i) {
            double xi = x_of(g, i);
            if (fabs(yj - value_of(g, nu[i])) > reach) continue;
            double wgt = exp(-((xi * xi) / two_s2 - emin));
            num = num + wgt * xi;
            den = den + wgt;
        }
        U[j] = num / den;
    }
}

void orc_mmse(const orc_params* p, const int64_t* nu, double* U, int64_t j0,
              int64_t j1) {
    geom g;
    if (make_geom(p, &g)) return;
    if (p->problem == 1) {
        mmse_uniform(&g, nu, U, j0, j1);
        return;
    }
    double two_s2 = 2.0 * p->sigma * p->sigma;
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
    for (int64_t j = j0; j < j1; ++j) {
        double yj = y_of(&g, j);
        double emin = INFINITY;
        for (int64_t i = 0; i < g.n_x; ++i) {
            double xi = x_of(&g, i), fi = value_of(&g, nu[i]);
            double e = (xi * xi) / two_s2 + ((yj - fi) * (yj - fi)) / 2.0;
            if (e < emin) emin = e;
        }
        double num = 0.0, den = 0.0;
        for (int64_t i = 0; i < g.n_x; ++i) {
            double xi = x_of(&g, i), fi = value_of(&g, nu[i]);
            double e = (xi * xi) / two_s2 + ((yj - fi) * (yj - fi)) / 2.0;
            double wgt = exp(-(e - emin));
            num = num + wgt * fi;
            den = den + wgt;
        }
        U[j] = num / den;
    }
}

/* ---- objective --------------------------------------------------------- */

double orc_J(const orc_params* p, const int64_t* nu, const double* U) {
    geom g;
    if (make_geom(p, &g)) return NAN;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    double* px = (double*)malloc(sizeof(double) * (size_t)g.n_x);
    double* terms = (double*)malloc(sizeof(double) * (size_t)g.n_x);
    phi_weights(&g, phi);
    orc_grids(p, NULL, px, NULL, NULL, NULL);
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
    for (int64_t i = 0; i < g.n_x; ++i)
        terms[i] = cost_of(&g, phi, U, i, nu[i]);
    double J = 0.0;
    for (int64_t i = 0; i < g.n_x; ++i) J = J + px[i] * terms[i];
    free(terms);
    free(px);
    free(phi);
    return J;
}

/* ---- whole solve ------------------------------------------------------- */

int orc_solve(const orc_params* p, int init_kind, const double* table,
              int n_sweeps, int64_t* nu_out, double* U_out, double* J_hist,
              int32_t* idx_hist) {
    geom g;
    if (make_geom(p, &g) || n_sweeps < 0) return -1;
    int64_t* a = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.n_x);
    int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.n_x);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)g.n_x);
    if (orc_init(p, init_kind, table, a)) {
        free(a); free(b); free(idx);
        return -1;
    }
    orc_mmse(p, a, U_out, 0, g.n_y);
    if (J_hist) J_hist[0] = orc_J(p, a, U_out);
    for (int s = 0; s < n_sweeps; ++s) {
        orc_search(p, a, U_out, b, idx, 0, g.n_x);
        int64_t* t = a; a = b; b = t;
        orc_mmse(p, a, U_out, 0, g.n_y);
        if (J_hist) J_hist[s + 1] = orc_J(p, a, U_out);
        if (idx_hist)
            memcpy(idx_hist + (size_t)s * (size_t)g.n_x, idx,
                   sizeof(int32_t) * (size_t)g.n_x);
    }
    memcpy(nu_out, a, sizeof(int64_t) * (size_t)g.n_x);
    free(a); free(b); free(idx);
    return 0;
}

/* ---- Algorithm 1: local update, adaptive split, outer loop ------------- */

/* g'/2 and g''/2 at u = value(nu) for x_i (see ucp_oracle.h): the same
 * positions, interpolation and summation order as S_of / cost_sc, each sum
 * factored by the cell width delta so that its terms need no division. */
static void derivs_of(const geom* g, const double* phi, const double* U, int64_t i,
                      int64_t nu, double* h1, double* h2) {
    int64_t cell = floor_div(nu, g->one);
    double t = ldexp((double)(nu - cell * g->one), -g->shift);
    int64_t jb = cell - g->hw + g->hy;
    double u = value_of(g, nu), x = x_of(g, i), dl = g->p.delta;
    double* a = (double*)malloc(sizeof(double) * (size_t)g->n_w);
    double* b = (double*)malloc(sizeof(double) * (size_t)g->n_w);
    for (int64_t l = 0; l < g->n_w; ++l) {
        int64_t j = jb + l;
        int64_t jl = j < 0 ? 0 : (j > g->n_y - 1 ? g->n_y - 1 : j);
        int64_t jr = j + 1 < 0 ? 0 : (j + 1 > g->n_y - 1 ? g->n_y - 1 : j + 1);
        double d = U[jr] - U[jl];
        double uh = U[jl] + t * d;
        if (g->p.problem == 1) {
            a[l] = phi[l] * ((uh - x) * d);
            b[l] = phi[l] * (d * d);
        } else {
            double e = u - uh, c = dl - d;
            a[l] = phi[l] * (e * c);
            b[l] = phi[l] * (c * c);
        }
    }
    double s1 = fixed_sum(a, g->n_w), s2 = fixed_sum(b, g->n_w);
    free(a);
    free(b);
    double lin = g->p.problem == 1 ? g->kk * u : g->kk * (u - x);
    *h1 = lin + s1 / dl;
    *h2 = g->kk + s2 / (dl * dl);
}

int orc_derivs(const orc_params* p, const double* U, int64_t i, int64_t nu,
               double* half_d1, double* half_d2) {
    geom g;
    if (make_geom(p, &g)) return -1;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
    derivs_of(&g, phi, U, i, nu, half_d1, half_d2);
    free(phi);
    return 0;
}

/* Local update of u0 (Section III-D, "Local Update"), every x_i from the
 * pre-update controller (Jacobi, as the partial exhaustion): Newton's step
 * where g'' > 0, else the gradient step with step size tau; the new value
 * is rounded to the controller lattice (value / delta * 2^shift, nearest,
 * halves away from zero), so that every later cost is evaluated at exact
 * positions.  A step to a non-finite or unrepresentable value keeps f_i. */
void orc_local_update(const orc_params* p, const int64_t* nu_pre, const double* U,
                      double tau, int64_t* nu_out, int64_t i0, int64_t i1) {
    geom g;
    if (make_geom(p, &g)) return;
    double* phi = (double*)malloc(sizeof(double) * (size_t)g.n_w);
    phi_weights(&g, phi);
#pragma omp parallel for schedule(dynamic, 8) num_threads(g_threads)
    for (int64_t i = i0; i < i1; ++i) {
        double h1, h2;
        derivs_of(&g, phi, U, i, nu_pre[i], &h1, &h2);
        double u = value_of(&g, nu_pre[i]);
        double un = h2 > 0.0 ? u - h1 / h2 : u - tau * (2.0 * h1);
        double v = un / p->delta * (double)g.one;
        nu_out[i] = fabs(v) < 9.0e15 ? (int64_t)llround(v) : nu_pre[i];
    }
    free(phi);
}

int orc_split(double I_L, double I_P, int N, int n_l) {
    if (!(I_L + I_P > 0.0)) return n_l;
    double r = floor(I_L * (double)N / (I_L + I_P));
    int nl = r < 1.0 ? 1 : (r > (double)(N - 1) ? N - 1 : (int)r);
    return nl;
}

int orc_algorithm1(const orc_params* p, int init_kind, const double* table, int N,
                   double precision, double tau, int max_rounds, int64_t* nu_out,
                   double* U_out, double* J_phase, int32_t* NL_rounds,
                   orc_alg1_report* rep) {
    geom g;
    if (make_geom(p, &g) || N < 2 || max_rounds < 0 || !(precision >= 0.0)) return -1;
    int64_t* a = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.n_x);
    int64_t* b = (int64_t*)malloc(sizeof(int64_t) * (size_t)g.n_x);
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)g.n_x);
    if (orc_init(p, init_kind, table, a)) {
        free(a); free(b); free(idx);
        return -1;
    }
    orc_mmse(p, a, U_out, 0, g.n_y);
    double Jc = orc_J(p, a, U_out);
    if (J_phase) J_phase[0] = Jc;
    double IL = precision, IP = precision;
    int NL = N / 2, NP = N - NL, rounds = 0, nloc = 0, nexh = 0;
    while (IL + IP > precision && rounds < max_rounds) {
        if (NL_rounds) NL_rounds[rounds] = NL;
        double J0 = Jc;
        for (int k = 0; k < NL; ++k) {            /* m = 0, then m = 1 */
            orc_local_update(p, a, U_out, tau, b, 0, g.n_x);
            int64_t* t = a; a = b; b = t;
            orc_mmse(p, a, U_out, 0, g.n_y);
            ++nloc;
        }
        Jc = orc_J(p, a, U_out);
        IL = fabs(J0 - Jc);
        if (J_phase) J_phase[1 + 2 * rounds] = Jc;
        double J1 = Jc;
        for (int k = 0; k < NP; ++k) {
            orc_search(p, a, U_out, b, idx, 0, g.n_x);
            int64_t* t = a; a = b; b = t;
            orc_mmse(p, a, U_out, 0, g.n_y);
            ++nexh;
        }
        Jc = orc_J(p, a, U_out);
        IP = fabs(J1 - Jc);
        if (J_phase) J_phase[2 + 2 * rounds] = Jc;
        NL = orc_split(IL, IP, N, NL);
        NP = N - NL;
        ++rounds;
    }
    memcpy(nu_out, a, sizeof(int64_t) * (size_t)g.n_x);
    if (rep) {
        rep->rounds = rounds;
        rep->converged = IL + IP <= precision;
        rep->local_iters = nloc;
        rep->exhaustion_iters = nexh;
        rep->N_L = NL;
        rep->N_P = NP;
        rep->J = Jc;
        rep->I_L = IL;
        rep->I_P = IP;
    }
    free(a); free(b); free(idx);
    return 0;
}
