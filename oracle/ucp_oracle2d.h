/*
 * ucp_oracle2d.h -- TEST INFRASTRUCTURE ONLY.
 *
 * The plain FP64 CPU oracle of the sweep on the 2-dimensional Witsenhausen
 * counterexample (Tseng, ACC 2020, Section V-D): the state x, the
 * controllers and the observations are vectors in R^2,
 *   x1 = x0 + u0(x0), y1 = x1 + w, x2 = x1 - u1(y1),
 *   J = (1/2) E[k^2 |u0|^2 + |x2|^2],  x0 ~ N(0, sigma^2 I), w ~ N(0, I).
 * The first controller is carried as f(x0) = x1 (two components) on a
 * square x0 grid; u1 as two tables on a square y grid, interpolated
 * bilinearly and held constant beyond the table.  Only tests/ and the
 * CPU-baseline leg of bench.py load this code; it shares nothing with the
 * CUDA library.
 *
 * Grids: one spacing delta for x0 (n x n points over [-x_half, x_half]^2),
 * w (m x m over [-w_half, w_half]^2) and y (ny x ny over [-y_half,
 * y_half]^2); point (a, b) of a grid is at ((a - h) delta, (b - h) delta)
 * and has flat index a n + b.  Weights: the prior p_ab ~ exp(-(x_a^2 +
 * x_b^2) / 2 sigma^2) normalised over the grid, the noise weights
 * phi_cd = phi_c phi_d, products of the normalised one-dimensional weights.
 *
 * Controller values lie on the lattice delta 2^-shift Z per component,
 * shift = n_levels (the refinement levels halve the step); they are passed
 * as int64 lattice indices, component 1 then component 2 (nu[2 i + k]).
 *
 * Candidate list of x0 point i (first strict minimum wins): the incumbent;
 * f at the points of the (2r + 1) x (2r + 1) window around i (row-major,
 * the centre skipped, points off the grid replaced by the incumbent); the
 * n_coarse x n_coarse coarse values (c_j1, c_j2), c_j = (2j - (n_coarse -
 * 1)) (q/2) delta with q = 2 ceil(cand_half / ((n_coarse - 1) delta)),
 * row-major; then n_levels levels of the 8 values best + (s h, t h),
 * (s, t) in {-1, 0, 1}^2 minus (0, 0) row-major, h = q delta 2^-level
 * around the best so far.
 */
#ifndef UCP_ORACLE2D_H
#define UCP_ORACLE2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double k, sigma, delta;
    double x_half, w_half, y_half, cand_half;
    int32_t n_coarse;   /* coarse values per axis                        */
    int32_t n_levels;   /* refinement levels (each halves the step)      */
    int32_t n_nbr;      /* r: the (2r + 1)^2 - 1 neighbouring samples    */
    int32_t reserved;
} orc2_params;

/* Sizes per axis, the candidate-list length and the lattice shift. */
int orc2_sizes(const orc2_params* p, int64_t* n_x, int64_t* n_w, int64_t* n_y,
               int64_t* n_cand, int32_t* shift);
/* Normalised weights: px (n_x^2), phi (n_w^2). */
int orc2_weights(const orc2_params* p, double* px, double* phi);
/* Identity start f(x) = x (kind 0) or a table of n_x^2 pairs (kind 2). */
int orc2_init(const orc2_params* p, int kind, const double* table, int64_t* nu_out);
/* S(u) = sum_cd phi_cd |u - U^(u + w_cd)|^2, u = value of (nu1, nu2). */
double orc2_S(const orc2_params* p, const double* U, int64_t nu1, int64_t nu2);
/* g(u; x_i) = k^2 |u - x_i|^2 + S(u). */
double orc2_cost(const orc2_params* p, const double* U, int64_t i, int64_t nu1, int64_t nu2);
/* Search of x0 points i0 .. i1 - 1 (Jacobi from nu_pre). */
void orc2_search(const orc2_params* p, const int64_t* nu_pre, const double* U,
                 int64_t* nu_out, int32_t* idx_out, int64_t i0, int64_t i1);
/* Every candidate of point i in list order with its cost; returns the
 * winner's position. */
int orc2_candidates(const orc2_params* p, const int64_t* nu_pre, const double* U,
                    int64_t i, int64_t* nu_list, double* g_list);
/* u1 update U(y) = E[x1 | y1 = y] at the targets t0 .. t1 - 1 (flat y
 * indices); U holds the two components, U[2 t + k]. */
void orc2_mmse(const orc2_params* p, const int64_t* nu, double* U, int64_t t0, int64_t t1);
/* J = (1/2) sum_i p_i g(f_i; x_i). */
double orc2_J(const orc2_params* p, const int64_t* nu, const double* U);

#ifdef __cplusplus
}
#endif
#endif
