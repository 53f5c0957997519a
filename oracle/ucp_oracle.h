/*
 * ucp_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Declarations of the plain, slow FP64 CPU oracle for the coordinate-descent
 * sweep of the generic UCP solver (Tseng, "A Generic Solver for Unconstrained
 * Control Problems with Integral Functional Objectives", ACC 2020) on
 * Witsenhausen's counterexample (Section V-A).  Only tests/, the smoke check
 * and the CPU-baseline leg of bench.py may load this library.  It shares no
 * code, header or table with the CUDA library.
 *
 * Notation (Section V-A): x1 = x0 + u0(x0), y1 = x1 + w, x2 = x1 - u1(y1),
 * J = E[k^2 u0^2 + x2^2], x0 ~ N(0, sigma^2), w ~ N(0, 1).  The first
 * controller is carried as f(x0) = x1 = x0 + u0(x0).
 *
 * Controller values live on the lattice  delta * 2^-shift * Z  with
 * shift = L * log2(n_refine / 2); they are passed as int64 lattice indices nu
 * (value = nu * delta * 2^-shift).  Every candidate the search generates lies
 * on this lattice, so positions on the y grid are exact.
 */
#ifndef UCP_ORACLE_H
#define UCP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double k;          /* control-cost weight, k > 0                           */
    double sigma;      /* prior std of x0, sigma > 0                           */
    double delta;      /* common spacing of the x0, w and y grids              */
    double x_half;     /* x0 grid is [-x_half, x_half]                         */
    double w_half;     /* w quadrature grid is [-w_half, w_half]               */
    double y_half;     /* u1 table grid is [-y_half, y_half]                   */
    double cand_half;  /* coarse candidates cover [-cand_half, cand_half]      */
    int32_t n_coarse;  /* number of coarse candidates (64)                     */
    int32_t n_refine;  /* candidates per refinement level (16)                 */
    int32_t n_levels;  /* refinement levels L                                  */
    int32_t n_nbr;     /* neighbours per side in the partial exhaustion (2)    */
    int32_t problem;   /* 0 Witsenhausen (Section V-A), 1 zero-delay source-
                          channel coding (Section V-B)                          */
} orc_params;

/* Problem 1 (Section V-B): x0 ~ N(0, sigma^2), x1 = u0(x0) + w,
 * w ~ U(-w_half, w_half), J = E[lambda u0^2 + (u1(x1) - x0)^2] with
 * lambda = k^2.  The first controller is carried as f = u0 itself; the
 * marginal cost of u0 at x_i is, up to p(x_i),
 *   g(u; x_i) = k^2 u^2 + sum_l phi_l (U^(u + w_l) - x_i)^2
 * with equal weights phi_l on the w grid, and u1(y) = E[x0 | x1 = y] is the
 * prior-weighted mean of the x_i whose |y - f_i| <= w_half (those nearest to
 * y when none is that close).  orc_S is defined for problem 0 only. */

/* Sizes; returns 0 on success, -1 on invalid parameters. */
int orc_sizes(const orc_params* p, int64_t* n_x, int64_t* n_w, int64_t* n_y,
              int64_t* n_cand, int32_t* shift);

/* Grids and normalised rectangle-rule weights. */
int orc_grids(const orc_params* p, double* x, double* px, double* w,
              double* phi, double* y);

/* Value of lattice index nu. */
double orc_value(const orc_params* p, int64_t nu);

/* Initial controller f: kind 0 identity, 1 odd staircase, 2 table. */
int orc_init(const orc_params* p, int kind, const double* table,
             int64_t* nu_out);

/* S(u) = sum_l phi_l (u - U^(u + w_l))^2 at u = value(nu). */
double orc_S(const orc_params* p, const double* U, int64_t nu);

/* g(u; x_i) = k^2 (u - x_i)^2 + S(u) (problem 1: the cost above). */
double orc_cost(const orc_params* p, const double* U, int64_t i, int64_t nu);

/* Candidate search for x_i, i in [i0, i1): Jacobi, reads nu_pre, writes
 * nu_out[i] and idx_out[i] (list position of the winner). */
void orc_search(const orc_params* p, const int64_t* nu_pre, const double* U,
                int64_t* nu_out, int32_t* idx_out, int64_t i0, int64_t i1);

/* Full candidate list for x_i with every cost, in list order (for tests). */
int orc_candidates(const orc_params* p, const int64_t* nu_pre, const double* U,
                   int64_t i, int64_t* nu_list, double* g_list);

/* u1 update U_j = E[x1 | y1 = y_j] (problem 1: E[x0 | x1 = y_j]) for j in
 * [j0, j1). */
void orc_mmse(const orc_params* p, const int64_t* nu, double* U, int64_t j0,
              int64_t j1);

/* J = sum_i px_i g(f_i; x_i). */
double orc_J(const orc_params* p, const int64_t* nu, const double* U);

/* init -> U = mmse(f) -> n_sweeps x {search, mmse, J}.  J_hist[0] is J of
 * the initial state, J_hist[s] after sweep s.  idx_hist may be NULL. */
int orc_solve(const orc_params* p, int init_kind, const double* table,
              int n_sweeps, int64_t* nu_out, double* U_out, double* J_hist,
              int32_t* idx_hist);

/* ---- Algorithm 1's outer loop (Sections III-B to III-D) ----------------
 *
 * Local update of u0 at x_i: with the linear interpolant of U the marginal
 * cost g(u; x_i) is a quadratic in u on each y-cell, and its derivatives
 * there are, with d_l = U[jr] - U[jl] the table step of the cell holding
 * u + w_l (0 beyond the table) and uh_l the interpolated value,
 *   problem 0: g'/2 = k^2 (u - x_i) + (1/delta) sum_l phi_l (u - uh_l)(delta - d_l)
 *              g''/2 = k^2 + (1/delta^2) sum_l phi_l (delta - d_l)^2
 *   problem 1: g'/2 = k^2 u + (1/delta) sum_l phi_l (uh_l - x_i) d_l
 *              g''/2 = k^2 + (1/delta^2) sum_l phi_l d_l^2
 * (the derivatives from the right at cell boundaries).  The sums are taken
 * in the fixed order of the w quadrature.  orc_derivs returns g'/2 and
 * g''/2.  The update is Newton's step u - g'/g'' where g'' > 0, else the
 * gradient step u - tau g' (never taken on these two problems, where
 * g'' >= 2 k^2), rounded to the controller lattice like a table start. */
int orc_derivs(const orc_params* p, const double* U, int64_t i, int64_t nu,
               double* half_d1, double* half_d2);
void orc_local_update(const orc_params* p, const int64_t* nu_pre, const double* U,
                      double tau, int64_t* nu_out, int64_t i0, int64_t i1);

/* Adaptive minimisation: the local-update share of the next round,
 * N_L = min(max(floor(I_L N / (I_L + I_P)), 1), N - 1) (kept as n_l when
 * I_L + I_P = 0). */
int orc_split(double I_L, double I_P, int N, int n_l);

typedef struct {
    int32_t rounds;            /* rounds run                                  */
    int32_t converged;         /* 1 if I_L + I_P <= precision at the end      */
    int32_t local_iters;       /* local-update iterations (Newton + u1 step)  */
    int32_t exhaustion_iters;  /* partial-exhaustion iterations (sweeps)      */
    int32_t N_L, N_P;          /* the split the next round would use          */
    double J, I_L, I_P;        /* final J and the last round's improvements   */
} orc_alg1_report;

/* Algorithm 1: init -> U = mmse(f) -> J_c; I_L = I_P = precision;
 * N_L = floor(N/2), N_P = N - N_L; while I_L + I_P > precision (and fewer
 * than max_rounds rounds): N_L local-update iterations (u0 by the local
 * update above, then u1 by its exact minimiser), J, I_L = |J before - J
 * after|; N_P partial-exhaustion iterations (the sweep of orc_search and
 * orc_mmse), J, I_P likewise; the next split by orc_split.  J_phase (may be
 * NULL, 1 + 2 max_rounds entries): the initial J, then J after every phase;
 * NL_rounds (may be NULL, max_rounds entries): N_L of every round run. */
int orc_algorithm1(const orc_params* p, int init_kind, const double* table, int N,
                   double precision, double tau, int max_rounds, int64_t* nu_out,
                   double* U_out, double* J_phase, int32_t* NL_rounds,
                   orc_alg1_report* rep);

/* Threads used by orc_search / orc_mmse / orc_solve (OpenMP; 1 = serial).
 * Results do not depend on the thread count. */
void orc_set_threads(int n);
int orc_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif
