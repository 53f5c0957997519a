// ucp_2d.h -- the 2-dimensional Witsenhausen counterexample (Section V-D):
// geometry of one instance and the device state behind ucp2_* (not part of
// the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ucp.h"

namespace ucp {

// Integer geometry: half widths in units of delta, sizes per axis, the
// controller lattice (value nu delta 2^-shift, shift = n_levels), the coarse
// spacing q (units of delta, even) and the candidate-list length.
// Screened search: the correlation tables cover first-tap cells
// [tab_lo, tab_lo + tab_n) per axis (tab_lo = -n_w - 1, tab_n = n_y + n_w + 2),
// their row pass ext_n = tab_n + n_w - 1 rows; eps_k scales the error bound
// of a table cost.
struct G2 {
    double k, kk, sigma, delta;
    int64_t hx, hw, hy, hr, n_x, n_w, n_y;
    int32_t shift;
    int64_t one, q, n_cand;
    int32_t n_coarse, n_levels, n_nbr, direct;
    int64_t tab_lo, tab_n, ext_n;
    double eps_k;
    int32_t u1_splits;   // source splits of the factorised u1 sums
    // Double-float table costs (n_levels <= 24): their error bound eps_df
    // (M + |g|), the lattice step delta 2^-shift as a float pair, 2^-shift.
    int32_t use_df;
    double eps_df;
    float eps_df_f;
    float us_hi, us_lo, inv_one_f, kk_hi, kk_lo;
};

// Fills g from p; nullptr or the reason p is invalid.
const char* make_g2(const ucp2_params& p, G2* g);

struct Dev2 {
    double* px;      // [n_x^2] prior weights
    double* phi1;    // [n_w] one-dimensional noise weights
    double* phi2;    // [n_w^2] phi_c phi_d
    double* U;       // [2 n_y^2] u1 table
    int64_t* nu[2];  // [2 n_x^2] controller, double buffered
    int32_t* idx;    // [n_x^2] winner positions of the last sweep
    double* terms;   // [n_x^2] J's terms
    double* scratch; // [8]: normalising sums, table constants, [4] live u1 pairs (count)
    double* table;   // [2 n_x^2] host table staging
    double* J;       // [J capacity] J history
    double* phin;    // [n_w] normalised one-dimensional noise weights
    double* H;       // [7 ext_n tab_n] row pass of the correlation tables
    double* tab;     // [tab_n^2 x 8] correlation tables, 8 slots per cell
    float2* tabf;    // the same as double-float pairs
    double* mins;    // [2 n_y + 1] exponent minima of the factorised u1 step
    double* fa;      // [n_y x n_x^2] prior x axis-1 factors, double-float pairs
    double* fb;      // [n_y x n_x^2] axis-2 factors, double-float pairs
    double* fa64;    // the same in FP64
    double* fb64;
    double* fv;      // [3 n_x^2] f values, then the prior factors
    double* part;    // [u1_splits x 3 x n_y^2] partial sums
    int32_t* list;   // [1 + n_y^2] count, then the targets of the FP64 pass
};

struct Prof;   // ucp_runtime.h: CUDA-event timers (null: none)

void launch2_setup(const G2& g, Dev2& d, int from_table, cudaStream_t s);
void launch2_sweep(const G2& g, Dev2& d, int cur, cudaStream_t s, Prof* prof = nullptr);
void launch2_mmse(const G2& g, Dev2& d, int buf, cudaStream_t s, Prof* prof = nullptr);
// J of controller buffer buf under the current u1 table into *out.  In the
// screened mode it first rebuilds the correlation tables of that u1 table
// (J's terms come from them, and the next search uses them), so it runs
// after every change of U.
void launch2_J(const G2& g, Dev2& d, int buf, double* out, cudaStream_t s,
               Prof* prof = nullptr);
void launch2_table(const G2& g, Dev2& d, int buf, cudaStream_t s);

}  // namespace ucp
