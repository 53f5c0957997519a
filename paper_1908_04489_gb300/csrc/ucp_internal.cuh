// ucp_internal.cuh -- shared declarations of the CUDA library (not part of
// the public ABI).  Geometry of one Witsenhausen instance (Section V-A) on
// the grids of Section III-D, and the launch wrappers of every kernel.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the library does not link libcuda)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ucp.h"

namespace ucp {

// Integer geometry of one instance.  Controller values are carried as int64
// lattice indices nu with value nu * delta * 2^-shift; the position of
// u + w_l on the y grid is then cell(nu) - hw + hy + l + frac(nu), exact.
struct Geom {
    double k, kk, sigma, delta, two_s2;
    int64_t hx, hw, hy, hr;     // half widths in units of delta
    int64_t n_x, n_w, n_y;
    int32_t shift;              // L * bits
    int32_t bits;               // log2(n_refine / 2)
    int64_t one;                // 2^shift
    int64_t q;                  // coarse spacing in units of delta (even)
    int32_t n_coarse, n_refine, n_levels, n_nbr;
    int32_t n_cand;             // 1 + 2 n_nbr + n_coarse + L n_refine
    int32_t u1_tile_min;        // fewest x0 points per tile of the u1 step
    int32_t problem;            // 0 Witsenhausen, 1 source-channel coding
    double w_noise;             // problem 1: noise half width (w_half)
    int32_t sc_fast;            // problem 1 at precision 1: screened search, warp u1 step
};

// Fills g from params; returns nullptr or a static reason string.
const char* make_geom(const ucp_params& p, Geom* g);

__host__ __device__ inline int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b) != 0 && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

// Device buffers of one instance (all owned by the instance).
struct DevState {
    double* px;       // [n_x] normalised prior weights p_i
    double* phi;      // [n_w] normalised quadrature weights phi_l
    double* U;        // [n_y] u1 table
    double* Ud;       // [n_y] U_{j+1} - U_j, 0 at the last entry
    int64_t* nu[2];   // [n_x] controller f, double buffered (Jacobi)
    int64_t* coarse;  // [n_coarse] coarse candidates (lattice indices)
    double* Sf;       // [n_x] S(f_i) under the current U
    double* Sc;       // [n_coarse] S at the coarse candidates
    int32_t* idx;     // [n_x] winner list position of the last sweep
    double* J;        // [1 + max_hist] J history
    double* scratch;  // reduction partials
    double* table;    // [n_x] staging for table inits / set_controllers
    double* sc_tab;   // problem 1 fast mode: [3 (n_y + n_w + 2)] tables A0, B0, B1
    double* sc_consts;// problem 1 fast mode: max |U|, the weight sum, exact re-costs
    double* sc_f;     // problem 1 fast mode: [n_x] f values
};

// Sizes of the fast path's buffers for one instance.
struct FastPlan {
    int64_t c_lo;      // lowest lattice cell covered by the tables
    int64_t n_pos;     // table positions (cells c_lo .. c_lo + n_pos - 1)
    int64_t jlo;       // y-index of table E-index 0
    int64_t n_e;       // length of E, E^2, E E_+ (n_pos + n_w + 1)
    int64_t tile;      // sources per tile of the u1 step (consecutive x0)
    int n_tiles;       // tiles; the u1 partial sums are kept per tile
    int64_t box_cap;   // 32-source chunk partials per tile (tile / 32 + kBoxMax)
    int run;           // targets per run of the u1 step
    int64_t n_runs;    // runs covering the y grid
    int64_t r_blocks;  // run blocks of the u1 kernel (kU1Runs runs each)
    int64_t J_blocks;  // blocks of the J reduction
    int64_t cell_blocks;  // blocks storing the cell coefficients (same launch)
    int64_t tc_na;     // table columns of the tensor-core build (128 positions each)
    int tc_ng;         // column groups (64 columns, one CTA row each)
    int tc_nch;        // tap chunks (kTcK taps each)
    int64_t tc_nblk;   // 128-value signal blocks sliced per sweep
};

struct dfloat;  // df.cuh

// Tensor-core correlation tables (kernels_tc.cu): 8-bit slices per operand,
// taps per chunk.
constexpr int kTcSlices = 6;
constexpr int kTcK = 128;

// u1 boxes: at most kBoxMax boxes per tile, kBoxTerms Taylor terms per box.
constexpr int kBoxMax = 32;
constexpr int kBoxTerms = 24;

// Everything the fast kernels read or write (device pointers + scalars).
struct FastView : FastPlan {
    const double* phi;   // [n_w] quadrature weights (FP64)
    const double* U;     // [n_y] u1 table
    const double* Ud;    // [n_y] U_{j+1} - U_j
    const int64_t* coarse;
    dfloat* C0;          // [n_pos - 1] cell quadratic S = C0 + t (C1 + t C2)
    dfloat* C1;
    dfloat* C2;
    float* Cb;           // [n_pos - 1] cell bound (tables, identity, E rounding)
    dfloat* P;           // [n_pos] correlation tables (double-float)
    dfloat* Q;
    dfloat* R;
    dfloat* E;           // [n_e] U^(y) - y on the extended grid
    dfloat* a;           // [n_w] phi_l w_l
    dfloat* phidf;       // [n_w] phi_l
    dfloat* wdf;         // [n_w] w_l
    dfloat* prior;       // [n_x] x_i^2 / (2 sigma^2)
    int64_t* src_nu;     // [n_x] lattice index of f_i this sweep
    dfloat* src_f;       // [n_x] f_i
    dfloat* src_F;       // [n_x] exp(delta f_i)
    dfloat* t64;         // [47] exp(k / 64), k = -23..23
    int32_t* box_cnt;    // [n_tiles] boxes of each tile
    int32_t* box_s0;     // [n_tiles * kBoxMax] first source of a box
    int32_t* box_n;      //   sources in the box
    float4* box_geo;     //   (c, h, pm, pmin): centre, half width, scale, min prior
    float4* box_rng;     //   (min f, max f, h if moments exist else inf, s)
    dfloat* box_C;       //   exp(delta c)
    dfloat* box_coef;    //   [2 kBoxTerms]: M_n / n!, then (c M_n + s M_{n+1}) / n!
    dfloat* box_part;    // [n_tiles * box_cap * (kBoxTerms + 1)] chunk partial moments
    float* run_lo;       // [n_runs] lower bound of min_i e_{i,j0} (scale)
    float* run_hi;       // [n_runs] upper bound of min_i e_ij over the run
    dfloat* partN;       // [n_tiles * n_y] numerator partials (double-float)
    dfloat* partD;       // [n_tiles * n_y] denominator partials
    double* Jpart;       // [J_blocks]
    uint16_t* tc_h;      // [2][tc_nch][kTcSlices][8][256] filter slices (bf16), shifted copies
    int32_t* tc_he;      // [2][tc_nch] filter chunk scales (exponents)
    uint16_t* tc_x;      // [3][kTcSlices][tc_nblk][128] signal slices (bf16)
    int32_t* tc_xe;      // [3][tc_nblk] signal block scales (exponents)
    float2* tc_part;     // [3][tc_nch][64 tc_ng][128] chunk partials (double-float)
    float* tc_bt;        // [tc_na + 1] per-column bound on the table error of S
    int32_t* tc_err;     // [0] set when a wait of the tensor-core kernel timed out;
                         // [1] test hook: the table kernel skips its filter copy
    CUtensorMap tc_map[3];  // TMA maps of tc_x per signal: rows of 128 bf16, 64 x 64 boxes
    int32_t* J_done;     // J blocks finished (reset by the last)
    double* W2_dev;      // sum phi_l w_l^2 (device copy)
    int32_t* n_exact;    // count of serial re-costings (near ties)
    int32_t* n_tier2;    // count of direct double-float quadratures (second tier)
    int32_t* defer_cnt;  // x0 points whose search was deferred this sweep
    void* defer_list;    // [n_x] their records (search position, carried winner)
    int64_t* n_pairs;    // [4] u1 work: direct (source, run) pairs, (box, run)
                         // expansions, double-float and FP32 Taylor terms
    float step_hi, step_lo;   // delta 2^-shift as double-float
    float delta_hi, delta_lo; // delta as double-float
    float kk_hi, kk_lo;       // k^2 as double-float
    float k_f;                // k (FP32, bound terms)
    float inv_one_f;          // 2^-shift
    float beta_rel;      // |table cost - serial cost| <= Cb = tc_bt(cell) + beta_rel M
    float beta_abs;      //   + beta_abs (2 sqrt(M) + 1)
    float beta_ctl;      //   + beta_ctl sqrt(control term) + ...
    float beta2_rel;     // direct double-float quadrature: beta2_rel S + ...
    float w_half;        // W (largest |w_l|)
    float y_abs;         // largest |y| on the extended grid of E
};

// Device-resident descriptor of one instance of a batch: everything a batched
// kernel needs, with the sweep state kept on the device so that one captured
// sweep serves every sweep.
struct InstDev {
    Geom g;
    FastView f;
    int64_t* nu[2];    // controller, double buffered
    int32_t* idx;      // winner list positions
    double* px;        // prior weights
    double* U;         // u1 table
    double* Ud;        // U_{j+1} - U_j
    double* J;         // J history
    int32_t cur;       // nu[cur] holds f
    int32_t sweeps;    // sweeps done (J history slot of the current J)
    int32_t defer_blocks;  // blocks of the deferred search for this instance
};

// Launch shapes that spread the same work differently over threads: every
// valid choice gives the same results, bit for bit (the autotuner's knobs).
constexpr int kSearchLanesDefault = 8;   // lanes per x0 point of the search
struct LaunchCfg {
    int search_lanes = 0;                 // lanes per x0 point in the search: 4, 8, 16 (0: 8)
    int u1_threads[5] = {0, 0, 0, 0, 0};  // threads per u1 run of 1, 2, 4, 8, 16 targets:
                                          // 1, 2 or 4, at most the run length (0: the rule)
    int defer_blocks = 0;                 // deferred-search blocks per instance (0: the rule)
};

// Block of a batched launch: which instance, which block of its own grid.
struct BlockRef {
    int32_t inst;
    int32_t local;
};

enum BatchKind {
    kBSearch = 0, kBTile, kBPerY, kBTabPart, kBBuildE, kBJPart, kBRun, kBTabComb,
    kBKinds
};

// Device arrays describing one batched sweep.
struct BatchLaunch {
    InstDev* insts;
    int n_inst;
    const BlockRef* map[kBKinds];  // per kernel kind (see BatchKind)
    int64_t n_blocks[kBKinds];
    const BlockRef* search_map;    // screening search
    int64_t search_blocks;
    const BlockRef* mmse_map[5];   // u1 main kernel per run length 1, 2, 4, 8, 16
    int64_t mmse_blocks[5];
    const BlockRef* defer_map;     // deferred (near-tie) search
    int64_t defer_blocks;
    int search_lanes;              // lanes per x0 point of the search (4, 8, 16)
    int u1_threads[5];             // threads per u1 run per run length (0: the rule)
};

// Set-up of a fast instance done by batched launches (instances created
// without their own set-up kernels): what those kernels read and write.
struct SetupDev {
    Geom g;
    FastView f;
    double* px;         // prior weights (exponentials, then normalised)
    double* phi;        // quadrature weights, likewise
    int64_t* coarse;    // coarse candidate list
    double* scratch;    // the two normalising sums
    int64_t* nu0;       // initial controller (lattice indices)
    int32_t* idx;       // winner positions (set to -1)
    const double* table;  // device copy of an init table (init_kind 2)
    int32_t init_kind;
    int64_t n7, lv[3];  // staircase step and levels (init_kind 1)
};

// Elementwise set-up blocks per instance (256 threads each): the largest of
// n_x, n_w, the coarse list and the fast path's constant table.
int64_t setup_elem_blocks(const Geom& g);
// Staircase step (units of delta) and level lattice indices of init kind 1.
void init_levels(const Geom& g, int kind, int64_t* n7, int64_t lv[3]);

struct SetupLaunch {
    const SetupDev* descs;
    const BlockRef* elem_map;     // setup_elem_blocks per instance
    int64_t elem_blocks;
    const BlockRef* inst_map;     // one block per instance
    int64_t inst_blocks;
    const BlockRef* filter_map;   // 2 tc_nch + 1 per instance (filter slices, W2)
    int64_t filter_blocks;
};
// kernels_plain.cu: exponentials, coarse list, init, counters; normalising
// sums; normalisation.  kernels_fast.cu: the fast path's constants.
// kernels_tc.cu: filter slices and W2.
void launch_batch_setup_plain(const SetupLaunch& sl, cudaStream_t s);
void launch_batch_setup_fast(const SetupLaunch& sl, cudaStream_t s);
void launch_batch_setup_tc(const SetupLaunch& sl, cudaStream_t s);

// Blocks of the deferred (near-tie) search per instance of a batch of 16 or
// more (smaller batches get 64 / n), and the bytes of one deferred-search
// record (kernels_fast.cu checks the size).
constexpr int kDeferBlocksBatch = 4;
constexpr size_t kDeferRecBytes = 64;

// Streaming multiprocessors of the current device (cached).
int sm_count();

// ---- plain FP64 path (kernels_plain.cu) --------------------------------
void launch_weights(const Geom& g, DevState& d, cudaStream_t s);
void launch_init(const Geom& g, DevState& d, int kind, int buf, cudaStream_t s);
void launch_table_to_lattice(const Geom& g, const double* table, int64_t* nu,
                             cudaStream_t s);
void launch_coarse_list(const Geom& g, DevState& d, cudaStream_t s);
void launch_mmse_plain(const Geom& g, DevState& d, int buf, cudaStream_t s);
void launch_udiff(const Geom& g, DevState& d, cudaStream_t s);
// out[k] = quadrature part of the cost of nus[k] (at_x: for x0 point k).
void launch_S_list(const Geom& g, DevState& d, const int64_t* nus, int64_t n,
                   double* out, cudaStream_t s, int at_x);
// The search of x0 points i_lo .. i_hi - 1 (i_hi < 0: all), Jacobi.
void launch_search_plain(const Geom& g, DevState& d, int buf_in, cudaStream_t s,
                         int64_t i_lo = 0, int64_t i_hi = -1);
void launch_J_plain(const Geom& g, DevState& d, int buf, int slot,
                    cudaStream_t s);
void launch_f_values(const Geom& g, const int64_t* nu, const double* x_or_null,
                     double* out, int as_u0, cudaStream_t s);
// Algorithm 1's local update of u0 (Section III-D): nu_out = Newton's step
// (gradient step tau where g'' <= 0) from nu_in under the u1 table U, every
// x0 point in parallel; exact FP64 in the w quadrature's fixed order.
size_t local_update_smem(const Geom& g);
cudaError_t launch_local_update(const Geom& g, const double* phi, const double* U,
                                const int64_t* nu_in, int64_t* nu_out, double tau,
                                cudaStream_t s);

}  // namespace ucp
