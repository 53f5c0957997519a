// ucp_fast.cuh -- state and launches of the fast path (kernels_fast.cu,
// kernels_u1.cu).
#pragma once

#include "ucp_internal.cuh"
#include "df.cuh"
#include "ucp_runtime.h"

namespace ucp {

// The constant table of the fast path (FastView::t64): entry k < 47 is
// exp((k - 23) / 64) (df_exp's table), entry 47 + n is 1 / n! for
// n <= kBoxTerms (the Taylor coefficients of the u1 boxes), in double-float.
constexpr int kConstTab = 47 + kBoxTerms + 1;
__device__ __forceinline__ dfloat const_table_entry(int k) {
    if (k < 47) return df_from_double(exp((double)(k - 23) / 64.0));
    double fact = 1.0;
    for (int m = 2; m <= k - 47; ++m) fact *= (double)m;   // n! (rounded above 22!)
    return df_from_double(1.0 / fact);
}

void fast_plan(const Geom& g, FastPlan* fp);
// u1 step (kernels_u1.cu): run length, tiles (at most max_tiles), buffers.
int mmse_run_length(const Geom& g);
void u1_plan(const Geom& g, int max_tiles, FastPlan* fp);
// Bytes of the u1 buffers (each rounded up to align) and their carving from
// an allocator get(ctx, bytes); false if an allocation failed.
size_t u1_scratch_bytes(const Geom& g, const FastPlan& fp, size_t align);
bool u1_carve(const Geom& g, FastView* f, void* (*get)(void*, size_t), void* ctx);
// One-time attribute of the batched u1 kernels (dynamic shared memory).
cudaError_t u1_init_attributes();
int64_t u1_batch_blocks(const Geom& g, const FastPlan& fp, int kind);
void launch_batch_u1(const BatchLaunch& bl, cudaStream_t s, Prof* prof = nullptr);
void launch_fast_setup(const Geom& g, const FastView& f, cudaStream_t s);
void launch_mmse_fast(const Geom& g, const FastView& f, const int64_t* nu,
                      double* U, cudaStream_t s, Prof* prof);
// Correlation tables on the tensor cores (kernels_tc.cu): plan, buffer
// sizes (7 arrays, each rounded up to align; sizes[] gets the raw sizes),
// block counts, one-time kernel attributes, per-instance filter slices, and
// the per-sweep build (E and slices, slice products, chunk sums + bound).
void tc_plan(const Geom& g, FastPlan* fp);
size_t tc_bytes(const FastPlan& fp, size_t align, size_t* sizes);
// TMA maps of the signal slices (after tc_x is allocated); false if the
// driver's encoder is unavailable or rejects them.
bool tc_encode_maps(FastView* f);
int64_t tc_build_E_blocks(const Geom& g, const FastPlan& fp);
int64_t tc_table_blocks(const FastPlan& fp);
int64_t tc_combine_blocks(const FastPlan& fp);
cudaError_t tc_init_attributes();
void launch_tc_setup(const Geom& g, const FastView& f, cudaStream_t s);
void launch_tables(const Geom& g, const FastView& f, const double* U, double* Ud,
                   cudaStream_t s, Prof* prof);
void launch_batch_tables(const BatchLaunch& bl, cudaStream_t s, Prof* prof = nullptr);
// The search of x0 points i_lo .. i_hi - 1 (i_hi < 0: all), from nu_in into
// nu_out (Jacobi).
void launch_search_fast(const Geom& g, const FastView& f, const int64_t* nu_in,
                        int64_t* nu_out, int32_t* idx, cudaStream_t s, int64_t i_lo = 0,
                        int64_t i_hi = -1, const LaunchCfg* cfg = nullptr);
// Blocks of the screened search with `lanes` lanes per x0 point.
int64_t search_blocks(const Geom& g, int lanes);
// Blocks of each batched kernel kind for one instance (fast_plan sizes).
int64_t batch_blocks(const Geom& g, const FastPlan& fp, int kind);
int64_t batch_mmse_blocks(const Geom& g, const FastPlan& fp);
// One sweep of every instance of the batch (search, u1, tables, J; then the
// device-side cur / sweep counters advance); or its search alone, or the rest.
// With a profiler, each kernel group is timed by CUDA events on `s`.
void launch_batch_sweep(const BatchLaunch& bl, cudaStream_t s, Prof* prof = nullptr);
void launch_batch_search(const BatchLaunch& bl, cudaStream_t s, Prof* prof = nullptr);
void launch_batch_rest(const BatchLaunch& bl, cudaStream_t s, Prof* prof = nullptr);
void launch_J_fast(const Geom& g, const FastView& f, const double* px,
                   const int64_t* nu, double* out, cudaStream_t s, Prof* prof);

}  // namespace ucp
