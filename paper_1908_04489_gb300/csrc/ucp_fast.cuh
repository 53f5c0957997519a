// ucp_fast.cuh -- state and launches of the fast path (kernels_fast.cu).
#pragma once

#include "ucp_internal.cuh"
#include "df.cuh"
#include "ucp_runtime.h"

namespace ucp {

void fast_plan(const Geom& g, FastPlan* fp);
int mmse_run_length(const Geom& g);
void launch_fast_setup(const Geom& g, const FastView& f, cudaStream_t s);
void launch_mmse_fast(const Geom& g, const FastView& f, const int64_t* nu,
                      double* U, cudaStream_t s, Prof* prof);
void launch_tables(const Geom& g, const FastView& f, const double* U, double* Ud,
                   cudaStream_t s, Prof* prof);
void launch_search_fast(const Geom& g, const FastView& f, const int64_t* nu_in,
                        int64_t* nu_out, int32_t* idx, cudaStream_t s);
// Blocks of each batched kernel kind for one instance (fast_plan sizes).
int64_t batch_blocks(const Geom& g, const FastPlan& fp, int kind);
int64_t batch_mmse_blocks(const Geom& g, const FastPlan& fp);
// One sweep of every instance of the batch (search, u1, tables, J; then the
// device-side cur / sweep counters advance).
void launch_batch_sweep(const BatchLaunch& bl, cudaStream_t s);
void launch_J_fast(const Geom& g, const FastView& f, const double* px,
                   const int64_t* nu, double* out, cudaStream_t s, Prof* prof);

}  // namespace ucp
