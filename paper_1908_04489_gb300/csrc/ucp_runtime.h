// ucp_runtime.h -- host-side runtime objects behind the C ABI: context,
// instance (device state + sweep driver), per-kernel event timers.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ucp_internal.cuh"

struct ucp_ctx {
    int device = 0;
    ucp_alloc_fn alloc = nullptr;
    ucp_free_fn free_fn = nullptr;
    void* user = nullptr;
    ucp::LaunchCfg cfg;   // launch shapes that new instances and batches start with
};

namespace ucp {

void set_error(const char* fmt, const char* a, const char* b);

// CUDA-event timers around every kernel launch of one stream.
struct Prof {
    struct Stat {
        const char* name;
        long long launches;
        double ms;
    };
    struct Pending {
        int stat;
        cudaEvent_t a, b;
    };
    bool on = false;
    cudaStream_t stream = nullptr;
    std::vector<Stat> stats;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    int begin(const char* name, cudaEvent_t* a);  // -1 when off
    void end(int stat, cudaEvent_t a);
    void drain();
    ~Prof();
};

// Times the launches made during its lifetime as one entry of `p` (no-op
// when p is null or off).
struct ProfScope {
    Prof* p;
    int k = -1;
    cudaEvent_t a = nullptr;
    ProfScope(Prof* p_, const char* name) : p(p_) {
        if (p) k = p->begin(name, &a);
    }
    ~ProfScope() {
        if (p) p->end(k, a);
    }
};

ucp_status prof_enable(Prof* p, cudaStream_t s, bool on);
int prof_collect(Prof* p, const char** names, int64_t* launches, double* ms,
                 int cap);

struct BatchSet;  // batch_set.h

// Owner of device allocations made through a context.  After reserve(n),
// get() carves 256-byte aligned pieces from that one allocation while it
// lasts (one allocator call per instance instead of one per buffer); carved
// pieces are returned with the slab by release_all().
struct Arena {
    ucp_ctx* ctx = nullptr;
    std::vector<void*> ptrs;
    size_t bytes = 0;
    char* slab = nullptr;
    size_t slab_size = 0, slab_used = 0;
    bool slab_owned = false;
    bool reserve(size_t n);   // false if the allocation failed (get() still works)
    void adopt(void* p, size_t n);   // carve from memory owned elsewhere
    void* get(size_t n);      // nullptr on failure
    void put(void* p);        // frees a separately allocated block; no-op in the slab
    void release_all();
};

}  // namespace ucp

struct ucp_inst {
    ucp_ctx* ctx = nullptr;
    ucp_params params{};
    ucp::Geom g{};
    ucp::DevState d{};
    ucp::Arena arena;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool poisoned = false;
    int cur = 0;                 // which nu buffer holds f
    long long sweeps_done = 0;   // J history slots used: sweeps_done + 1
    long long hist_cap = 0;
    size_t bytes = 0;
    ucp::Prof prof;
    bool fast = false;           // precision 1
    double fbound = 0.0;         // largest |f| or |U| set by the caller
    ucp::FastView fv{};
    // fast path on a non-default stream: one sweep captured as a CUDA graph
    // per buffer parity (the search with this instance's own launch
    // parameters, the rest over a one-member batch set with device-side
    // sweep state), replayed
    ucp::BatchSet* solo = nullptr;
    cudaGraphExec_t solo_graph[2] = {nullptr, nullptr};
    bool solo_tried = false;
    bool solo_failed = false;   // the one-member batch set could not be built
    ucp::LaunchCfg cfg;         // launch shapes (results do not depend on them)
};

namespace ucp {

// Device bytes one instance allocates (matches inst_init).
size_t inst_bytes(const Geom& g, int precision);
// Set up an instance on `stream`: buffers, then (own_setup) the grids,
// weights, init, the first u1 update, tables and J (J history slot 0).  A
// fast instance created without own_setup gets its buffers and host-side
// state only; its set-up kernels and first step come from batched launches
// (batchset_setup) before its first sweep.
// `slab`: inst_bytes(g, precision) bytes of device memory owned by the
// caller (a batch), carved for the buffers instead of an allocation.
ucp_status inst_init(ucp_inst* in, ucp_ctx* ctx, const ucp_params& p,
                     const Geom& g, cudaStream_t stream, bool own_setup = true,
                     void* slab = nullptr);
// ucp_create with the choices above (validates the parameters).
ucp_status inst_create(ucp_ctx* ctx, const ucp_params* params, cudaStream_t stream,
                       bool own_setup, ucp_inst** out, void* slab = nullptr);
ucp_status inst_sweep(ucp_inst* in, int n);
// n local-update iterations of Algorithm 1 (u0 by the local update, then u1
// by its exact minimiser, then J), recorded in the J history like sweeps.
ucp_status inst_local_update(ucp_inst* in, int n, double tau);
// Checks a public launch configuration; nullptr or the reason it is invalid.
const char* launch_cfg_from(const ucp_launch_config* c, LaunchCfg* out);
// New launch shapes for later sweeps (graphs and block maps rebuilt).
ucp_status inst_set_launch_cfg(ucp_inst* in, const LaunchCfg& cfg);
// One sweep split by x0 ranges: the search of a range (its new f to host
// memory), then the full new f and the rest of the sweep.
ucp_status inst_sweep_part(ucp_inst* in, int64_t i0, int64_t i1, double* f_host);
ucp_status inst_sweep_finish(ucp_inst* in, const double* f_host);
// Algorithm 1's outer loop on the host around the two kinds of iteration.
ucp_status inst_solve(ucp_inst* in, const ucp_solve_params& sp, ucp_solve_report* rep,
                      double* J_phase, int32_t* NL_rounds);
// N_L of the next round: min(max(floor(I_L N / (I_L + I_P)), 1), N - 1),
// n_l when I_L + I_P = 0.
int alg1_split(double I_L, double I_P, int N, int n_l);
// Make room in the J history for `need` entries (synchronises on growth).
ucp_status grow_history(ucp_inst* in, long long need);
ucp_status inst_sync(ucp_inst* in);
ucp_status inst_read(ucp_inst* in, const void* dev, void* host, size_t bytes);
ucp_status inst_get(ucp_inst* in, double* f, double* u1, int as_u0, int32_t* idx);
ucp_status inst_set(ucp_inst* in, const double* f, const double* u1);
void inst_release(ucp_inst* in);

}  // namespace ucp
