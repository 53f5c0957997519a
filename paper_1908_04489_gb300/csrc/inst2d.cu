// inst2d.cu -- one instance of the 2-dimensional Witsenhausen counterexample
// (Section V-D) behind the ucp2_* calls: device buffers, the start, sweeps
// (u0 step, u1 step, J) and the J history.  Kernels: kernels_2d.cu.
#include <math.h>
#include <string.h>

#include <vector>

#include "ucp_2d.h"
#include "ucp_runtime.h"

using namespace ucp;

struct ucp_inst2 {
    ucp_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    G2 g{};
    Dev2 d{};
    std::vector<void*> bufs;
    int cur = 0;
    long long sweeps = 0, J_cap = 0;
    bool poisoned = false;
    Prof prof;   // CUDA-event timers per kernel group (ucp2_profile)
};

static void* alloc2(ucp_inst2* in, size_t bytes) {
    void* p = nullptr;
    if (in->ctx->alloc) p = in->ctx->alloc(bytes, in->ctx->user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) in->bufs.push_back(p);
    return p;
}

static void free2(ucp_inst2* in) {
    for (void* p : in->bufs) {
        if (in->ctx->free_fn) in->ctx->free_fn(p, in->ctx->user);
        else cudaFree(p);
    }
    in->bufs.clear();
}

static ucp_status cuda_check(ucp_inst2* in, const char* where) {
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return UCP_OK;
    in->poisoned = true;
    set_error("%s: %s", where, cudaGetErrorString(e));
    return UCP_E_CUDA;
}

// J history slot `slot` (grown by copying when full).
static ucp_status ensure_J(ucp_inst2* in, long long need) {
    if (need <= in->J_cap) return UCP_OK;
    const long long cap = need * 2 + 64;
    double* nj = (double*)alloc2(in, 8 * (size_t)cap);
    if (!nj) return UCP_E_NOMEM;
    if (in->J_cap)
        cudaMemcpyAsync(nj, in->d.J, 8 * (size_t)in->J_cap, cudaMemcpyDeviceToDevice, in->stream);
    in->d.J = nj;
    in->J_cap = cap;
    return UCP_OK;
}

// Every value of a host controller table finite and within the lattice's
// int64 range once scaled by 2^shift / delta.
static bool f_in_range(const G2& g, const double* f, size_t n2) {
    for (size_t k = 0; k < n2; ++k)
        if (!(fabs(f[k] / g.delta * (double)g.one) < 9.0e15)) return false;
    return true;
}

extern "C" ucp_status ucp2_plan(const ucp2_params* p, uint64_t* n_x, uint64_t* n_w,
                                uint64_t* n_y, uint64_t* n_cand) {
    if (!p) return UCP_E_ARG;
    G2 g;
    if (const char* why = make_g2(*p, &g)) {
        set_error("ucp2_plan: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (n_x) *n_x = (uint64_t)g.n_x;
    if (n_w) *n_w = (uint64_t)g.n_w;
    if (n_y) *n_y = (uint64_t)g.n_y;
    if (n_cand) *n_cand = (uint64_t)g.n_cand;
    return UCP_OK;
}

extern "C" ucp_status ucp2_create(ucp_ctx* ctx, const ucp2_params* p, const double* init_f,
                                  void* stream, ucp_inst2** out) {
    if (!p || !out) return UCP_E_ARG;
    G2 g;
    if (const char* why = make_g2(*p, &g)) {
        set_error("ucp2_create: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (!ctx) {
        set_error("ucp2_create: %s%s", "a context is required", "");
        return UCP_E_ARG;
    }
    if (init_f && !f_in_range(g, init_f, 2 * (size_t)(g.n_x * g.n_x))) {
        set_error("ucp2_create: %s%s", "init_f value not finite or out of range", "");
        return UCP_E_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return UCP_E_CUDA;
    ucp_inst2* in = new ucp_inst2();
    in->ctx = ctx;
    in->stream = (cudaStream_t)stream;
    in->g = g;
    const size_t n = (size_t)(g.n_x * g.n_x), nw = (size_t)g.n_w, ny2 = (size_t)(g.n_y * g.n_y);
    Dev2& d = in->d;
    d.px = (double*)alloc2(in, 8 * n);
    d.phi1 = (double*)alloc2(in, 8 * nw);
    d.phi2 = (double*)alloc2(in, 8 * nw * nw);
    d.U = (double*)alloc2(in, 16 * ny2);
    d.nu[0] = (int64_t*)alloc2(in, 16 * n);
    d.nu[1] = (int64_t*)alloc2(in, 16 * n);
    d.idx = (int32_t*)alloc2(in, 4 * n);
    d.terms = (double*)alloc2(in, 8 * n);
    d.scratch = (double*)alloc2(in, 64);
    d.table = (double*)alloc2(in, 16 * n);
    d.phin = (double*)alloc2(in, 8 * nw);
    const bool screened = !(g.direct & 1), factorised = !(g.direct & 2);
    if (screened) {
        d.H = (double*)alloc2(in, 8 * 7 * (size_t)(g.ext_n * g.tab_n));
        d.tab = (double*)alloc2(in, 64 * (size_t)(g.tab_n * g.tab_n));
        d.tabf = (float2*)alloc2(in, 64 * (size_t)(g.tab_n * g.tab_n));
    }
    if (factorised) {
        d.mins = (double*)alloc2(in, 8 * (size_t)(2 * g.n_y + 1));
        d.fa = (double*)alloc2(in, 8 * n * (size_t)g.n_y);
        d.fb = (double*)alloc2(in, 8 * n * (size_t)g.n_y);
        d.part = (double*)alloc2(in, 24 * (size_t)g.u1_splits * (size_t)(g.n_y * g.n_y));
        d.fa64 = (double*)alloc2(in, 8 * n * (size_t)g.n_y);
        d.fb64 = (double*)alloc2(in, 8 * n * (size_t)g.n_y);
        d.fv = (double*)alloc2(in, 24 * n);
        d.list = (int32_t*)alloc2(in, 4 * (1 + (size_t)(g.n_y * g.n_y)));
    }
    if ((screened && (!d.H || !d.tab || !d.tabf)) ||
        (factorised && (!d.mins || !d.fa || !d.fb || !d.part || !d.fa64 || !d.fb64 || !d.fv ||
                        !d.list)) ||
        !d.phin || !d.px || !d.phi1 || !d.phi2 || !d.U || !d.nu[0] || !d.nu[1] || !d.idx || !d.terms ||
        !d.scratch || !d.table || ensure_J(in, 64) != UCP_OK) {
        free2(in);
        delete in;
        return UCP_E_NOMEM;
    }
    cudaStream_t s = in->stream;
    if (init_f) {
        cudaMemcpyAsync(d.table, init_f, 16 * n, cudaMemcpyHostToDevice, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {   // the caller's buffer is free after return
            free2(in);
            delete in;
            return UCP_E_CUDA;
        }
    }
    cudaMemsetAsync(d.idx, 0xff, 4 * n, s);
    cudaMemsetAsync(d.scratch, 0, 64, s);   // sums, constants, the live-pair count
    launch2_setup(g, d, init_f != nullptr, s);
    launch2_mmse(g, d, 0, s);
    launch2_J(g, d, 0, d.J, s);
    const ucp_status st = cuda_check(in, "ucp2_create");
    if (st != UCP_OK) {
        cudaStreamSynchronize(s);
        free2(in);
        delete in;
        return st;
    }
    *out = in;
    return UCP_OK;
}

extern "C" ucp_status ucp2_sweep(ucp_inst2* in, int32_t n) {
    if (!in || n < 0) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (ensure_J(in, in->sweeps + 1 + n) != UCP_OK) return UCP_E_NOMEM;
    for (int k = 0; k < n; ++k) {
        Prof* pr = in->prof.on ? &in->prof : nullptr;
        launch2_sweep(in->g, in->d, in->cur, in->stream, pr);
        in->cur ^= 1;
        in->sweeps += 1;
        launch2_mmse(in->g, in->d, in->cur, in->stream, pr);
        launch2_J(in->g, in->d, in->cur, in->d.J + in->sweeps, in->stream, pr);
    }
    return cuda_check(in, "ucp2_sweep");
}

extern "C" ucp_status ucp2_J_history(ucp_inst2* in, double* out, uint64_t n,
                                     uint64_t* n_written) {
    if (!in || (!out && n)) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    uint64_t m = (uint64_t)in->sweeps + 1;
    if (n < m) m = n;
    if (m) cudaMemcpyAsync(out, in->d.J, 8 * m, cudaMemcpyDeviceToHost, in->stream);
    if (cudaStreamSynchronize(in->stream) != cudaSuccess) return cuda_check(in, "ucp2_J_history");
    if (n_written) *n_written = m;
    return UCP_OK;
}

extern "C" ucp_status ucp2_get_controllers(ucp_inst2* in, double* f, uint64_t f_len,
                                           double* u1, uint64_t u1_len, int32_t* idx,
                                           uint64_t idx_len) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    const G2& g = in->g;
    const size_t n = (size_t)(g.n_x * g.n_x);
    if ((f && f_len < 2 * n) || (u1 && u1_len < 2 * (uint64_t)(g.n_y * g.n_y)) ||
        (idx && idx_len < n)) {
        set_error("ucp2_get_controllers: %s%s", "a buffer is shorter than the instance's size", "");
        return UCP_E_ARG;
    }
    std::vector<int64_t> nu(f ? 2 * n : 0);
    if (f) cudaMemcpyAsync(nu.data(), in->d.nu[in->cur], 16 * n, cudaMemcpyDeviceToHost, in->stream);
    if (u1) cudaMemcpyAsync(u1, in->d.U, 16 * (size_t)(g.n_y * g.n_y), cudaMemcpyDeviceToHost,
                            in->stream);
    if (idx) cudaMemcpyAsync(idx, in->d.idx, 4 * n, cudaMemcpyDeviceToHost, in->stream);
    if (cudaStreamSynchronize(in->stream) != cudaSuccess)
        return cuda_check(in, "ucp2_get_controllers");
    for (size_t k = 0; f && k < 2 * n; ++k) f[k] = ldexp((double)nu[k] * g.delta, -g.shift);
    return UCP_OK;
}

extern "C" ucp_status ucp2_set_controllers(ucp_inst2* in, const double* f, uint64_t f_len,
                                           const double* u1, uint64_t u1_len) {
    if (!in || !f) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    const G2& g = in->g;
    const size_t n = (size_t)(g.n_x * g.n_x);
    if (f_len != 2 * n || (u1 && u1_len != 2 * (uint64_t)(g.n_y * g.n_y))) {
        set_error("ucp2_set_controllers: %s%s", "a buffer's length is not the instance's size", "");
        return UCP_E_ARG;
    }
    if (!f_in_range(g, f, 2 * n)) {
        set_error("ucp2_set_controllers: %s%s", "f value not finite or out of range", "");
        return UCP_E_ARG;
    }
    cudaMemcpyAsync(in->d.table, f, 16 * n, cudaMemcpyHostToDevice, in->stream);
    if (u1) cudaMemcpyAsync(in->d.U, u1, 16 * (size_t)(g.n_y * g.n_y), cudaMemcpyHostToDevice,
                            in->stream);
    launch2_table(g, in->d, in->cur, in->stream);
    if (!u1) launch2_mmse(g, in->d, in->cur, in->stream);
    launch2_J(g, in->d, in->cur, in->d.J + in->sweeps, in->stream);
    if (cudaStreamSynchronize(in->stream) != cudaSuccess) {
        in->poisoned = true;
        set_error("ucp2_set_controllers: %s%s", "stream synchronisation failed", "");
        return UCP_E_CUDA;
    }
    return cuda_check(in, "ucp2_set_controllers");
}

extern "C" ucp_status ucp2_profile(ucp_inst2* in, int32_t enable) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    return prof_enable(&in->prof, in->stream, enable != 0);
}

extern "C" int32_t ucp2_kernel_times(ucp_inst2* in, const char** names, int64_t* launches,
                                     double* total_ms, int32_t cap) {
    if (!in || cap < 0) return -1;
    if (cudaStreamSynchronize(in->stream) != cudaSuccess) return -1;
    return prof_collect(&in->prof, names, launches, total_ms, cap);
}

extern "C" ucp_status ucp2_work_counters(ucp_inst2* in, int64_t* live_pairs) {
    if (!in || !live_pairs) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, in->d.scratch + 4, sizeof(v), cudaMemcpyDeviceToHost, in->stream);
    if (cudaStreamSynchronize(in->stream) != cudaSuccess)
        return cuda_check(in, "ucp2_work_counters");
    *live_pairs = (int64_t)v;
    return UCP_OK;
}

extern "C" ucp_status ucp2_destroy(ucp_inst2* in) {
    if (!in) return UCP_E_ARG;
    cudaStreamSynchronize(in->stream);
    free2(in);
    delete in;
    return UCP_OK;
}
