// ucp_capi.cu -- the C ABI of libucp.so (declared in include/ucp.h):
// argument validation, device memory, the per-instance sweep driver and the
// per-kernel CUDA-event timers.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "ucp_internal.cuh"
#include "ucp_runtime.h"

namespace ucp {

static thread_local char g_last_error[512] = "";

void set_error(const char* fmt, const char* a, const char* b) {
    snprintf(g_last_error, sizeof(g_last_error), fmt, a ? a : "", b ? b : "");
}

static int half_steps(double half, double delta, int64_t* out) {
    const double r = half / delta;
    const double n = floor(r + 0.5);
    if (!(n >= 0.0) || fabs(r - n) > 1e-9 * (n > 1.0 ? n : 1.0)) return -1;
    *out = (int64_t)n;
    return 0;
}

const char* make_geom(const ucp_params& p, Geom* g) {
    memset(g, 0, sizeof(*g));
    if (!(p.k > 0.0) || !isfinite(p.k)) return "k must be a positive number";
    if (!(p.sigma > 0.0) || !isfinite(p.sigma)) return "sigma must be positive";
    if (!(p.delta > 0.0) || !isfinite(p.delta)) return "delta must be positive";
    if (half_steps(p.x_half, p.delta, &g->hx) || g->hx < 1)
        return "x_half must be a positive multiple of delta";
    if (half_steps(p.w_half, p.delta, &g->hw) || g->hw < 1)
        return "w_half must be a positive multiple of delta";
    if (half_steps(p.y_half, p.delta, &g->hy) || g->hy < 1)
        return "y_half must be a positive multiple of delta";
    if (half_steps(p.cand_half, p.delta, &g->hr))
        return "cand_half must be a multiple of delta";
    if (p.n_coarse < 2 || p.n_coarse > 4096) return "n_coarse must be in [2, 4096]";
    if (p.n_refine != 2 && p.n_refine != 4 && p.n_refine != 8 &&
        p.n_refine != 16 && p.n_refine != 32)
        return "n_refine must be 2, 4, 8, 16 or 32";
    if (p.n_levels < 0 || p.n_levels > 8) return "n_levels must be in [0, 8]";
    if (p.n_nbr < 0 || p.n_nbr > 8) return "n_nbr must be in [0, 8]";
    if (p.flags != 0) return "flags must be 0";
    if (p.reserved != 0) return "reserved must be 0";
    if (p.problem != 0 && p.problem != 1) return "problem must be 0 or 1";
    if (p.precision != 0 && p.precision != 1) return "precision must be 0 or 1";
    if (p.delta * (p.x_half + p.y_half + p.cand_half) > 200.0)
        return "delta * (x_half + y_half + cand_half) must be <= 200";
    if (p.init_kind < 0 || p.init_kind > 2) return "init_kind must be 0, 1 or 2";
    int bits = 0;
    while ((1 << bits) < p.n_refine / 2) ++bits;
    g->bits = bits;
    g->shift = bits * p.n_levels;
    if (g->shift > 30) return "n_levels * log2(n_refine/2) must be <= 30";
    g->one = (int64_t)1 << g->shift;
    g->n_x = 2 * g->hx + 1;
    g->n_w = 2 * g->hw + 1;
    g->n_y = 2 * g->hy + 1;
    if (g->n_x > (1 << 26) || g->n_w > (1 << 24) || g->n_y > (1 << 26))
        return "grid too large";
    const int64_t nc1 = p.n_coarse - 1;
    int64_t c = (g->hr + nc1 - 1) / nc1;
    if (c < 1) c = 1;
    g->q = 2 * c;
    // lattice indices of every reachable value must stay far inside int64
    const double reach = (double)(g->hr + g->hx + g->hy + 2 * g->q) * (double)g->one;
    if (reach > 8.0e12) return "grid extent too large for the candidate lattice";
    g->k = p.k;
    g->kk = p.k * p.k;
    g->sigma = p.sigma;
    g->delta = p.delta;
    g->two_s2 = 2.0 * p.sigma * p.sigma;
    g->n_coarse = p.n_coarse;
    g->n_refine = p.n_refine;
    g->n_levels = p.n_levels;
    g->n_nbr = p.n_nbr;
    g->n_cand = 1 + 2 * p.n_nbr + p.n_coarse + p.n_levels * p.n_refine;
    g->problem = p.problem;
    g->sc_fast = p.problem == 1 && p.precision == 1;
    g->w_noise = p.w_half;
    // A tile of the u1 step holds at most 32 boxes of f-width 0.1: controllers
    // that vary steadily across x0 (the identity start, or a table start
    // whose increments are mostly nonzero, and their first sweeps) need
    // narrow tiles to keep their sources in boxes (256 points); piecewise flat
    // ones (the staircase, flat tables) fill few boxes, and wider tiles (512
    // points) keep the number of per-tile partial sums down.
    bool steady = p.init_kind == 0;
    if (p.init_kind == 2 && p.init_table && p.init_len == (uint64_t)g->n_x && g->n_x > 1) {
        int64_t moving = 0;
        for (int64_t i = 0; i + 1 < g->n_x; ++i)
            moving += p.init_table[i + 1] != p.init_table[i];
        steady = 2 * moving > g->n_x - 1;
    }
    g->u1_tile_min = steady ? 256 : 512;
    if (p.init_kind == 1) {
        int64_t n7;
        if (half_steps(7.0, p.delta, &n7) || n7 < 1)
            return "staircase init needs 7 to be a multiple of delta";
    }
    if (p.init_kind == 2) {
        if (!p.init_table) return "init_kind 2 needs init_table";
        if (p.init_len != (uint64_t)g->n_x) return "init_len must equal n_x";
    }
    return nullptr;
}

}  // namespace ucp

using namespace ucp;

// ---- status / version ---------------------------------------------------

extern "C" const char* ucp_status_str(ucp_status s) {
    switch (s) {
        case UCP_OK: return "ok";
        case UCP_PENDING: return "pending";
        case UCP_E_ARG: return "invalid argument";
        case UCP_E_NOMEM: return "out of device memory";
        case UCP_E_BUDGET: return "request exceeds the server budget";
        case UCP_E_CUDA: return "CUDA error";
        case UCP_E_TIMEOUT: return "device wait timed out";
        case UCP_E_STATE: return "object poisoned, destroyed or busy";
        case UCP_E_NOTFOUND: return "unknown ticket";
    }
    return "unknown status";
}

extern "C" const char* ucp_last_error(void) { return g_last_error; }

extern "C" const char* ucp_version(void) { return "ucp 0.1 sm_103a"; }

extern "C" ucp_status ucp_plan(const ucp_params* params, uint64_t* n_x,
                               uint64_t* n_w, uint64_t* n_y, uint64_t* n_cand,
                               uint64_t* device_bytes) {
    if (!params) {
        set_error("ucp_plan: %s%s", "NULL params", "");
        return UCP_E_ARG;
    }
    Geom g;
    if (const char* why = make_geom(*params, &g)) {
        set_error("ucp_plan: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (n_x) *n_x = (uint64_t)g.n_x;
    if (n_w) *n_w = (uint64_t)g.n_w;
    if (n_y) *n_y = (uint64_t)g.n_y;
    if (n_cand) *n_cand = (uint64_t)g.n_cand;
    if (device_bytes) *device_bytes = (uint64_t)inst_bytes(g, params->precision);
    return UCP_OK;
}

// ---- context ----------------------------------------------------------

extern "C" ucp_status ucp_ctx_create(int32_t device, ucp_alloc_fn alloc,
                                     ucp_free_fn free_fn, void* user,
                                     ucp_ctx** out) {
    if (!out || ((alloc == nullptr) != (free_fn == nullptr))) {
        set_error("ucp_ctx_create: %s%s", "out must be non-NULL and alloc/free ",
                  "given together");
        return UCP_E_ARG;
    }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        set_error("ucp_ctx_create: no such CUDA device (%s)%s",
                  cudaGetErrorString(e), "");
        return e != cudaSuccess ? UCP_E_CUDA : UCP_E_ARG;
    }
    ucp_ctx* c = new ucp_ctx();
    c->device = device;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    *out = c;
    return UCP_OK;
}

extern "C" ucp_status ucp_ctx_destroy(ucp_ctx* ctx) {
    if (!ctx) return UCP_E_ARG;
    delete ctx;
    return UCP_OK;
}

// ---- instance ---------------------------------------------------------

ucp_status ucp::inst_create(ucp_ctx* ctx, const ucp_params* params, cudaStream_t stream,
                            bool own_setup, ucp_inst** out, void* slab) {
    if (!params || !out) {
        set_error("ucp_create: %s%s", "NULL argument", "");
        return UCP_E_ARG;
    }
    *out = nullptr;
    Geom g;
    if (const char* why = make_geom(*params, &g)) {
        set_error("ucp_create: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (!ctx) {
        set_error("ucp_create: %s%s", "NULL context", "");
        return UCP_E_ARG;
    }
    ucp_inst* in = new ucp_inst();
    ucp_status st = inst_init(in, ctx, *params, g, stream, own_setup, slab);
    if (st != UCP_OK) {
        inst_release(in);
        delete in;
        return st;
    }
    *out = in;
    return UCP_OK;
}

extern "C" ucp_status ucp_create(ucp_ctx* ctx, const ucp_params* params,
                                 void* stream, ucp_inst** out) {
    return inst_create(ctx, params, (cudaStream_t)stream, true, out);
}

extern "C" ucp_status ucp_sizes(const ucp_inst* in, uint64_t* n_x, uint64_t* n_w,
                                uint64_t* n_y, uint64_t* n_cand,
                                uint64_t* device_bytes) {
    if (!in) return UCP_E_ARG;
    if (n_x) *n_x = (uint64_t)in->g.n_x;
    if (n_w) *n_w = (uint64_t)in->g.n_w;
    if (n_y) *n_y = (uint64_t)in->g.n_y;
    if (n_cand) *n_cand = (uint64_t)in->g.n_cand;
    if (device_bytes) *device_bytes = (uint64_t)in->bytes;
    return UCP_OK;
}

extern "C" ucp_status ucp_sweep(ucp_inst* in, int32_t n_sweeps) {
    if (!in || n_sweeps < 0) {
        set_error("ucp_sweep: %s%s", "NULL instance or negative count", "");
        return UCP_E_ARG;
    }
    if (in->poisoned) return UCP_E_STATE;
    return inst_sweep(in, n_sweeps);
}

static ucp_status arg_error(const char* where, const char* why) {
    set_error("%s: %s", where, why);
    return UCP_E_ARG;
}

namespace ucp {
const char* launch_cfg_from(const ucp_launch_config* c, LaunchCfg* out) {
    if (!c) return "NULL configuration";
    if (c->search_lanes != 0 && c->search_lanes != 4 && c->search_lanes != 8 &&
        c->search_lanes != 16)
        return "search_lanes must be 0, 4, 8 or 16";
    for (int r = 0; r < 5; ++r) {
        const int P = c->u1_threads[r];
        if (P != 0 && P != 1 && P != 2 && P != 4) return "u1_threads must be 0, 1, 2 or 4";
        if (P > (1 << r)) return "u1_threads above the run length";
    }
    if (c->defer_blocks < 0 || c->defer_blocks > 4096)
        return "defer_blocks must be in 0..4096";
    out->search_lanes = c->search_lanes;
    for (int r = 0; r < 5; ++r) out->u1_threads[r] = c->u1_threads[r];
    out->defer_blocks = c->defer_blocks;
    return nullptr;
}
}  // namespace ucp

extern "C" ucp_status ucp_ctx_set_launch_config(ucp_ctx* ctx, const ucp_launch_config* c) {
    if (!ctx) return UCP_E_ARG;
    LaunchCfg cfg;
    if (const char* why = launch_cfg_from(c, &cfg))
        return arg_error("ucp_ctx_set_launch_config", why);
    ctx->cfg = cfg;
    return UCP_OK;
}

extern "C" ucp_status ucp_set_launch_config(ucp_inst* in, const ucp_launch_config* c) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    LaunchCfg cfg;
    if (const char* why = launch_cfg_from(c, &cfg)) return arg_error("ucp_set_launch_config", why);
    return inst_set_launch_cfg(in, cfg);
}

extern "C" ucp_status ucp_sweep_part(ucp_inst* in, int64_t i0, int64_t i1, double* f_part) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (i0 < 0 || i1 < i0 || i1 > in->g.n_x || (i1 > i0 && !f_part))
        return arg_error("ucp_sweep_part", "need 0 <= i0 <= i1 <= n_x and a host buffer");
    return inst_sweep_part(in, i0, i1, f_part);
}

extern "C" ucp_status ucp_sweep_finish(ucp_inst* in, const double* f, uint64_t n_x) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (!f || n_x != (uint64_t)in->g.n_x)
        return arg_error("ucp_sweep_finish", "f must hold n_x values");
    for (uint64_t k = 0; k < n_x; ++k)
        if (!(fabs(f[k] / in->g.delta * (double)in->g.one) < 9.0e15))
            return arg_error("ucp_sweep_finish", "f value not finite or out of range");
    return inst_sweep_finish(in, f);
}

extern "C" ucp_status ucp_local_update(ucp_inst* in, int32_t n, double tau) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (n < 0 || !std::isfinite(tau))
        return arg_error("ucp_local_update", "n must be >= 0 and tau finite");
    if (!local_update_smem(in->g))
        return arg_error("ucp_local_update", "w grid too long for the local update");
    return inst_local_update(in, n, tau);
}

extern "C" ucp_status ucp_solve(ucp_inst* in, const ucp_solve_params* sp,
                                ucp_solve_report* rep, double* J_phase, int32_t* NL_rounds) {
    if (!in || !sp) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (sp->N < 2 || sp->max_rounds < 0 || !(sp->precision >= 0.0) ||
        !std::isfinite(sp->precision) || !std::isfinite(sp->tau))
        return arg_error("ucp_solve", "N >= 2, max_rounds >= 0, finite precision >= 0 "
                                      "and finite tau required");
    if (!local_update_smem(in->g))
        return arg_error("ucp_solve", "w grid too long for the local update");
    return inst_solve(in, *sp, rep, J_phase, NL_rounds);
}

extern "C" ucp_status ucp_eval_J(ucp_inst* in, double* J_out) {
    if (!in || !J_out) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    double J = 0.0;
    ucp_status st = inst_read(in, in->d.J + in->sweeps_done, &J, sizeof(double));
    if (st == UCP_OK) *J_out = J;
    return st;
}

extern "C" ucp_status ucp_J_history(ucp_inst* in, double* out, uint64_t n,
                                    uint64_t* n_written) {
    if (!in || (!out && n)) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    uint64_t m = (uint64_t)in->sweeps_done + 1;
    if (n < m) m = n;
    ucp_status st = m ? inst_read(in, in->d.J, out, m * sizeof(double)) : inst_sync(in);
    if (st == UCP_OK && n_written) *n_written = m;
    return st;
}

extern "C" ucp_status ucp_get_controllers(ucp_inst* in, double* f, uint64_t n_x,
                                          double* u1, uint64_t n_y,
                                          int32_t as_paper_u0, int32_t* idx) {
    if (!in) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if ((f || idx) && n_x != (uint64_t)in->g.n_x) {
        set_error("ucp_get_controllers: %s%s", "n_x does not match", "");
        return UCP_E_ARG;
    }
    if (u1 && n_y != (uint64_t)in->g.n_y) {
        set_error("ucp_get_controllers: %s%s", "n_y does not match", "");
        return UCP_E_ARG;
    }
    return inst_get(in, f, u1, as_paper_u0, idx);
}

extern "C" ucp_status ucp_set_controllers(ucp_inst* in, const double* f,
                                          uint64_t n_x, const double* u1,
                                          uint64_t n_y) {
    if (!in || !f || n_x != (uint64_t)in->g.n_x ||
        (u1 && n_y != (uint64_t)in->g.n_y)) {
        set_error("ucp_set_controllers: %s%s", "bad buffer or size", "");
        return UCP_E_ARG;
    }
    if (in->poisoned) return UCP_E_STATE;
    for (uint64_t i = 0; i < n_x; ++i)
        if (!(fabs(f[i] / in->g.delta) * (double)in->g.one < 4.0e15)) {
            set_error("ucp_set_controllers: %s%s", "f value out of range", "");
            return UCP_E_ARG;
        }
    return inst_set(in, f, u1);
}

extern "C" ucp_status ucp_destroy(ucp_inst* in) {
    if (!in) return UCP_E_ARG;
    cudaStreamSynchronize(in->stream);
    inst_release(in);
    delete in;
    return UCP_OK;
}

extern "C" ucp_status ucp_profile(ucp_inst* in, int32_t enable) {
    if (!in) return UCP_E_ARG;
    return prof_enable(&in->prof, in->stream, enable != 0);
}

extern "C" int32_t ucp_kernel_times(ucp_inst* in, const char** names,
                                    int64_t* launches, double* total_ms,
                                    int32_t cap) {
    if (!in) return -1;
    return prof_collect(&in->prof, names, launches, total_ms, cap);
}

extern "C" ucp_status ucp_tie_recosts(ucp_inst* in, int64_t* out) {
    if (!in || !out) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    if (in->g.sc_fast) {   // problem 1's fast mode counts its exact re-costs
        unsigned long long v = 0;
        ucp_status st = inst_read(in, in->d.sc_consts + 2, &v, sizeof(v));
        if (st == UCP_OK) *out = (int64_t)v;
        return st;
    }
    if (!in->fast) { *out = 0; return UCP_OK; }
    int32_t v = 0;
    ucp_status st = inst_read(in, in->fv.n_exact, &v, sizeof(v));
    if (st == UCP_OK) *out = v;
    return st;
}

extern "C" ucp_status ucp_test_tc_skip_copy(ucp_inst* in, int32_t on) {
    if (!in || on < 0 || on > 2) return UCP_E_ARG;
    if (in->poisoned || !in->fast) return UCP_E_STATE;
    const int32_t v = on;
    cudaMemcpyAsync(in->fv.tc_err + 1, &v, sizeof(v), cudaMemcpyHostToDevice, in->stream);
    return inst_sync(in);
}

extern "C" ucp_status ucp_get_tables(ucp_inst* in, double* P, double* Q, double* R,
                                     int64_t n_pos, float* bound, int64_t n_cols,
                                     int64_t* sizes) {
    if (!in || !sizes) return UCP_E_ARG;
    if (in->poisoned || !in->fast) return UCP_E_STATE;
    const FastView& f = in->fv;
    sizes[0] = f.n_pos;
    sizes[1] = f.tc_na;
    sizes[2] = f.c_lo;
    sizes[3] = f.jlo;
    const bool want_tab = P || Q || R;
    if ((want_tab && (!P || !Q || !R || n_pos < f.n_pos)) || (bound && n_cols < f.tc_na)) {
        set_error("ucp_get_tables: %s%s", "NULL table buffer or buffers shorter than the ",
                  "instance's tables");
        return UCP_E_ARG;
    }
    std::vector<float2> h(want_tab ? (size_t)f.n_pos * 3 : 0);
    if (want_tab) {
        const dfloat* src[3] = {f.P, f.Q, f.R};
        for (int k = 0; k < 3; ++k)
            cudaMemcpyAsync(h.data() + (size_t)k * f.n_pos, src[k], 8 * (size_t)f.n_pos,
                            cudaMemcpyDeviceToHost, in->stream);
    }
    if (bound)
        cudaMemcpyAsync(bound, f.tc_bt, 4 * (size_t)f.tc_na, cudaMemcpyDeviceToHost,
                        in->stream);
    const ucp_status st = inst_sync(in);
    if (st != UCP_OK) return st;
    double* dst[3] = {P, Q, R};
    if (want_tab)
        for (int k = 0; k < 3; ++k)
            for (int64_t p = 0; p < f.n_pos; ++p) {
                const float2 v = h[(size_t)k * f.n_pos + p];
                dst[k][p] = (double)v.x + (double)v.y;
            }
    return UCP_OK;
}

extern "C" ucp_status ucp_work_counters(ucp_inst* in, int64_t* out, int32_t n) {
    if (!in || n < 0 || n > UCP_N_COUNTERS || (n > 0 && !out)) return UCP_E_ARG;
    if (in->poisoned) return UCP_E_STATE;
    int32_t r = 0, t2 = 0;
    int64_t p[4] = {0, 0, 0, 0};
    if (in->fast) {
        cudaMemcpyAsync(&r, in->fv.n_exact, 4, cudaMemcpyDeviceToHost, in->stream);
        cudaMemcpyAsync(&t2, in->fv.n_tier2, 4, cudaMemcpyDeviceToHost, in->stream);
        ucp_status st = inst_read(in, in->fv.n_pairs, p, sizeof(p));
        if (st != UCP_OK) return st;
    }
    const int64_t all[UCP_N_COUNTERS] = {r, p[0], p[1], p[2], p[3], t2};
    for (int32_t k = 0; k < n; ++k) out[k] = all[k];
    return UCP_OK;
}
