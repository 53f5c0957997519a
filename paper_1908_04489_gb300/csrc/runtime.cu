// runtime.cu -- instance lifecycle and the sweep driver (host side).
//
// Sweep order (Algorithm 1's partial-exhaustion phase for u0, then the
// closed-form u1 update, then J; Section IV-A's Jacobi parallelism):
//   search(f_pre, U) -> f ; U <- E[x1 | y1] ; S at the coarse list and at f
//   under the new U ; J.
#include <math.h>

#include <vector>
#include <string.h>

#include "ucp_fast.cuh"
#include "ucp_runtime.h"
#include "batch_set.h"
#include "fixed_sum.cuh"

namespace ucp {

// ---- event timers -------------------------------------------------------

int Prof::begin(const char* name, cudaEvent_t* a) {
    if (!on) return -1;
    int k = -1;
    for (size_t s = 0; s < stats.size(); ++s)
        if (strcmp(stats[s].name, name) == 0) { k = (int)s; break; }
    if (k < 0) {
        stats.push_back({name, 0, 0.0});
        k = (int)stats.size() - 1;
    }
    if (pending.size() >= 4096) drain();
    if (pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        pool.push_back(e);
    }
    *a = pool.back();
    pool.pop_back();
    cudaEventRecord(*a, stream);
    return k;
}

void Prof::end(int stat, cudaEvent_t a) {
    if (stat < 0) return;
    cudaEvent_t b;
    if (pool.empty()) {
        if (cudaEventCreate(&b) != cudaSuccess) { pool.push_back(a); return; }
    } else {
        b = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(b, stream);
    pending.push_back({stat, a, b});
}

void Prof::drain() {
    if (pending.empty()) return;
    cudaStreamSynchronize(stream);
    for (auto& p : pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            stats[p.stat].launches += 1;
            stats[p.stat].ms += ms;
        }
        pool.push_back(p.a);
        pool.push_back(p.b);
    }
    pending.clear();
}

Prof::~Prof() {
    for (auto& p : pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
}

ucp_status prof_enable(Prof* p, cudaStream_t s, bool on) {
    p->drain();
    p->stream = s;
    p->on = on;
    p->stats.clear();
    return UCP_OK;
}

int prof_collect(Prof* p, const char** names, int64_t* launches, double* ms,
                 int cap) {
    p->drain();
    int n = (int)p->stats.size();
    for (int k = 0; k < n && k < cap; ++k) {
        if (names) names[k] = p->stats[k].name;
        if (launches) launches[k] = p->stats[k].launches;
        if (ms) ms[k] = p->stats[k].ms;
    }
    return n;
}

#define UCP_LAUNCH(in, NAME, CALL)                                  \
    do {                                                            \
        cudaEvent_t ucp_ev_a_;                                      \
        const int ucp_k_ = (in)->prof.begin(NAME, &ucp_ev_a_);      \
        CALL;                                                       \
        (in)->prof.end(ucp_k_, ucp_ev_a_);                          \
    } while (0)

// ---- device memory --------------------------------------------------------

static void* raw_alloc(ucp_ctx* ctx, size_t n) {
    void* p = nullptr;
    if (ctx && ctx->alloc) {
        p = ctx->alloc(n, ctx->user);
    } else if (cudaMalloc(&p, n) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void raw_free(ucp_ctx* ctx, void* p) {
    if (ctx && ctx->free_fn) ctx->free_fn(p, ctx->user);
    else cudaFree(p);
}

bool Arena::reserve(size_t n) {
    if (slab) return false;
    n = (n + 255) & ~(size_t)255;
    slab = (char*)raw_alloc(ctx, n);
    if (!slab) return false;
    slab_size = n;
    slab_used = 0;
    slab_owned = true;
    bytes += n;
    return true;
}

void Arena::adopt(void* p, size_t n) {
    if (slab || !p) return;
    slab = (char*)p;
    slab_size = n;
    slab_used = 0;
    slab_owned = false;
    bytes += n;
}

void* Arena::get(size_t n) {
    n = (n + 255) & ~(size_t)255;
    if (slab && slab_used + n <= slab_size) {
        void* p = slab + slab_used;
        slab_used += n;
        return p;
    }
    void* p = raw_alloc(ctx, n);
    if (p) { ptrs.push_back(p); bytes += n; }
    return p;
}

void Arena::put(void* p) {
    if (slab && (char*)p >= slab && (char*)p < slab + slab_size) return;
    for (size_t k = 0; k < ptrs.size(); ++k)
        if (ptrs[k] == p) {
            raw_free(ctx, p);
            ptrs.erase(ptrs.begin() + k);
            return;
        }
}

void Arena::release_all() {
    for (void* p : ptrs) raw_free(ctx, p);
    ptrs.clear();
    if (slab && slab_owned) raw_free(ctx, slab);
    slab = nullptr;
    slab_size = slab_used = 0;
    slab_owned = false;
    bytes = 0;
}

// ---- instance -------------------------------------------------------------

static ucp_status check(ucp_inst* in, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        in->poisoned = true;
        set_error("%s: %s", where, cudaGetErrorString(e));
        return UCP_E_CUDA;
    }
    return UCP_OK;
}

static ucp_status refresh_costs(ucp_inst* in, int slot) {
    const Geom& g = in->g;
    DevState& d = in->d;
    UCP_LAUNCH(in, "udiff", launch_udiff(g, d, in->stream));
    // S at the coarse candidates is shared by every x0 point in problem 0;
    // problem 1's estimation error depends on x0 and is formed in the search
    if (g.problem == 0)
        UCP_LAUNCH(in, "S_coarse", launch_S_list(g, d, d.coarse, g.n_coarse, d.Sc, in->stream, 0));
    UCP_LAUNCH(in, "S_f", launch_S_list(g, d, d.nu[in->cur], g.n_x, d.Sf, in->stream, 1));
    UCP_LAUNCH(in, "J", launch_J_plain(g, d, in->cur, slot, in->stream));
    return check(in, "refresh");
}

ucp_status grow_history(ucp_inst* in, long long need) {
    if (need <= in->hist_cap) return UCP_OK;
    long long cap = in->hist_cap;
    while (cap < need) cap *= 2;
    double* nh = (double*)in->arena.get(sizeof(double) * (size_t)cap);
    if (!nh) {
        set_error("%s%s", "J history: out of device memory", "");
        return UCP_E_NOMEM;
    }
    cudaMemcpyAsync(nh, in->d.J, sizeof(double) * (size_t)(in->sweeps_done + 1),
                    cudaMemcpyDeviceToDevice, in->stream);
    if (cudaStreamSynchronize(in->stream) != cudaSuccess) return check(in, "history");
    in->arena.put(in->d.J);
    in->d.J = nh;
    in->hist_cap = cap;
    in->bytes = in->arena.bytes;
    return UCP_OK;
}

static size_t rnd(size_t n) { return (n + 255) & ~(size_t)255; }

size_t inst_bytes(const Geom& g, int precision) {
    const size_t nx = (size_t)g.n_x, ny = (size_t)g.n_y, nw = (size_t)g.n_w;
    const size_t nc = (size_t)g.n_coarse;
    size_t b = 6 * rnd(8 * nx) + rnd(4 * nx) + 2 * rnd(8 * ny) + rnd(8 * nw) +
               2 * rnd(8 * nc) + rnd(8 * 64) + rnd(8 * 4096);
    if (g.sc_fast) b += rnd(8 * 3 * (size_t)(g.n_y + g.n_w + 2)) + rnd(8 * 4) + rnd(8 * nx);
    if (precision == 1 && g.problem == 0) {
        FastPlan fp;
        fast_plan(g, &fp);
        size_t tcs[7];
        b += 6 * rnd(8 * (size_t)fp.n_pos) + rnd(4 * (size_t)fp.n_pos) + rnd(8 * (size_t)fp.n_e) +
             3 * rnd(8 * nw) + rnd(8 * nx) + rnd(8 * kConstTab) +
             rnd(8 * (size_t)fp.J_blocks) + rnd(8) + 3 * rnd(4) + rnd(kDeferRecBytes * nx) + rnd(32) +
             tc_bytes(fp, 256, tcs) + rnd(4) +
             u1_scratch_bytes(g, fp, 256);
    }
    return b;
}

// Largest |f| the search can produce from the current state, and |U|.
static double value_bound(const Geom& g, double fmax) {
    const double reach = (double)(g.hr + 2 * g.q) * g.delta;
    const double x = (double)g.hx * g.delta;
    double b = reach > x ? reach : x;
    return b > fmax ? b : fmax;
}

// Error-bound coefficients of the screened table costs (kernels_fast.cu).
static void fast_bounds(ucp_inst* in, double B) {
    const Geom& g = in->g;
    FastView& f = in->fv;
    const double u = 0x1p-53, uf2 = 0x1p-48;
    // the plain path's sum in the fixed order (a term passes through at most
    // 31 additions in its chunk and one per level); the tables' own error and
    // the rounding of the cell quadratic are bounded per cell on the device
    const double levels = ceil(log2((double)sum_chunks(g.n_w) + 1.0));
    const double ser = (kSumChunk - 1 + levels + 1) * u;
    const double rel = ser;
    f.beta_rel = (float)(1.25 * rel);
    // rounding of grid positions, of E = U - y and of the residuals of both
    // evaluations: |d(residual)| <= u A
    const double W = (double)g.hw * g.delta;
    const double y0 = (double)(f.jlo - g.hy) * g.delta;
    const double y1 = (double)(f.jlo + f.n_e - g.hy) * g.delta;
    const double Y = fabs(y0) > fabs(y1) ? fabs(y0) : fabs(y1);
    const double A = 3.0 * W + 4.0 * Y + 9.0 * B + 8.0;
    f.beta_abs = (float)(1.25 * u * A);
    const double X = (double)g.hx * g.delta;
    f.beta_ctl = (float)(4.0 * u * (2.0 * B + X) * g.k);
    // direct quadrature (second screening tier): the plain path's sum
    // error, the double-float term products (24 uf^2), 8-term double-float
    // blocks (16 uf^2) and the FP64 sum of the blocks
    f.beta2_rel = (float)(1.25 * (ser + 8.0 * u + 40.0 * uf2 +
                                  ((double)g.n_w / 16.0 + 8.0) * u));
    f.w_half = (float)W;
    f.y_abs = (float)Y * (1.0f + 0x1p-20f);
}

static ucp_status fast_alloc(ucp_inst* in) {
    const Geom& g = in->g;
    FastView& f = in->fv;
    DevState& d = in->d;
    Arena& A = in->arena;
    fast_plan(g, &f);
    f.phi = d.phi;
    f.U = d.U;
    f.Ud = d.Ud;
    f.coarse = d.coarse;
    const size_t nx = (size_t)g.n_x, nw = (size_t)g.n_w;
    f.C0 = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.C1 = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.C2 = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.Cb = (float*)A.get(4 * (size_t)f.n_pos);
    f.P = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.Q = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.R = (dfloat*)A.get(8 * (size_t)f.n_pos);
    f.E = (dfloat*)A.get(8 * (size_t)f.n_e);
    f.a = (dfloat*)A.get(8 * nw);
    f.phidf = (dfloat*)A.get(8 * nw);
    f.wdf = (dfloat*)A.get(8 * nw);
    f.prior = (dfloat*)A.get(8 * nx);
    f.t64 = (dfloat*)A.get(8 * kConstTab);
    f.Jpart = (double*)A.get(8 * (size_t)f.J_blocks);
    size_t tcs[7];
    tc_bytes(f, 256, tcs);
    f.tc_h = (uint16_t*)A.get(tcs[0]);
    f.tc_he = (int32_t*)A.get(tcs[1]);
    f.tc_x = (uint16_t*)A.get(tcs[2]);
    f.tc_xe = (int32_t*)A.get(tcs[3]);
    f.tc_part = (float2*)A.get(tcs[4]);
    f.tc_bt = (float*)A.get(tcs[5]);
    f.tc_err = (int32_t*)A.get(tcs[6]);
    f.J_done = (int32_t*)A.get(4);
    f.W2_dev = (double*)A.get(8);
    f.n_exact = (int32_t*)A.get(4);
    f.n_tier2 = (int32_t*)A.get(4);
    f.defer_cnt = (int32_t*)A.get(4);
    f.defer_list = A.get(kDeferRecBytes * nx);
    f.n_pairs = (int64_t*)A.get(32);
    const bool u1_ok = u1_carve(
        g, &f, [](void* a, size_t n) { return ((Arena*)a)->get(n); }, &A);
    if (!f.C0 || !f.C1 || !f.C2 || !f.Cb || !f.P || !f.Q || !f.R || !f.E || !f.a || !f.phidf || !f.wdf ||
        !f.prior || !f.t64 || !u1_ok || !f.Jpart || !f.tc_h || !f.tc_he || !f.tc_x ||
        !f.tc_xe || !f.tc_part || !f.tc_bt || !f.tc_err || !f.J_done || !f.W2_dev ||
        !f.n_exact || !f.n_tier2 || !f.defer_cnt || !f.defer_list || !f.n_pairs) {
        set_error("%s%s", "ucp_create: out of device memory (fast path)", "");
        return UCP_E_NOMEM;
    }
    if (!tc_encode_maps(&f)) {
        set_error("%s%s", "ucp_create: TMA tensor maps of the table signals ",
                  "could not be encoded");
        return UCP_E_CUDA;
    }
    const double step = ldexp(g.delta, -g.shift);
    const dfloat sd = df_from_double(step), kd = df_from_double(g.kk);
    f.step_hi = sd.hi;
    f.step_lo = sd.lo;
    const dfloat dd = df_from_double(g.delta);
    f.delta_hi = dd.hi;
    f.delta_lo = dd.lo;
    f.kk_hi = kd.hi;
    f.kk_lo = kd.lo;
    f.k_f = (float)g.k * 1.0000001f;
    f.inv_one_f = (float)ldexp(1.0, -g.shift);
    in->fbound = 0.0;
    fast_bounds(in, value_bound(g, 0.0));
    return UCP_OK;
}

static ucp_status fast_refresh(ucp_inst* in, int slot) {
    const Geom& g = in->g;
    DevState& d = in->d;
    launch_tables(g, in->fv, d.U, d.Ud, in->stream, &in->prof);
    launch_J_fast(g, in->fv, d.px, d.nu[in->cur], d.J + slot, in->stream, &in->prof);
    return check(in, "refresh");
}

ucp_status inst_init(ucp_inst* in, ucp_ctx* ctx, const ucp_params& p,
                     const Geom& g, cudaStream_t stream, bool own_setup, void* slab) {
    in->ctx = ctx;
    in->cfg = ctx->cfg;
    in->params = p;
    in->params.init_table = nullptr;
    in->g = g;
    in->arena.ctx = ctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return check(in, "set device");
    in->stream = stream;  // NULL: the default stream
    in->prof.stream = in->stream;
    in->hist_cap = 64;
    DevState& d = in->d;
    Arena& A = in->arena;
    const size_t nx = (size_t)g.n_x, ny = (size_t)g.n_y, nw = (size_t)g.n_w;
    // every buffer below from one allocation (inst_bytes counts them all)
    if (slab) A.adopt(slab, inst_bytes(g, p.precision));
    else A.reserve(inst_bytes(g, p.precision));
    d.px = (double*)A.get(8 * nx);
    d.phi = (double*)A.get(8 * nw);
    d.U = (double*)A.get(8 * ny);
    d.Ud = (double*)A.get(8 * ny);
    d.nu[0] = (int64_t*)A.get(8 * nx);
    d.nu[1] = (int64_t*)A.get(8 * nx);
    d.coarse = (int64_t*)A.get(8 * (size_t)g.n_coarse);
    d.Sf = (double*)A.get(8 * nx);
    d.Sc = (double*)A.get(8 * (size_t)g.n_coarse);
    d.idx = (int32_t*)A.get(4 * nx);
    d.J = (double*)A.get(8 * (size_t)in->hist_cap);
    d.scratch = (double*)A.get(8 * 4096);
    d.table = (double*)A.get(8 * nx);
    if (g.sc_fast) {
        d.sc_tab = (double*)A.get(8 * 3 * (size_t)(g.n_y + g.n_w + 2));
        d.sc_consts = (double*)A.get(8 * 4);
        d.sc_f = (double*)A.get(8 * nx);
    }
    if (!d.px || !d.phi || !d.U || !d.Ud || !d.nu[0] || !d.nu[1] || !d.coarse ||
        !d.Sf || !d.Sc || !d.idx || !d.J || !d.scratch || !d.table ||
        (g.sc_fast && (!d.sc_tab || !d.sc_consts || !d.sc_f))) {
        set_error("%s%s", "ucp_create: out of device memory", "");
        return UCP_E_NOMEM;
    }
    in->fast = p.precision == 1 && p.problem == 0;
    if (g.sc_fast) cudaMemsetAsync(d.sc_consts, 0, 8 * 4, stream);
    if (in->fast) {
        if (tc_init_attributes() != cudaSuccess) return check(in, "tensor-core kernel attributes");
        if (u1_init_attributes() != cudaSuccess) return check(in, "u1 kernel attributes");
        ucp_status st = fast_alloc(in);
        if (st != UCP_OK) return st;
    }
    in->bytes = A.bytes;
    cudaStream_t s = in->stream;
    if (in->fast && !own_setup) {
        // the set-up kernels and the first step come from batched launches
        // (batchset_setup); only the host-side state and the table copy here
        if (p.init_kind == 2) {
            double fm = 0.0;
            for (int64_t i = 0; i < g.n_x; ++i)
                fm = fabs(p.init_table[i]) > fm ? fabs(p.init_table[i]) : fm;
            in->fbound = fm;
            fast_bounds(in, value_bound(g, fm));
            cudaMemcpyAsync(d.table, p.init_table, 8 * nx, cudaMemcpyHostToDevice, s);
            // the caller's host buffer must not be read after we return
            if (cudaStreamSynchronize(s) != cudaSuccess) return check(in, "init copy");
        }
        in->cur = 0;
        in->sweeps_done = 0;
        return check(in, "set-up");
    }
    UCP_LAUNCH(in, "weights", launch_weights(g, d, s));
    UCP_LAUNCH(in, "coarse", launch_coarse_list(g, d, s));
    if (in->fast) {
        UCP_LAUNCH(in, "fast_setup", launch_fast_setup(g, in->fv, s));
        UCP_LAUNCH(in, "tc_setup", launch_tc_setup(g, in->fv, s));
        cudaMemsetAsync(in->fv.n_exact, 0, 4, s);
        cudaMemsetAsync(in->fv.n_tier2, 0, 4, s);
        cudaMemsetAsync(in->fv.defer_cnt, 0, 4, s);
        cudaMemsetAsync(in->fv.J_done, 0, 4, s);
        cudaMemsetAsync(in->fv.tc_err, 0, 8, s);   // the error flag and the test hook
        cudaMemsetAsync(in->fv.n_pairs, 0, 32, s);
        if (p.init_kind == 2) {
            double fm = 0.0;
            for (int64_t i = 0; i < g.n_x; ++i)
                fm = fabs(p.init_table[i]) > fm ? fabs(p.init_table[i]) : fm;
            in->fbound = fm;
            fast_bounds(in, value_bound(g, fm));
        }
    }
    if (p.init_kind == 2) {
        cudaMemcpyAsync(d.table, p.init_table, 8 * nx, cudaMemcpyHostToDevice, s);
        UCP_LAUNCH(in, "init", launch_table_to_lattice(g, d.table, d.nu[0], s));
        // the caller's host buffer must not be read after we return
        if (cudaStreamSynchronize(s) != cudaSuccess) return check(in, "init copy");
    } else {
        UCP_LAUNCH(in, "init", launch_init(g, d, p.init_kind, 0, s));
    }
    cudaMemsetAsync(d.idx, 0xff, 4 * nx, s);
    in->cur = 0;
    in->sweeps_done = 0;
    if (in->fast) {
        launch_mmse_fast(g, in->fv, d.nu[0], d.U, s, &in->prof);
        return fast_refresh(in, 0);
    }
    UCP_LAUNCH(in, "mmse", launch_mmse_plain(g, d, 0, s));
    return refresh_costs(in, 0);
}

// Fast-path sweeps replayed from captured graphs (non-default stream,
// profiler off).  Returns false when the graphs are not available (the
// caller launches kernel by kernel); the kernels are the same computations
// either way, so the results are too.
static void solo_drop(ucp_inst* in) {
    for (int c = 0; c < 2; ++c) {
        if (in->solo_graph[c]) cudaGraphExecDestroy(in->solo_graph[c]);
        in->solo_graph[c] = nullptr;
    }
    in->solo_tried = false;
}

// The one-member batch set that the fast path's sweeps launch the u1 step,
// the tables and J over (built on first use; false if it cannot be).
static bool solo_ensure(ucp_inst* in) {
    if (in->solo) return true;
    if (in->solo_failed) return false;
    in->solo = new BatchSet();
    in->solo->arena = &in->arena;
    in->solo->cfg = in->cfg;
    std::vector<ucp_inst*> one{in};
    if (batchset_build(*in->solo, one, in->stream) != UCP_OK) {
        cudaGetLastError();
        delete in->solo;
        in->solo = nullptr;
        in->solo_failed = true;
        return false;
    }
    return true;
}

static bool solo_sweeps(ucp_inst* in, int n) {
    if (!in->stream || in->prof.on) return false;
    if (!in->solo_tried) {
        in->solo_tried = true;
        if (!solo_ensure(in)) return false;
        for (int c = 0; c < 2; ++c) {
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(in->stream, cudaStreamCaptureModeThreadLocal) !=
                cudaSuccess)
                break;
            launch_search_fast(in->g, in->fv, in->d.nu[c], in->d.nu[c ^ 1], in->d.idx,
                               in->stream, 0, -1, &in->cfg);
            launch_batch_rest(in->solo->bl, in->stream);
            if (cudaStreamEndCapture(in->stream, &graph) == cudaSuccess && graph) {
                if (cudaGraphInstantiate(&in->solo_graph[c], graph, 0) != cudaSuccess)
                    in->solo_graph[c] = nullptr;
                cudaGraphDestroy(graph);
            }
        }
        cudaGetLastError();  // a failed capture falls back to plain launches
    }
    if (!in->solo_graph[0] || !in->solo_graph[1]) return false;
    std::vector<ucp_inst*> one{in};
    if (batchset_refresh(*in->solo, one, in->stream) != UCP_OK) return false;
    for (int k = 0; k < n; ++k) {
        cudaGraphLaunch(in->solo_graph[in->cur], in->stream);
        in->cur ^= 1;
    }
    in->sweeps_done += n;
    return true;
}

// The same launches as the graphs, kernel by kernel (default stream, or the
// profiler on: each kernel group timed by events).
static bool solo_launches(ucp_inst* in, int n) {
    if (!solo_ensure(in)) return false;
    std::vector<ucp_inst*> one{in};
    if (batchset_refresh(*in->solo, one, in->stream) != UCP_OK) return false;
    Prof* prof = in->prof.on ? &in->prof : nullptr;
    for (int k = 0; k < n; ++k) {
        UCP_LAUNCH(in, "search", launch_search_fast(in->g, in->fv, in->d.nu[in->cur],
                                                    in->d.nu[in->cur ^ 1], in->d.idx,
                                                    in->stream, 0, -1, &in->cfg));
        launch_batch_rest(in->solo->bl, in->stream, prof);
        in->cur ^= 1;
    }
    in->sweeps_done += n;
    return true;
}

ucp_status inst_set_launch_cfg(ucp_inst* in, const LaunchCfg& cfg) {
    in->cfg = cfg;
    solo_drop(in);
    if (in->solo) {
        in->solo->cfg = cfg;
        std::vector<ucp_inst*> one{in};
        if (batchset_build(*in->solo, one, in->stream) != UCP_OK) return check(in, "launch config");
    }
    return UCP_OK;
}

ucp_status inst_sweep(ucp_inst* in, int n) {
    if (n == 0) return UCP_OK;
    ucp_status st = grow_history(in, in->sweeps_done + 1 + n);
    if (st != UCP_OK) return st;
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    if (in->fast && solo_sweeps(in, n)) return check(in, "sweep");
    if (in->fast && solo_launches(in, n)) return check(in, "sweep");
    if (in->fast) {
        for (int k = 0; k < n; ++k) {
            UCP_LAUNCH(in, "search", launch_search_fast(g, in->fv, d.nu[in->cur],
                                                        d.nu[in->cur ^ 1], d.idx, s, 0, -1,
                                                        &in->cfg));
            in->cur ^= 1;
            launch_mmse_fast(g, in->fv, d.nu[in->cur], d.U, s, &in->prof);
            in->sweeps_done += 1;
            st = fast_refresh(in, (int)in->sweeps_done);
            if (st != UCP_OK) return st;
        }
        return UCP_OK;
    }
    for (int k = 0; k < n; ++k) {
        UCP_LAUNCH(in, "search", launch_search_plain(g, d, in->cur, s));
        in->cur ^= 1;
        UCP_LAUNCH(in, "mmse", launch_mmse_plain(g, d, in->cur, s));
        in->sweeps_done += 1;
        st = refresh_costs(in, (int)in->sweeps_done);
        if (st != UCP_OK) return st;
    }
    return UCP_OK;
}

ucp_status inst_local_update(ucp_inst* in, int n, double tau) {
    if (n == 0) return UCP_OK;
    ucp_status st = grow_history(in, in->sweeps_done + 1 + n);
    if (st != UCP_OK) return st;
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    for (int k = 0; k < n; ++k) {
        cudaError_t e = cudaSuccess;
        UCP_LAUNCH(in, "local_update", e = launch_local_update(g, d.phi, d.U, d.nu[in->cur],
                                                               d.nu[in->cur ^ 1], tau, s));
        if (e != cudaSuccess) return check(in, "local update");
        in->cur ^= 1;
        in->sweeps_done += 1;
        if (in->fast) {
            launch_mmse_fast(g, in->fv, d.nu[in->cur], d.U, s, &in->prof);
            st = fast_refresh(in, (int)in->sweeps_done);
        } else {
            UCP_LAUNCH(in, "mmse", launch_mmse_plain(g, d, in->cur, s));
            st = refresh_costs(in, (int)in->sweeps_done);
        }
        if (st != UCP_OK) return st;
    }
    return check(in, "local update");
}

// One sweep split over several processes (Section IV-A: the x0 points are
// independent for a fixed controller).  Part: the search of points i0..i1-1
// from the current state into the next buffer, their new values copied to
// host memory.  Finish: the full new controller (every part) from host
// memory into the next buffer, then the rest of the sweep (u1 step, tables
// or costs, J).  Part over every point + finish == one ucp_sweep.
ucp_status inst_sweep_part(ucp_inst* in, int64_t i0, int64_t i1, double* f_host) {
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    if (in->fast) {
        UCP_LAUNCH(in, "search", launch_search_fast(g, in->fv, d.nu[in->cur],
                                                    d.nu[in->cur ^ 1], d.idx, s, i0, i1,
                                                    &in->cfg));
    } else {
        UCP_LAUNCH(in, "search", launch_search_plain(g, d, in->cur, s, i0, i1));
    }
    const size_t n = (size_t)(i1 - i0);
    if (n == 0) return check(in, "sweep part");
    std::vector<int64_t> nu(n);
    ucp_status st = inst_read(in, d.nu[in->cur ^ 1] + i0, nu.data(), 8 * n);
    if (st != UCP_OK) return st;
    for (size_t k = 0; k < n; ++k) f_host[k] = ldexp((double)nu[k] * g.delta, -g.shift);
    return UCP_OK;
}

ucp_status inst_sweep_finish(ucp_inst* in, const double* f_host) {
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    ucp_status st = grow_history(in, in->sweeps_done + 2);
    if (st != UCP_OK) return st;
    cudaMemcpyAsync(d.table, f_host, 8 * (size_t)g.n_x, cudaMemcpyHostToDevice, s);
    UCP_LAUNCH(in, "init", launch_table_to_lattice(g, d.table, d.nu[in->cur ^ 1], s));
    // the caller's host buffer must not be read after we return
    if (cudaStreamSynchronize(s) != cudaSuccess) return check(in, "sweep finish copy");
    in->cur ^= 1;
    in->sweeps_done += 1;
    if (in->fast) {
        launch_mmse_fast(g, in->fv, d.nu[in->cur], d.U, s, &in->prof);
        return fast_refresh(in, (int)in->sweeps_done);
    }
    UCP_LAUNCH(in, "mmse", launch_mmse_plain(g, d, in->cur, s));
    return refresh_costs(in, (int)in->sweeps_done);
}

int alg1_split(double I_L, double I_P, int N, int n_l) {
    if (!(I_L + I_P > 0.0)) return n_l;
    const double r = floor(I_L * (double)N / (I_L + I_P));
    return r < 1.0 ? 1 : (r > (double)(N - 1) ? N - 1 : (int)r);
}

// Algorithm 1 (Sections III-B to III-D): rounds of N_L local-update
// iterations and N_P partial-exhaustion iterations (sweeps), J read after
// each phase, I_L and I_P the absolute changes of J over the two phases,
// the next split proportional to them (each phase at least once), until
// I_L + I_P <= p.  Starts from the instance's current state.
ucp_status inst_solve(ucp_inst* in, const ucp_solve_params& sp, ucp_solve_report* rep,
                      double* J_phase, int32_t* NL_rounds) {
    auto J_now = [&](double* J) {
        return inst_read(in, in->d.J + in->sweeps_done, J, sizeof(double));
    };
    double Jc = 0.0;
    ucp_status st = J_now(&Jc);
    if (st != UCP_OK) return st;
    if (J_phase) J_phase[0] = Jc;
    const int N = sp.N;
    double IL = sp.precision, IP = sp.precision;
    int NL = N / 2, NP = N - NL, rounds = 0, nloc = 0, nexh = 0;
    while (IL + IP > sp.precision && rounds < sp.max_rounds) {
        if (NL_rounds) NL_rounds[rounds] = NL;
        const double J0 = Jc;
        if ((st = inst_local_update(in, NL, sp.tau)) != UCP_OK) return st;
        nloc += NL;
        if ((st = J_now(&Jc)) != UCP_OK) return st;
        IL = fabs(J0 - Jc);
        if (J_phase) J_phase[1 + 2 * rounds] = Jc;
        const double J1 = Jc;
        if ((st = inst_sweep(in, NP)) != UCP_OK) return st;
        nexh += NP;
        if ((st = J_now(&Jc)) != UCP_OK) return st;
        IP = fabs(J1 - Jc);
        if (J_phase) J_phase[2 + 2 * rounds] = Jc;
        NL = alg1_split(IL, IP, N, NL);
        NP = N - NL;
        ++rounds;
    }
    if (rep) {
        rep->rounds = rounds;
        rep->converged = IL + IP <= sp.precision;
        rep->local_iters = nloc;
        rep->exhaustion_iters = nexh;
        rep->N_L = NL;
        rep->N_P = NP;
        rep->J = Jc;
        rep->I_L = IL;
        rep->I_P = IP;
    }
    return UCP_OK;
}

ucp_status inst_sync(ucp_inst* in) {
    if (cudaStreamSynchronize(in->stream) != cudaSuccess) return check(in, "sync");
    if (in->fast) {
        int32_t e = 0;
        if (cudaMemcpy(&e, in->fv.tc_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return check(in, "sync");
        if (e) {
            in->poisoned = true;
            set_error("%s%s", "sync: a tensor-core wait timed out", "");
            return UCP_E_TIMEOUT;
        }
    }
    return check(in, "sync");
}

ucp_status inst_read(ucp_inst* in, const void* dev, void* host, size_t bytes) {
    cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, in->stream);
    return inst_sync(in);
}

ucp_status inst_get(ucp_inst* in, double* f, double* u1, int as_u0, int32_t* idx) {
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    if (f) {
        UCP_LAUNCH(in, "f_values", launch_f_values(g, d.nu[in->cur], nullptr, d.table, as_u0, s));
        cudaMemcpyAsync(f, d.table, 8 * (size_t)g.n_x, cudaMemcpyDeviceToHost, s);
    }
    if (u1) cudaMemcpyAsync(u1, d.U, 8 * (size_t)g.n_y, cudaMemcpyDeviceToHost, s);
    if (idx) cudaMemcpyAsync(idx, d.idx, 4 * (size_t)g.n_x, cudaMemcpyDeviceToHost, s);
    return inst_sync(in);
}

ucp_status inst_set(ucp_inst* in, const double* f, const double* u1) {
    const Geom& g = in->g;
    DevState& d = in->d;
    cudaStream_t s = in->stream;
    if (in->stream) cudaStreamSynchronize(in->stream);
    solo_drop(in);   // the captured searches hold the screening bounds by value
    if (in->fast) {
        double fm = in->fbound;
        for (int64_t i = 0; i < g.n_x; ++i) fm = fabs(f[i]) > fm ? fabs(f[i]) : fm;
        if (u1)
            for (int64_t j = 0; j < g.n_y; ++j) fm = fabs(u1[j]) > fm ? fabs(u1[j]) : fm;
        in->fbound = fm;
        fast_bounds(in, value_bound(g, fm));
    }
    cudaMemcpyAsync(d.table, f, 8 * (size_t)g.n_x, cudaMemcpyHostToDevice, s);
    UCP_LAUNCH(in, "init", launch_table_to_lattice(g, d.table, d.nu[in->cur], s));
    if (u1) {
        cudaMemcpyAsync(d.U, u1, 8 * (size_t)g.n_y, cudaMemcpyHostToDevice, s);
    } else if (in->fast) {
        launch_mmse_fast(g, in->fv, d.nu[in->cur], d.U, s, &in->prof);
    } else {
        UCP_LAUNCH(in, "mmse", launch_mmse_plain(g, d, in->cur, s));
    }
    cudaMemsetAsync(d.idx, 0xff, 4 * (size_t)g.n_x, s);
    in->sweeps_done = 0;
    ucp_status st = in->fast ? fast_refresh(in, 0) : refresh_costs(in, 0);
    if (st != UCP_OK) return st;
    return inst_sync(in);  // host buffers are not read after return
}

void inst_release(ucp_inst* in) {
    if (in->stream) cudaStreamSynchronize(in->stream);
    solo_drop(in);
    delete in->solo;
    in->solo = nullptr;
    in->prof.drain();
    in->arena.release_all();
    if (in->own_stream && in->stream) cudaStreamDestroy(in->stream);
    in->stream = nullptr;
}

}  // namespace ucp
