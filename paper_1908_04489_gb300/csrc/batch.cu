// batch.cu -- many Witsenhausen instances swept together (ucp_batch_*).
//
// Instances of different sizes (k, sigma, delta, grid widths) are created as
// ordinary fast-path instances; a batched sweep then runs each kernel kind
// once for all of them, every block mapped to (instance, block of that
// instance's own grid) by a host-built table.  The sweep state lives on the
// device, so one sweep is captured once as a CUDA graph and replayed.  The
// solver arithmetic is the single-instance fast path's, kernel body for
// kernel body: each instance gets the same results alone or in a batch.
#include <string.h>

#include <vector>

#include "batch_set.h"

using namespace ucp;

struct ucp_batch {
    ucp_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<ucp_inst*> members;
    Arena arena;
    BatchSet bs;
    double* J_gather = nullptr;   // [2 n] device: J, then the tensor-core error flags
    bool poisoned = false;
    cudaGraphExec_t graph = nullptr;
    bool graph_tried = false;
    Prof prof;   // per-kernel events (sweeps launch kernel by kernel while on)
    SetupSet ss;
};

namespace ucp {

InstDev describe_inst(const ucp_inst* in) {
    InstDev d;
    memset(&d, 0, sizeof(d));
    d.g = in->g;
    d.f = in->fv;
    d.nu[0] = in->d.nu[0];
    d.nu[1] = in->d.nu[1];
    d.idx = in->d.idx;
    d.px = in->d.px;
    d.U = in->d.U;
    d.Ud = in->d.Ud;
    d.J = in->d.J;
    d.cur = in->cur;
    d.sweeps = (int32_t)in->sweeps_done;
    return d;
}

static int run_slot(int R) {
    return R >= 16 ? 4 : (R >= 8 ? 3 : (R >= 4 ? 2 : (R >= 2 ? 1 : 0)));
}

static int defer_blocks_per_inst(size_t n, const LaunchCfg& cfg) {
    if (cfg.defer_blocks > 0) return cfg.defer_blocks;
    return n >= 16 ? kDeferBlocksBatch : (int)(64 / n);
}

ucp_status batchset_refresh(BatchSet& bs, const std::vector<ucp_inst*>& members,
                            cudaStream_t s) {
    const size_t n = members.size();
    bs.desc.resize(n);
    for (size_t k = 0; k < n; ++k) {
        bs.desc[k] = describe_inst(members[k]);
        bs.desc[k].defer_blocks = defer_blocks_per_inst(n, bs.cfg);
    }
    if (n) cudaMemcpyAsync(bs.insts, bs.desc.data(), sizeof(InstDev) * n,
                           cudaMemcpyHostToDevice, s);
    return cudaGetLastError() == cudaSuccess ? UCP_OK : UCP_E_CUDA;
}

ucp_status batchset_build(BatchSet& bs, const std::vector<ucp_inst*>& members,
                          cudaStream_t s) {
    const size_t n = members.size();
    std::vector<BlockRef> maps[kBKinds], smap, mmaps[5], dmap;
    const int defer_blocks = defer_blocks_per_inst(n, bs.cfg);
    const int lanes = bs.cfg.search_lanes ? bs.cfg.search_lanes : kSearchLanesDefault;
    for (size_t k = 0; k < n; ++k) {
        const ucp_inst* in = members[k];
        for (int kind = 1; kind < kBKinds; ++kind) {
            const int64_t nb = batch_blocks(in->g, in->fv, kind);
            for (int64_t x = 0; x < nb; ++x) maps[kind].push_back({(int32_t)k, (int32_t)x});
        }
        const int64_t ns = search_blocks(in->g, lanes);
        for (int64_t x = 0; x < ns; ++x) smap.push_back({(int32_t)k, (int32_t)x});
        for (int x = 0; x < defer_blocks; ++x) dmap.push_back({(int32_t)k, x});
        std::vector<BlockRef>& mm = mmaps[run_slot(in->fv.run)];
        const int64_t nm = batch_mmse_blocks(in->g, in->fv);
        for (int64_t x = 0; x < nm; ++x) mm.push_back({(int32_t)k, (int32_t)x});
    }
    bs.host_maps.clear();
    size_t off[kBKinds], moff[5];
    for (int kind = 0; kind < kBKinds; ++kind) {
        off[kind] = bs.host_maps.size();
        bs.host_maps.insert(bs.host_maps.end(), maps[kind].begin(), maps[kind].end());
    }
    const size_t soff = bs.host_maps.size();
    bs.host_maps.insert(bs.host_maps.end(), smap.begin(), smap.end());
    for (int r = 0; r < 5; ++r) {
        moff[r] = bs.host_maps.size();
        bs.host_maps.insert(bs.host_maps.end(), mmaps[r].begin(), mmaps[r].end());
    }
    const size_t doff = bs.host_maps.size();
    bs.host_maps.insert(bs.host_maps.end(), dmap.begin(), dmap.end());
    // grow the device buffers (after the stream drains, as they may be in use)
    if (n > bs.insts_cap || bs.host_maps.size() > bs.maps_cap) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return UCP_E_CUDA;
        if (n > bs.insts_cap) {
            if (bs.insts) bs.arena->put(bs.insts);
            bs.insts_cap = n + n / 2 + 8;
            bs.insts = (InstDev*)bs.arena->get(sizeof(InstDev) * bs.insts_cap);
        }
        if (bs.host_maps.size() > bs.maps_cap) {
            if (bs.maps) bs.arena->put(bs.maps);
            bs.maps_cap = bs.host_maps.size() + bs.host_maps.size() / 2 + 64;
            bs.maps = (BlockRef*)bs.arena->get(sizeof(BlockRef) * bs.maps_cap);
        }
        if (!bs.insts || !bs.maps) {
            bs.insts_cap = bs.maps_cap = 0;
            return UCP_E_NOMEM;
        }
    }
    if (!bs.host_maps.empty())
        cudaMemcpyAsync(bs.maps, bs.host_maps.data(), sizeof(BlockRef) * bs.host_maps.size(),
                        cudaMemcpyHostToDevice, s);
    BatchLaunch& bl = bs.bl;
    bl.insts = bs.insts;
    bl.n_inst = (int)n;
    for (int kind = 0; kind < kBKinds; ++kind) {
        bl.map[kind] = bs.maps + off[kind];
        bl.n_blocks[kind] = (int64_t)maps[kind].size();
    }
    bl.search_map = bs.maps + soff;
    bl.search_blocks = (int64_t)smap.size();
    bl.defer_map = bs.maps + doff;
    bl.defer_blocks = (int64_t)dmap.size();
    bl.search_lanes = lanes;
    for (int r = 0; r < 5; ++r) bl.u1_threads[r] = bs.cfg.u1_threads[r];
    for (int r = 0; r < 5; ++r) {
        bl.mmse_map[r] = bs.maps + moff[r];
        bl.mmse_blocks[r] = (int64_t)mmaps[r].size();
    }
    return batchset_refresh(bs, members, s);
}

// Grow a device array of `cap` elements to hold n (after the stream drains,
// as the old one may be in use).
template <typename T>
static ucp_status grow(Arena* arena, T*& p, size_t& cap, size_t n, cudaStream_t s) {
    if (n <= cap && p) return UCP_OK;
    if (cudaStreamSynchronize(s) != cudaSuccess) return UCP_E_CUDA;
    if (p) arena->put(p);
    cap = n + n / 2 + 8;
    p = (T*)arena->get(sizeof(T) * cap);
    if (!p) {
        cap = 0;
        return UCP_E_NOMEM;
    }
    return UCP_OK;
}

ucp_status batchset_setup(SetupSet& ss, BatchSet& bs, const std::vector<ucp_inst*>& members,
                          cudaStream_t s) {
    const size_t n = members.size();
    if (n == 0) return UCP_OK;
    ss.desc.resize(n);
    std::vector<BlockRef> elem, inst, filt;
    for (size_t k = 0; k < n; ++k) {
        const ucp_inst* in = members[k];
        SetupDev& d = ss.desc[k];
        memset(&d, 0, sizeof(d));
        d.g = in->g;
        d.f = in->fv;
        d.px = in->d.px;
        d.phi = in->d.phi;
        d.coarse = in->d.coarse;
        d.scratch = in->d.scratch;
        d.nu0 = in->d.nu[0];
        d.idx = in->d.idx;
        d.table = in->d.table;
        d.init_kind = in->params.init_kind;
        init_levels(in->g, d.init_kind, &d.n7, d.lv);
        const int64_t ne = setup_elem_blocks(in->g);
        for (int64_t x = 0; x < ne; ++x) elem.push_back({(int32_t)k, (int32_t)x});
        inst.push_back({(int32_t)k, 0});
        for (int64_t x = 0; x < 2 * (int64_t)in->fv.tc_nch + 1; ++x)
            filt.push_back({(int32_t)k, (int32_t)x});
    }
    ss.host_maps.clear();
    ss.host_maps.insert(ss.host_maps.end(), elem.begin(), elem.end());
    ss.host_maps.insert(ss.host_maps.end(), inst.begin(), inst.end());
    ss.host_maps.insert(ss.host_maps.end(), filt.begin(), filt.end());
    ucp_status st = grow(ss.arena, ss.descs, ss.descs_cap, n, s);
    if (st == UCP_OK) st = grow(ss.arena, ss.maps, ss.maps_cap, ss.host_maps.size(), s);
    if (st != UCP_OK) return st;
    cudaMemcpyAsync(ss.descs, ss.desc.data(), sizeof(SetupDev) * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(ss.maps, ss.host_maps.data(), sizeof(BlockRef) * ss.host_maps.size(),
                    cudaMemcpyHostToDevice, s);
    SetupLaunch sl;
    sl.descs = ss.descs;
    sl.elem_map = ss.maps;
    sl.elem_blocks = (int64_t)elem.size();
    sl.inst_map = ss.maps + elem.size();
    sl.inst_blocks = (int64_t)inst.size();
    sl.filter_map = ss.maps + elem.size() + inst.size();
    sl.filter_blocks = (int64_t)filt.size();
    launch_batch_setup_plain(sl, s);
    launch_batch_setup_fast(sl, s);
    launch_batch_setup_tc(sl, s);
    if (cudaGetLastError() != cudaSuccess) return UCP_E_CUDA;
    // the first step: the rest of a sweep under descriptors that make it act
    // on nu[0] (the initial f) and store J in history slot 0; its last kernel
    // then leaves cur = 0 and sweeps = 0 on the device, the host-side state
    for (InstDev& d : bs.desc) {
        d.cur = 1;
        d.sweeps = -1;
    }
    cudaMemcpyAsync(bs.insts, bs.desc.data(), sizeof(InstDev) * bs.desc.size(),
                    cudaMemcpyHostToDevice, s);
    launch_batch_rest(bs.bl, s);
    if (cudaGetLastError() != cudaSuccess) return UCP_E_CUDA;
    return batchset_refresh(bs, members, s);
}

}  // namespace ucp

namespace {

ucp_status fail(ucp_batch* b, const char* where) {
    const cudaError_t e = cudaGetLastError();
    b->poisoned = true;
    set_error("%s: %s", where, cudaGetErrorString(e));
    return UCP_E_CUDA;
}

__global__ void k_gather_J(const InstDev* insts, int n, double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) {
        out[b] = insts[b].J[insts[b].sweeps];
        out[n + b] = (double)*insts[b].f.tc_err;
    }
}

}  // namespace

extern "C" UCP_API ucp_status ucp_batch_create(ucp_ctx* ctx, const ucp_params* params,
                                               int32_t n, void* stream,
                                               ucp_batch** out) {
    if (!ctx || !params || !out || n < 1) {
        set_error("ucp_batch_create: %s%s", "NULL argument or n < 1", "");
        return UCP_E_ARG;
    }
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        Geom g;
        if (const char* why = make_geom(params[k], &g)) {
            set_error("ucp_batch_create: %s%s", why, "");
            return UCP_E_ARG;
        }
        if (params[k].precision != 1 || params[k].problem != 0) {
            set_error("ucp_batch_create: %s%s", "batched instances use the fast path "
                      "(precision 1) of Witsenhausen's problem (problem 0)", "");
            return UCP_E_ARG;
        }
    }
    ucp_batch* b = new ucp_batch();
    b->ctx = ctx;
    b->stream = (cudaStream_t)stream;
    b->arena.ctx = ctx;
    // one allocation holds every member's buffers (the members carve it)
    std::vector<size_t> off((size_t)n + 1, 0);
    for (int k = 0; k < n; ++k) {
        Geom g;
        make_geom(params[k], &g);
        off[k + 1] = off[k] + ((inst_bytes(g, 1) + 255) & ~(size_t)255);
    }
    char* slab = (char*)b->arena.get(off[n]);
    if (!slab) {
        set_error("%s%s", "ucp_batch_create: out of device memory", "");
        delete b;
        return UCP_E_NOMEM;
    }
    for (int k = 0; k < n; ++k) {
        ucp_inst* in = nullptr;
        ucp_status st = inst_create(ctx, &params[k], (cudaStream_t)stream, false, &in,
                                    slab + off[k]);
        if (st != UCP_OK) {
            for (ucp_inst* m : b->members) ucp_destroy(m);
            cudaStreamSynchronize(b->stream);
            b->arena.release_all();
            delete b;
            return st;
        }
        b->members.push_back(in);
    }
    b->bs.arena = &b->arena;
    b->bs.cfg = ctx->cfg;
    b->ss.arena = &b->arena;
    b->J_gather = (double*)b->arena.get(2 * sizeof(double) * (size_t)n);
    ucp_status st = b->J_gather ? batchset_build(b->bs, b->members, b->stream) : UCP_E_NOMEM;
    // every member's set-up and first u1 update, tables and J, batched
    if (st == UCP_OK) st = batchset_setup(b->ss, b->bs, b->members, b->stream);
    if (st != UCP_OK) {
        set_error("%s%s", "ucp_batch_create: could not build the batch", "");
        for (ucp_inst* m : b->members) ucp_destroy(m);
        cudaStreamSynchronize(b->stream);
        b->arena.release_all();
        delete b;
        return st;
    }
    *out = b;
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_sweep(ucp_batch* b, int32_t n_sweeps) {
    if (!b || n_sweeps < 0) return UCP_E_ARG;
    if (b->poisoned) return UCP_E_STATE;
    if (n_sweeps == 0) return UCP_OK;
    for (ucp_inst* in : b->members) {
        if (in->poisoned) return UCP_E_STATE;
        ucp_status st = grow_history(in, in->sweeps_done + 1 + n_sweeps);
        if (st != UCP_OK) return st;
    }
    if (batchset_refresh(b->bs, b->members, b->stream) != UCP_OK)
        return fail(b, "ucp_batch_sweep");
    // capture one sweep as a graph on a capturable (non-default) stream
    if (!b->graph_tried && b->stream) {
        b->graph_tried = true;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            launch_batch_sweep(b->bs.bl, b->stream);
            if (cudaStreamEndCapture(b->stream, &graph) == cudaSuccess && graph) {
                if (cudaGraphInstantiate(&b->graph, graph, 0) != cudaSuccess)
                    b->graph = nullptr;
                cudaGraphDestroy(graph);
            }
        }
        cudaGetLastError();  // a failed capture falls back to plain launches
    }
    for (int s = 0; s < n_sweeps; ++s) {
        if (b->prof.on) launch_batch_sweep(b->bs.bl, b->stream, &b->prof);
        else if (b->graph) cudaGraphLaunch(b->graph, b->stream);
        else launch_batch_sweep(b->bs.bl, b->stream);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(b, "ucp_batch_sweep");
    for (ucp_inst* in : b->members) {
        in->sweeps_done += n_sweeps;
        in->cur ^= (n_sweeps & 1);
    }
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_eval_J(ucp_batch* b, double* J_out) {
    if (!b || !J_out) return UCP_E_ARG;
    if (b->poisoned) return UCP_E_STATE;
    const int n = (int)b->members.size();
    if (batchset_refresh(b->bs, b->members, b->stream) != UCP_OK)
        return fail(b, "ucp_batch_eval_J");
    k_gather_J<<<(n + 127) / 128, 128, 0, b->stream>>>(b->bs.insts, n, b->J_gather);
    std::vector<double> flags((size_t)n);
    cudaMemcpyAsync(J_out, b->J_gather, sizeof(double) * (size_t)n,
                    cudaMemcpyDeviceToHost, b->stream);
    cudaMemcpyAsync(flags.data(), b->J_gather + n, sizeof(double) * (size_t)n,
                    cudaMemcpyDeviceToHost, b->stream);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(b, "ucp_batch_eval_J");
    for (double e : flags)
        if (e != 0.0) {
            b->poisoned = true;
            set_error("%s%s", "ucp_batch_eval_J: a tensor-core wait timed out", "");
            return UCP_E_TIMEOUT;
        }
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_set_launch_config(ucp_batch* b,
                                                          const ucp_launch_config* c) {
    if (!b) return UCP_E_ARG;
    if (b->poisoned) return UCP_E_STATE;
    LaunchCfg cfg;
    if (const char* why = launch_cfg_from(c, &cfg)) {
        set_error("ucp_batch_set_launch_config: %s%s", why, "");
        return UCP_E_ARG;
    }
    // the captured sweep holds the old block maps: drop it, rebuild them
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(b, "ucp_batch_set_launch_config");
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_tried = false;
    b->bs.cfg = cfg;
    if (batchset_build(b->bs, b->members, b->stream) != UCP_OK)
        return fail(b, "ucp_batch_set_launch_config");
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_profile(ucp_batch* b, int32_t enable) {
    if (!b) return UCP_E_ARG;
    return prof_enable(&b->prof, b->stream, enable != 0);
}

extern "C" UCP_API int32_t ucp_batch_kernel_times(ucp_batch* b, const char** names,
                                                  int64_t* launches, double* total_ms,
                                                  int32_t cap) {
    if (!b) return -1;
    return prof_collect(&b->prof, names, launches, total_ms, cap);
}

extern "C" UCP_API ucp_status ucp_batch_instance(ucp_batch* b, int32_t k, ucp_inst** out) {
    if (!b || !out || k < 0 || k >= (int32_t)b->members.size()) return UCP_E_ARG;
    *out = b->members[k];
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_destroy(ucp_batch* b) {
    if (!b) return UCP_E_ARG;
    cudaStreamSynchronize(b->stream);
    b->prof.drain();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (ucp_inst* m : b->members) ucp_destroy(m);
    b->arena.release_all();
    delete b;
    return UCP_OK;
}
