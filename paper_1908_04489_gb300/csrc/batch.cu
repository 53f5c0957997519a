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

#include "ucp_fast.cuh"
#include "ucp_runtime.h"

using namespace ucp;

struct ucp_batch {
    ucp_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<ucp_inst*> members;
    Arena arena;
    BatchLaunch bl{};
    std::vector<InstDev> desc;
    double* J_gather = nullptr;   // [n] device
    bool poisoned = false;
    cudaGraphExec_t graph = nullptr;
    bool graph_tried = false;
};

namespace {

ucp_status fail(ucp_batch* b, const char* where) {
    const cudaError_t e = cudaGetLastError();
    b->poisoned = true;
    set_error("%s: %s", where, cudaGetErrorString(e));
    return UCP_E_CUDA;
}

InstDev describe(const ucp_inst* in) {
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

int run_slot(int R) { return R >= 16 ? 4 : (R >= 8 ? 3 : (R >= 4 ? 2 : (R >= 2 ? 1 : 0))); }

__global__ void k_gather_J(const InstDev* insts, int n, double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) out[b] = insts[b].J[insts[b].sweeps];
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
        if (params[k].precision != 1) {
            set_error("ucp_batch_create: %s%s", "batched instances use the fast path "
                      "(precision 1)", "");
            return UCP_E_ARG;
        }
        if (params[k].n_refine != params[0].n_refine) {
            set_error("ucp_batch_create: %s%s", "all instances must share n_refine", "");
            return UCP_E_ARG;
        }
    }
    ucp_batch* b = new ucp_batch();
    b->ctx = ctx;
    b->stream = (cudaStream_t)stream;
    b->arena.ctx = ctx;
    for (int k = 0; k < n; ++k) {
        ucp_inst* in = nullptr;
        ucp_status st = ucp_create(ctx, &params[k], stream, &in);
        if (st != UCP_OK) {
            for (ucp_inst* m : b->members) ucp_destroy(m);
            delete b;
            return st;
        }
        b->members.push_back(in);
    }
    // block maps
    std::vector<BlockRef> maps[8], mmaps[5];
    for (int k = 0; k < n; ++k) {
        const ucp_inst* in = b->members[k];
        for (int kind = 0; kind < 8; ++kind) {
            const int64_t nb = batch_blocks(in->g, in->fv, kind);
            for (int64_t x = 0; x < nb; ++x) maps[kind].push_back({k, (int32_t)x});
        }
        const int64_t nb = batch_mmse_blocks(in->g, in->fv);
        std::vector<BlockRef>& mm = mmaps[run_slot(in->fv.run)];
        for (int64_t x = 0; x < nb; ++x) mm.push_back({k, (int32_t)x});
    }
    BatchLaunch& bl = b->bl;
    bl.n_inst = n;
    bl.G = params[0].n_refine;
    bl.insts = (InstDev*)b->arena.get(sizeof(InstDev) * (size_t)n);
    b->J_gather = (double*)b->arena.get(sizeof(double) * (size_t)n);
    bool ok = bl.insts && b->J_gather;
    for (int kind = 0; kind < 8 && ok; ++kind) {
        BlockRef* p = (BlockRef*)b->arena.get(sizeof(BlockRef) * maps[kind].size());
        ok = p != nullptr;
        if (ok) cudaMemcpyAsync(p, maps[kind].data(), sizeof(BlockRef) * maps[kind].size(),
                                cudaMemcpyHostToDevice, b->stream);
        bl.map[kind] = p;
        bl.n_blocks[kind] = (int64_t)maps[kind].size();
    }
    for (int r = 0; r < 5 && ok; ++r) {
        bl.mmse_blocks[r] = (int64_t)mmaps[r].size();
        bl.mmse_map[r] = nullptr;
        if (mmaps[r].empty()) continue;
        BlockRef* p = (BlockRef*)b->arena.get(sizeof(BlockRef) * mmaps[r].size());
        ok = p != nullptr;
        if (ok) cudaMemcpyAsync(p, mmaps[r].data(), sizeof(BlockRef) * mmaps[r].size(),
                                cudaMemcpyHostToDevice, b->stream);
        bl.mmse_map[r] = p;
    }
    if (!ok) {
        set_error("%s%s", "ucp_batch_create: out of device memory", "");
        for (ucp_inst* m : b->members) ucp_destroy(m);
        cudaStreamSynchronize(b->stream);
        b->arena.release_all();
        delete b;
        return UCP_E_NOMEM;
    }
    // the host-side maps must stay valid until the copies are done
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        ucp_status st = fail(b, "ucp_batch_create");
        for (ucp_inst* m : b->members) ucp_destroy(m);
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
    const int n = (int)b->members.size();
    b->desc.resize(n);
    for (int k = 0; k < n; ++k) {
        ucp_inst* in = b->members[k];
        if (in->poisoned) return UCP_E_STATE;
        ucp_status st = grow_history(in, in->sweeps_done + 1 + n_sweeps);
        if (st != UCP_OK) return st;
        b->desc[k] = describe(in);
    }
    cudaMemcpyAsync(b->bl.insts, b->desc.data(), sizeof(InstDev) * (size_t)n,
                    cudaMemcpyHostToDevice, b->stream);
    // capture one sweep as a graph on a capturable (non-default) stream
    if (!b->graph_tried && b->stream) {
        b->graph_tried = true;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            launch_batch_sweep(b->bl, b->stream);
            if (cudaStreamEndCapture(b->stream, &graph) == cudaSuccess && graph) {
                if (cudaGraphInstantiate(&b->graph, graph, 0) != cudaSuccess)
                    b->graph = nullptr;
                cudaGraphDestroy(graph);
            }
        }
        cudaGetLastError();  // a failed capture falls back to plain launches
    }
    for (int s = 0; s < n_sweeps; ++s) {
        if (b->graph) cudaGraphLaunch(b->graph, b->stream);
        else launch_batch_sweep(b->bl, b->stream);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(b, "ucp_batch_sweep");
    for (ucp_inst* in : b->members) {
        in->sweeps_done += n_sweeps;
        in->cur ^= (n_sweeps & 1);
    }
    // the descriptors' host copy must outlive the upload
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(b, "ucp_batch_sweep");
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_eval_J(ucp_batch* b, double* J_out) {
    if (!b || !J_out) return UCP_E_ARG;
    if (b->poisoned) return UCP_E_STATE;
    const int n = (int)b->members.size();
    b->desc.resize(n);
    for (int k = 0; k < n; ++k) b->desc[k] = describe(b->members[k]);
    cudaMemcpyAsync(b->bl.insts, b->desc.data(), sizeof(InstDev) * (size_t)n,
                    cudaMemcpyHostToDevice, b->stream);
    k_gather_J<<<(n + 127) / 128, 128, 0, b->stream>>>(b->bl.insts, n, b->J_gather);
    cudaMemcpyAsync(J_out, b->J_gather, sizeof(double) * (size_t)n,
                    cudaMemcpyDeviceToHost, b->stream);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(b, "ucp_batch_eval_J");
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_instance(ucp_batch* b, int32_t k, ucp_inst** out) {
    if (!b || !out || k < 0 || k >= (int32_t)b->members.size()) return UCP_E_ARG;
    *out = b->members[k];
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_batch_destroy(ucp_batch* b) {
    if (!b) return UCP_E_ARG;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (ucp_inst* m : b->members) ucp_destroy(m);
    b->arena.release_all();
    delete b;
    return UCP_OK;
}
