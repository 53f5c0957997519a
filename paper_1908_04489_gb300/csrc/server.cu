// server.cu -- continuous batching of solve requests (ucp_srv_*, ucp_submit,
// ucp_poll).
//
// A server thread owns the GPU work.  Each step it (1) admits queued
// requests in arrival order while a slot is free and their device bytes fit
// the HBM budget, setting each up as a fast-path instance, (2) runs one
// batched sweep over every admitted instance (requests of different sizes
// and sweep counts share the launches), and (3) retires the instances that
// reached their sweep count: their J, f and u1 are copied to host memory and
// the slot and bytes are freed.  Requests that arrive while others are on
// the GPU join at the next step.  The arithmetic is the single-instance fast
// path's, so every result equals the same request solved alone.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_set.h"

using namespace ucp;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    ucp_params p{};
    std::vector<double> table;   // init table (init_kind 2), owned copy
    int sweeps = 0;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    bool done = false;
    ucp_status status = UCP_PENDING;
    double J = 0.0;
    std::vector<double> f, U;
    ucp_inst* inst = nullptr;
};

// Device memory of served instances: freed blocks are kept by size and
// reused, so steady serving does not call cudaMalloc / cudaFree (the latter
// synchronises the device).
struct Pool {
    std::mutex mu;
    std::unordered_map<size_t, std::vector<void*>> free_blocks;
    std::unordered_map<void*, size_t> size_of;
    std::vector<void*> all;
};

// Block sizes are rounded up to buckets spaced by an eighth of their power of
// two, so that instances of nearby sizes (sigma and the grid widths vary
// continuously across requests) reuse each other's blocks.  Admission counts
// the bytes a request uses; the pooled blocks holding them are at most 12.5%
// larger.
size_t pool_bucket(size_t n) {
    n = (n + 255) & ~(size_t)255;
    size_t b = 256;
    while (b * 2 <= n) b *= 2;
    const size_t step = b / 8 > 256 ? b / 8 : 256;
    return (n + step - 1) / step * step;
}

void pool_free(void* q, void* user);
void* pool_alloc(size_t n, void* user) {
    Pool* p = (Pool*)user;
    n = pool_bucket(n);
    {
        std::lock_guard<std::mutex> lock(p->mu);
        auto it = p->free_blocks.find(n);
        if (it != p->free_blocks.end() && !it->second.empty()) {
            void* q = it->second.back();
            it->second.pop_back();
            return q;
        }
    }
    void* q = nullptr;
    if (cudaMalloc(&q, n) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(p->mu);
    p->all.push_back(q);
    p->size_of[q] = n;
    return q;
}

void pool_free(void* q, void* user) {
    Pool* p = (Pool*)user;
    std::lock_guard<std::mutex> lock(p->mu);
    p->free_blocks[p->size_of[q]].push_back(q);
}

}  // namespace

struct ucp_srv {
    ucp_ctx* ctx = nullptr;       // the caller's context (device)
    ucp_ctx own;                  // same device, pooled allocator
    Pool pool;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    std::vector<std::shared_ptr<Request>> active;   // server thread only
    size_t used = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool poisoned = false;
    bool fail_next = false;
    ucp_status fail_status = UCP_OK;
    std::thread th;
    Arena arena;
    BatchSet bs;    // the active requests (one batched sweep per step)
    BatchSet adm;   // the requests admitted in a step (their set-up)
    SetupSet ss;
    Clock::time_point t0;
    uint64_t steps = 0, completed = 0;
    int max_active = 0;

    double now() const {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
};

namespace {

void finish(ucp_srv* s, const std::shared_ptr<Request>& r, ucp_status st) {
    std::lock_guard<std::mutex> lock(s->mu);
    r->status = st;
    r->done = true;
    r->t_done = s->now();
    s->completed += 1;
}

void fail_all(ucp_srv* s, ucp_status st) {
    for (auto& r : s->active) {
        if (r->inst) ucp_destroy(r->inst);
        r->inst = nullptr;
        finish(s, r, st);
    }
    s->active.clear();
    std::lock_guard<std::mutex> lock(s->mu);
    s->used = 0;
    s->poisoned = true;
    s->fail_status = st;
    for (auto& r : s->queue) {
        r->status = st;
        r->done = true;
        r->t_done = s->now();
    }
    s->queue.clear();
}

void loop(ucp_srv* s) {
    if (cudaSetDevice(s->ctx->device) != cudaSuccess) {
        fail_all(s, UCP_E_CUDA);
        return;
    }
    bool membership_changed = true;
    for (;;) {
        std::vector<std::shared_ptr<Request>> admitted;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->active.empty() && s->queue.empty() && !s->stop)
                s->cv.wait_for(lock, std::chrono::milliseconds(20));
            if (s->stop) break;
            while (!s->queue.empty() && (int)s->active.size() + (int)admitted.size() < s->max_slots &&
                   s->used + s->queue.front()->bytes <= s->budget) {
                auto r = s->queue.front();
                s->queue.pop_front();
                s->used += r->bytes;
                r->t_admit = s->now();
                admitted.push_back(r);
            }
        }
        std::vector<ucp_inst*> fresh;
        for (auto& r : admitted) {
            if (!r->table.empty()) r->p.init_table = r->table.data();
            ucp_inst* in = nullptr;
            ucp_status st = inst_create(&s->own, &r->p, s->stream, false, &in);
            if (st == UCP_OK) st = grow_history(in, r->sweeps + 1);
            if (st != UCP_OK) {
                if (in) ucp_destroy(in);
                {
                    std::lock_guard<std::mutex> lock(s->mu);
                    s->used -= r->bytes;
                }
                finish(s, r, st);
                continue;
            }
            r->inst = in;
            s->active.push_back(r);
            fresh.push_back(in);
            membership_changed = true;
        }
        if (!fresh.empty()) {
            // the admitted requests' first u1 update, tables and J, batched
            ucp_status st = batchset_build(s->adm, fresh, s->stream);
            if (st == UCP_OK) st = batchset_setup(s->ss, s->adm, fresh, s->stream);
            if (st != UCP_OK) {
                fail_all(s, st);
                continue;
            }
        }
        if (s->active.empty()) continue;
        bool inject = false;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            inject = s->fail_next;
            s->fail_next = false;
        }
        if (inject) {
            // host-side fault injection: behave as if the step's launch failed
            set_error("%s%s", "ucp server: injected step failure", "");
            fail_all(s, UCP_E_CUDA);
            continue;
        }
        // retire the requests that reached their sweep count (results to
        // host memory, slot and bytes freed)
        {
            std::vector<std::shared_ptr<Request>> keep;
            for (auto& r : s->active) {
                if (r->inst->sweeps_done < r->sweeps) {
                    keep.push_back(r);
                    continue;
                }
                r->f.resize((size_t)r->inst->g.n_x);
                r->U.resize((size_t)r->inst->g.n_y);
                ucp_status g1 = ucp_get_controllers(r->inst, r->f.data(), r->f.size(),
                                                    r->U.data(), r->U.size(), 0, nullptr);
                ucp_status g2 = g1 == UCP_OK ? ucp_eval_J(r->inst, &r->J) : g1;
                ucp_destroy(r->inst);
                r->inst = nullptr;
                finish(s, r, g2);
                {
                    std::lock_guard<std::mutex> lock(s->mu);
                    s->used -= r->bytes;
                }
                membership_changed = true;
            }
            s->active.swap(keep);
        }
        if (s->active.empty()) continue;
        std::vector<ucp_inst*> members;
        members.reserve(s->active.size());
        for (auto& r : s->active) members.push_back(r->inst);
        ucp_status st = membership_changed ? batchset_build(s->bs, members, s->stream)
                                           : batchset_refresh(s->bs, members, s->stream);
        if (st != UCP_OK) {
            fail_all(s, st);
            continue;
        }
        membership_changed = false;
        if ((int)s->active.size() > s->max_active) s->max_active = (int)s->active.size();
        launch_batch_sweep(s->bs.bl, s->stream);
        if (cudaGetLastError() != cudaSuccess) {
            fail_all(s, UCP_E_CUDA);
            continue;
        }
        for (auto& r : s->active) {
            r->inst->sweeps_done += 1;
            r->inst->cur ^= 1;
        }
        s->steps += 1;
    }
    for (auto& r : s->active)
        if (r->inst) ucp_destroy(r->inst);
    s->active.clear();
}

}  // namespace

extern "C" UCP_API ucp_status ucp_srv_create(ucp_ctx* ctx, uint64_t hbm_budget_bytes,
                                             int32_t max_slots, void* stream,
                                             ucp_srv** out) {
    if (!ctx || !out || max_slots < 1 || hbm_budget_bytes == 0) {
        set_error("ucp_srv_create: %s%s", "bad context, budget or slot count", "");
        return UCP_E_ARG;
    }
    ucp_srv* s = new ucp_srv();
    s->ctx = ctx;
    s->stream = (cudaStream_t)stream;
    s->budget = (size_t)hbm_budget_bytes;
    s->max_slots = max_slots;
    s->own.device = ctx->device;
    s->own.alloc = pool_alloc;
    s->own.free_fn = pool_free;
    s->own.user = &s->pool;
    s->arena.ctx = &s->own;
    s->bs.arena = &s->arena;
    s->adm.arena = &s->arena;
    s->ss.arena = &s->arena;
    s->t0 = Clock::now();
    s->th = std::thread(loop, s);
    *out = s;
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_submit(ucp_srv* s, const ucp_params* params,
                                         int32_t n_sweeps, uint64_t* ticket) {
    if (!s || !params || !ticket || n_sweeps < 0) return UCP_E_ARG;
    Geom g;
    if (const char* why = make_geom(*params, &g)) {
        set_error("ucp_submit: %s%s", why, "");
        return UCP_E_ARG;
    }
    if (params->precision != 1 || params->problem != 0) {
        set_error("ucp_submit: %s%s", "served requests use the fast path (precision 1) of "
                  "Witsenhausen's problem (problem 0)", "");
        return UCP_E_ARG;
    }
    auto r = std::make_shared<Request>();
    r->p = *params;
    if (params->init_kind == 2)
        r->table.assign(params->init_table, params->init_table + g.n_x);
    r->p.init_table = nullptr;
    r->sweeps = n_sweeps;
    r->bytes = inst_bytes(g, 1) + (size_t)8 * (size_t)(n_sweeps + 1);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->poisoned || s->stop) return UCP_E_STATE;
    if (r->bytes > s->budget) {
        set_error("ucp_submit: %s%s", "request alone exceeds the HBM budget", "");
        return UCP_E_BUDGET;
    }
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    s->table[r->ticket] = r;
    s->queue.push_back(r);
    s->cv.notify_one();
    *ticket = r->ticket;
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_poll(ucp_srv* s, uint64_t ticket, ucp_result* res,
                                       double* f, uint64_t n_x, double* u1,
                                       uint64_t n_y) {
    if (!s) return UCP_E_ARG;
    std::shared_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        auto it = s->table.find(ticket);
        if (it == s->table.end()) return UCP_E_NOTFOUND;
        r = it->second;
        if (!r->done) return UCP_PENDING;
        if ((f && n_x != r->f.size() && r->status == UCP_OK) ||
            (u1 && n_y != r->U.size() && r->status == UCP_OK)) {
            set_error("ucp_poll: %s%s", "output size does not match the request", "");
            return UCP_E_ARG;
        }
        s->table.erase(it);
    }
    if (res) {
        res->J = r->J;
        res->t_submit = r->t_submit;
        res->t_admit = r->t_admit;
        res->t_done = r->t_done;
        res->sweeps = r->sweeps;
        res->status = r->status;
    }
    if (r->status == UCP_OK) {
        if (f) memcpy(f, r->f.data(), sizeof(double) * r->f.size());
        if (u1) memcpy(u1, r->U.data(), sizeof(double) * r->U.size());
    }
    return r->status;
}

extern "C" UCP_API ucp_status ucp_srv_stats(ucp_srv* s, ucp_srv_info* info) {
    if (!s || !info) return UCP_E_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    info->queued = (int64_t)s->queue.size();
    info->in_flight = (int64_t)(s->table.size() - s->queue.size());
    info->steps = (int64_t)s->steps;
    info->completed = (int64_t)s->completed;
    info->max_active = s->max_active;
    info->bytes_in_use = (uint64_t)s->used;
    info->now = s->now();
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_srv_fail_next_step(ucp_srv* s) {
    if (!s) return UCP_E_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->fail_next = true;
    return UCP_OK;
}

extern "C" UCP_API ucp_status ucp_srv_destroy(ucp_srv* s) {
    if (!s) return UCP_E_ARG;
    bool pending = false;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        for (auto& kv : s->table)
            if (!kv.second->done) pending = true;
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    s->arena.release_all();
    {
        std::lock_guard<std::mutex> lock(s->pool.mu);
        for (void* q : s->pool.all) cudaFree(q);
    }
    delete s;
    return pending ? UCP_E_STATE : UCP_OK;
}
