// Serving runtime: continuous batching of symmetric MTTKRP requests.
//
// A native scheduler thread owns `max_slots` CUDA streams (half of them high
// priority).  Requests queue on submission; whenever a slot and HBM budget are
// free, the scheduler admits the next requests (FIFO; a blocked head may be
// passed by later requests that fit, until it has waited 5 ms), launches each on
// its slot's stream, and polls completion events.  Requests that arrive while
// others run are admitted as soon as room frees up, so their kernels overlap
// on the device; small requests go to high-priority streams so they are not
// stuck behind large ones.  Each response carries the FP64 CP-fit residual when
// asked for, and host steady-clock timestamps for submit, admission and
// completion.  Nothing here waits on the device without a bound: the scheduler
// only queries events, and destroy drains with a time limit.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    uint64_t ticket;
    sym_request r;
    size_t bytes;
    uint64_t t_submit;
    bool small;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool high = false;
    bool busy = false;
    Pending req{};
    uint64_t t_admit = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* res_dev = nullptr;
    double* res_host = nullptr;  // pinned
    sym_status launch_status = SYM_OK;
};

size_t request_bytes(const sym_request& r) {
    const sym_tensor_s* X = r.X;
    const size_t esz = r.bdt == SYM_BF16 ? 2 : 4;
    return X->info.arena_used + (size_t)X->n * (size_t)r.ldb * esz + (size_t)X->n * (size_t)r.ldm * 4;
}

}  // namespace

struct sym_server_s {
    sym_server_cfg cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Pending> queue;
    std::vector<Slot> slots;
    std::unordered_map<uint64_t, sym_result> done;
    std::unordered_set<uint64_t> live;
    size_t inflight_bytes = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool orphaned = false;  // destroy timed out: the scheduler releases everything when it exits
    std::thread th;
    sym_server_stats stats{};
    int64_t inflight = 0;

    void run();
    void finish(Slot& s, sym_status st);
    void launch(Slot& s);
    void release();
};

// Streams, events and pinned buffers of the slots (host-side resources only).
void sym_server_s::release() {
    for (auto& s : slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.res_host) cudaFreeHost(s.res_host);
        s.stream = nullptr;
        s.done = nullptr;
        s.res_host = nullptr;
    }
}

void sym_server_s::finish(Slot& s, sym_status st) {
    sym_result res{};
    res.status = st;
    res.residual = (st == SYM_OK && s.req.r.want_residual) ? *s.res_host : 0.0;
    res.user_tag = s.req.r.user_tag;
    res.t_submit_ns = s.req.t_submit;
    res.t_admit_ns = s.t_admit;
    res.t_done_ns = now_ns();
    {
        std::lock_guard<std::mutex> lk(mu);
        done[s.req.ticket] = res;
        live.erase(s.req.ticket);
        inflight_bytes -= s.req.bytes;
        inflight -= 1;
        stats.completed += 1;
    }
    s.busy = false;
    cv_done.notify_all();
}

void sym_server_s::launch(Slot& s) {
    using namespace symgpu;
    const sym_request& r = s.req.r;
    const bool bf16 = r.bdt == SYM_BF16;
    sym_status st = mttkrp_core(r.X, r.B, bf16, r.rank, r.ldb, r.M, r.ldm, s.stream);
    if (st == SYM_OK && r.want_residual) {
        st = residual_launch(r.X, r.B, bf16, r.rank, r.ldb, r.M, r.ldm, s.res_dev, s.ws, s.ws_bytes, s.stream);
        if (st == SYM_OK)
            st = cuda_status(cudaMemcpyAsync(s.res_host, s.res_dev, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
    }
    if (st == SYM_OK) st = cuda_status(cudaEventRecord(s.done, s.stream));
    s.launch_status = st;
}

void sym_server_s::run() {
    cudaSetDevice(device);
    const uint64_t pass_limit_ns = 5'000'000;  // a blocked head may be passed for this long
    for (;;) {
        bool progressed = false;
        // 1. completions
        for (auto& s : slots) {
            if (!s.busy) continue;
            if (s.launch_status != SYM_OK) {
                finish(s, s.launch_status);
                progressed = true;
                continue;
            }
            cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            finish(s, q == cudaSuccess ? SYM_OK : symgpu::cuda_status(q));
            progressed = true;
        }
        // 2. admission
        std::vector<Slot*> to_launch;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop && queue.empty() && inflight == 0) break;
            const uint64_t t = now_ns();
            for (auto it = queue.begin(); it != queue.end();) {
                if (inflight_bytes + it->bytes > cfg.hbm_budget_bytes) {
                    // head blocked on budget: later requests may pass it for a while
                    if (it == queue.begin() && t - it->t_submit > pass_limit_ns) break;
                    ++it;
                    continue;
                }
                Slot* pick = nullptr;
                for (auto& s : slots)  // small -> prefer high priority; large -> prefer low
                    if (!s.busy && s.high == it->small) {
                        pick = &s;
                        break;
                    }
                if (!pick)
                    for (auto& s : slots)
                        if (!s.busy) {
                            pick = &s;
                            break;
                        }
                if (!pick) break;
                pick->busy = true;
                pick->req = *it;
                pick->t_admit = t;
                inflight_bytes += it->bytes;
                inflight += 1;
                stats.admitted += 1;
                stats.peak_inflight = std::max<int64_t>(stats.peak_inflight, inflight);
                stats.peak_bytes = std::max<int64_t>(stats.peak_bytes, (int64_t)inflight_bytes);
                to_launch.push_back(pick);
                it = queue.erase(it);
            }
            if (to_launch.empty() && !progressed) {
                if (inflight == 0)
                    cv_sched.wait_for(lk, std::chrono::milliseconds(20),
                                      [&] { return stop || !queue.empty(); });
            }
        }
        for (Slot* s : to_launch) {
            launch(*s);
            std::lock_guard<std::mutex> lk(mu);
            stats.launches += 1;
        }
        if (to_launch.empty() && !progressed) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    bool self_release;
    {
        std::lock_guard<std::mutex> lk(mu);
        self_release = orphaned;
    }
    if (self_release) {  // nobody joins this thread any more: the last in-flight request has completed
        release();
        delete this;
    }
}

using namespace symgpu;

extern "C" size_t sym_server_arena_bytes(const sym_server_cfg* cfg) {
    if (!cfg || cfg->max_slots < 1 || cfg->max_rank < 4) return 0;
    const size_t per = align_up(residual_ws_bytes(cfg->max_rank), 256) + 256;
    return per * (size_t)cfg->max_slots;
}

extern "C" sym_status sym_server_create(const sym_server_cfg* cfg, void* arena, size_t arena_bytes, int device,
                                        sym_server* out) {
    if (!out) return SYM_E_INVALID;
    *out = nullptr;
    if (!cfg || cfg->max_slots < 1 || cfg->max_slots > 256 || cfg->max_rank < 4 || cfg->max_rank > 128 ||
        cfg->max_rank % 4 || cfg->hbm_budget_bytes == 0)
        return SYM_E_INVALID;
    if (!arena || !aligned(arena, 256)) return SYM_E_INVALID;
    if (arena_bytes < sym_server_arena_bytes(cfg)) return SYM_E_NOMEM;
    sym_server_s* S = new (std::nothrow) sym_server_s();
    if (!S) return SYM_E_NOMEM;
    S->cfg = *cfg;
    if (S->cfg.wait_limit_ns <= 0) S->cfg.wait_limit_ns = 10'000'000'000LL;
    S->device = device;
    sym_status st = cuda_status(cudaSetDevice(device));
    int lo = 0, hi = 0;
    if (st == SYM_OK) st = cuda_status(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    S->slots.resize((size_t)cfg->max_slots);
    const size_t per = align_up(residual_ws_bytes(cfg->max_rank), 256) + 256;
    for (int k = 0; k < cfg->max_slots && st == SYM_OK; ++k) {
        Slot& s = S->slots[(size_t)k];
        s.high = k < (cfg->max_slots + 1) / 2;
        st = cuda_status(cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, s.high ? hi : lo));
        if (st == SYM_OK) st = cuda_status(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
        if (st == SYM_OK) st = cuda_status(cudaHostAlloc((void**)&s.res_host, sizeof(double), cudaHostAllocDefault));
        char* base = static_cast<char*>(arena) + per * (size_t)k;
        s.res_dev = reinterpret_cast<double*>(base);
        s.ws = base + 256;
        s.ws_bytes = per - 256;
    }
    if (st != SYM_OK) {
        for (auto& s : S->slots) {
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.done) cudaEventDestroy(s.done);
            if (s.res_host) cudaFreeHost(s.res_host);
        }
        delete S;
        return st;
    }
    try {
        S->th = std::thread([S] { S->run(); });
    } catch (...) {
        for (auto& s : S->slots) {
            cudaStreamDestroy(s.stream);
            cudaEventDestroy(s.done);
            cudaFreeHost(s.res_host);
        }
        delete S;
        return SYM_E_NOMEM;
    }
    *out = S;
    return SYM_OK;
}

extern "C" sym_status sym_batch_submit(sym_server S, const sym_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return SYM_E_INVALID;
    if (!req->X) return SYM_E_BADREQ;
    if (validate_mttkrp_args(req->X, req->B, req->bdt, req->rank, req->ldb, req->M, req->ldm) != SYM_OK)
        return SYM_E_BADREQ;
    if (req->rank > S->cfg.max_rank) return SYM_E_BADREQ;
    const size_t bytes = request_bytes(*req);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return SYM_E_INVALID;
        if (bytes > S->cfg.hbm_budget_bytes) {
            S->stats.rejected += 1;
            return SYM_E_BUDGET;
        }
        Pending p{S->next_ticket++, *req, bytes, now_ns(), req->X->nnz <= S->cfg.small_nnz};
        S->queue.push_back(p);
        S->live.insert(p.ticket);
        S->stats.submitted += 1;
        *ticket = p.ticket;
    }
    S->cv_sched.notify_one();
    return SYM_OK;
}

extern "C" sym_status sym_batch_poll(sym_server S, uint64_t ticket, sym_result* out) {
    if (!S || !out) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it != S->done.end()) {
        *out = it->second;
        S->done.erase(it);
        return SYM_OK;
    }
    if (S->live.count(ticket)) {
        out->status = SYM_PENDING;
        return SYM_PENDING;
    }
    return SYM_E_NOTFOUND;
}

extern "C" sym_status sym_batch_wait(sym_server S, uint64_t ticket, int64_t timeout_ns, sym_result* out) {
    if (!S || !out) return SYM_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns > 0 ? timeout_ns : 0);
    for (;;) {
        auto it = S->done.find(ticket);
        if (it != S->done.end()) {
            *out = it->second;
            S->done.erase(it);
            return SYM_OK;
        }
        if (!S->live.count(ticket)) return SYM_E_NOTFOUND;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = S->done.find(ticket);
            if (it2 != S->done.end()) {
                *out = it2->second;
                S->done.erase(it2);
                return SYM_OK;
            }
            return SYM_E_TIMEOUT;
        }
    }
}

extern "C" sym_status sym_server_stats_get(sym_server S, sym_server_stats* out) {
    if (!S || !out) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return SYM_OK;
}

extern "C" sym_status sym_server_destroy(sym_server S) {
    if (!S) return SYM_OK;
    sym_status st = SYM_OK;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->stop = true;
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(S->cfg.wait_limit_ns);
        S->cv_sched.notify_all();
        while (!(S->queue.empty() && S->inflight == 0)) {
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
                if (S->queue.empty() && S->inflight == 0) break;  // finished just as the limit ran out
                st = SYM_E_TIMEOUT;
                // drop queued requests; in-flight ones finish on their own, and the scheduler thread
                // (which exits once they have) then releases the server itself
                for (auto& p : S->queue) S->live.erase(p.ticket);
                S->queue.clear();
                S->orphaned = true;
                break;
            }
        }
    }
    S->cv_sched.notify_all();
    if (st != SYM_OK) {
        S->th.detach();  // S is released by the scheduler thread; do not touch it after this
        return st;
    }
    S->th.join();
    S->release();
    delete S;
    return st;
}
