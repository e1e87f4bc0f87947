// Serving runtime: continuous batching of symmetric MTTKRP requests.
//
// A native scheduler thread owns `max_slots` CUDA streams (half of them high
// priority).  Requests queue on submission; whenever a slot and HBM budget are
// free, the scheduler admits the next requests (FIFO; a blocked head may be
// passed by later requests that fit, until it has waited 5 ms), launches each on
// its slot's stream, and polls completion events.  Requests that arrive while
// others run are admitted as soon as room frees up, so their kernels overlap
// on the device; small requests go to high-priority streams so they are not
// stuck behind large ones.  With coalesce_small, the small requests admitted
// in one scheduler pass share one slot: they run back to back on its stream
// with one completion event (a grouped launch), so a burst of small requests
// does not take every slot.  Each response carries the FP64 CP-fit residual
// when asked for, and host steady-clock timestamps for submit, admission and
// completion.
//
// Registered tensors: a caller may hand the server the host image of a tensor
// (sym_tensor_save) instead of a resident tensor.  The server keeps such
// tensors in a device pool carved from its arena: a request for a tensor that
// is not resident loads it (one host-to-device copy of its canonical arrays);
// when the pool is full, the
// least recently used resident tensors that no request in flight uses are
// dropped (the host image is the master copy, so nothing is copied back).
// Loads run on a stream of their own (at most two at a time) and take no
// slot: a request is admitted once its tensor's copy has landed.  The
// pool and the factors / outputs of the requests in flight together stay
// within the HBM budget.  Admission prefers requests whose tensor is resident:
// a request that would need a load waits (up to cfg.affinity_wait_ns) while
// others can run, so the requests for one tensor that queue meanwhile share
// its load.  A request may declare its factor unchanged since an earlier
// request (want_residual 2): the residual then reuses the Gram matrix B^T B
// cached from that request instead of recomputing it.
//
// Nothing here waits on the device without a bound: the scheduler only queries
// events, and destroy drains with a time limit (releasing the server then
// waits for the load stream's last copy, a host-to-device copy that ends by
// itself).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
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

constexpr int kMaxGroup = 16;  // requests in one grouped launch
constexpr int kGramSlots = 512;  // cached Gram matrices (B^T B) of recently used factors
constexpr int kMaxLoads = 2;     // registered-tensor loads in flight at once

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// A registered tensor: its host image and, while resident, its pool range.
struct Entry {
    const void* image = nullptr;
    size_t bytes = 0;      // device bytes when loaded
    bool resident = false;
    size_t off = 0;        // pool offset while resident
    sym_tensor_s* X = nullptr;  // handle into the pool while resident
    cudaEvent_t ready = nullptr;  // recorded after the load
    int inuse = 0;         // requests in flight on it
    bool loading = false;  // its copy into the pool is in flight (on the load stream)
    uint64_t last_use = 0;
};

struct Pending {
    uint64_t ticket;
    sym_request r;
    int64_t reg = -1;  // registered tensor index, or -1 (r.X is a resident tensor)
    size_t bytes;
    uint64_t t_submit;
    bool small;
    int gram = -1;     // Gram cache slot the request reads or fills, or -1
};

// The Gram matrix of one factor (identified by its device pointer, shape,
// stride and type), kept for requests that declare the factor unchanged.
struct GramSlot {
    const void* B = nullptr;
    int64_t n = 0, ldb = 0;
    int32_t rank = 0;
    sym_dtype bdt = SYM_F32;
    double* G = nullptr;          // packed upper triangle, FP64 (server arena)
    cudaEvent_t ready = nullptr;  // recorded after it is computed
    bool valid = false;
    int inuse = 0;                // requests in flight reading or filling it
    uint64_t last_use = 0;
    bool same(const sym_request& r, int64_t nn) const {
        return valid && B == r.B && n == nn && ldb == r.ldb && rank == r.rank && bdt == r.bdt;
    }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool high = false;
    bool busy = false;
    std::vector<Pending> reqs;  // one request, or a group of small ones
    uint64_t t_admit = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* res_dev = nullptr;   // kMaxGroup residuals
    double* res_host = nullptr;  // pinned, kMaxGroup
    sym_status launch_status = SYM_OK;
};

size_t factor_bytes(const sym_request& r, int64_t n) {
    const size_t esz = r.bdt == SYM_BF16 ? 2 : 4;
    return (size_t)n * (size_t)r.ldb * esz + (size_t)n * (size_t)r.ldm * 4;
}

size_t slot_bytes(const sym_server_cfg* cfg) {
    return symgpu::align_up(symgpu::residual_ws_bytes(cfg->max_rank), 256) +
           symgpu::align_up(sizeof(double) * kMaxGroup, 256);
}

size_t gram_bytes(const sym_server_cfg* cfg) {
    return symgpu::align_up(sizeof(double) * (size_t)cfg->max_rank * (cfg->max_rank + 1) / 2, 256);
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
    // registered tensors and their device pool
    char* pool = nullptr;
    size_t pool_bytes = 0;
    std::map<size_t, size_t> free_ranges;  // offset -> size, coalesced
    std::vector<Entry> entries;
    uint64_t tick = 0;
    size_t resident_bytes = 0;
    GramSlot grams[kGramSlots];  // touched by the scheduler thread only
    uint64_t gram_tick = 0;
    cudaStream_t load_stream = nullptr;  // copies of registered tensors into the pool
    int loads_in_flight = 0;

    void run();
    void finish(Slot& s, sym_status st);
    void launch(Slot& s);
    void release();
    bool pool_alloc(size_t bytes, size_t* off);
    void pool_free(size_t off, size_t bytes);
    bool make_resident(Entry& E, cudaStream_t s, sym_status* err);
    void fail_queued(std::deque<Pending>::iterator& it, sym_status st);
};

bool sym_server_s::pool_alloc(size_t bytes, size_t* off) {
    for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
        if (it->second < bytes) continue;
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_ranges.erase(it);
        if (rest) free_ranges[at] = rest;
        return true;
    }
    return false;
}

void sym_server_s::pool_free(size_t off, size_t bytes) {
    auto it = free_ranges.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_ranges.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        free_ranges.erase(nx);
    }
    if (it != free_ranges.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            free_ranges.erase(it);
        }
    }
}

// Called with mu held.  Loads E into the pool (evicting least recently used
// idle entries as needed) with its copies on stream s; false when the pool
// cannot make room now (every resident entry is in use).
bool sym_server_s::make_resident(Entry& E, cudaStream_t s, sym_status* err) {
    *err = SYM_OK;
    size_t off = 0;
    while (!pool_alloc(E.bytes, &off)) {
        Entry* victim = nullptr;
        for (auto& c : entries)
            if (c.resident && c.inuse == 0 && !c.loading && (!victim || c.last_use < victim->last_use)) victim = &c;
        if (!victim) return false;
        pool_free(victim->off, victim->bytes);
        sym_tensor_destroy(victim->X);
        victim->X = nullptr;
        victim->resident = false;
        resident_bytes -= victim->bytes;
        stats.evictions += 1;
    }
    sym_tensor X = nullptr;
    sym_status st = sym_tensor_load(E.image, pool + off, E.bytes, reinterpret_cast<sym_stream_t>(s), &X);
    if (st == SYM_OK) st = symgpu::cuda_status(cudaEventRecord(E.ready, s));
    if (st != SYM_OK) {
        if (X) sym_tensor_destroy(X);
        pool_free(off, E.bytes);
        *err = st;
        return true;  // admitted, fails at launch
    }
    E.X = X;
    E.off = off;
    E.resident = true;
    resident_bytes += E.bytes;
    stats.loads += 1;
    stats.peak_resident_bytes = std::max<int64_t>(stats.peak_resident_bytes, (int64_t)resident_bytes);
    return true;
}

// Called with mu held: a queued request that can never run (its tensor failed
// to load) completes with that status; `it` moves to the next request.
void sym_server_s::fail_queued(std::deque<Pending>::iterator& it, sym_status st) {
    sym_result res{};
    res.status = st;
    res.user_tag = it->r.user_tag;
    res.t_submit_ns = it->t_submit;
    res.t_admit_ns = res.t_done_ns = now_ns();
    done[it->ticket] = res;
    live.erase(it->ticket);
    stats.admitted += 1;
    stats.completed += 1;
    it = queue.erase(it);
    cv_done.notify_all();
}

// Streams, events and pinned buffers of the slots and of the registered tensors.
void sym_server_s::release() {
    if (load_stream) {
        cudaStreamSynchronize(load_stream);  // no copy into the caller's arena is left in flight
        cudaStreamDestroy(load_stream);
        load_stream = nullptr;
    }
    for (auto& s : slots) {
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.res_host) cudaFreeHost(s.res_host);
        s.stream = nullptr;
        s.done = nullptr;
        s.res_host = nullptr;
    }
    for (auto& e : entries) {
        if (e.X) sym_tensor_destroy(e.X);
        if (e.ready) cudaEventDestroy(e.ready);
        e.X = nullptr;
        e.ready = nullptr;
    }
    for (auto& g : grams) {
        if (g.ready) cudaEventDestroy(g.ready);
        g.ready = nullptr;
    }
}

void sym_server_s::finish(Slot& s, sym_status st) {
    const uint64_t t_done = now_ns();
    {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t k = 0; k < s.reqs.size(); ++k) {
            const Pending& p = s.reqs[k];
            sym_result res{};
            res.status = st;
            res.residual = (st == SYM_OK && p.r.want_residual) ? s.res_host[k] : 0.0;
            res.user_tag = p.r.user_tag;
            res.t_submit_ns = p.t_submit;
            res.t_admit_ns = s.t_admit;
            res.t_done_ns = t_done;
            done[p.ticket] = res;
            live.erase(p.ticket);
            inflight_bytes -= p.bytes;
            inflight -= 1;
            stats.completed += 1;
            if (p.reg >= 0) entries[(size_t)p.reg].inuse -= 1;
            if (p.gram >= 0) grams[p.gram].inuse -= 1;
        }
    }
    s.reqs.clear();
    s.busy = false;
    cv_done.notify_all();
}

void sym_server_s::launch(Slot& s) {
    using namespace symgpu;
    sym_status st = s.launch_status;
    for (size_t k = 0; k < s.reqs.size() && st == SYM_OK; ++k) {
        const sym_request& r = s.reqs[k].r;
        const bool bf16 = r.bdt == SYM_BF16;
        const sym_tensor_s* X = r.X;
        if (s.reqs[k].reg >= 0) {
            Entry& E = entries[(size_t)s.reqs[k].reg];
            X = E.X;
            st = cuda_status(cudaStreamWaitEvent(s.stream, E.ready, 0));  // its load may run on another slot
        }
        if (st == SYM_OK) st = mttkrp_core(X, r.B, bf16, r.rank, r.ldb, r.M, r.ldm, s.stream);
        if (st == SYM_OK && r.want_residual) {
            // Gram of the factor: reused when the request declares the factor unchanged (want_residual 2) and
            // the cache holds it, else computed into an idle cache slot (the least recently used one)
            const double* G_in = nullptr;
            double* G_out = nullptr;
            int gi = -1;
            for (int g = 0; g < kGramSlots && gi < 0; ++g)
                if (grams[g].same(r, X->n)) gi = g;
            if (gi >= 0 && r.want_residual == 2) {
                st = cuda_status(cudaStreamWaitEvent(s.stream, grams[gi].ready, 0));
                G_in = grams[gi].G;
                stats.gram_hits += 1;
            } else {
                if (gi >= 0 && grams[gi].inuse > 0) {  // stale copy still read: retire it, fill another slot
                    grams[gi].valid = false;
                    gi = -1;
                }
                if (gi < 0)
                    for (int g = 0; g < kGramSlots; ++g)
                        if (grams[g].inuse == 0 && (gi < 0 || grams[g].last_use < grams[gi].last_use)) gi = g;
                if (gi >= 0) {
                    GramSlot& G = grams[gi];
                    G.B = r.B;
                    G.n = X->n;
                    G.ldb = r.ldb;
                    G.rank = r.rank;
                    G.bdt = r.bdt;
                    G.valid = true;
                    G_out = G.G;
                }
            }
            if (gi >= 0) {
                grams[gi].inuse += 1;
                grams[gi].last_use = ++gram_tick;
                s.reqs[k].gram = gi;
            }
            if (st == SYM_OK)
                st = residual_launch_gram(X, r.B, bf16, r.rank, r.ldb, r.M, r.ldm, s.res_dev + k, s.ws, s.ws_bytes,
                                          G_in, G_out, s.stream);
            if (st == SYM_OK && G_out) st = cuda_status(cudaEventRecord(grams[gi].ready, s.stream));
            if (st != SYM_OK && G_out) grams[gi].valid = false;
            if (st == SYM_OK)
                st = cuda_status(
                    cudaMemcpyAsync(s.res_host + k, s.res_dev + k, sizeof(double), cudaMemcpyDeviceToHost, s.stream));
        }
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
            Slot* group = nullptr;  // the slot collecting this pass's small requests
            // Phase 0 admits requests whose tensor is on the device (or not registered) and registered
            // requests that have waited longer than cfg.affinity_wait_ns; phase 1, with the slots left, the
            // rest (each loading its tensor, after which the queued requests for that tensor are resident too).
            const uint64_t affinity_ns = (uint64_t)std::max<int64_t>(0, cfg.affinity_wait_ns);
            if (loads_in_flight > 0)  // loads that have landed make their tensors admissible
                for (auto& E : entries)
                    if (E.loading && cudaEventQuery(E.ready) != cudaErrorNotReady) {
                        cudaGetLastError();
                        E.loading = false;
                        --loads_in_flight;
                        progressed = true;
                    }
            bool slots_left = true;
            for (int phase = 0; phase < 2 && slots_left; ++phase) {
                for (auto it = queue.begin(); it != queue.end();) {
                    if (phase == 0 && it->reg >= 0 && !entries[(size_t)it->reg].resident &&
                        t - it->t_submit < affinity_ns) {
                        ++it;
                        continue;
                    }
                    if (inflight_bytes + it->bytes > cfg.hbm_budget_bytes) {
                        // head blocked on budget: later requests may pass it for a while
                        if (it == queue.begin() && t - it->t_submit > pass_limit_ns) break;
                        ++it;
                        continue;
                    }
                    if (it->reg >= 0) {
                        // A tensor that is not resident is loaded on the load stream without taking a slot; its
                        // requests are admitted once the copy has landed, so slots keep serving resident work.
                        Entry& E = entries[(size_t)it->reg];
                        if (E.loading) {
                            ++it;
                            continue;
                        }
                        if (!E.resident) {
                            if (loads_in_flight < kMaxLoads) {
                                sym_status err = SYM_OK;
                                if (make_resident(E, load_stream, &err)) {  // false: no room in the pool yet
                                    if (err != SYM_OK) {
                                        fail_queued(it, err);
                                        continue;
                                    }
                                    E.loading = true;
                                    ++loads_in_flight;
                                }
                            }
                            ++it;
                            continue;
                        }
                    }
                    const bool join =
                        cfg.coalesce_small && it->small && group && (int)group->reqs.size() < kMaxGroup;
                    Slot* pick = join ? group : nullptr;
                    if (!pick) {
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
                    }
                    if (!pick) {  // no slot free: both phases end
                        slots_left = false;
                        break;
                    }
                    if (!pick->busy) pick->launch_status = SYM_OK;
                    if (it->reg >= 0) {  // resident and loaded (checked above)
                        Entry& E = entries[(size_t)it->reg];
                        E.inuse += 1;
                        E.last_use = ++tick;
                    }
                    if (!pick->busy) {
                        pick->busy = true;
                        pick->t_admit = t;
                        to_launch.push_back(pick);
                        stats.launches += 1;
                        if (cfg.coalesce_small && it->small) group = pick;
                    } else if ((int)pick->reqs.size() == 1) {
                        stats.grouped_launches += 1;  // the slot's first request now leads a group
                    }
                    pick->reqs.push_back(*it);
                    inflight_bytes += it->bytes;
                    inflight += 1;
                    stats.admitted += 1;
                    stats.peak_inflight = std::max<int64_t>(stats.peak_inflight, inflight);
                    stats.peak_bytes = std::max<int64_t>(stats.peak_bytes, (int64_t)(inflight_bytes + resident_bytes));
                    it = queue.erase(it);
                }
            }
            // Loads need no slot: requests that have waited out the affinity wait get their tensor's load
            // started even while every slot is busy.
            for (auto it = queue.begin(); it != queue.end() && loads_in_flight < kMaxLoads;) {
                if (it->reg >= 0 && t - it->t_submit >= affinity_ns) {
                    Entry& E = entries[(size_t)it->reg];
                    if (!E.resident && !E.loading) {
                        sym_status err = SYM_OK;
                        if (make_resident(E, load_stream, &err)) {
                            if (err != SYM_OK) {
                                fail_queued(it, err);
                                continue;
                            }
                            E.loading = true;
                            ++loads_in_flight;
                        }
                    }
                }
                ++it;
            }
            if (to_launch.empty() && !progressed) {
                if (inflight == 0 && loads_in_flight == 0)
                    cv_sched.wait_for(lk, std::chrono::milliseconds(20), [&] { return stop || !queue.empty(); });
            }
        }
        for (Slot* s : to_launch) launch(*s);
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
    return slot_bytes(cfg) * (size_t)cfg->max_slots + gram_bytes(cfg) * kGramSlots + align_up(cfg->pool_bytes, 256);
}

extern "C" sym_status sym_server_create(const sym_server_cfg* cfg, void* arena, size_t arena_bytes, int device,
                                        sym_server* out) {
    if (!out) return SYM_E_INVALID;
    *out = nullptr;
    if (!cfg || cfg->max_slots < 1 || cfg->max_slots > 256 || cfg->max_rank < 4 || cfg->max_rank > 128 ||
        cfg->max_rank % 4 || cfg->hbm_budget_bytes == 0 || cfg->affinity_wait_ns < 0)
        return SYM_E_INVALID;
    if (cfg->pool_bytes > cfg->hbm_budget_bytes) return SYM_E_BUDGET;
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
    const size_t per = slot_bytes(cfg);
    for (int k = 0; k < cfg->max_slots && st == SYM_OK; ++k) {
        Slot& s = S->slots[(size_t)k];
        s.high = k < (cfg->max_slots + 1) / 2;
        st = cuda_status(cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, s.high ? hi : lo));
        if (st == SYM_OK) st = cuda_status(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
        if (st == SYM_OK)
            st = cuda_status(cudaHostAlloc((void**)&s.res_host, sizeof(double) * kMaxGroup, cudaHostAllocDefault));
        char* base = static_cast<char*>(arena) + per * (size_t)k;
        s.res_dev = reinterpret_cast<double*>(base);
        s.ws = base + align_up(sizeof(double) * kMaxGroup, 256);
        s.ws_bytes = per - align_up(sizeof(double) * kMaxGroup, 256);
    }
    if (st == SYM_OK) st = cuda_status(cudaStreamCreateWithPriority(&S->load_stream, cudaStreamNonBlocking, lo));
    char* gram_base = static_cast<char*>(arena) + per * (size_t)cfg->max_slots;
    for (int g = 0; g < kGramSlots && st == SYM_OK; ++g) {
        S->grams[g].G = reinterpret_cast<double*>(gram_base + gram_bytes(cfg) * (size_t)g);
        st = cuda_status(cudaEventCreateWithFlags(&S->grams[g].ready, cudaEventDisableTiming));
    }
    S->pool = gram_base + gram_bytes(cfg) * kGramSlots;
    S->pool_bytes = align_up(cfg->pool_bytes, 256);
    if (S->pool_bytes) S->free_ranges[0] = S->pool_bytes;
    if (st != SYM_OK) {
        S->release();
        delete S;
        return st;
    }
    try {
        S->th = std::thread([S] { S->run(); });
    } catch (...) {
        S->release();
        delete S;
        return SYM_E_NOMEM;
    }
    *out = S;
    return SYM_OK;
}

extern "C" sym_status sym_server_register(sym_server S, const void* image, uint64_t* id) {
    if (!S || !image || !id) return SYM_E_INVALID;
    const size_t bytes = sym_tensor_load_bytes(image);
    if (bytes == 0) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return SYM_E_INVALID;
    if (align_up(bytes, 256) > S->pool_bytes) return SYM_E_BUDGET;  // could never be resident
    Entry e;
    e.image = image;
    e.bytes = align_up(bytes, 256);
    if (cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming) != cudaSuccess) return SYM_E_CUDA;
    S->entries.push_back(e);
    *id = (uint64_t)(S->entries.size() - 1);
    return SYM_OK;
}

static sym_status enqueue(sym_server S, const sym_request& r, int64_t reg, int64_t n, int64_t nnz, size_t tensor_bytes,
                          uint64_t* ticket) {
    const size_t bytes = tensor_bytes + factor_bytes(r, n);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return SYM_E_INVALID;
        if (bytes + (reg >= 0 ? S->pool_bytes : 0) > S->cfg.hbm_budget_bytes) {
            S->stats.rejected += 1;
            return SYM_E_BUDGET;
        }
        Pending p{S->next_ticket++, r, reg, bytes, now_ns(), nnz <= S->cfg.small_nnz};
        S->queue.push_back(p);
        S->live.insert(p.ticket);
        S->stats.submitted += 1;
        *ticket = p.ticket;
    }
    S->cv_sched.notify_one();
    return SYM_OK;
}

extern "C" sym_status sym_batch_submit(sym_server S, const sym_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return SYM_E_INVALID;
    if (!req->X) return SYM_E_BADREQ;
    if (validate_mttkrp_args(req->X, req->B, req->bdt, req->rank, req->ldb, req->M, req->ldm) != SYM_OK)
        return SYM_E_BADREQ;
    if (req->rank > S->cfg.max_rank || req->want_residual < 0 || req->want_residual > 2) return SYM_E_BADREQ;
    return enqueue(S, *req, -1, req->X->n, req->X->nnz, req->X->info.arena_used, ticket);
}

extern "C" sym_status sym_batch_submit_registered(sym_server S, uint64_t id, const sym_request* req,
                                                  uint64_t* ticket) {
    if (!S || !req || !ticket) return SYM_E_INVALID;
    int64_t n = 0, nnz = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (id >= S->entries.size()) return SYM_E_NOTFOUND;
        // the header fields the checks need, without touching the device
        const size_t lb = sym_tensor_load_bytes(S->entries[(size_t)id].image);
        if (lb == 0) return SYM_E_BADREQ;
        sym_tensor_info_t inf;
        if (sym_tensor_image_info(S->entries[(size_t)id].image, &inf) != SYM_OK) return SYM_E_BADREQ;
        n = inf.n;
        nnz = inf.nnz;
    }
    if (!req->B || !req->M || (req->bdt != SYM_F32 && req->bdt != SYM_BF16)) return SYM_E_BADREQ;
    if (req->want_residual < 0 || req->want_residual > 2) return SYM_E_BADREQ;
    if (req->rank < 4 || req->rank > 128 || req->rank % 4 || req->rank > S->cfg.max_rank) return SYM_E_BADREQ;
    if (req->ldb < req->rank || req->ldm < req->rank || req->ldb % 4 || req->ldm % 4) return SYM_E_BADREQ;
    if (!aligned(req->B, req->bdt == SYM_BF16 ? 8 : 16) || !aligned(req->M, 16)) return SYM_E_BADREQ;
    sym_request r = *req;
    r.X = nullptr;
    return enqueue(S, r, (int64_t)id, n, nnz, 0, ticket);
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
    out->resident_bytes = (int64_t)S->resident_bytes;
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
