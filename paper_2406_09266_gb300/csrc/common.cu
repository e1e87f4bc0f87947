// Status strings, CUDA error capture, device queries and the opt-in per-kernel
// event profiler.
#include <atomic>
#include <mutex>
#include <string.h>
#include <string>
#include <vector>

#include "common.cuh"

namespace symgpu {

static thread_local int g_last_cuda_error = 0;

sym_status cuda_status(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return e == cudaSuccess ? SYM_OK : SYM_E_CUDA;
}

int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return 0;
    return d;
}

sym_status raise_smem_limit(const void* func, size_t bytes) {
    if (bytes <= 48 * 1024) return SYM_OK;  // within the default limit of every kernel
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void*, int>, size_t>> raised;
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(mu);
    for (auto& r : raised)
        if (r.first.first == func && r.first.second == dev) {
            if (r.second >= bytes) return SYM_OK;
            SYM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
            r.second = bytes;
            return SYM_OK;
        }
    SYM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    raised.push_back({{func, dev}, bytes});
    return SYM_OK;
}

int sm_count() {
    static int cached[64] = {0};
    int d = current_device();
    if (d < 0 || d >= 64) d = 0;
    if (cached[d] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) v = 148;
        cached[d] = v;
    }
    return cached[d];
}

namespace {

struct PendingEvent {
    std::string name;
    cudaEvent_t a, b;
};
struct Totals {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
};

std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
std::vector<PendingEvent> g_pending;
std::vector<cudaEvent_t> g_free_events;
std::vector<Totals> g_totals;

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void drain_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Totals* t = nullptr;
            for (auto& x : g_totals)
                if (x.name == p.name) t = &x;
            if (!t) {
                g_totals.push_back(Totals{p.name, 0, 0.0});
                t = &g_totals.back();
            }
            t->launches += 1;
            t->ms += ms;
        }
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace

ProfScope::ProfScope(const char* n, cudaStream_t s) : name(n), stream(s), start(nullptr) {
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = take_event();
    if (e && cudaEventRecord(e, s) == cudaSuccess) start = e;
}

ProfScope::~ProfScope() {
    if (!start) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = take_event();
    if (e && cudaEventRecord(e, stream) == cudaSuccess) {
        g_pending.push_back(PendingEvent{name, (cudaEvent_t)start, e});
        if (g_pending.size() > 4096) drain_locked();
    }
}

std::vector<sym_status (*)(unsigned long long*)>& bc_setters() {
    static std::vector<sym_status (*)(unsigned long long*)> v;  // filled during static initialisation
    return v;
}

void bc_register_setter(sym_status (*set)(unsigned long long*)) { bc_setters().push_back(set); }

}  // namespace symgpu

extern "C" int sym_bounds_check_enabled(void) {
#ifdef SYM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

extern "C" sym_status sym_bounds_check_attach(unsigned long long* counter) {
#ifdef SYM_BOUNDS_CHECK
    if (counter && !symgpu::aligned(counter, 8)) return SYM_E_INVALID;
    for (auto set : symgpu::bc_setters()) {
        const sym_status st = set(counter);
        if (st != SYM_OK) return st;
    }
    return SYM_OK;
#else
    (void)counter;
    return SYM_E_UNSUPPORTED;
#endif
}

extern "C" sym_status sym_profile_enable(int on) {
    symgpu::g_prof_on.store(on ? 1 : 0);
    return SYM_OK;
}

extern "C" int sym_profile_read(sym_profile_entry* out, int max_entries) {
    std::lock_guard<std::mutex> lk(symgpu::g_prof_mu);
    symgpu::drain_locked();
    int k = 0;
    for (auto& t : symgpu::g_totals) {
        if (k >= max_entries || !out) break;
        memset(&out[k], 0, sizeof(out[k]));
        strncpy(out[k].name, t.name.c_str(), sizeof(out[k].name) - 1);
        out[k].launches = t.launches;
        out[k].total_ms = t.ms;
        ++k;
    }
    return k;
}

extern "C" sym_status sym_profile_reset(void) {
    std::lock_guard<std::mutex> lk(symgpu::g_prof_mu);
    symgpu::drain_locked();
    symgpu::g_totals.clear();
    return SYM_OK;
}

extern "C" const char* sym_status_string(sym_status s) {
    switch (s) {
        case SYM_OK: return "ok";
        case SYM_E_INVALID: return "invalid argument";
        case SYM_E_NONCANONICAL: return "input is not canonical";
        case SYM_E_RANGE: return "index out of range";
        case SYM_E_DUPLICATE: return "duplicate entry";
        case SYM_E_NOMEM: return "arena or workspace too small";
        case SYM_E_BUDGET: return "request exceeds the HBM budget";
        case SYM_E_TIMEOUT: return "bounded wait timed out";
        case SYM_E_CUDA: return "CUDA runtime error";
        case SYM_E_BADREQ: return "malformed request";
        case SYM_E_UNSUPPORTED: return "unsupported shape";
        case SYM_E_NOTFOUND: return "unknown ticket";
        case SYM_PENDING: return "pending";
    }
    return "unknown status";
}

extern "C" int sym_last_cuda_error(void) { return symgpu::g_last_cuda_error; }

extern "C" int sym_version(void) { return SYMGPU_VERSION; }
