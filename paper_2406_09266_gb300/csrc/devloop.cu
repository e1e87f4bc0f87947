// Device-resident request loop: symmetric MTTKRP (Sec. 4.3, Sec. 5.2.6) and
// SSYMV / SYPRD (Sec. 3.1, Sec. 5.2.1, Sec. 5.2.3) requests served by one
// persistent kernel that takes them from a ring in mapped host memory (the
// paper has no serving layer; the arithmetic is that of the single calls).
//
// Protocol.  The host writes request r into ring slot r mod S and publishes it
// by raising `tail` (release order).  Every CTA of the loop kernel runs the
// same loop: its thread 0 reads `cur`, the request the CTA takes work from,
// and, once that request is published, claims its next chunk with a
// compare-and-swap on the slot's claim word (request index in the high half,
// chunks claimed in the low half).  A request is cut into zero chunks (its
// output cleared) followed by compute chunks (entries of the tensor or of the
// CSR); a compute chunk starts once every zero chunk of its request is done
// (those were claimed before it by running CTAs that wait for nothing, so the
// wait ends).  When every chunk of `cur` is claimed, or its slot already holds
// a later request, the next CAS moves `cur` on.  The CTA that completes a
// request's last chunk writes SYPRD, resets the slot's counters for request
// r + S, stamps the completion time (%globaltimer) and stores r + 1 in the
// slot's completion word in mapped host memory, which the host polls.
//
// Requests of any order, rank and factor type share the kernel, so the MTTKRP
// chunks use the per-entry form (each canonical entry updates the output row of
// every distinct index of its tuple, weighted by its arrangement count), not the
// fiber-factorised kernels of the single call.
//
// Inputs are read with L2-only loads (ld.global.cg): a persistent kernel keeps
// its L1 lines across requests, and a caller may rewrite a factor or x between
// two requests.  Outputs are cleared with L2-only stores and formed with L2
// reductions.
//
// Every wait is bounded: a CTA leaves the loop after idle_ns without a published
// request (the host relaunches the kernel for the next one) or when the host
// raises `stop`; the wait for a request's zero chunks gives up after wait_ns and
// the request completes with SYM_E_TIMEOUT.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace symgpu {
namespace {

constexpr int DL_THREADS = 256;
constexpr int DL_WARPS = DL_THREADS / 32;
constexpr int64_t DL_SV_PER_THREAD = 16;                        // CSR entries per thread of an SSYMV chunk
constexpr int64_t DL_SV_CHUNK = DL_SV_PER_THREAD * DL_THREADS;  // 4,096
constexpr int64_t DL_MT_PER_GROUP = 8;                          // tensor entries per lane group of a chunk
constexpr int64_t DL_ZERO = 32768;                              // output floats cleared per zero chunk
constexpr int32_t DL_MTTKRP = 1, DL_SSYMV = 2;

// One request as the loop kernel reads it (host-written, mapped memory).
struct DLReq {
    int32_t kind, order, kw, bits;
    int32_t bf16, rank, lanes;
    int32_t hook;     // test hook: 1 = the zero chunks are done but not counted (the compute chunks' wait runs out)
    int64_t n, nnz;
    int64_t zchunks;  // zero chunks (first), then compute chunks
    int64_t nchunks;  // all chunks
    int64_t zrows;    // output rows (MTTKRP) or floats (SSYMV) per zero chunk
    int64_t chunk;    // entries per compute chunk
    const uint64_t* klo;
    const uint64_t* khi;
    const float* val;
    const int32_t* rowptr;
    const int32_t* col;
    const void* B;  // factor (MTTKRP) or x (SSYMV)
    int64_t ldb;
    float* M;       // output (MTTKRP) or y (SSYMV)
    int64_t ldm;
    double* syprd;  // SSYMV: x^T A x, or null
};
static_assert(sizeof(DLReq) % 8 == 0, "DLReq is copied as 8-byte words");
constexpr int DL_REQ_WORDS = (int)(sizeof(DLReq) / 8);

// Host-written control words (mapped memory).
struct DLCtl {
    uint64_t tail;  // requests published
    uint32_t stop;  // leave the loop now
    uint32_t pad;
};

struct DLArgs {
    const DLReq* ring;             // [S] mapped
    const DLCtl* ctl;              // mapped
    unsigned long long* done_seq;  // [S] mapped: r + 1 once request r is complete
    unsigned long long* t_done;    // [S] mapped: %globaltimer at completion
    int* status;                   // [S] mapped: SYM_OK or SYM_E_TIMEOUT
    unsigned long long* cur;       // device: request the CTAs take work from
    unsigned long long* claim;     // [S] device: (request index mod 2^32) << 32 | chunks claimed
    unsigned* done;                // [S] device: chunks finished
    unsigned* zdone;               // [S] device: zero chunks finished
    unsigned* err;                 // [S] device: a wait of the request ran out
    double* acc;                   // [S] device: SYPRD sum
    unsigned long long mask;       // S - 1
    uint64_t idle_ns, wait_ns;
};

__device__ __forceinline__ uint64_t dl_now() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint64_t dl_ld_acquire_sys(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dl_st_release_sys(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <bool BF16>
__device__ __forceinline__ float4 dl_row4(const void* B, int64_t row, int64_t ldb, int col) {
    if constexpr (BF16) {
        const uint2 u = __ldcg(reinterpret_cast<const uint2*>(static_cast<const __nv_bfloat16*>(B) + row * ldb + col));
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                           __uint_as_float(u.y & 0xffff0000u));
    } else {
        return __ldcg(reinterpret_cast<const float4*>(static_cast<const float*>(B) + row * ldb + col));
    }
}

// Thread 0: claims the next chunk.  False: leave the loop (stop, or idle for
// idle_ns, both seen only when no published chunk is left to claim).  `tail_seen` caches the last published count read (it only grows),
// so a busy loop does not read mapped memory for every claim.
__device__ bool dl_claim(const DLArgs& a, DLReq* sreq, long long* cached, uint64_t* tail_seen,
                         unsigned long long* out_r, unsigned* out_k) {
    bool idle = false;
    uint64_t idle0 = 0;
    unsigned nap = 128;  // idle back-off, up to 4 us between reads of the mapped tail
    for (;;) {
        const unsigned long long r = *reinterpret_cast<volatile unsigned long long*>(a.cur);
        if (r >= *tail_seen) *tail_seen = dl_ld_acquire_sys(&a.ctl->tail);
        if (r >= *tail_seen) {
            // nothing published to take: leave on `stop` (read only here, so a busy loop does not
            // read mapped memory per claim; the host raises it once its requests are done) or when idle
            if (*reinterpret_cast<const volatile uint32_t*>(&a.ctl->stop)) return false;
            const uint64_t t = dl_now();
            if (!idle) {
                idle = true;
                idle0 = t;
            } else if (t - idle0 > a.idle_ns) {
                return false;
            }
            __nanosleep(nap);
            nap = min(2 * nap, 4096u);
            continue;
        }
        idle = false;
        nap = 128;
        const unsigned long long slot = r & a.mask;
        if (*cached != (long long)r) {
            const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(a.ring + slot);
            unsigned long long* dst = reinterpret_cast<unsigned long long*>(sreq);
            for (int w = 0; w < DL_REQ_WORDS; ++w) dst[w] = src[w];
            *cached = (long long)r;
        }
        const unsigned long long c = *reinterpret_cast<volatile unsigned long long*>(a.claim + slot);
        const unsigned k = (unsigned)(c & 0xffffffffull);
        if ((c >> 32) != (r & 0xffffffffull) || k >= (unsigned)sreq->nchunks) {
            // every chunk of r is claimed, or r is complete and its slot reset for r + S
            atomicCAS(a.cur, r, r + 1);
            continue;
        }
        if (atomicCAS(a.claim + slot, c, c + 1) == c) {
            *out_r = r;
            *out_k = k;
            return true;
        }
    }
}

// Thread 0: waits until the request's zero chunks are done (bounded).
__device__ bool dl_wait_zero(const DLArgs& a, unsigned long long slot, unsigned z) {
    const volatile unsigned* p = a.zdone + slot;
    if (*p >= z) return true;
    const uint64_t t0 = dl_now();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (*p >= z) return true;
        if (dl_now() - t0 > a.wait_ns) return false;
        __nanosleep(128);
    }
}

__device__ void dl_zero(const DLReq& q, int64_t z) {
    if (q.kind == DL_MTTKRP) {
        const int64_t r0 = z * q.zrows, r1 = min(q.n, r0 + q.zrows);
        const int per = q.rank / 4;
        const int64_t cnt = (r1 - r0) * per;
        for (int64_t t = threadIdx.x; t < cnt; t += DL_THREADS) {
            const int64_t row = r0 + t / per;
            const int c4 = 4 * (int)(t % per);
            __stcg(reinterpret_cast<float4*>(q.M + row * q.ldm + c4), f4_zero());
        }
    } else {
        const int64_t a0 = z * q.zrows, a1 = min(q.n, a0 + q.zrows);
        for (int64_t t = a0 + threadIdx.x; t < a1; t += DL_THREADS) __stcg(q.M + t, 0.f);
    }
}

// MTTKRP compute chunk: entries [e0, e1) of the canonical stream, one entry
// per lane group of q.lanes lanes (4 columns per lane).  For the sorted tuple
// c of an entry with value v, the output row of each distinct index u gets
// v * W_u * prod over the other positions of B rows, W_u = (N-1)! m_u / prod_t m_t!
// (the arrangements of the tuple with u first; m_t are the run lengths).
template <int N, int KW, bool BF16>
__device__ void dl_mttkrp_chunk(const DLReq& q, int64_t e0, int64_t e1) {
    const int L = q.lanes;
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane & (L - 1));
    if (col >= q.rank) return;
    const int gpw = 32 / L;
    const int group = (int)(threadIdx.x >> 5) * gpw + lane / L;
    const int G = DL_WARPS * gpw;
    const int64_t n = q.n, ldb = q.ldb, ldm = q.ldm;
    const void* B = q.B;
    float* M = q.M;
    const int bits = q.bits;
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    for (int64_t e = e0 + group; e < e1; e += G) {
        int32_t c[N];
        unpack_key<N, KW>(KeyWords{__ldcg(q.klo + e), KW == 2 ? __ldcg(q.khi + e) : 0ull}, bits, c);
        bool ok = true;
#pragma unroll
        for (int p = 0; p < N; ++p) ok = ok && (uint32_t)c[p] < (uint64_t)n;
        if (!ok) continue;  // (tensors are range-checked at creation)
        const float v = __ldcg(q.val + e);
        float4 b[N];
#pragma unroll
        for (int p = 0; p < N; ++p) b[p] = dl_row4<BF16>(B, c[p], ldb, col);
        float4 pre[N + 1], suf[N + 1];
        pre[0] = make_float4(1.f, 1.f, 1.f, 1.f);
        suf[N] = pre[0];
#pragma unroll
        for (int p = 0; p < N; ++p) pre[p + 1] = f4_mul(pre[p], b[p]);
#pragma unroll
        for (int p = N - 1; p >= 0; --p) suf[p] = f4_mul(suf[p + 1], b[p]);
        int den = 1, run = 1;
#pragma unroll
        for (int p = 1; p < N; ++p) {
            if (c[p] == c[p - 1]) {
                ++run;
            } else {
                den *= fact[run];
                run = 1;
            }
        }
        den *= fact[run];
#pragma unroll
        for (int p = 0; p < N; ++p) {
            if (p > 0 && c[p] == c[p - 1]) continue;  // not the first position of its run
            int m = 1;
#pragma unroll
            for (int t = p + 1; t < N; ++t)
                if (c[t] == c[p]) ++m;
            const float W = (float)(fact[N - 1] * m / den);
            red_add_f4(M + (int64_t)c[p] * ldm + col, f4_scale(f4_mul(pre[p], suf[p + 1]), W * v));
        }
    }
}

__device__ void dl_mttkrp(const DLReq& q, int64_t e0, int64_t e1) {
    const int key = q.order * 4 + (q.kw == 2 ? 2 : 0) + (q.bf16 ? 1 : 0);
    switch (key) {
        case 8: dl_mttkrp_chunk<2, 1, false>(q, e0, e1); break;
        case 9: dl_mttkrp_chunk<2, 1, true>(q, e0, e1); break;
        case 12: dl_mttkrp_chunk<3, 1, false>(q, e0, e1); break;
        case 13: dl_mttkrp_chunk<3, 1, true>(q, e0, e1); break;
        case 14: dl_mttkrp_chunk<3, 2, false>(q, e0, e1); break;
        case 15: dl_mttkrp_chunk<3, 2, true>(q, e0, e1); break;
        case 16: dl_mttkrp_chunk<4, 1, false>(q, e0, e1); break;
        case 17: dl_mttkrp_chunk<4, 1, true>(q, e0, e1); break;
        case 18: dl_mttkrp_chunk<4, 2, false>(q, e0, e1); break;
        case 19: dl_mttkrp_chunk<4, 2, true>(q, e0, e1); break;
        case 20: dl_mttkrp_chunk<5, 1, false>(q, e0, e1); break;
        case 21: dl_mttkrp_chunk<5, 1, true>(q, e0, e1); break;
        case 22: dl_mttkrp_chunk<5, 2, false>(q, e0, e1); break;
        case 23: dl_mttkrp_chunk<5, 2, true>(q, e0, e1); break;
        default: break;  // (the host accepts orders 2..5 only)
    }
}

// SSYMV compute chunk: CSR entries [e0, e1), 16 consecutive entries per
// thread.  a_ij adds a x_j to y_i (summed over the thread's run of row i, one
// reduction per run) and, for j > i, a x_i to y_j; returns the thread's SYPRD
// terms (off-diagonal ones twice) in FP32.
__device__ float dl_ssymv_chunk(const DLReq& q, int64_t e0, int64_t e1) {
    const int64_t b = e0 + (int64_t)threadIdx.x * DL_SV_PER_THREAD;
    const int64_t end = min(b + DL_SV_PER_THREAD, e1);
    float sp = 0.f;
    if (b >= end) return sp;
    const int64_t n = q.n;
    const int32_t* rowptr = q.rowptr;
    const int32_t* col = q.col;
    const float* val = q.val;
    const float* x = static_cast<const float*>(q.B);
    float* y = q.M;
    // row of entry b: the last i with rowptr[i] <= b
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)__ldcg(rowptr + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    int64_t i = lo;
    int64_t next = __ldcg(rowptr + i + 1);
    float xi = __ldcg(x + i);
    float run = 0.f;
    for (int64_t e = b; e < end; ++e) {
        while (e >= next && i < n - 1) {
            if (run != 0.f) atomicAdd(y + i, run);
            run = 0.f;
            ++i;
            next = __ldcg(rowptr + i + 1);
            xi = __ldcg(x + i);
        }
        const int32_t j = __ldcg(col + e);
        if ((uint32_t)j >= (uint64_t)n) continue;  // (the CSR is trusted; never read outside x)
        const float av = __ldcg(val + e);
        const float t = av * __ldcg(x + j);
        run += t;
        if (j != i) atomicAdd(y + j, av * xi);
        sp = fmaf(j != i ? 2.f * t : t, xi, sp);
    }
    if (run != 0.f) atomicAdd(y + i, run);
    return sp;
}

// Thread 0 of the CTA that finished request r's last chunk.
__device__ void dl_finish(const DLArgs& a, const DLReq& q, unsigned long long r, unsigned long long slot) {
    __threadfence();
    const bool failed = *reinterpret_cast<volatile unsigned*>(a.err + slot) != 0;
    if (q.kind == DL_SSYMV && q.syprd)
        *q.syprd = failed ? __longlong_as_double(0x7ff8000000000000ll)
                          : *reinterpret_cast<volatile double*>(a.acc + slot);
    *reinterpret_cast<volatile double*>(a.acc + slot) = 0.0;
    *reinterpret_cast<volatile unsigned*>(a.err + slot) = 0u;
    *reinterpret_cast<volatile unsigned*>(a.done + slot) = 0u;
    *reinterpret_cast<volatile unsigned*>(a.zdone + slot) = 0u;
    *reinterpret_cast<volatile unsigned long long*>(a.claim + slot) = ((r + a.mask + 1) & 0xffffffffull) << 32;
    __threadfence_system();
    *reinterpret_cast<volatile int*>(a.status + slot) = failed ? (int)SYM_E_TIMEOUT : (int)SYM_OK;
    *reinterpret_cast<volatile unsigned long long*>(a.t_done + slot) = dl_now();
    __threadfence_system();
    dl_st_release_sys(a.done_seq + slot, r + 1);
}

__global__ void __launch_bounds__(DL_THREADS) k_devloop(DLArgs a) {
    __shared__ DLReq s_req;
    __shared__ long long s_cached;
    __shared__ uint64_t s_tail;
    __shared__ unsigned long long s_r;
    __shared__ unsigned s_k;
    __shared__ int s_go, s_ok;
    __shared__ double s_part[DL_WARPS];
    if (threadIdx.x == 0) {
        s_cached = -1;
        s_tail = 0;
    }
    for (;;) {
        if (threadIdx.x == 0) {
            long long cached = s_cached;
            uint64_t tail = s_tail;
            unsigned long long r = 0;
            unsigned k = 0;
            const bool go = dl_claim(a, &s_req, &cached, &tail, &r, &k);
            s_cached = cached;
            s_tail = tail;
            s_r = r;
            s_k = k;
            s_go = go ? 1 : 0;
            s_ok = (go && k >= (unsigned)s_req.zchunks) ? (dl_wait_zero(a, r & a.mask, (unsigned)s_req.zchunks) ? 1 : 0)
                                                         : 1;
        }
        __syncthreads();
        if (!s_go) break;
        const unsigned long long r = s_r, slot = r & a.mask;
        const int64_t k = s_k, Z = s_req.zchunks;
        const bool ok = s_ok != 0;
        const bool sv = s_req.kind == DL_SSYMV;
        float sp = 0.f;
        if (k < Z) {
            dl_zero(s_req, k);
        } else if (ok) {
            const int64_t e0 = (k - Z) * s_req.chunk, e1 = min(s_req.nnz, e0 + s_req.chunk);
            if (sv) sp = dl_ssymv_chunk(s_req, e0, e1);
            else dl_mttkrp(s_req, e0, e1);
        }
        const bool want_sp = sv && k >= Z && s_req.syprd != nullptr;  // uniform over the CTA
        if (want_sp) {
            const double w = warp_sum((double)sp);
            if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = w;
        }
        __threadfence();  // this thread's stores and reductions before the chunk is counted
        __syncthreads();
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(a.err + slot, 1u);
            if (want_sp) {
                double s = 0.0;
                for (int w = 0; w < DL_WARPS; ++w) s += s_part[w];
                atomicAdd(a.acc + slot, s);
            }
            __threadfence();
            if (k < Z && s_req.hook != 1) atomicAdd(a.zdone + slot, 1u);
            const unsigned prev = atomicAdd(a.done + slot, 1u);
            if (prev + 1 == (unsigned)s_req.nchunks) dl_finish(a, s_req, r, slot);
        }
    }
}

// One thread writes %globaltimer into mapped memory (clock calibration).
__global__ void k_dl_clock(unsigned long long* out) {
    *reinterpret_cast<volatile unsigned long long*>(out) = dl_now();
    __threadfence_system();
}

uint64_t host_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Flight {
    size_t bytes;
    uint64_t t_submit, t_admit, tag;
};

struct Queued {
    DLReq q;
    size_t bytes;
    uint64_t t_submit, tag, ticket;
};

}  // namespace
}  // namespace symgpu

using namespace symgpu;

struct sym_devloop_s {
    std::mutex mu;
    sym_devloop_cfg cfg{};
    int device = 0;
    int ctas = 0;
    uint64_t S = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_exit = nullptr;
    bool launched = false;
    // mapped host memory: ring, control, completion words, completion times, statuses
    void* host_block = nullptr;
    DLReq* ring_h = nullptr;
    DLCtl* ctl_h = nullptr;
    unsigned long long* done_seq_h = nullptr;
    unsigned long long* t_done_h = nullptr;
    int* status_h = nullptr;
    unsigned long long* clock_h = nullptr;
    DLArgs args{};
    void* dev_block = nullptr;
    int64_t gt_minus_host = 0;  // %globaltimer - host steady clock (ns)
    uint64_t next_ticket = 0;   // tickets are request indices, published in submission order
    std::deque<Queued> queue;   // submitted, not yet published (ring slot or budget not free)
    std::unordered_map<uint64_t, Flight> flight;
    std::unordered_map<uint64_t, sym_result> results;
    size_t inflight_bytes = 0;
    int hook = 0;  // test hook copied into the requests submitted while it is set
    sym_devloop_stats stats{};
};

namespace {

// Launches the loop kernel if it is not running (mu held).
sym_status dl_ensure_running(sym_devloop L) {
    if (L->launched) {
        const cudaError_t q = cudaEventQuery(L->ev_exit);
        if (q == cudaErrorNotReady) return SYM_OK;
        if (q != cudaSuccess) return cuda_status(q);
    }
    // launch on the loop's device whatever device the calling thread has current
    int prev = -1;
    SYM_CUDA(cudaGetDevice(&prev));
    if (prev != L->device) SYM_CUDA(cudaSetDevice(L->device));
    k_devloop<<<L->ctas, DL_THREADS, 0, L->stream>>>(L->args);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(L->ev_exit, L->stream);
    if (prev != L->device) cudaSetDevice(prev);
    SYM_CUDA(e);
    L->launched = true;
    L->stats.launches += 1;
    return SYM_OK;
}

// Retires completed requests and publishes queued ones in order (mu held).
sym_status dl_progress(sym_devloop L) {
    for (auto it = L->flight.begin(); it != L->flight.end();) {
        const uint64_t r = it->first, slot = r & (L->S - 1);
        const unsigned long long d = __atomic_load_n(&L->done_seq_h[slot], __ATOMIC_ACQUIRE);
        if (d != r + 1) {
            ++it;
            continue;
        }
        sym_result res{};
        res.status = (sym_status)__atomic_load_n(&L->status_h[slot], __ATOMIC_ACQUIRE);
        res.residual = 0.0;
        res.user_tag = it->second.tag;
        res.t_submit_ns = it->second.t_submit;
        res.t_admit_ns = it->second.t_admit;
        const int64_t td = (int64_t)__atomic_load_n(&L->t_done_h[slot], __ATOMIC_ACQUIRE) - L->gt_minus_host;
        res.t_done_ns = std::max<uint64_t>((uint64_t)std::max<int64_t>(td, 0), res.t_admit_ns);
        L->inflight_bytes -= it->second.bytes;
        L->results[r] = res;
        L->stats.completed += 1;
        it = L->flight.erase(it);
    }
    bool published = false;
    while (!L->queue.empty()) {
        Queued& h = L->queue.front();
        const uint64_t r = h.ticket, slot = r & (L->S - 1);
        // slot free once request r - S has been retired; budget for the bytes it touches
        if (r >= L->S && L->flight.count(r - L->S)) break;
        if (L->inflight_bytes + h.bytes > L->cfg.hbm_budget_bytes && !L->flight.empty()) break;
        L->ring_h[slot] = h.q;
        L->inflight_bytes += h.bytes;
        L->flight[r] = Flight{h.bytes, h.t_submit, host_ns(), h.tag};
        __atomic_store_n(&L->ctl_h->tail, r + 1, __ATOMIC_RELEASE);
        L->stats.published += 1;
        L->stats.peak_inflight = std::max<int64_t>(L->stats.peak_inflight, (int64_t)L->flight.size());
        L->stats.peak_bytes = std::max<int64_t>(L->stats.peak_bytes, (int64_t)L->inflight_bytes);
        L->queue.pop_front();
        published = true;
    }
    if (published || !L->flight.empty()) return dl_ensure_running(L);
    return SYM_OK;
}

sym_status dl_submit(sym_devloop L, const DLReq& q, size_t bytes, uint64_t tag, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(L->mu);
    if (bytes > L->cfg.hbm_budget_bytes) {
        L->stats.rejected += 1;
        return SYM_E_BUDGET;
    }
    Queued h{q, bytes, host_ns(), tag, L->next_ticket++};
    h.q.hook = L->hook;
    L->queue.push_back(h);
    L->stats.submitted += 1;
    *ticket = h.ticket;
    return dl_progress(L);
}

void dl_free(sym_devloop L) {
    if (L->ev_exit) cudaEventDestroy(L->ev_exit);
    if (L->stream) cudaStreamDestroy(L->stream);
    if (L->dev_block) cudaFree(L->dev_block);
    if (L->host_block) cudaFreeHost(L->host_block);
    delete L;
}

}  // namespace

extern "C" sym_status sym_devloop_create(const sym_devloop_cfg* cfg, int device, sym_devloop* out) {
    if (!cfg || !out) return SYM_E_INVALID;
    const int S = cfg->ring_slots;
    if (S < 16 || S > 4096 || (S & (S - 1)) != 0) return SYM_E_INVALID;
    if (cfg->ctas < 0 || cfg->ctas > 8 * 1024 || cfg->idle_exit_ns <= 0 || cfg->wait_limit_ns <= 0)
        return SYM_E_INVALID;
    int prev = -1;
    SYM_CUDA(cudaGetDevice(&prev));
    SYM_CUDA(cudaSetDevice(device));
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{prev};
    sym_devloop L = new (std::nothrow) sym_devloop_s();
    if (!L) return SYM_E_INVALID;
    L->cfg = *cfg;
    L->device = device;
    L->S = (uint64_t)S;
    L->ctas = cfg->ctas > 0 ? cfg->ctas : 2 * sm_count();
    // mapped host block: ring | control | done_seq | t_done | status | clock word
    const size_t ring_b = align_up(sizeof(DLReq) * S, 128), ctl_b = 128, seq_b = align_up(8 * (size_t)S, 128),
                 st_b = align_up(4 * (size_t)S, 128);
    const size_t host_bytes = ring_b + ctl_b + 2 * seq_b + st_b + 128;
    auto fail = [&](cudaError_t e) {
        dl_free(L);
        return cuda_status(e);
    };
    cudaError_t e = cudaHostAlloc(&L->host_block, host_bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return fail(e);
    memset(L->host_block, 0, host_bytes);
    char* h = static_cast<char*>(L->host_block);
    L->ring_h = reinterpret_cast<DLReq*>(h);
    L->ctl_h = reinterpret_cast<DLCtl*>(h + ring_b);
    L->done_seq_h = reinterpret_cast<unsigned long long*>(h + ring_b + ctl_b);
    L->t_done_h = reinterpret_cast<unsigned long long*>(h + ring_b + ctl_b + seq_b);
    L->status_h = reinterpret_cast<int*>(h + ring_b + ctl_b + 2 * seq_b);
    L->clock_h = reinterpret_cast<unsigned long long*>(h + ring_b + ctl_b + 2 * seq_b + st_b);
    void* hd = nullptr;
    if ((e = cudaHostGetDevicePointer(&hd, L->host_block, 0)) != cudaSuccess) return fail(e);
    char* d = static_cast<char*>(hd);
    L->args.ring = reinterpret_cast<const DLReq*>(d);
    L->args.ctl = reinterpret_cast<const DLCtl*>(d + ring_b);
    L->args.done_seq = reinterpret_cast<unsigned long long*>(d + ring_b + ctl_b);
    L->args.t_done = reinterpret_cast<unsigned long long*>(d + ring_b + ctl_b + seq_b);
    L->args.status = reinterpret_cast<int*>(d + ring_b + ctl_b + 2 * seq_b);
    unsigned long long* clock_d = reinterpret_cast<unsigned long long*>(d + ring_b + ctl_b + 2 * seq_b + st_b);
    // device block: cur | claim[S] | acc[S] | done[S] | zdone[S] | err[S]
    const size_t dev_bytes = 256 + 8 * (size_t)S * 2 + 4 * (size_t)S * 3;
    if ((e = cudaMalloc(&L->dev_block, dev_bytes)) != cudaSuccess) return fail(e);
    char* g = static_cast<char*>(L->dev_block);
    L->args.cur = reinterpret_cast<unsigned long long*>(g);
    L->args.claim = reinterpret_cast<unsigned long long*>(g + 256);
    L->args.acc = reinterpret_cast<double*>(g + 256 + 8 * (size_t)S);
    L->args.done = reinterpret_cast<unsigned*>(g + 256 + 16 * (size_t)S);
    L->args.zdone = reinterpret_cast<unsigned*>(g + 256 + 16 * (size_t)S + 4 * (size_t)S);
    L->args.err = reinterpret_cast<unsigned*>(g + 256 + 16 * (size_t)S + 8 * (size_t)S);
    std::vector<unsigned long long> claim0((size_t)S);
    for (int s = 0; s < S; ++s) claim0[(size_t)s] = (unsigned long long)s << 32;  // slot s first serves request s
    if ((e = cudaMemset(L->dev_block, 0, dev_bytes)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(L->args.claim, claim0.data(), 8 * (size_t)S, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);
    L->args.mask = (unsigned long long)(S - 1);
    L->args.idle_ns = (uint64_t)cfg->idle_exit_ns;
    L->args.wait_ns = (uint64_t)cfg->wait_limit_ns;
    if ((e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreateWithFlags(&L->ev_exit, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
    // %globaltimer against the host clock: the tightest of a few round trips
    int64_t best_span = INT64_MAX;
    for (int k = 0; k < 5; ++k) {
        const uint64_t t0 = host_ns();
        k_dl_clock<<<1, 1, 0, L->stream>>>(clock_d);
        if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(L->stream)) != cudaSuccess)
            return fail(e);
        const uint64_t t1 = host_ns();
        const uint64_t gt = __atomic_load_n(L->clock_h, __ATOMIC_ACQUIRE);
        if ((int64_t)(t1 - t0) < best_span) {
            best_span = (int64_t)(t1 - t0);
            L->gt_minus_host = (int64_t)gt - (int64_t)((t0 + t1) / 2);
        }
    }
    *out = L;
    return SYM_OK;
}

extern "C" sym_status sym_devloop_submit_mttkrp(sym_devloop L, const sym_request* req, uint64_t* ticket) {
    if (!L || !req || !ticket) return SYM_E_INVALID;
    const sym_tensor_s* X = req->X;
    if (!X || req->want_residual != 0) return SYM_E_BADREQ;
    if (validate_mttkrp_args(X, req->B, req->bdt, req->rank, req->ldb, req->M, req->ldm) != SYM_OK)
        return SYM_E_BADREQ;
    if (X->order < 2 || X->order > 5 || X->device != L->device) return SYM_E_BADREQ;
    int lanes = 1;
    while (4 * lanes < req->rank) lanes <<= 1;
    DLReq q{};
    q.kind = DL_MTTKRP;
    q.order = X->order;
    q.kw = X->kw;
    q.bits = X->bits;
    q.bf16 = req->bdt == SYM_BF16 ? 1 : 0;
    q.rank = req->rank;
    q.lanes = lanes;
    q.n = X->n;
    q.nnz = X->nnz;
    q.zrows = std::max<int64_t>(1, DL_ZERO / req->rank);
    q.zchunks = std::max<int64_t>(1, (X->n + q.zrows - 1) / q.zrows);
    q.chunk = (int64_t)DL_WARPS * (32 / lanes) * DL_MT_PER_GROUP;
    q.nchunks = q.zchunks + (X->nnz + q.chunk - 1) / q.chunk;
    if (q.nchunks >= (int64_t)0x7fffffff) return SYM_E_BADREQ;
    q.klo = X->klo;
    q.khi = X->khi;
    q.val = X->val;
    q.B = req->B;
    q.ldb = req->ldb;
    q.M = req->M;
    q.ldm = req->ldm;
    const size_t esz = req->bdt == SYM_BF16 ? 2 : 4;
    const size_t bytes = X->info.arena_used + (size_t)X->n * (size_t)req->ldb * esz + (size_t)X->n * (size_t)req->ldm * 4;
    return dl_submit(L, q, bytes, req->user_tag, ticket);
}

extern "C" sym_status sym_devloop_submit_ssymv(sym_devloop L, const sym_csr_upper* A, const float* x, float* y,
                                               double* syprd, uint64_t user_tag, uint64_t* ticket) {
    if (!L || !A || !ticket) return SYM_E_INVALID;
    if (A->n < 0 || A->nnz < 0 || A->nnz > (int64_t)0x7fffffff || A->n > (int64_t)0x7fffffff) return SYM_E_BADREQ;
    if (A->n > 0 && (!A->rowptr || !x || !y)) return SYM_E_BADREQ;
    if (A->nnz > 0 && (!A->col || !A->val)) return SYM_E_BADREQ;
    if (A->n == 0 && A->nnz > 0) return SYM_E_BADREQ;
    if ((y && !aligned(y, 4)) || (x && !aligned(x, 4)) || (syprd && !aligned(syprd, 8))) return SYM_E_BADREQ;
    DLReq q{};
    q.kind = DL_SSYMV;
    q.n = A->n;
    q.nnz = A->nnz;
    q.zrows = DL_ZERO;
    q.zchunks = std::max<int64_t>(1, (A->n + DL_ZERO - 1) / DL_ZERO);
    q.chunk = DL_SV_CHUNK;
    q.nchunks = q.zchunks + (A->nnz + DL_SV_CHUNK - 1) / DL_SV_CHUNK;
    q.rowptr = A->rowptr;
    q.col = A->col;
    q.val = A->val;
    q.B = x;
    q.M = y;
    q.syprd = syprd;
    const size_t bytes = (size_t)(A->n + 1) * 4 + (size_t)A->nnz * 8 + (size_t)A->n * 8 + (syprd ? 8 : 0);
    return dl_submit(L, q, bytes, user_tag, ticket);
}

extern "C" sym_status sym_devloop_poll(sym_devloop L, uint64_t ticket, sym_result* out) {
    if (!L || !out) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(L->mu);
    const sym_status ps = dl_progress(L);
    auto it = L->results.find(ticket);
    if (it != L->results.end()) {
        *out = it->second;
        L->results.erase(it);
        return SYM_OK;
    }
    if (ps != SYM_OK) return ps;
    if (L->flight.count(ticket)) {
        out->status = SYM_PENDING;
        return SYM_PENDING;
    }
    for (const Queued& h : L->queue)
        if (h.ticket == ticket) {
            out->status = SYM_PENDING;
            return SYM_PENDING;
        }
    return SYM_E_NOTFOUND;
}

extern "C" sym_status sym_devloop_wait(sym_devloop L, uint64_t ticket, int64_t timeout_ns, sym_result* out) {
    if (!L || !out) return SYM_E_INVALID;
    const uint64_t deadline = host_ns() + (uint64_t)std::max<int64_t>(timeout_ns, 0);
    for (;;) {
        const sym_status s = sym_devloop_poll(L, ticket, out);
        if (s != SYM_PENDING) return s;
        if (host_ns() > deadline) return SYM_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
}

extern "C" sym_status sym_devloop_set_test_hook(sym_devloop L, int hook) {
    if (!L || hook < 0 || hook > 1) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(L->mu);
    L->hook = hook;
    return SYM_OK;
}

extern "C" sym_status sym_devloop_stats_get(sym_devloop L, sym_devloop_stats* out) {
    if (!L || !out) return SYM_E_INVALID;
    std::lock_guard<std::mutex> lk(L->mu);
    *out = L->stats;
    return SYM_OK;
}

extern "C" sym_status sym_devloop_destroy(sym_devloop L) {
    if (!L) return SYM_E_INVALID;
    const uint64_t deadline = host_ns() + (uint64_t)L->cfg.wait_limit_ns;
    sym_status st = SYM_OK;
    {
        // drain: everything submitted completes (bounded)
        std::unique_lock<std::mutex> lk(L->mu);
        for (;;) {
            const sym_status ps = dl_progress(L);
            if (ps != SYM_OK) {
                st = ps;
                break;
            }
            if (L->flight.empty() && L->queue.empty()) break;
            if (host_ns() > deadline) {
                st = SYM_E_TIMEOUT;
                break;
            }
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
        __atomic_store_n(&L->ctl_h->stop, 1u, __ATOMIC_RELEASE);
    }
    // the loop kernel leaves at its next claim; wait for it (bounded)
    if (L->launched) {
        for (;;) {
            const cudaError_t q = cudaEventQuery(L->ev_exit);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) {
                st = cuda_status(q);
                break;
            }
            if (host_ns() > deadline + 2000000000ull) {
                return SYM_E_TIMEOUT;  // the kernel still runs: keep its memory (leaked with the handle)
            }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
    }
    dl_free(L);
    return st;
}
