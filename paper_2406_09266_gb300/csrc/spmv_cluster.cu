// One-launch SSYMV + SYPRD for small matrices (Sec. 3.1: each stored a_ij,
// i < j, feeds y_i and y_j; Sec. 3.2.2: SYPRD weights the off-diagonal terms 2).
//
// For an n of a few thousand the multi-block form (memset of y, the SSYMV
// kernel, the FP64 SYPRD finaliser) is three dependent launches of a few
// microseconds each.  Here one thread-block cluster of CL_CTAS CTAs does all of
// it in one launch:
//   * every CTA copies x and rowptr into its shared memory, plus an equal
//     share of the entries (col, val) — all copies issued at once (cp.async),
//     so the whole input costs one memory latency;
//   * every CTA adds its row sums and mirrored updates a_ij x_i into a full-
//     length partial y of its own (shared-memory atomics: no memset, no global
//     atomics);
//   * CTA r owns rows [r S, (r+1) S) of y.  Every CTA pushes slice c of its
//     partial y into an inbox in CTA c's shared memory with one bulk copy per
//     peer, counted on the receiver's mbarrier; the owner waits for its
//     CL_CTAS - 1 slices (a bounded wait), sums the CL_CTAS partials in CTA
//     order and writes its rows of y;
//   * SYPRD: FP32 per thread, FP64 across warps, pushed to CTA 0 the same way
//     and summed there in CTA order.
// The only cluster-wide barrier follows the mbarrier initialisation (so that
// no copy reaches an uninitialised barrier) and overlaps the input copies.  A
// CTA leaves once its inbox is full and its outgoing copies have been read, so
// no peer touches its shared memory afterwards.  If the inbox does not fill
// within about 2 s the CTA writes NaN to its rows of y (and CTA 0 to SYPRD).
#include <algorithm>

#include "common.cuh"
#include "spmv.cuh"

namespace symgpu {

namespace {

constexpr int CL_CTAS = 8;
constexpr int CL_THREADS = 512;
constexpr int CL_WARPS = CL_THREADS / 32;
// Size limits of the one-launch form (set, not tuned: the crossover with the
// multi-block form has not been measured).
constexpr int CL_MAX_N = 8192;
constexpr size_t CL_SMEM_CAP = 160 * 1024;

struct ClusterShape {
    int slice = 0;  // rows of y each CTA owns (multiple of 4)
    int per = 0;    // entries per CTA (multiple of 4)
    int xw = 0, rw = 0;  // 32-bit words of x and of rowptr (multiples of 4)
    size_t smem = 0;
};

// Shared memory layout, in 32-bit words from the start (all 16-byte aligned):
// x [xw] | partial y [CTAS S] | rowptr [rw] | col [per] | val [per] |
// inbox [(CTAS - 1) S] | SYPRD inbox [CTAS x 4] | warp partials [2 WARPS] | mbarrier [4]
inline size_t cluster_smem_words(int slice, int per, int xw, int rw) {
    return (size_t)xw + (size_t)CL_CTAS * slice + rw + 2 * (size_t)per + (size_t)(CL_CTAS - 1) * slice +
           4 * CL_CTAS + 2 * CL_WARPS + 4;
}

inline int round4(int64_t v) { return (int)((v + 3) & ~(int64_t)3); }

bool cluster_shape(const sym_csr_upper* A, ClusterShape* sh) {
    if (A->n <= 0 || A->n > CL_MAX_N) return false;
    sh->slice = round4((A->n + CL_CTAS - 1) / CL_CTAS);
    sh->per = round4((A->nnz + CL_CTAS - 1) / CL_CTAS);
    sh->xw = round4(A->n);
    sh->rw = round4(A->n + 1);
    sh->smem = 4 * cluster_smem_words(sh->slice, sh->per, sh->xw, sh->rw);
    return sh->smem <= CL_SMEM_CAP;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// Issues the copy of `count` 32-bit words (16 bytes per copy where the global
// source is 16-byte aligned; the shared destination always is).
__device__ __forceinline__ void copy_words(uint32_t dst, const void* src, int count, int tid) {
    const char* g = static_cast<const char*>(src);
    int k0 = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        const int c4 = count >> 2;
        for (int k = tid; k < c4; k += CL_THREADS) cp_async16(dst + 16u * k, g + 16 * (size_t)k);
        k0 = 4 * c4;
    }
    for (int k = k0 + tid; k < count; k += CL_THREADS) cp_async4(dst + 4u * k, g + 4 * (size_t)k);
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}

// Address of the same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t a, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase 0 of `bar` to complete; gives up after `limit_ns` (2 s in
// normal runs).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint64_t limit_ns) {
    if (mbar_try_wait(bar, 0)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, 0)) return true;
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
}

// Shared (this CTA) -> shared (CTA of dst) bulk copy, completion counted on the
// destination CTA's mbarrier; addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_s2c(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Largest i in [lo, n) with rp[i] <= v, or lo - 1.
__device__ __forceinline__ int last_le(const int32_t* rp, int lo, int n, int v) {
    int a = lo, b = n;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (rp[mid] <= v) a = mid + 1;
        else b = mid;
    }
    return a - 1;
}

// CTA r of the cluster takes the entries [r per, (r+1) per); each of its
// threads takes a contiguous run of E of them (E odd, so that the lanes' runs
// start in different banks), finds the row of its first entry by binary search
// and keeps the row sum in a register until the row changes (a row split
// between threads or CTAs adds one partial sum per piece).
// wait_ns bounds the inbox wait.  skip_to >= 0 is a test hook: no CTA pushes
// anything into CTA skip_to's inbox, so its wait runs out with no copy in
// flight towards it; it then writes NaN to its rows (and to SYPRD if it is CTA 0).
template <bool SYPRD>
__global__ void __cluster_dims__(CL_CTAS, 1, 1) __launch_bounds__(CL_THREADS, 1)
    k_ssymv_cluster(int n, int nnz, int per, int slice, int xw, int rw, const int32_t* __restrict__ rowptr,
                    const int32_t* __restrict__ col, const float* __restrict__ val, const float* __restrict__ x,
                    float* __restrict__ y, double* __restrict__ syprd, uint64_t wait_ns, int skip_to) {
    extern __shared__ __align__(16) unsigned char cl_smem[];
    float* xs = reinterpret_cast<float*>(cl_smem);
    float* yp = xs + xw;  // this CTA's partial y, CL_CTAS slices
    int32_t* rp = reinterpret_cast<int32_t*>(yp + CL_CTAS * slice);
    int32_t* cs = rp + rw;
    float* vs = reinterpret_cast<float*>(cs + per);
    float* inbox = vs + per;  // CL_CTAS - 1 slices of this CTA's rows from the peers
    double* sinbox = reinterpret_cast<double*>(inbox + (CL_CTAS - 1) * slice);  // 16 bytes per CTA
    double* wpart = sinbox + 2 * CL_CTAS;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(wpart + CL_WARPS);

    const int tid = threadIdx.x;
    const uint32_t rank = cluster_rank();
    const uint32_t slice_bytes = 16u * (uint32_t)(slice >> 2);
    if (tid == 0) {
        mbar_init(smem_u32(mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        const uint32_t in_bytes = (CL_CTAS - 1) * (slice_bytes + (SYPRD && rank == 0 ? 16u : 0u));
        mbar_arrive_expect_tx(smem_u32(mbar), in_bytes);
    }
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");  // waited on before the first push

    const int e0 = min(nnz, (int)rank * per), e1 = min(nnz, e0 + per);
    copy_words(smem_u32(xs), x, n, tid);
    copy_words(smem_u32(rp), rowptr, n + 1, tid);
    copy_words(smem_u32(cs), col + e0, e1 - e0, tid);
    copy_words(smem_u32(vs), val + e0, e1 - e0, tid);
    for (int k = tid; k < CL_CTAS * slice; k += CL_THREADS) yp[k] = 0.f;
    cp_async_wait_all();
    __syncthreads();

    // Every shared-memory index below stays in bounds whatever rowptr holds:
    // q in [0, e1 - e0), rows in [0, n).
    const int cnt = e1 - e0;
    const int E = ((cnt + CL_THREADS - 1) / CL_THREADS) | 1;
    const int q0 = min(cnt, tid * E), q1 = min(cnt, q0 + E);
    float syp = 0.f;
    if (q0 < q1) {
        int i = max(0, last_le(rp, 0, n, e0 + q0));
        int next = rp[i + 1];  // first entry past row i
        float xi = xs[i], rowsum = 0.f, sr = 0.f;
        for (int q = q0; q < q1; ++q) {
            const int p = e0 + q;
            if (p >= next && i < n - 1) {
                if (rowsum != 0.f) atomicAdd(&yp[i], rowsum);
                if (SYPRD) syp += sr * xi;
                rowsum = 0.f;
                sr = 0.f;
                ++i;
                if (p >= rp[i + 1] && i < n - 1) i = max(i, last_le(rp, i + 1, n, p));  // skip empty rows
                next = rp[i + 1];
                xi = xs[i];
            }
            const int j = cs[q];
            if ((unsigned)j >= (unsigned)n) {  // a column outside the matrix: skipped (and counted when checked)
                (void)SYM_INDEX_OK(j, n);
                continue;
            }
            const float a = vs[q];
            const float t = a * xs[j];
            rowsum += t;
            if (j != i) {
                atomicAdd(&yp[j], a * xi);
                if (SYPRD) sr += 2.f * t;
            } else if (SYPRD) {
                sr += t;
            }
        }
        if (rowsum != 0.f) atomicAdd(&yp[i], rowsum);
        if (SYPRD) syp += sr * xi;
    }
    if (SYPRD) {
        const float w = warp_sum(syp);
        if ((tid & 31) == 0) wpart[tid >> 5] = (double)w;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // partial y visible to the bulk copies
    __syncthreads();
    if (SYPRD && tid < 32) {
        // FP64 sum of the warp partials: a fixed shuffle tree over lanes 0..15.
        double t = tid < CL_WARPS ? wpart[tid] : 0.0;
#pragma unroll
        for (int o = CL_WARPS >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) {
            sinbox[2 * rank] = t;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
    }
    asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory");  // every peer's mbarrier is initialised
    if (tid == 0) {
        const uint32_t bar = smem_u32(mbar);
        for (uint32_t c = 0; c < CL_CTAS; ++c) {
            if (c == rank || (int)c == skip_to) continue;
            const uint32_t slot = rank < c ? rank : rank - 1;  // this CTA's slot in the inbox of CTA c
            bulk_s2c(map_rank(smem_u32(inbox + slot * slice), c), smem_u32(yp + c * slice), slice_bytes,
                     map_rank(bar, c));
        }
        if (SYPRD && rank != 0 && skip_to != 0)
            bulk_s2c(map_rank(smem_u32(sinbox + 2 * rank), 0), smem_u32(sinbox + 2 * rank), 16u, map_rank(bar, 0));
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    }
    const bool ok = mbar_wait_bounded(smem_u32(mbar), wait_ns);

    // Rows [r slice, (r+1) slice): the CL_CTAS partials summed in CTA order.
    const int r0 = (int)rank * slice;
    for (int k = 4 * tid; k < slice && r0 + k < n; k += 4 * CL_THREADS) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < CL_CTAS; ++c) {
            const float4 v = c == (int)rank
                                 ? *reinterpret_cast<const float4*>(yp + r0 + k)
                                 : *reinterpret_cast<const float4*>(inbox + (c < (int)rank ? c : c - 1) * slice + k);
            t.x += v.x;
            t.y += v.y;
            t.z += v.z;
            t.w += v.w;
        }
        if (!ok) t = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                                 __int_as_float(0x7fc00000));
        const int m = min(4, n - (r0 + k));
        y[r0 + k] = t.x;
        if (m > 1) y[r0 + k + 1] = t.y;
        if (m > 2) y[r0 + k + 2] = t.z;
        if (m > 3) y[r0 + k + 3] = t.w;
    }
    if (SYPRD && rank == 0 && tid == 0) {
        double t = 0.0;
        for (int c = 0; c < CL_CTAS; ++c) t += sinbox[2 * c];
        *syprd = ok ? t : __longlong_as_double(0x7ff8000000000000ll);
    }
    if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");  // outgoing copies have read yp
}

sym_status launch_cluster(const sym_csr_upper* A, const ClusterShape& sh, const float* x, float* y, double* syprd,
                          cudaStream_t s, uint64_t wait_ns = 2000000000ull, int skip_to = -1) {
    SYM_PROF("ssymv_cluster", s);
    if (syprd) {
        SYM_TRY(raise_smem_limit(k_ssymv_cluster<true>, sh.smem));
        k_ssymv_cluster<true><<<CL_CTAS, CL_THREADS, sh.smem, s>>>((int)A->n, (int)A->nnz, sh.per, sh.slice, sh.xw,
                                                                   sh.rw, A->rowptr, A->col, A->val, x, y, syprd,
                                                                   wait_ns, skip_to);
    } else {
        SYM_TRY(raise_smem_limit(k_ssymv_cluster<false>, sh.smem));
        k_ssymv_cluster<false><<<CL_CTAS, CL_THREADS, sh.smem, s>>>((int)A->n, (int)A->nnz, sh.per, sh.slice, sh.xw,
                                                                    sh.rw, A->rowptr, A->col, A->val, x, y, syprd,
                                                                    wait_ns, skip_to);
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

}  // namespace

bool ssymv_single_launch(const sym_csr_upper* A) {
    ClusterShape sh;
    return cluster_shape(A, &sh);
}

sym_status ssymv_cluster_launch(const sym_csr_upper* A, const float* x, float* y, double* syprd, cudaStream_t s) {
    ClusterShape sh;
    if (!cluster_shape(A, &sh)) return SYM_E_UNSUPPORTED;
    return launch_cluster(A, sh, x, y, syprd, s);
}

}  // namespace symgpu

extern "C" int sym_spmv_single_launch(const sym_csr_upper* A) {
    if (symgpu::validate_csr(A) != SYM_OK) return 0;
    return symgpu::ssymv_single_launch(A) ? 1 : 0;
}

extern "C" sym_status sym_spmv_cluster_bounded(const sym_csr_upper* A, const float* x, float* y, double* syprd,
                                               int64_t wait_limit_ns, int skip_to, sym_stream_t stream) {
    using namespace symgpu;
    sym_status st = validate_csr(A);
    if (st != SYM_OK) return st;
    if (A->n > 0 && (!x || !y)) return SYM_E_INVALID;
    if (skip_to < -1 || skip_to >= CL_CTAS) return SYM_E_INVALID;
    ClusterShape sh;
    if (A->n == 0 || !cluster_shape(A, &sh)) return SYM_E_UNSUPPORTED;
    const uint64_t limit = wait_limit_ns > 0 ? (uint64_t)wait_limit_ns : 2000000000ull;
    return launch_cluster(A, sh, x, y, syprd, as_stream(stream), limit, skip_to);
}
