// Symmetric tensor handles: canonicalisation of a coordinate list into the
// device layout used by the MTTKRP kernels.
//
// Canonical triangle (Sec. 2.1, Def. "Canonical", upper triangle): every tuple
// is stored sorted, i_1 <= ... <= i_N, and entries are kept in lexicographic
// order, which is the traversal order of a CSF tree rooted at i_1 (Sec. 2.2).
// Diagonal splitting (Sec. 4.2.9): entries with all indices distinct form the
// STRICT stream; entries with a repeated index form the DIAGONAL stream.  Both
// live in one array, strict first, each in lexicographic order.
//
// Layout per entry: the sorted tuple packed into a key of ORDER * bits bits
// (c_1 most significant), 64-bit words (a second word when ORDER*bits > 64),
// plus a float value.  Keys are what the radix sort orders and what the
// kernels decode.
#include <new>
#include <string.h>

#include "common.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

constexpr int CT = 256;

struct DevCounters {
    unsigned long long range_bad;
    unsigned long long dup_seen;       // entries equal to their predecessor
    unsigned long long dup_mismatch;   // ... whose value bits differ
    unsigned long long by_pattern[16];
    unsigned long long expanded;
    unsigned long long root_fibers;
    unsigned long long l2_fibers;
    unsigned long long nnz_strict;
    unsigned long long nnz_kept;
    double normsq;
};

template <int N>
__device__ __forceinline__ void sort_small(int32_t* c) {
#pragma unroll
    for (int a = 1; a < N; ++a)
#pragma unroll
        for (int b = a; b > 0; --b) {
            int32_t x = c[b - 1], y = c[b];
            c[b - 1] = min(x, y);
            c[b] = max(x, y);
        }
}

// Number of distinct permutations N!/prod(m_t!) from a sorted tuple's runs.
template <int N>
__device__ __forceinline__ int distinct_perms(const int32_t* c) {
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    int den = 1, run = 1;
#pragma unroll
    for (int q = 1; q < N; ++q) {
        if (c[q] == c[q - 1]) {
            ++run;
        } else {
            den *= fact[run];
            run = 1;
        }
    }
    den *= fact[run];
    return fact[N] / den;
}

// Each thread packs PACK_EPT entries, CT apart, with all their coordinate loads
// issued before any is used: when the coordinate list is read in place from
// host memory over the host link, the extra loads in flight hide its latency.
constexpr int PACK_EPT = 4;

template <int N, int KW>
__global__ void __launch_bounds__(CT) k_pack(const int32_t* __restrict__ idx, int64_t ld, int64_t nnz, int64_t n,
                                             int bits, uint64_t* __restrict__ klo, uint64_t* __restrict__ khi,
                                             uint32_t* __restrict__ pay, DevCounters* cnt) {
    const int64_t e0 = (int64_t)blockIdx.x * (CT * PACK_EPT) + threadIdx.x;
    int32_t c[PACK_EPT][N];
#pragma unroll
    for (int u = 0; u < PACK_EPT; ++u) {
        const int64_t e = e0 + (int64_t)u * CT;
#pragma unroll
        for (int q = 0; q < N; ++q) c[u][q] = e < nnz ? idx[(int64_t)q * ld + e] : 0;
    }
    int bad = 0;
#pragma unroll
    for (int u = 0; u < PACK_EPT; ++u) {
        const int64_t e = e0 + (int64_t)u * CT;
        if (e >= nnz) continue;
        bool out = false;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (c[u][q] < 0 || c[u][q] >= n) {
                out = true;
                c[u][q] = 0;
            }
        }
        bad += out ? 1 : 0;
        sort_small<N>(c[u]);
        KeyWords k = pack_key<N, KW>(c[u], bits);
        klo[e] = k.lo;
        if (KW == 2) khi[e] = k.hi;
        pay[e] = (uint32_t)e;
    }
    // entries with an out-of-range coordinate (each counted once)
    unsigned m = __ballot_sync(0xffffffffu, bad != 0);
    if (m) {
        int tot = bad;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&cnt->range_bad, (unsigned long long)tot);
    }
}

// Marks kept entries (first of each equal-key run), classifies them and takes
// the exact counts.  flag_s / flag_d: 1 when the entry goes to that stream.
template <int N, int KW>
__global__ void __launch_bounds__(CT) k_mark(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                                             const uint32_t* __restrict__ pay, const float* __restrict__ val,
                                             int64_t nnz, int bits, int policy, uint32_t* __restrict__ flag_s,
                                             uint32_t* __restrict__ flag_d, DevCounters* cnt) {
    // Grid-stride over the sorted entries; every warp keeps its counts in
    // registers and the CTA sends them to the global counters once, so the
    // same-address global atomics scale with the grid, not with nnz.
    constexpr int NP = 1 << (N - 1);
    __shared__ unsigned long long s_pat[16];
    __shared__ unsigned long long s_misc[7];  // expanded, root, l2, strict, kept, dups, mismatches
    __shared__ double s_norm[CT / 32];
    if (threadIdx.x < 16) s_pat[threadIdx.x] = 0;
    if (threadIdx.x < 7) s_misc[threadIdx.x] = 0;
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned long long w_ex = 0, w_root = 0, w_l2 = 0, w_strict = 0, w_keep = 0, w_dup = 0, w_mis = 0;
    unsigned long long w_pat[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) w_pat[q] = 0;
    double nrm = 0.0;
    const int64_t stride = (int64_t)gridDim.x * CT;
    for (int64_t base = (int64_t)blockIdx.x * CT + (threadIdx.x & ~31); base < nnz; base += stride) {
        const int64_t p = base + lane;  // the loop bound is per warp: the ballots below see every lane
        bool dup = false, mismatch = false, keep = false, new_root = false, new_l2 = false;
        int pat = -1;
        unsigned ex = 0;
        if (p < nnz) {
            KeyWords k{klo[p], KW == 2 ? khi[p] : 0ull};
            int32_t c[N], pc[N];
            unpack_key<N, KW>(k, bits, c);
            if (p > 0) {
                KeyWords kp{klo[p - 1], KW == 2 ? khi[p - 1] : 0ull};
                dup = (kp.lo == k.lo) && (kp.hi == k.hi);
                unpack_key<N, KW>(kp, bits, pc);
                if (dup && policy == SYM_DUP_KEEP_EQUAL)
                    mismatch = __float_as_uint(val[pay[p]]) != __float_as_uint(val[pay[p - 1]]);
            }
            keep = !dup;
            pat = 0;
#pragma unroll
            for (int q = 0; q + 1 < N; ++q) pat |= (c[q] == c[q + 1]) ? (1 << q) : 0;
            flag_s[p] = (keep && pat == 0) ? 1u : 0u;
            flag_d[p] = (keep && pat != 0) ? 1u : 0u;
            if (keep) {
                ex = (unsigned)distinct_perms<N>(c);
                new_root = (p == 0 || pc[0] != c[0]);
                new_l2 = (p == 0 || pc[0] != c[0] || pc[1] != c[1]);
                const double v = (double)val[pay[p]];
                nrm += (double)ex * v * v;
            }
        }
        w_ex += __reduce_add_sync(full, ex);
        w_root += __popc(__ballot_sync(full, new_root));
        w_l2 += __popc(__ballot_sync(full, new_l2));
        w_strict += __popc(__ballot_sync(full, keep && pat == 0));
        w_keep += __popc(__ballot_sync(full, keep));
        w_dup += __popc(__ballot_sync(full, dup));
        w_mis += __popc(__ballot_sync(full, mismatch));
#pragma unroll
        for (int q = 0; q < NP; ++q) w_pat[q] += __popc(__ballot_sync(full, keep && pat == q));
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NP; ++q)
            if (w_pat[q]) atomicAdd(&s_pat[q], w_pat[q]);
        if (w_ex) atomicAdd(&s_misc[0], w_ex);
        if (w_root) atomicAdd(&s_misc[1], w_root);
        if (w_l2) atomicAdd(&s_misc[2], w_l2);
        if (w_strict) atomicAdd(&s_misc[3], w_strict);
        if (w_keep) atomicAdd(&s_misc[4], w_keep);
        if (w_dup) atomicAdd(&s_misc[5], w_dup);
        if (w_mis) atomicAdd(&s_misc[6], w_mis);
    }
    nrm = warp_sum(nrm);
    if (lane == 0) s_norm[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x < 16 && s_pat[threadIdx.x]) atomicAdd(&cnt->by_pattern[threadIdx.x], s_pat[threadIdx.x]);
    if (threadIdx.x == 16) {
        atomicAdd(&cnt->expanded, s_misc[0]);
        atomicAdd(&cnt->root_fibers, s_misc[1]);
        atomicAdd(&cnt->l2_fibers, s_misc[2]);
        atomicAdd(&cnt->nnz_strict, s_misc[3]);
        atomicAdd(&cnt->nnz_kept, s_misc[4]);
        atomicAdd(&cnt->dup_seen, s_misc[5]);
        atomicAdd(&cnt->dup_mismatch, s_misc[6]);
    }
    if (threadIdx.x == 32) {
        double t = 0.0;
        for (int w = 0; w < CT / 32; ++w) t += s_norm[w];
        atomicAdd(&cnt->normsq, t);
    }
}

template <int KW>
__global__ void k_compact(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                          const uint32_t* __restrict__ pay, const float* __restrict__ val, int64_t nnz,
                          const uint32_t* __restrict__ flag_s, const uint32_t* __restrict__ flag_d,
                          const uint32_t* __restrict__ pos_s, const uint32_t* __restrict__ pos_d,
                          const DevCounters* cnt, uint64_t* __restrict__ out_lo, uint64_t* __restrict__ out_hi,
                          float* __restrict__ out_val) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    int64_t dst = -1;
    if (flag_s[p]) dst = pos_s[p];
    else if (flag_d[p]) dst = (int64_t)cnt->nnz_strict + pos_d[p];
    if (dst < 0) return;
    out_lo[dst] = klo[p];
    if (KW == 2) out_hi[dst] = khi[p];
    out_val[dst] = val[pay[p]];
}

template <int N, int KW>
__global__ void k_export(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                         const float* __restrict__ val, int64_t nnz, int bits, int32_t* __restrict__ cidx,
                         int64_t ld, float* __restrict__ cval) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    int32_t c[N];
    unpack_key<N, KW>(KeyWords{klo[p], KW == 2 ? khi[p] : 0ull}, bits, c);
#pragma unroll
    for (int q = 0; q < N; ++q) cidx[(int64_t)q * ld + p] = c[q];
    cval[p] = val[p];
}

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_gen_coords(int order, int64_t n, int64_t count, uint64_t seed, int32_t* __restrict__ idx,
                             int64_t ld, float* __restrict__ val) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    uint64_t s1 = 0, s2 = 0;
    for (int q = 0; q < order; ++q) {
        uint64_t k = (uint64_t)e * order + q + 1;
        uint64_t z = sm64_mix(seed + k * gamma);
        uint64_t r = ((z >> 32) * (uint64_t)n) >> 32;
        idx[(int64_t)q * ld + e] = (int32_t)r;
        s1 += r;
        s2 += sm64_mix(r + seed);
    }
    uint64_t h = sm64_mix(s1 * gamma + s2);
    int32_t m = (int32_t)(h >> 40);
    val[e] = (float)(m - (1 << 23)) * (1.0f / 8388608.0f);
}

// ---------------------------------------------------------------- order-2 -> upper CSR

__global__ void k_csr_counts(const uint64_t* __restrict__ klo, int64_t nnz, int64_t nnz_strict, int bits,
                             unsigned long long* __restrict__ cnt, unsigned long long* __restrict__ scnt,
                             int* __restrict__ has_diag) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    int32_t c[2];
    unpack_key<2, 1>(KeyWords{klo[p], 0ull}, bits, c);
    atomicAdd(&cnt[c[0]], 1ull);
    if (p < nnz_strict)
        atomicAdd(&scnt[c[0]], 1ull);
    else
        has_diag[c[0]] = 1;
}

__global__ void k_csr_fill(const uint64_t* __restrict__ klo, const float* __restrict__ val, int64_t nnz,
                           int64_t nnz_strict, int bits, const int64_t* __restrict__ rowptr,
                           const int64_t* __restrict__ sstart, const int* __restrict__ has_diag,
                           int32_t* __restrict__ col, float* __restrict__ oval) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    int32_t c[2];
    unpack_key<2, 1>(KeyWords{klo[p], 0ull}, bits, c);
    const int64_t dst = (p < nnz_strict) ? rowptr[c[0]] + has_diag[c[0]] + (p - sstart[c[0]]) : rowptr[c[0]];
    col[dst] = c[1];
    oval[dst] = val[p];
}

__global__ void k_u64_to_i64(const unsigned long long* __restrict__ a, int64_t n, int64_t* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (int64_t)a[i];
}

// ---------------------------------------------------------------- batched matrix generator

__global__ void k_gen_batch(int64_t count, const int64_t* __restrict__ row_off, const int64_t* __restrict__ draw_off,
                            int64_t total, uint64_t seed, int32_t* __restrict__ idx, int64_t ld,
                            float* __restrict__ val) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= total) return;
    int64_t lo = 0, hi = count;  // instance b with draw_off[b] <= d < draw_off[b+1]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (draw_off[mid] <= d) lo = mid; else hi = mid;
    }
    const int64_t b = lo;
    const int64_t n = row_off[b + 1] - row_off[b];
    const int64_t slots = n * (n + 1) / 2;
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    const uint64_t z = sm64_mix(seed + (uint64_t)(d + 1) * gamma);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    int64_t sl = (int64_t)floor(u * (double)slots);
    if (sl >= slots) sl = slots - 1;
    const double t = (double)(2 * n + 1);
    int64_t i = (int64_t)floor((t - sqrt(t * t - 8.0 * (double)sl)) * 0.5);
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    auto start = [n](int64_t r) { return r * (2 * n - r + 1) / 2; };
    while (i > 0 && start(i) > sl) --i;
    while (i + 1 < n && start(i + 1) <= sl) ++i;
    const int64_t j = i + (sl - start(i));
    const uint64_t gi = (uint64_t)(row_off[b] + i), gj = (uint64_t)(row_off[b] + j);
    idx[d] = (int32_t)gi;
    idx[ld + d] = (int32_t)gj;
    const uint64_t s1 = gi + gj;
    const uint64_t s2 = sm64_mix(gi + seed) + sm64_mix(gj + seed);
    const uint64_t h = sm64_mix(s1 * gamma + s2);
    const int32_t m = (int32_t)(h >> 40);
    val[d] = (float)(m - (1 << 23)) * (1.0f / 8388608.0f);
}

// ---------------------------------------------------------------- leaf index

template <int N, int KW>
__global__ void k_reverse_pack(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, int64_t ns,
                               int bits, uint64_t* __restrict__ olo, uint64_t* __restrict__ ohi,
                               uint32_t* __restrict__ pay) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= ns) return;
    int32_t c[N], r[N];
    unpack_key<N, KW>(KeyWords{klo[p], KW == 2 ? khi[p] : 0ull}, bits, c);
#pragma unroll
    for (int q = 0; q < N; ++q) r[q] = c[N - 1 - q];
    const KeyWords k = pack_key<N, KW>(r, bits);
    olo[p] = k.lo;
    if (KW == 2) ohi[p] = k.hi;
    pay[p] = (uint32_t)p;
}

__global__ void k_gather_f32(const float* __restrict__ src, const uint32_t* __restrict__ pay, int64_t m,
                             float* __restrict__ dst) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) dst[k] = src[pay[k]];
}

int bits_for(int64_t n) {
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b < 1 ? 1 : b;
}

struct CreatePlan {
    int kw;
    int bits;
};

// Workspace layout of sym_tensor_create (shared by the size query and the call).
template <typename C>
void layout_ws(C& c, int64_t nnz, int kw, uint64_t** lo0, uint64_t** hi0, uint32_t** p0, uint64_t** lo1,
               uint64_t** hi1, uint32_t** p1, uint32_t** fs, uint32_t** fd, uint32_t** ps, uint32_t** pd,
               DevCounters** cnt, void** radix, void** scan, float** vcopy) {
    size_t m = nnz > 0 ? (size_t)nnz : 1;
    *lo0 = c.template take<uint64_t>(m);
    *hi0 = kw == 2 ? c.template take<uint64_t>(m) : nullptr;
    *p0 = c.template take<uint32_t>(m);
    *lo1 = c.template take<uint64_t>(m);
    *hi1 = kw == 2 ? c.template take<uint64_t>(m) : nullptr;
    *p1 = c.template take<uint32_t>(m);
    *fs = c.template take<uint32_t>(m);
    *fd = c.template take<uint32_t>(m);
    *ps = c.template take<uint32_t>(m);
    *pd = c.template take<uint32_t>(m);
    *cnt = c.template take<DevCounters>(1);
    *radix = c.template take<char>(radix_ws_bytes((int64_t)m, kw));
    *scan = c.template take<char>(scan_ws_bytes((int64_t)m));
    *vcopy = c.template take<float>(m);  // device copy of values given in host memory
}

struct NullCarver {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

template <typename C>
void layout_arena(C& c, int64_t nnz, int kw, uint64_t** lo, uint64_t** hi, float** val) {
    size_t m = nnz > 0 ? (size_t)nnz : 1;
    *lo = c.template take<uint64_t>(m);
    *hi = kw == 2 ? c.template take<uint64_t>(m) : nullptr;
    *val = c.template take<float>(m);
}

// Copy of host values issued on a side stream once the keys are packed.
struct SideCopy {
    cudaStream_t side = nullptr;
    cudaEvent_t start = nullptr, done = nullptr;
    const float* host = nullptr;
    float* dev = nullptr;
    size_t bytes = 0;
    sym_status issue(cudaStream_t s) {  // after the packing kernel on s
        if (!side) return SYM_OK;
        SYM_CUDA(cudaEventRecord(start, s));
        SYM_CUDA(cudaStreamWaitEvent(side, start, 0));
        SYM_CUDA(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, side));
        SYM_CUDA(cudaEventRecord(done, side));
        return SYM_OK;
    }
    ~SideCopy() {
        if (side) cudaStreamSynchronize(side);  // on every path the copy into the workspace has landed
        if (start) cudaEventDestroy(start);
        if (done) cudaEventDestroy(done);
        if (side) cudaStreamDestroy(side);
    }
};

template <int N>
sym_status launch_create_kernels(int kw, const int32_t* idx, int64_t ld, const float* val, int64_t nnz, int64_t n,
                                 int bits, int policy, uint64_t* lo0, uint64_t* hi0, uint32_t* p0, uint64_t* lo1,
                                 uint64_t* hi1, uint32_t* p1, uint32_t* fs, uint32_t* fd, uint32_t* ps,
                                 uint32_t* pd, DevCounters* cnt, void* radix, void* scan, uint64_t* out_lo,
                                 uint64_t* out_hi, float* out_val, SideCopy& vals, cudaStream_t s) {
    unsigned g = (unsigned)((nnz + CT - 1) / CT);
    const unsigned gp = (unsigned)((nnz + CT * PACK_EPT - 1) / (CT * PACK_EPT));
    if (kw == 1)
        k_pack<N, 1><<<gp, CT, 0, s>>>(idx, ld, nnz, n, bits, lo0, hi0, p0, cnt);
    else
        k_pack<N, 2><<<gp, CT, 0, s>>>(idx, ld, nnz, n, bits, lo0, hi0, p0, cnt);
    SYM_CHECK_LAUNCH();
    SYM_TRY(vals.issue(s));
    uint64_t *slo, *shi;
    uint32_t* sp;
    sym_status st = radix_sort_pairs(kw, lo0, hi0, p0, lo1, hi1, p1, nnz, N * bits, radix, s, &slo, &shi, &sp);
    if (st != SYM_OK) return st;
    const unsigned gm = (unsigned)std::min<int64_t>((int64_t)g, (int64_t)sm_count() * 8);
    if (vals.done) SYM_CUDA(cudaStreamWaitEvent(s, vals.done, 0));  // values copied during the sort
    if (kw == 1)
        k_mark<N, 1><<<gm, CT, 0, s>>>(slo, shi, sp, val, nnz, bits, policy, fs, fd, cnt);
    else
        k_mark<N, 2><<<gm, CT, 0, s>>>(slo, shi, sp, val, nnz, bits, policy, fs, fd, cnt);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_u32(fs, ps, nnz, scan, s);
    if (st != SYM_OK) return st;
    st = exclusive_scan_u32(fd, pd, nnz, scan, s);
    if (st != SYM_OK) return st;
    if (kw == 1)
        k_compact<1><<<g, CT, 0, s>>>(slo, shi, sp, val, nnz, fs, fd, ps, pd, cnt, out_lo, out_hi, out_val);
    else
        k_compact<2><<<g, CT, 0, s>>>(slo, shi, sp, val, nnz, fs, fd, ps, pd, cnt, out_lo, out_hi, out_val);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

}  // namespace

}  // namespace symgpu

using namespace symgpu;

extern "C" sym_status sym_tensor_create_bytes(int order, int64_t n, int64_t nnz, size_t* arena_bytes,
                                              size_t* ws_bytes) {
    if (order < 2 || order > 5 || n < 1 || n > 0x7fffffffLL || nnz < 0 || nnz > 0xffffffffLL) return SYM_E_INVALID;
    int bits = bits_for(n);
    if (order * bits > 128) return SYM_E_UNSUPPORTED;
    int kw = order * bits > 64 ? 2 : 1;
    NullCarver a, w;
    uint64_t *lo, *hi;
    float* v;
    layout_arena(a, nnz, kw, &lo, &hi, &v);
    uint64_t *l0, *h0, *l1, *h1;
    uint32_t *p0, *p1, *fs, *fd, *ps, *pd;
    DevCounters* c;
    void *r, *sc;
    float* vc;
    layout_ws(w, nnz, kw, &l0, &h0, &p0, &l1, &h1, &p1, &fs, &fd, &ps, &pd, &c, &r, &sc, &vc);
    if (arena_bytes) *arena_bytes = a.s.used;
    if (ws_bytes) *ws_bytes = w.s.used;
    return SYM_OK;
}

extern "C" sym_status sym_tensor_create(int order, int64_t n, int64_t nnz, const int32_t* idx, int64_t ld_idx,
                                        const float* val, sym_dup_policy dup, void* arena, size_t arena_bytes,
                                        void* ws, size_t ws_bytes, sym_stream_t stream, sym_tensor* out) {
    if (!out) return SYM_E_INVALID;
    *out = nullptr;
    size_t need_a = 0, need_w = 0;
    sym_status st = sym_tensor_create_bytes(order, n, nnz, &need_a, &need_w);
    if (st != SYM_OK) return st;
    if (nnz > 0 && (!idx || !val || ld_idx < nnz)) return SYM_E_INVALID;
    if (dup != SYM_DUP_ERROR && dup != SYM_DUP_KEEP_EQUAL) return SYM_E_INVALID;
    bool val_host = false;
    if (nnz > 0) {
        // idx may be page-locked host memory (read in place by the packing kernel through its device
        // address); val may be device memory or page-locked host memory (copied during the sort)
        // (a pointer the runtime cannot classify, e.g. some virtual-memory mappings, is taken as device memory)
        cudaPointerAttributes ai{}, av{};
        if (cudaPointerGetAttributes(&ai, idx) != cudaSuccess) {
            cudaGetLastError();
            ai.type = cudaMemoryTypeDevice;
        }
        if (cudaPointerGetAttributes(&av, val) != cudaSuccess) {
            cudaGetLastError();
            av.type = cudaMemoryTypeDevice;
        }
        if (av.type == cudaMemoryTypeHost) {
            val_host = true;  // page-locked: copied into the workspace on a side stream during the sort
        } else if (av.type != cudaMemoryTypeDevice && av.type != cudaMemoryTypeManaged) {
            return SYM_E_INVALID;
        }
        if (ai.type == cudaMemoryTypeHost) {
            if (!ai.devicePointer) return SYM_E_INVALID;
            idx = static_cast<const int32_t*>(ai.devicePointer);
        } else if (ai.type != cudaMemoryTypeDevice && ai.type != cudaMemoryTypeManaged) {
            return SYM_E_INVALID;
        }
    }
    if (!arena || !ws || !aligned(arena, 256) || !aligned(ws, 256)) return SYM_E_INVALID;
    if (arena_bytes < need_a || ws_bytes < need_w) return SYM_E_NOMEM;
    const int bits = bits_for(n);
    const int kw = order * bits > 64 ? 2 : 1;
    cudaStream_t s = as_stream(stream);

    Carver A(arena, arena_bytes), W(ws, ws_bytes);
    uint64_t *out_lo, *out_hi;
    float* out_val;
    layout_arena(A, nnz, kw, &out_lo, &out_hi, &out_val);
    uint64_t *l0, *h0, *l1, *h1;
    uint32_t *p0, *p1, *fs, *fd, *ps, *pd;
    DevCounters* cnt;
    void *radix, *scan;
    float* vcopy;
    layout_ws(W, nnz, kw, &l0, &h0, &p0, &l1, &h1, &p1, &fs, &fd, &ps, &pd, &cnt, &radix, &scan, &vcopy);
    SYM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), s));
    // Values in page-locked host memory cross the host link on a side stream while the keys are sorted
    // (after the packing kernel, which reads the coordinates over the same link); the first kernel that
    // reads them waits for the copy.  The side stream and events live for this call only (it synchronises
    // `s`, which waits for them, before returning).
    SideCopy sc;
    if (val_host) {
        SYM_CUDA(cudaStreamCreateWithFlags(&sc.side, cudaStreamNonBlocking));
        SYM_CUDA(cudaEventCreateWithFlags(&sc.start, cudaEventDisableTiming));
        SYM_CUDA(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming));
        sc.host = val;
        sc.dev = vcopy;
        sc.bytes = (size_t)nnz * sizeof(float);
        val = vcopy;
    }
    if (nnz > 0) {
        switch (order) {
            case 2: st = launch_create_kernels<2>(kw, idx, ld_idx, val, nnz, n, bits, dup, l0, h0, p0, l1, h1, p1, fs, fd, ps, pd, cnt, radix, scan, out_lo, out_hi, out_val, sc, s); break;
            case 3: st = launch_create_kernels<3>(kw, idx, ld_idx, val, nnz, n, bits, dup, l0, h0, p0, l1, h1, p1, fs, fd, ps, pd, cnt, radix, scan, out_lo, out_hi, out_val, sc, s); break;
            case 4: st = launch_create_kernels<4>(kw, idx, ld_idx, val, nnz, n, bits, dup, l0, h0, p0, l1, h1, p1, fs, fd, ps, pd, cnt, radix, scan, out_lo, out_hi, out_val, sc, s); break;
            default: st = launch_create_kernels<5>(kw, idx, ld_idx, val, nnz, n, bits, dup, l0, h0, p0, l1, h1, p1, fs, fd, ps, pd, cnt, radix, scan, out_lo, out_hi, out_val, sc, s); break;
        }
        if (st != SYM_OK) return st;
    }
    DevCounters h;
    SYM_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    if (h.range_bad) return SYM_E_RANGE;
    if (dup == SYM_DUP_ERROR && h.dup_seen) return SYM_E_DUPLICATE;
    if (dup == SYM_DUP_KEEP_EQUAL && h.dup_mismatch) return SYM_E_DUPLICATE;

    sym_tensor_s* t = new (std::nothrow) sym_tensor_s();
    if (!t) return SYM_E_NOMEM;
    t->order = order;
    t->bits = bits;
    t->kw = kw;
    t->n = n;
    t->nnz = (int64_t)h.nnz_kept;
    t->nnz_strict = (int64_t)h.nnz_strict;
    t->klo = out_lo;
    t->khi = out_hi;
    t->val = out_val;
    t->rklo = nullptr;
    t->rkhi = nullptr;
    t->rval = nullptr;
    sym_mttkrp_default_config(&t->cfg);
    t->device = current_device();
    sym_tensor_info_t& I = t->info;
    memset(&I, 0, sizeof(I));
    I.order = order;
    I.key_bits = bits;
    I.n = n;
    I.nnz = t->nnz;
    I.nnz_strict = t->nnz_strict;
    I.nnz_diag = t->nnz - t->nnz_strict;
    I.duplicates_dropped = (int64_t)h.dup_seen;
    for (int p = 0; p < 16; ++p) I.counts_by_pattern[p] = (int64_t)h.by_pattern[p];
    I.expanded_nnz = (int64_t)h.expanded;
    I.root_fibers = (int64_t)h.root_fibers;
    I.l2_fibers = (int64_t)h.l2_fibers;
    I.normsq = h.normsq;
    I.arena_used = A.used;
    *out = t;
    return SYM_OK;
}

extern "C" sym_status sym_tensor_info(sym_tensor X, sym_tensor_info_t* out) {
    if (!X || !out) return SYM_E_INVALID;
    *out = X->info;
    return SYM_OK;
}

extern "C" sym_status sym_tensor_export(sym_tensor X, int32_t* cidx, int64_t ld_out, float* cval,
                                        sym_stream_t stream) {
    if (!X || (X->nnz > 0 && (!cidx || !cval)) || ld_out < X->nnz) return SYM_E_INVALID;
    if (X->nnz == 0) return SYM_OK;
    cudaStream_t s = as_stream(stream);
    unsigned g = (unsigned)((X->nnz + 255) / 256);
#define SYM_EXPORT_CASE(N)                                                                                    \
    if (X->kw == 1)                                                                                           \
        k_export<N, 1><<<g, 256, 0, s>>>(X->klo, X->khi, X->val, X->nnz, X->bits, cidx, ld_out, cval);      \
    else                                                                                                      \
        k_export<N, 2><<<g, 256, 0, s>>>(X->klo, X->khi, X->val, X->nnz, X->bits, cidx, ld_out, cval);
    switch (X->order) {
        case 2: SYM_EXPORT_CASE(2) break;
        case 3: SYM_EXPORT_CASE(3) break;
        case 4: SYM_EXPORT_CASE(4) break;
        default: SYM_EXPORT_CASE(5) break;
    }
#undef SYM_EXPORT_CASE
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_tensor_destroy(sym_tensor X) {
    delete X;
    return SYM_OK;
}

extern "C" sym_status sym_gen_coords(int order, int64_t n, int64_t count, uint64_t seed, int32_t* idx,
                                     int64_t ld_idx, float* val, sym_stream_t stream) {
    if (order < 1 || order > 5 || n < 1 || n > 0x7fffffffLL || count < 0 || ld_idx < count) return SYM_E_INVALID;
    if (count == 0) return SYM_OK;
    if (!idx || !val) return SYM_E_INVALID;
    k_gen_coords<<<(unsigned)((count + 255) / 256), 256, 0, as_stream(stream)>>>(order, n, count, seed, idx, ld_idx,
                                                                                 val);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" size_t sym_tensor_upper_csr_ws_bytes(sym_tensor X) {
    if (!X || X->order != 2) return 0;
    Sizer z;
    z.take<unsigned long long>((size_t)X->n + 1);
    z.take<unsigned long long>((size_t)X->n + 1);
    z.take<int64_t>((size_t)X->n + 1);
    z.take<int>((size_t)X->n + 1);
    z.take<char>(scan_ws_bytes(X->n + 1));
    return z.used;
}

extern "C" sym_status sym_tensor_upper_csr(sym_tensor X, int64_t* rowptr, int32_t* col, float* val, void* ws,
                                           size_t ws_bytes, sym_stream_t stream) {
    if (!X || X->order != 2 || X->kw != 1 || !rowptr || (X->nnz > 0 && (!col || !val)) || !ws) return SYM_E_INVALID;
    if (ws_bytes < sym_tensor_upper_csr_ws_bytes(X)) return SYM_E_NOMEM;
    cudaStream_t s = as_stream(stream);
    const int64_t n = X->n;
    Carver W(ws, ws_bytes);
    unsigned long long* cnt = W.take<unsigned long long>((size_t)n + 1);
    unsigned long long* scnt = W.take<unsigned long long>((size_t)n + 1);
    int64_t* sstart = W.take<int64_t>((size_t)n + 1);
    int* hd = W.take<int>((size_t)n + 1);
    void* scan = W.take<char>(scan_ws_bytes(n + 1));
    SYM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s));
    SYM_CUDA(cudaMemsetAsync(scnt, 0, sizeof(unsigned long long) * (n + 1), s));
    SYM_CUDA(cudaMemsetAsync(hd, 0, sizeof(int) * (n + 1), s));
    if (X->nnz > 0) {
        k_csr_counts<<<(unsigned)((X->nnz + 255) / 256), 256, 0, s>>>(X->klo, X->nnz, X->nnz_strict, X->bits, cnt, scnt,
                                                                      hd);
        SYM_CHECK_LAUNCH();
    }
    const unsigned gn = (unsigned)((n + 1 + 255) / 256);
    k_u64_to_i64<<<gn, 256, 0, s>>>(cnt, n + 1, rowptr);
    SYM_CHECK_LAUNCH();
    sym_status st = exclusive_scan_i64(rowptr, rowptr, n + 1, scan, s);
    if (st != SYM_OK) return st;
    k_u64_to_i64<<<gn, 256, 0, s>>>(scnt, n + 1, sstart);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_i64(sstart, sstart, n + 1, scan, s);
    if (st != SYM_OK) return st;
    if (X->nnz > 0) {
        k_csr_fill<<<(unsigned)((X->nnz + 255) / 256), 256, 0, s>>>(X->klo, X->val, X->nnz, X->nnz_strict, X->bits,
                                                                    rowptr, sstart, hd, col, val);
        SYM_CHECK_LAUNCH();
    }
    return SYM_OK;
}

extern "C" sym_status sym_gen_batch_coords(int64_t count, const int64_t* row_off, const int64_t* draw_off,
                                           int64_t total_draws, uint64_t seed, int32_t* idx, int64_t ld_idx,
                                           float* val, sym_stream_t stream) {
    if (count < 1 || !row_off || !draw_off || total_draws < 0 || ld_idx < total_draws) return SYM_E_INVALID;
    if (total_draws == 0) return SYM_OK;
    if (!idx || !val) return SYM_E_INVALID;
    k_gen_batch<<<(unsigned)((total_draws + 255) / 256), 256, 0, as_stream(stream)>>>(count, row_off, draw_off,
                                                                                     total_draws, seed, idx, ld_idx,
                                                                                     val);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

namespace {

template <typename C>
void layout_leaf(C& a, C& w, int64_t ns, int kw, uint64_t** rlo, uint64_t** rhi, float** rval, uint64_t** l0,
                 uint64_t** h0, uint32_t** p0, uint64_t** l1, uint64_t** h1, uint32_t** p1, void** radix) {
    const size_t m = ns > 0 ? (size_t)ns : 1;
    *rlo = a.template take<uint64_t>(m);
    *rhi = kw == 2 ? a.template take<uint64_t>(m) : nullptr;
    *rval = a.template take<float>(m);
    *l0 = w.template take<uint64_t>(m);
    *h0 = kw == 2 ? w.template take<uint64_t>(m) : nullptr;
    *p0 = w.template take<uint32_t>(m);
    *l1 = w.template take<uint64_t>(m);
    *h1 = kw == 2 ? w.template take<uint64_t>(m) : nullptr;
    *p1 = w.template take<uint32_t>(m);
    *radix = w.template take<char>(radix_ws_bytes((int64_t)m, kw));
}

template <int N>
sym_status build_leaf(sym_tensor_s* X, uint64_t* rlo, uint64_t* rhi, float* rval, uint64_t* l0, uint64_t* h0,
                      uint32_t* p0, uint64_t* l1, uint64_t* h1, uint32_t* p1, void* radix, cudaStream_t s) {
    const int64_t ns = X->nnz_strict;
    const unsigned g = (unsigned)((ns + 255) / 256);
    if (X->kw == 1)
        k_reverse_pack<N, 1><<<g, 256, 0, s>>>(X->klo, X->khi, ns, X->bits, l0, h0, p0);
    else
        k_reverse_pack<N, 2><<<g, 256, 0, s>>>(X->klo, X->khi, ns, X->bits, l0, h0, p0);
    SYM_CHECK_LAUNCH();
    uint64_t *slo, *shi;
    uint32_t* sp;
    sym_status st = radix_sort_pairs(X->kw, l0, h0, p0, l1, h1, p1, ns, N * X->bits, radix, s, &slo, &shi, &sp);
    if (st != SYM_OK) return st;
    SYM_CUDA(cudaMemcpyAsync(rlo, slo, sizeof(uint64_t) * ns, cudaMemcpyDeviceToDevice, s));
    if (X->kw == 2) SYM_CUDA(cudaMemcpyAsync(rhi, shi, sizeof(uint64_t) * ns, cudaMemcpyDeviceToDevice, s));
    k_gather_f32<<<g, 256, 0, s>>>(X->val, sp, ns, rval);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

}  // namespace

extern "C" sym_status sym_tensor_leaf_index_bytes(sym_tensor X, size_t* arena_bytes, size_t* ws_bytes) {
    if (!X || X->order < 3) return SYM_E_INVALID;
    NullCarver a, w;
    uint64_t *rlo, *rhi, *l0, *h0, *l1, *h1;
    float* rv;
    uint32_t *p0, *p1;
    void* radix;
    layout_leaf(a, w, X->nnz_strict, X->kw, &rlo, &rhi, &rv, &l0, &h0, &p0, &l1, &h1, &p1, &radix);
    if (arena_bytes) *arena_bytes = a.s.used;
    if (ws_bytes) *ws_bytes = w.s.used;
    return SYM_OK;
}

extern "C" sym_status sym_tensor_add_leaf_index(sym_tensor X, void* arena, size_t arena_bytes, void* ws,
                                                size_t ws_bytes, sym_stream_t stream) {
    size_t na = 0, nw = 0;
    sym_status st = sym_tensor_leaf_index_bytes(X, &na, &nw);
    if (st != SYM_OK) return st;
    if (!arena || !ws || !aligned(arena, 256) || !aligned(ws, 256)) return SYM_E_INVALID;
    if (arena_bytes < na || ws_bytes < nw) return SYM_E_NOMEM;
    Carver A(arena, arena_bytes), W(ws, ws_bytes);
    uint64_t *rlo, *rhi, *l0, *h0, *l1, *h1;
    float* rv;
    uint32_t *p0, *p1;
    void* radix;
    layout_leaf(A, W, X->nnz_strict, X->kw, &rlo, &rhi, &rv, &l0, &h0, &p0, &l1, &h1, &p1, &radix);
    cudaStream_t s = as_stream(stream);
    if (X->nnz_strict > 0) {
        switch (X->order) {
            case 3: st = build_leaf<3>(X, rlo, rhi, rv, l0, h0, p0, l1, h1, p1, radix, s); break;
            case 4: st = build_leaf<4>(X, rlo, rhi, rv, l0, h0, p0, l1, h1, p1, radix, s); break;
            default: st = build_leaf<5>(X, rlo, rhi, rv, l0, h0, p0, l1, h1, p1, radix, s); break;
        }
        if (st != SYM_OK) return st;
    }
    SYM_CUDA(cudaStreamSynchronize(s));
    X->rklo = rlo;
    X->rkhi = rhi;
    X->rval = rv;
    X->info.arena_used += A.used;
    return SYM_OK;
}
