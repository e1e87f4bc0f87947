// Non-symmetric baseline: the fully expanded tensor (every distinct permutation
// of every canonical entry, i.e. all nonzeros of the full symmetric tensor),
// sorted lexicographically, and a plain mode-1 MTTKRP over it that uses no
// symmetry.  This is what the symmetric kernels are measured against: the
// paper's "naive" kernels read the full tensor (Sec. 5.2, Sec. 5.2.6).
#include <algorithm>
#include <new>

#include "common.cuh"
#include "tensor.cuh"

struct sym_expanded_s {
    int order, bits, kw;
    int64_t n, nnz;
    uint64_t* klo;
    uint64_t* khi;
    float* val;
};

namespace symgpu {

namespace {

template <int N>
__device__ __forceinline__ int perm_count(const int32_t* c) {
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
    return fact[N] / (den * fact[run]);
}

// Next lexicographic arrangement of a[0..N); false after the last one.
template <int N>
__device__ __forceinline__ bool next_arrangement(int32_t* a) {
    int i = N - 2;
    while (i >= 0 && a[i] >= a[i + 1]) --i;
    if (i < 0) return false;
    int j = N - 1;
    while (a[j] <= a[i]) --j;
    int32_t t = a[i];
    a[i] = a[j];
    a[j] = t;
    for (int l = i + 1, r = N - 1; l < r; ++l, --r) {
        t = a[l];
        a[l] = a[r];
        a[r] = t;
    }
    return true;
}

template <int N, int KW>
__global__ void k_count_perms(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, int64_t nnz,
                              int bits, int64_t* __restrict__ cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int32_t c[N];
    unpack_key<N, KW>(KeyWords{klo[e], KW == 2 ? khi[e] : 0ull}, bits, c);
    cnt[e] = perm_count<N>(c);
}

template <int N, int KW>
__global__ void k_expand(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, int64_t nnz, int bits,
                         const int64_t* __restrict__ off, uint64_t* __restrict__ olo, uint64_t* __restrict__ ohi,
                         uint32_t* __restrict__ pay) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int32_t c[N];
    unpack_key<N, KW>(KeyWords{klo[e], KW == 2 ? khi[e] : 0ull}, bits, c);  // ascending
    int64_t k = off[e];
    do {
        KeyWords w = pack_key<N, KW>(c, bits);
        olo[k] = w.lo;
        if (KW == 2) ohi[k] = w.hi;
        pay[k] = (uint32_t)e;
        ++k;
    } while (next_arrangement<N>(c));
}

__global__ void k_gather_val(const float* __restrict__ src, const uint32_t* __restrict__ pay, int64_t m,
                             float* __restrict__ dst) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) dst[k] = src[pay[k]];
}

template <int N, int KW>
__global__ void k_export_exp(const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi,
                             const float* __restrict__ val, int64_t m, int bits, int32_t* __restrict__ out,
                             int64_t ld, float* __restrict__ oval) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    int32_t c[N];
    unpack_key<N, KW>(KeyWords{klo[k], KW == 2 ? khi[k] : 0ull}, bits, c);
#pragma unroll
    for (int q = 0; q < N; ++q) out[(int64_t)q * ld + k] = c[q];
    oval[k] = val[k];
}

constexpr int EX_THREADS = 256;

// Mode-1 MTTKRP over the expanded tensor: M[c_1] += v * prod_{q>=2} B[c_q].
// Entries are sorted by c_1, so each group keeps a register accumulator for
// the current output row and reduces it to memory only when the row changes.
template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(EX_THREADS) k_mttkrp_expanded(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, int64_t chunk) {
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t warp = ((int64_t)blockIdx.x * EX_THREADS + threadIdx.x) >> 5;
    const int64_t start = warp * chunk;
    if (start >= nnz) return;
    const int64_t end = min(start + chunk, nnz);
    int32_t cur = -1;
    float4 acc = f4_zero();
    for (int64_t b0 = start; b0 < end; b0 += 32) {
        const int64_t e = b0 + lane;
        uint64_t mlo = 0, mhi = 0;
        float mv = 0.f;
        if (e < end) {
            mlo = klo[e];
            if (KW == 2) mhi = khi[e];
            mv = val[e];
        }
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            const int src = g * L + t;
            const uint64_t lo = __shfl_sync(0xffffffffu, mlo, src);
            const uint64_t hi = (KW == 2) ? __shfl_sync(0xffffffffu, mhi, src) : 0ull;
            const float v = __shfl_sync(0xffffffffu, mv, src);
            if (b0 + src >= end || !on) continue;
            int32_t c[N];
            unpack_key<N, KW>(KeyWords{lo, hi}, bits, c);
            if (c[0] != cur) {
                if (cur >= 0) red_add_f4(M + (int64_t)cur * ldm + col, acc);
                acc = f4_zero();
                cur = c[0];
            }
            float4 p = load_row4<BF16>(B, c[1], ldb, col);
#pragma unroll
            for (int q = 2; q < N; ++q) p = f4_mul(p, load_row4<BF16>(B, c[q], ldb, col));
            acc = f4_fmas(p, v, acc);
        }
    }
    if (on && cur >= 0) red_add_f4(M + (int64_t)cur * ldm + col, acc);
}

template <typename C>
void layout_exp_arena(C& c, int64_t m, int kw, uint64_t** lo, uint64_t** hi, float** val) {
    size_t k = m > 0 ? (size_t)m : 1;
    *lo = c.template take<uint64_t>(k);
    *hi = kw == 2 ? c.template take<uint64_t>(k) : nullptr;
    *val = c.template take<float>(k);
}

template <typename C>
void layout_exp_ws(C& c, int64_t nnz, int64_t m, int kw, int64_t** cnt, int64_t** off, uint64_t** lo0,
                   uint64_t** hi0, uint32_t** p0, uint32_t** p1, void** radix, void** scan) {
    size_t k = m > 0 ? (size_t)m : 1;
    *cnt = c.template take<int64_t>((size_t)nnz + 1);
    *off = c.template take<int64_t>((size_t)nnz + 1);
    *lo0 = c.template take<uint64_t>(k);
    *hi0 = kw == 2 ? c.template take<uint64_t>(k) : nullptr;
    *p0 = c.template take<uint32_t>(k);
    *p1 = c.template take<uint32_t>(k);
    *radix = c.template take<char>(radix_ws_bytes((int64_t)k, kw));
    *scan = c.template take<char>(scan_ws_bytes(nnz + 1));
}

struct NullCarver {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

template <int N>
sym_status expand_order(const sym_tensor_s* X, sym_expanded_s* E, Carver& W, cudaStream_t s) {
    int64_t *cnt, *off;
    uint64_t *lo0, *hi0;
    uint32_t *p0, *p1;
    void *radix, *scan;
    layout_exp_ws(W, X->nnz, E->nnz, X->kw, &cnt, &off, &lo0, &hi0, &p0, &p1, &radix, &scan);
    if (!scan) return SYM_E_NOMEM;
    const unsigned g = (unsigned)((X->nnz + 255) / 256);
    if (X->kw == 1)
        k_count_perms<N, 1><<<g, 256, 0, s>>>(X->klo, X->khi, X->nnz, X->bits, cnt);
    else
        k_count_perms<N, 2><<<g, 256, 0, s>>>(X->klo, X->khi, X->nnz, X->bits, cnt);
    SYM_CHECK_LAUNCH();
    sym_status st = exclusive_scan_i64(cnt, off, X->nnz, scan, s);
    if (st != SYM_OK) return st;
    // expanded keys land directly in the arena arrays, sorted into the alternates
    if (X->kw == 1)
        k_expand<N, 1><<<g, 256, 0, s>>>(X->klo, X->khi, X->nnz, X->bits, off, E->klo, E->khi, p0);
    else
        k_expand<N, 2><<<g, 256, 0, s>>>(X->klo, X->khi, X->nnz, X->bits, off, E->klo, E->khi, p0);
    SYM_CHECK_LAUNCH();
    uint64_t *slo, *shi;
    uint32_t* sp;
    st = radix_sort_pairs(X->kw, E->klo, E->khi, p0, lo0, hi0, p1, E->nnz, N * X->bits, radix, s, &slo, &shi, &sp);
    if (st != SYM_OK) return st;
    if (slo != E->klo) {
        SYM_CUDA(cudaMemcpyAsync(E->klo, slo, sizeof(uint64_t) * E->nnz, cudaMemcpyDeviceToDevice, s));
        if (X->kw == 2)
            SYM_CUDA(cudaMemcpyAsync(E->khi, shi, sizeof(uint64_t) * E->nnz, cudaMemcpyDeviceToDevice, s));
    }
    k_gather_val<<<(unsigned)((E->nnz + 255) / 256), 256, 0, s>>>(X->val, sp, E->nnz, E->val);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

template <int N, int KW, bool BF16>
sym_status launch_exp(const sym_expanded_s* E, const void* B, int R, int64_t ldb, float* M, int64_t ldm,
                      cudaStream_t s) {
    const int64_t chunk = 256;
    const int64_t warps = (E->nnz + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((warps * 32 + EX_THREADS - 1) / EX_THREADS);
    int L = 1;
    while (4 * L < R) L <<= 1;
    SYM_PROF("mttkrp_expanded", s);
#define SYM_EXP_L(LL)                                                                                         \
    case LL:                                                                                                  \
        k_mttkrp_expanded<N, KW, LL, BF16><<<grid, EX_THREADS, 0, s>>>(E->klo, E->khi, E->val, E->nnz, E->bits, \
                                                                       B, ldb, R, M, ldm, chunk);             \
        break;
    switch (L) {
        SYM_EXP_L(1)
        SYM_EXP_L(2)
        SYM_EXP_L(4)
        SYM_EXP_L(8)
        SYM_EXP_L(16)
        SYM_EXP_L(32)
        default: return SYM_E_UNSUPPORTED;
    }
#undef SYM_EXP_L
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

template <int N>
sym_status launch_exp_order(const sym_expanded_s* E, const void* B, bool bf16, int R, int64_t ldb, float* M,
                            int64_t ldm, cudaStream_t s) {
    if (E->kw == 1)
        return bf16 ? launch_exp<N, 1, true>(E, B, R, ldb, M, ldm, s) : launch_exp<N, 1, false>(E, B, R, ldb, M, ldm, s);
    return bf16 ? launch_exp<N, 2, true>(E, B, R, ldb, M, ldm, s) : launch_exp<N, 2, false>(E, B, R, ldb, M, ldm, s);
}

}  // namespace

sym_status validate_mttkrp_args(const sym_tensor_s* X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                const float* M, int64_t ldm);

}  // namespace symgpu

using namespace symgpu;

extern "C" sym_status sym_expanded_bytes(sym_tensor X, size_t* arena_bytes, size_t* ws_bytes) {
    if (!X) return SYM_E_INVALID;
    const int64_t m = X->info.expanded_nnz;
    if (m > 0xffffffffLL) return SYM_E_UNSUPPORTED;
    NullCarver a, w;
    uint64_t *lo, *hi;
    float* v;
    layout_exp_arena(a, m, X->kw, &lo, &hi, &v);
    int64_t *cnt, *off;
    uint64_t *lo0, *hi0;
    uint32_t *p0, *p1;
    void *radix, *scan;
    layout_exp_ws(w, X->nnz, m, X->kw, &cnt, &off, &lo0, &hi0, &p0, &p1, &radix, &scan);
    if (arena_bytes) *arena_bytes = a.s.used;
    if (ws_bytes) *ws_bytes = w.s.used;
    return SYM_OK;
}

extern "C" sym_status sym_expanded_create(sym_tensor X, void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                                          sym_stream_t stream, sym_expanded* out) {
    if (!X || !out || !arena || !ws || !aligned(arena, 256) || !aligned(ws, 256)) return SYM_E_INVALID;
    *out = nullptr;
    size_t na = 0, nw = 0;
    sym_status st = sym_expanded_bytes(X, &na, &nw);
    if (st != SYM_OK) return st;
    if (arena_bytes < na || ws_bytes < nw) return SYM_E_NOMEM;
    sym_expanded_s* E = new (std::nothrow) sym_expanded_s();
    if (!E) return SYM_E_NOMEM;
    E->order = X->order;
    E->bits = X->bits;
    E->kw = X->kw;
    E->n = X->n;
    E->nnz = X->info.expanded_nnz;
    Carver A(arena, arena_bytes), W(ws, ws_bytes);
    layout_exp_arena(A, E->nnz, E->kw, &E->klo, &E->khi, &E->val);
    cudaStream_t s = as_stream(stream);
    if (E->nnz > 0) {
        switch (X->order) {
            case 2: st = expand_order<2>(X, E, W, s); break;
            case 3: st = expand_order<3>(X, E, W, s); break;
            case 4: st = expand_order<4>(X, E, W, s); break;
            default: st = expand_order<5>(X, E, W, s); break;
        }
    }
    if (st == SYM_OK) st = cuda_status(cudaStreamSynchronize(s));
    if (st != SYM_OK) {
        delete E;
        return st;
    }
    *out = E;
    return SYM_OK;
}

extern "C" sym_status sym_expanded_info(sym_expanded E, int64_t* nnz) {
    if (!E || !nnz) return SYM_E_INVALID;
    *nnz = E->nnz;
    return SYM_OK;
}

extern "C" sym_status sym_expanded_export(sym_expanded E, int32_t* eidx, int64_t ld_out, float* evals,
                                          sym_stream_t stream) {
    if (!E || ld_out < E->nnz || (E->nnz > 0 && (!eidx || !evals))) return SYM_E_INVALID;
    if (E->nnz == 0) return SYM_OK;
    cudaStream_t s = as_stream(stream);
    const unsigned g = (unsigned)((E->nnz + 255) / 256);
#define SYM_EXE(N)                                                                                          \
    if (E->kw == 1)                                                                                         \
        k_export_exp<N, 1><<<g, 256, 0, s>>>(E->klo, E->khi, E->val, E->nnz, E->bits, eidx, ld_out, evals); \
    else                                                                                                    \
        k_export_exp<N, 2><<<g, 256, 0, s>>>(E->klo, E->khi, E->val, E->nnz, E->bits, eidx, ld_out, evals);
    switch (E->order) {
        case 2: SYM_EXE(2) break;
        case 3: SYM_EXE(3) break;
        case 4: SYM_EXE(4) break;
        default: SYM_EXE(5) break;
    }
#undef SYM_EXE
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_expanded(sym_expanded E, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                          float* M, int64_t ldm, sym_stream_t stream) {
    if (!E || !B || !M) return SYM_E_INVALID;
    if (bdt != SYM_F32 && bdt != SYM_BF16) return SYM_E_INVALID;
    if (rank < 4 || rank > 128 || rank % 4 != 0 || ldb < rank || ldm < rank || ldb % 4 || ldm % 4)
        return SYM_E_INVALID;
    if (!aligned(B, bdt == SYM_BF16 ? 8 : 16) || !aligned(M, 16)) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    if (ldm == rank)
        SYM_CUDA(cudaMemsetAsync(M, 0, sizeof(float) * (size_t)E->n * rank, s));
    else
        SYM_CUDA(cudaMemset2DAsync(M, sizeof(float) * ldm, 0, sizeof(float) * rank, E->n, s));
    if (E->nnz == 0) return SYM_OK;
    const bool bf16 = bdt == SYM_BF16;
    switch (E->order) {
        case 2: return launch_exp_order<2>(E, B, bf16, rank, ldb, M, ldm, s);
        case 3: return launch_exp_order<3>(E, B, bf16, rank, ldb, M, ldm, s);
        case 4: return launch_exp_order<4>(E, B, bf16, rank, ldb, M, ldm, s);
        default: return launch_exp_order<5>(E, B, bf16, rank, ldb, M, ldm, s);
    }
}

namespace symgpu {
namespace {

// Plain mode-1 TTM over the expanded 3-way tensor: with A stored in full and
// sorted by (c_1, c_2, c_3), C[c_1, c_2, :] = sum over the (c_1, c_2) fiber of
// v B[c_3, :] (A[k, j, l] = A[j, l, k] for the full tensor), summed in
// registers and flushed once per fiber; every output position, n x n, is
// computed.  No symmetry is used.
template <int KW, int L, bool BF16>
__global__ void __launch_bounds__(256) k_ttm3_expanded(const uint64_t* __restrict__ klo,
                                                       const uint64_t* __restrict__ khi,
                                                       const float* __restrict__ val, int64_t nnz, int bits,
                                                       int64_t n, const void* __restrict__ B, int64_t ldb, int R,
                                                       float* __restrict__ C) {
    constexpr int64_t CHUNK = 256;
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t start = warp * CHUNK;
    const int64_t end = min(start + CHUNK, nnz);
    if (start >= end) return;
    int32_t ca = -1, cb = -1;
    float4 acc = f4_zero();
    for (int64_t b0 = start; b0 < end; b0 += 32) {
        const int64_t e = b0 + lane;
        uint64_t mlo = 0, mhi = 0;
        float mv = 0.f;
        if (e < end) {
            mlo = __ldcs(klo + e);
            if (KW == 2) mhi = __ldcs(khi + e);
            mv = __ldcs(val + e);
        }
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            const int src = g * L + t;
            const uint64_t lo = __shfl_sync(0xffffffffu, mlo, src);
            const uint64_t hi = (KW == 2) ? __shfl_sync(0xffffffffu, mhi, src) : 0ull;
            const float v = __shfl_sync(0xffffffffu, mv, src);
            if (b0 + src >= end) continue;
            int32_t c[3];
            unpack_key<3, KW>(KeyWords{lo, hi}, bits, c);
            if (c[0] != ca || c[1] != cb) {
                if (ca >= 0 && on) red_add_f4(C + ((int64_t)ca * n + cb) * R + col, acc);
                acc = f4_zero();
                ca = c[0];
                cb = c[1];
            }
            if (on) acc = f4_fmas(load_row4<BF16>(B, c[2], ldb, col), v, acc);
        }
    }
    if (ca >= 0 && on) red_add_f4(C + ((int64_t)ca * n + cb) * R + col, acc);
}

template <int KW, int L>
void launch_ttm_exp(const sym_expanded_s* E, const void* B, bool bf16, int64_t ldb, int R, float* C, cudaStream_t s) {
    const int64_t warps = (E->nnz + 255) / 256;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    if (bf16)
        k_ttm3_expanded<KW, L, true><<<grid, 256, 0, s>>>(E->klo, E->khi, E->val, E->nnz, E->bits, E->n, B, ldb, R, C);
    else
        k_ttm3_expanded<KW, L, false><<<grid, 256, 0, s>>>(E->klo, E->khi, E->val, E->nnz, E->bits, E->n, B, ldb, R, C);
}

template <int KW>
void launch_ttm_exp_l(const sym_expanded_s* E, const void* B, bool bf16, int64_t ldb, int R, float* C,
                      cudaStream_t s) {
    const int q = R / 4;
    if (q <= 1) launch_ttm_exp<KW, 1>(E, B, bf16, ldb, R, C, s);
    else if (q <= 2) launch_ttm_exp<KW, 2>(E, B, bf16, ldb, R, C, s);
    else if (q <= 4) launch_ttm_exp<KW, 4>(E, B, bf16, ldb, R, C, s);
    else if (q <= 8) launch_ttm_exp<KW, 8>(E, B, bf16, ldb, R, C, s);
    else if (q <= 16) launch_ttm_exp<KW, 16>(E, B, bf16, ldb, R, C, s);
    else launch_ttm_exp<KW, 32>(E, B, bf16, ldb, R, C, s);
}

}  // namespace
}  // namespace symgpu

extern "C" sym_status sym_ttm_expanded(sym_expanded E, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C,
                                       sym_stream_t stream) {
    if (!E || !B || !C) return SYM_E_INVALID;
    if (E->order != 3 || E->kw != 1) return SYM_E_UNSUPPORTED;
    if (bdt != SYM_F32 && bdt != SYM_BF16) return SYM_E_INVALID;
    if (rank < 4 || rank > 128 || rank % 4 != 0 || ldb < rank || ldb % 4) return SYM_E_INVALID;
    if (!aligned(B, bdt == SYM_BF16 ? 8 : 16) || !aligned(C, 16)) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    SYM_CUDA(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)E->n * E->n * rank, s));
    if (E->nnz == 0) return SYM_OK;
    SYM_PROF("ttm_expanded", s);
    launch_ttm_exp_l<1>(E, B, bdt == SYM_BF16, ldb, rank, C, s);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_expanded_destroy(sym_expanded E) {
    delete E;
    return SYM_OK;
}
