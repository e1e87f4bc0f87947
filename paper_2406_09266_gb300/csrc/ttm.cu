// Mode-1 TTM of a fully symmetric 3-way tensor with visible output symmetry
// (Sec. 4.2, TTM listing and the two output-symmetry listings; Sec. 5.2.5):
//   C[i, j, l] = sum_k A[k, j, l] B[k, i]
// reading only the canonical triangle of A and writing only the canonical
// triangle (j <= l) of C, which is symmetric in (j, l).
//
// For a canonical entry a <= b <= c with value v, the distinct permutations
// (k, j, l) of (a, b, c) with j <= l are one per distinct value taken as k:
//   k = c:  C[a, b] += v B[c]       (every pattern)
//   k = b:  C[a, c] += v B[b]       (unless b == c: then (a, c) = (a, b), counted above)
//   k = a:  C[b, c] += v B[a]       (unless a == b: then (b, c) = (a, c), counted above)
// i.e. 3 updates for a strict entry (half of its 6 assignments), 2 for
// a = b < c and a < b = c, 1 for a = b = c.  The first update is the leaf of
// the (a, b) fiber of the sorted stream and is summed in registers across the
// fiber; the other two are 16-byte vector reductions.  Strict and diagonal
// streams are processed by the same rule in one pass.
//
// With the tensor's leaf index (the strict entries again, each tuple reversed
// to (c, b, a) and sorted), the k = a update of the strict entries becomes a
// fiber sum too: C[b, c] += sum over the (c, b) fiber of v B[a], flushed once
// per fiber by a second pass, so the first pass keeps one reduction per entry.
//
// Schedule: each warp takes chunks of `entries_per_warp` consecutive entries;
// with ctas_per_sm > 0 the grid is persistent and warp w takes chunks
// w, w + W, w + 2W, ... (W warps in the grid), so the whole GPU walks the
// sorted stream front to back and the output rows being updated at any time
// stay within a window that L2 can hold.
//
// Output layouts (rank index fastest, R floats per output position):
//   SYM_TTM_PACKED: the canonical triangle only, position (j, l), j <= l, at
//                   p = j n - j (j - 1) / 2 + (l - j)   (n (n + 1) / 2 positions);
//   SYM_TTM_FULL:   n x n positions; the canonical triangle is computed in
//                   place, then a replication pass copies C[l, j] to C[j, l]
//                   for j > l (the copy loop of the output-symmetry listing).
#include <algorithm>

#include "common.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

constexpr int TTM_THREADS = 256;

template <bool FULL>
__device__ __forceinline__ int64_t out_pos(int64_t j, int64_t l, int64_t n) {
    if constexpr (FULL) return j * n + l;
    return j * n - j * (j - 1) / 2 + (l - j);
}

// Loads the next 32 entries of [b0, end) into the lanes (evict-first: the
// stream is read once).
__device__ __forceinline__ void ttm_load32(const uint64_t* __restrict__ klo, const float* __restrict__ val, int64_t e,
                                           int64_t end, uint64_t* key, float* v) {
    *key = 0;
    *v = 0.f;
    if (e < end) {
        *key = __ldcs(klo + e);
        *v = __ldcs(val + e);
    }
}

// First pass, over the canonical stream (strict then diagonal, one-word keys).
// LEAF_SPLIT: the k = a update of strict entries is left to the leaf pass.
template <int L, bool BF16, bool FULL, bool LEAF_SPLIT>
__global__ void __launch_bounds__(TTM_THREADS) k_ttm3(const uint64_t* __restrict__ klo, const float* __restrict__ val,
                                                      int64_t nnz, int bits, int64_t n, const void* __restrict__ B,
                                                      int64_t ldb, int R, float* __restrict__ C, int64_t chunk) {
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t start = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * chunk; start < nnz;
         start += W * chunk) {
        const int64_t end = min(start + chunk, nnz);
        int32_t ca = -1, cb = -1;
        float4 Ba = f4_zero(), Bb = f4_zero(), acc = f4_zero();
        for (int64_t b0 = start; b0 < end; b0 += 32) {
            uint64_t mk;
            float mv;
            ttm_load32(klo, val, b0 + lane, end, &mk, &mv);
#pragma unroll 1
            for (int t = 0; t < L; ++t) {
                const int src = g * L + t;
                const uint64_t key = __shfl_sync(0xffffffffu, mk, src);
                const float v = __shfl_sync(0xffffffffu, mv, src);
                if (b0 + src >= end) continue;
                int32_t c[3];
                unpack_key<3, 1>(KeyWords{key, 0ull}, bits, c);
                if (c[0] != ca || c[1] != cb) {
                    if (ca >= 0 && on) red_add_f4(C + out_pos<FULL>(ca, cb, n) * R + col, acc);
                    acc = f4_zero();
                    if (c[0] != ca) Ba = on ? load_row4<BF16>(B, c[0], ldb, col) : f4_zero();
                    Bb = (c[1] == c[0]) ? Ba : (on ? load_row4<BF16>(B, c[1], ldb, col) : f4_zero());
                    ca = c[0];
                    cb = c[1];
                }
                const float4 bc = on ? load_row4<BF16>(B, c[2], ldb, col) : f4_zero();
                acc = f4_fmas(bc, v, acc);
                if (on && c[1] != c[2]) red_add_f4(C + out_pos<FULL>(c[0], c[2], n) * R + col, f4_scale(Bb, v));
                const bool ka = LEAF_SPLIT ? (c[0] != c[1] && c[1] == c[2]) : (c[0] != c[1]);
                if (on && ka) red_add_f4(C + out_pos<FULL>(c[1], c[2], n) * R + col, f4_scale(Ba, v));
            }
        }
        if (ca >= 0 && on) red_add_f4(C + out_pos<FULL>(ca, cb, n) * R + col, acc);
    }
}

// Second pass, over the leaf index: strict entries as (c, b, a), sorted, so
// the (c, b) fiber sums v B[a] into C[b, c] in registers.
template <int L, bool BF16, bool FULL>
__global__ void __launch_bounds__(TTM_THREADS) k_ttm3_leaf(const uint64_t* __restrict__ rklo,
                                                           const float* __restrict__ rval, int64_t nnz, int bits,
                                                           int64_t n, const void* __restrict__ B, int64_t ldb, int R,
                                                           float* __restrict__ C, int64_t chunk) {
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t start = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * chunk; start < nnz;
         start += W * chunk) {
        const int64_t end = min(start + chunk, nnz);
        int32_t cc = -1, cb = -1;
        float4 acc = f4_zero();
        for (int64_t b0 = start; b0 < end; b0 += 32) {
            uint64_t mk;
            float mv;
            ttm_load32(rklo, rval, b0 + lane, end, &mk, &mv);
#pragma unroll 1
            for (int t = 0; t < L; ++t) {
                const int src = g * L + t;
                const uint64_t key = __shfl_sync(0xffffffffu, mk, src);
                const float v = __shfl_sync(0xffffffffu, mv, src);
                if (b0 + src >= end) continue;
                int32_t c[3];  // (c, b, a), c > b > a
                unpack_key<3, 1>(KeyWords{key, 0ull}, bits, c);
                if (c[0] != cc || c[1] != cb) {
                    if (cc >= 0 && on) red_add_f4(C + out_pos<FULL>(cb, cc, n) * R + col, acc);
                    acc = f4_zero();
                    cc = c[0];
                    cb = c[1];
                }
                if (on) acc = f4_fmas(load_row4<BF16>(B, c[2], ldb, col), v, acc);
            }
        }
        if (cc >= 0 && on) red_add_f4(C + out_pos<FULL>(cb, cc, n) * R + col, acc);
    }
}

// C[j, l, :] = C[l, j, :] for j > l in the full n x n layout, by P x P tiles
// of positions staged in shared memory so that both the read (row l of the
// upper triangle) and the write (row j of the lower one) touch P consecutive
// positions (P R floats) at a time.  Tile (tj, tl), tl <= tj, is numbered
// row-major over the lower tile triangle; each CTA walks tiles with a stride.
__global__ void __launch_bounds__(256) k_ttm_mirror(float* __restrict__ C, int64_t n, int R, int P) {
    extern __shared__ float4 tile[];  // [l in tile][j in tile][R/4]
    const int per = R / 4;
    const int run = P * per;           // float4 of one tile row (P positions), <= 256
    const int rows_per_pass = blockDim.x / run;
    const int r_in = threadIdx.x % run, r_row = threadIdx.x / run;
    const int r_pos = r_in / per;      // position inside the run
    const int64_t nt = (n + P - 1) / P;
    const int64_t tiles = nt * (nt + 1) / 2;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // t -> (tj, tl), tl <= tj: tj is the largest row with tj (tj + 1) / 2 <= t (integer search)
        int64_t lo = 0, hi = nt - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (mid * (mid + 1) / 2 <= t) lo = mid; else hi = mid - 1;
        }
        const int64_t j0 = lo * P, l0 = (t - lo * (lo + 1) / 2) * P;
        const int pj = (int)(n - j0 < P ? n - j0 : P), pl = (int)(n - l0 < P ? n - l0 : P);
        __syncthreads();
        // source rows l: C[l, j0 + r_pos], contiguous over the run
        if (r_row < rows_per_pass && r_pos < pj) {
            const int64_t j = j0 + r_pos;
            for (int ll = r_row; ll < pl; ll += rows_per_pass) {
                const int64_t l = l0 + ll;
                if (j > l) tile[ll * run + r_in] = *reinterpret_cast<const float4*>(C + (l * n + j0) * R + 4 * r_in);
            }
        }
        __syncthreads();
        // destination rows j: C[j, l0 + r_pos], contiguous over the run
        if (r_row < rows_per_pass && r_pos < pl) {
            const int64_t l = l0 + r_pos;
            const int c = r_in - r_pos * per;
            for (int jj = r_row; jj < pj; jj += rows_per_pass) {
                const int64_t j = j0 + jj;
                if (j > l)
                    *reinterpret_cast<float4*>(C + (j * n + l0) * R + 4 * r_in) = tile[r_pos * run + jj * per + c];
            }
        }
    }
}

struct TtmLaunch {
    const sym_tensor_s* X;
    const void* B;
    int64_t ldb;
    int R;
    float* C;
    bool full;
    bool leaf;      // two passes (leaf index present and wanted)
    int64_t chunk;  // entries per warp chunk
    int ctas_per_sm;
    cudaStream_t s;
};

inline unsigned ttm_grid(const TtmLaunch& a, int64_t nnz) {
    const int64_t warps = (nnz + a.chunk - 1) / a.chunk;
    const int64_t need = (warps * 32 + TTM_THREADS - 1) / TTM_THREADS;
    if (a.ctas_per_sm <= 0) return (unsigned)std::max<int64_t>(1, need);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sm_count() * a.ctas_per_sm));
}

template <int L, bool BF16, bool FULL>
void launch_ttm3(const TtmLaunch& a) {
    const sym_tensor_s* X = a.X;
    if (a.leaf) {
        k_ttm3<L, BF16, FULL, true><<<ttm_grid(a, X->nnz), TTM_THREADS, 0, a.s>>>(X->klo, X->val, X->nnz, X->bits,
                                                                                 X->n, a.B, a.ldb, a.R, a.C, a.chunk);
        if (X->nnz_strict > 0)
            k_ttm3_leaf<L, BF16, FULL><<<ttm_grid(a, X->nnz_strict), TTM_THREADS, 0, a.s>>>(
                X->rklo, X->rval, X->nnz_strict, X->bits, X->n, a.B, a.ldb, a.R, a.C, a.chunk);
    } else {
        k_ttm3<L, BF16, FULL, false><<<ttm_grid(a, X->nnz), TTM_THREADS, 0, a.s>>>(X->klo, X->val, X->nnz, X->bits,
                                                                                  X->n, a.B, a.ldb, a.R, a.C, a.chunk);
    }
}

template <int L, bool BF16>
void launch_ttm3_f(const TtmLaunch& a) {
    if (a.full) launch_ttm3<L, BF16, true>(a);
    else launch_ttm3<L, BF16, false>(a);
}

template <bool BF16>
void launch_ttm3_l(const TtmLaunch& a) {
    const int q = a.R / 4;  // float4 columns
    if (q <= 1) launch_ttm3_f<1, BF16>(a);
    else if (q <= 2) launch_ttm3_f<2, BF16>(a);
    else if (q <= 4) launch_ttm3_f<4, BF16>(a);
    else if (q <= 8) launch_ttm3_f<8, BF16>(a);
    else if (q <= 16) launch_ttm3_f<16, BF16>(a);
    else launch_ttm3_f<32, BF16>(a);
}

}  // namespace

}  // namespace symgpu

using namespace symgpu;

extern "C" int64_t sym_ttm_output_elems(int64_t n, int rank, sym_ttm_layout layout) {
    if (n < 0 || rank <= 0) return -1;
    if (layout == SYM_TTM_PACKED) return n * (n + 1) / 2 * rank;
    if (layout == SYM_TTM_FULL) return n * n * rank;
    return -1;
}

extern "C" sym_status sym_ttm_default_config(sym_ttm_cfg* out) {
    if (!out) return SYM_E_INVALID;
    out->entries_per_warp = 64;
    out->ctas_per_sm = 0;
    out->leaf_index = -1;
    return SYM_OK;
}

extern "C" sym_status sym_ttm(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C,
                              sym_ttm_layout layout, const sym_ttm_cfg* cfg, sym_stream_t stream) {
    if (!X || !B || !C) return SYM_E_INVALID;
    if (X->order != 3) return SYM_E_UNSUPPORTED;
    // two-word keys mean n > 2^21: the dense output (>= 2^41 positions) cannot exist
    if (X->kw != 1) return SYM_E_UNSUPPORTED;
    if (bdt != SYM_F32 && bdt != SYM_BF16) return SYM_E_INVALID;
    if (layout != SYM_TTM_PACKED && layout != SYM_TTM_FULL) return SYM_E_INVALID;
    if (rank < 4 || rank > 128 || rank % 4 != 0) return SYM_E_INVALID;
    if (ldb < rank || ldb % 4 != 0) return SYM_E_INVALID;
    if (!aligned(B, bdt == SYM_BF16 ? 8 : 16) || !aligned(C, 16)) return SYM_E_INVALID;
    sym_ttm_cfg c;
    sym_ttm_default_config(&c);
    if (cfg) c = *cfg;
    if (c.entries_per_warp < 32 || c.entries_per_warp % 32 != 0 || c.entries_per_warp > (1 << 20)) return SYM_E_INVALID;
    if (c.ctas_per_sm < 0 || c.ctas_per_sm > 8) return SYM_E_INVALID;
    if (c.leaf_index < -1 || c.leaf_index > 1) return SYM_E_INVALID;
    if (c.leaf_index == 1 && !X->rklo) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    TtmLaunch a{X, B, ldb, rank, C, layout == SYM_TTM_FULL, c.leaf_index != 0 && X->rklo != nullptr,
                c.entries_per_warp, c.ctas_per_sm, s};
    const int64_t elems = sym_ttm_output_elems(X->n, rank, layout);
    SYM_CUDA(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)elems, s));
    if (X->nnz > 0) {
        SYM_PROF("ttm", s);
        if (bdt == SYM_BF16)
            launch_ttm3_l<true>(a);
        else
            launch_ttm3_l<false>(a);
        SYM_CHECK_LAUNCH();
    }
    if (a.full && X->n > 1) {
        SYM_PROF("ttm_mirror", s);
        const int P = rank <= 32 ? 16 : 8;  // tile <= 16 x 16 x 32 or 8 x 8 x 128 floats = 32 KB
        const int64_t nt = (X->n + P - 1) / P;
        const int64_t tiles = nt * (nt + 1) / 2;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 8, tiles));
        k_ttm_mirror<<<grid, 256, sizeof(float) * (size_t)P * P * rank, s>>>(C, X->n, rank, P);
        SYM_CHECK_LAUNCH();
    }
    return SYM_OK;
}
