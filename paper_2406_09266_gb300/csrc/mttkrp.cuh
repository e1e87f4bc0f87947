// Symmetric MTTKRP kernels (Sec. 4.3 "MTTKRP Demonstration", Sec. 5.2.6):
//   M[i, r] = sum over the full tensor X[i, k, l, ..] B[k, r] B[l, r] ...
// read from the canonical triangle only.
//
// STRICT stream (all indices distinct, Sec. 4.2.9 diagonal splitting): each
// entry c_1 < ... < c_N with value v stands for N! full-tensor entries, and
// the N!/N = (N-1)! of them that start with c_p all add the same term
// v * prod_{q != p} B[c_q] to row c_p (distributive assignment grouping,
// Sec. 4.2.7: the factor 2 of the 3-way split loop nest).  The kernel walks the
// sorted entries as a CSF tree (Sec. 2.2) and factorises the sums level by
// level (workspace transformation, Sec. 4.2.8, applied at every level):
//   P_q  = B[c_1] * ... * B[c_q]                    (prefix products, cached)
//   T_q  = sum over the subtree below (c_1..c_q) of v * prod_{t > q} B[c_t]
//   row c_q receives (N-1)! * P_{q-1} * T_q once per fiber (not per entry),
//   the leaf row c_N receives (N-1)! * v * P_{N-1} per entry.
// So an entry costs one factor-row gather, one FMA row and one vector
// reduction; the upper levels cost per fiber.
//
// DIAGONAL stream (some index repeated): per entry with runs u_t of
// multiplicity m_t, row u_t receives the integer weight
// W_t = (N-1)! m_t / prod_s m_s! times v * prod over all positions but one
// occurrence of u_t of B[c_q] (the per-run form of the simplicial lookup
// table of Sec. 4.2.5 — integer weights instead of the table's per-position
// fractions such as 1/3).
//
// Thread mapping: a group of L lanes owns one entry at a time, each lane 4
// consecutive columns of the rank (float4 / 4 x bf16 gathers, 16-byte vector
// reductions).  A warp loads 32 consecutive entries with coalesced 64-bit key
// and 32-bit value loads; group g processes the L entries held by its own
// lanes, so each group walks a strided but ordered subsequence of the warp's
// contiguous chunk and keeps its fiber state in registers across batches.
#pragma once

#include <algorithm>

#include "common.cuh"
#include "tensor.cuh"

namespace symgpu {

constexpr int MT_THREADS = 256;

template <int N, int KW>
__device__ __forceinline__ void decode_entry(uint64_t lo, uint64_t hi, int bits, int32_t* c) {
    unpack_key<N, KW>(KeyWords{lo, hi}, bits, c);
}

template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(MT_THREADS) k_mttkrp_strict(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk) {
    static_assert(N >= 2 && N <= 5, "order");
    constexpr int LV = N - 1;  // fiber levels above the leaf
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t warp = ((int64_t)blockIdx.x * MT_THREADS + threadIdx.x) >> 5;
    const int64_t start = warp * chunk;
    if (start >= nnz) return;
    const int64_t end = min(start + chunk, nnz);

    int32_t cur[LV];
    float4 Brow[LV], P[LV], T[LV];
#pragma unroll
    for (int q = 0; q < LV; ++q) {
        cur[q] = -1;
        Brow[q] = f4_zero();
        P[q] = f4_zero();
        T[q] = f4_zero();
    }
    bool have = false;

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
            if (b0 + src >= end) continue;
            int32_t c[N];
            decode_entry<N, KW>(lo, hi, bits, c);
            // first fiber level whose coordinate changed (LV: same prefix)
            int d = LV;
#pragma unroll
            for (int q = LV - 1; q >= 0; --q)
                if (!have || c[q] != cur[q]) d = q;
            if (d < LV) {
                if (have) {
#pragma unroll
                    for (int q = LV - 1; q >= 0; --q) {
                        if (q >= d) {
                            float4 out = (q > 0) ? f4_mul(P[q - 1], T[q]) : T[q];
                            if (on) red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
                            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
                            T[q] = f4_zero();
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < LV; ++q) {
                    if (q >= d) {
                        cur[q] = c[q];
                        Brow[q] = on ? load_row4<BF16>(B, c[q], ldb, col) : f4_zero();
                        P[q] = (q > 0) ? f4_mul(P[q - 1], Brow[q]) : Brow[q];
                    }
                }
                have = true;
            }
            const float4 bl = on ? load_row4<BF16>(B, c[N - 1], ldb, col) : f4_zero();
            T[LV - 1] = f4_fmas(bl, v, T[LV - 1]);
            if (on) red_add_f4(M + (int64_t)c[N - 1] * ldm + col, f4_scale(P[LV - 1], w * v));
        }
    }
    if (have) {
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
            float4 out = (q > 0) ? f4_mul(P[q - 1], T[q]) : T[q];
            if (on) red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
        }
    }
}

// One entry per lane group, any equality pattern (used for the diagonal
// stream; with all-distinct entries it is the unfactorised per-entry form).
template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(MT_THREADS) k_mttkrp_entries(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t cnt,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm) {
    constexpr int GPW = 32 / L;
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t group = (((int64_t)blockIdx.x * MT_THREADS + threadIdx.x) >> 5) * GPW + lane / L;
    const int64_t ngroups = ((int64_t)gridDim.x * MT_THREADS >> 5) * GPW;
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    for (int64_t e = group; e < cnt; e += ngroups) {
        int32_t c[N];
        decode_entry<N, KW>(klo[e], KW == 2 ? khi[e] : 0ull, bits, c);
        const float v = val[e];
        if (!on) continue;
        float4 b[N];
#pragma unroll
        for (int q = 0; q < N; ++q) b[q] = load_row4<BF16>(B, c[q], ldb, col);
        // prefix / suffix products over positions
        float4 pre[N + 1], suf[N + 1];
        pre[0] = make_float4(1.f, 1.f, 1.f, 1.f);
        suf[N] = pre[0];
#pragma unroll
        for (int q = 0; q < N; ++q) pre[q + 1] = f4_mul(pre[q], b[q]);
#pragma unroll
        for (int q = N - 1; q >= 0; --q) suf[q] = f4_mul(suf[q + 1], b[q]);
        // run multiplicities
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
#pragma unroll
        for (int p = 0; p < N; ++p) {
            if (p > 0 && c[p] == c[p - 1]) continue;  // not the first position of its run
            int m = 1;
#pragma unroll
            for (int q = p + 1; q < N; ++q)
                if (c[q] == c[p]) ++m;
            const float W = (float)(fact[N - 1] * m / den);
            red_add_f4(M + (int64_t)c[p] * ldm + col, f4_scale(f4_mul(pre[p], suf[p + 1]), W * v));
        }
    }
}

// Per-order launchers (one translation unit per order instantiates its kernels).
template <int N, int KW, int L, bool BF16>
sym_status launch_mttkrp_shape(const sym_tensor_s* X, const void* B, int R, int64_t ldb, float* M, int64_t ldm,
                               int chunk, bool factorised, cudaStream_t s) {
    const int64_t ns = X->nnz_strict, nd = X->nnz - X->nnz_strict;
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    const int64_t groups_per_cta = (MT_THREADS / 32) * (32 / L);
    const int64_t max_ctas = (int64_t)sm_count() * 16;
    if (ns > 0) {
        if (factorised) {
            const int64_t warps = (ns + chunk - 1) / chunk;
            const unsigned grid = (unsigned)((warps * 32 + MT_THREADS - 1) / MT_THREADS);
            SYM_PROF("mttkrp_strict", s);
            k_mttkrp_strict<N, KW, L, BF16><<<grid, MT_THREADS, 0, s>>>(X->klo, X->khi, X->val, ns, X->bits, B, ldb,
                                                                        R, M, ldm, (float)fact[N - 1], chunk);
        } else {
            const unsigned grid = (unsigned)std::min<int64_t>((ns + groups_per_cta - 1) / groups_per_cta, max_ctas);
            SYM_PROF("mttkrp_strict_entries", s);
            k_mttkrp_entries<N, KW, L, BF16><<<grid, MT_THREADS, 0, s>>>(X->klo, X->khi, X->val, ns, X->bits, B, ldb,
                                                                         R, M, ldm);
        }
        SYM_CHECK_LAUNCH();
    }
    if (nd > 0) {
        const unsigned grid = (unsigned)std::min<int64_t>((nd + groups_per_cta - 1) / groups_per_cta, max_ctas);
        SYM_PROF("mttkrp_diag", s);
        k_mttkrp_entries<N, KW, L, BF16><<<grid, MT_THREADS, 0, s>>>(
            X->klo + ns, X->khi ? X->khi + ns : nullptr, X->val + ns, nd, X->bits, B, ldb, R, M, ldm);
        SYM_CHECK_LAUNCH();
    }
    return SYM_OK;
}

inline int lanes_for_rank(int R) {
    int L = 1;
    while (4 * L < R) L <<= 1;
    return L;
}

template <int N, int KW, bool BF16>
sym_status launch_mttkrp_kw(const sym_tensor_s* X, const void* B, int R, int64_t ldb, float* M, int64_t ldm,
                            int chunk, bool factorised, cudaStream_t s) {
    switch (lanes_for_rank(R)) {
        case 1: return launch_mttkrp_shape<N, KW, 1, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        case 2: return launch_mttkrp_shape<N, KW, 2, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        case 4: return launch_mttkrp_shape<N, KW, 4, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        case 8: return launch_mttkrp_shape<N, KW, 8, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        case 16: return launch_mttkrp_shape<N, KW, 16, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        case 32: return launch_mttkrp_shape<N, KW, 32, BF16>(X, B, R, ldb, M, ldm, chunk, factorised, s);
        default: return SYM_E_UNSUPPORTED;
    }
}

template <int N>
sym_status launch_mttkrp_impl(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                              int64_t ldm, int chunk, bool factorised, cudaStream_t s) {
    if (X->kw == 1)
        return bf16 ? launch_mttkrp_kw<N, 1, true>(X, B, R, ldb, M, ldm, chunk, factorised, s)
                    : launch_mttkrp_kw<N, 1, false>(X, B, R, ldb, M, ldm, chunk, factorised, s);
    return bf16 ? launch_mttkrp_kw<N, 2, true>(X, B, R, ldb, M, ldm, chunk, factorised, s)
                : launch_mttkrp_kw<N, 2, false>(X, B, R, ldb, M, ldm, chunk, factorised, s);
}

template <int N>
sym_status launch_mttkrp_order(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                               int64_t ldm, int chunk, bool factorised, cudaStream_t s);

}  // namespace symgpu

namespace symgpu {
// Entry points shared with the serving runtime (defined in mttkrp.cu).
sym_status mttkrp_core(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M, int64_t ldm,
                       int chunk, bool factorised, cudaStream_t s);
sym_status residual_launch(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, const float* M,
                           int64_t ldm, double* residual, void* ws, size_t ws_bytes, cudaStream_t s);
size_t residual_ws_bytes(int R);
sym_status validate_mttkrp_args(const sym_tensor_s* X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                const float* M, int64_t ldm);
int default_chunk(const sym_tensor_s* X);
}  // namespace symgpu
