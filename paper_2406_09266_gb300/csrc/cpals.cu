// One symmetric CP-ALS update of the shared factor (the decomposition the
// symmetric MTTKRP serves, Sec. 5.2.6: one factor B for every mode):
//   M     = MTTKRP(X, B)                                  (symmetric kernels)
//   H     = (B^T B) raised elementwise to N-1, + ridge I   (FP64)
//   B_new = M H^{-1}
// H is R x R (R <= 128): one CTA factorises it (right-looking Cholesky, FP64,
// in shared memory); R warps spread over R/8 CTAs then solve one column of
// H^{-1} = L^{-T} L^{-1} each (FP64 is slow per SM on this part, so the
// O(R^3) inverse is not left to one CTA); the n x R product with M runs in
// FP32 with H^{-1} staged in shared memory.  A non-positive pivot is reported
// in *info (1-based column) and leaves B_new = 0.
#include <algorithm>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

__device__ __forceinline__ int tri_index(int r, int s, int R) {  // r <= s
    return r * R - r * (r - 1) / 2 + (s - r);
}

// H = G^(o(N-1)) + ridge I, factorised H = L L^T in place (right-looking
// Cholesky, FP64, one CTA of 32 x 32 threads, the whole matrix in shared
// memory).  Writes L and L^T (row-major, FP64) and the reciprocals of L's
// diagonal for the column solves, and the 1-based column of the first
// non-positive pivot to *info (0 on success).
__global__ void __launch_bounds__(1024) k_cholesky(const double* __restrict__ G, int R, int power, double ridge,
                                                   double* __restrict__ Lg, double* __restrict__ LTg,
                                                   double* __restrict__ dinv, int* __restrict__ fail_out,
                                                   int* __restrict__ info_out) {
    extern __shared__ double A[];  // R x R
    __shared__ int s_fail;
    __shared__ double s_rd;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_fail = 0;
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) {
        const int r = k / R, c = k % R;
        const double g = G[r <= c ? tri_index(r, c, R) : tri_index(c, r, R)];
        double h = 1.0;
        for (int q = 0; q < power; ++q) h *= g;
        A[k] = h + (r == c ? ridge : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * R + j];
            if (!(d > 0.0)) {
                s_fail = j + 1;
            } else {
                const double sd = sqrt(d);
                A[j * R + j] = sd;
                s_rd = 1.0 / sd;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const double rd = s_rd;
        for (int i = j + 1 + threadIdx.x; i < R; i += blockDim.x) A[i * R + j] *= rd;
        __syncthreads();
        // trailing lower triangle: A[i][k] -= A[i][j] A[k][j], j < k <= i
        for (int i = j + 1 + ty; i < R; i += 32) {
            const double aij = A[i * R + j];
            for (int k = j + 1 + tx; k <= i; k += 32) A[i * R + k] -= aij * A[k * R + j];
        }
        __syncthreads();
    }
    const int fail = s_fail;
    if (threadIdx.x == 0) {
        *fail_out = fail;
        if (info_out) *info_out = fail;
    }
    if (fail) return;
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) {
        const int r = k / R, c = k % R;
        const double v = (c <= r) ? A[k] : 0.0;
        Lg[k] = v;             // L[r][c]
        LTg[c * R + r] = v;    // L^T[c][r]
    }
    for (int i = threadIdx.x; i < R; i += blockDim.x) dinv[i] = 1.0 / A[i * R + i];
}

constexpr int INV_WARPS = 8;  // columns per CTA

// Column c of H^{-1} = L^{-T} L^{-1} e_c, one warp per column: forward solve
// L y = e_c (y_i = 0 for i < c), then back solve L^T x = y; each step is a
// dot product over the warp's lanes with a row of L (then of L^T) staged in
// shared memory.  H^{-1} is symmetric, so the column is written as row c.
// After a failed factorisation the output is 0.
__global__ void __launch_bounds__(INV_WARPS * 32) k_inverse_columns(const double* __restrict__ L,
                                                                   const double* __restrict__ LT,
                                                                   const double* __restrict__ dinv, int R,
                                                                   const int* __restrict__ fail,
                                                                   float* __restrict__ Hinv) {
    extern __shared__ double sm[];  // R x R factor, then INV_WARPS x R solution vectors
    double* F = sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * INV_WARPS + w;
    double* y = sm + (size_t)R * R + (size_t)w * R;
    const bool live = c < R;
    if (*fail) {
        if (live)
            for (int i = lane; i < R; i += 32) Hinv[(int64_t)c * R + i] = 0.f;
        return;
    }
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) F[k] = L[k];
    if (live)
        for (int i = lane; i < R; i += 32) y[i] = 0.0;
    __syncthreads();
    if (live) {
        for (int i = c; i < R; ++i) {
            double t = 0.0;
            for (int k = c + lane; k < i; k += 32) t += F[i * R + k] * y[k];
            t = warp_sum(t);
            if (lane == 0) y[i] = ((i == c ? 1.0 : 0.0) - t) * dinv[i];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) F[k] = LT[k];
    __syncthreads();
    if (live) {
        for (int i = R - 1; i >= 0; --i) {
            double t = 0.0;
            for (int k = i + 1 + lane; k < R; k += 32) t += F[i * R + k] * y[k];
            t = warp_sum(t);
            if (lane == 0) y[i] = (y[i] - t) * dinv[i];
            __syncwarp();
        }
        for (int i = lane; i < R; i += 32) Hinv[(int64_t)c * R + i] = (float)y[i];
    }
}

// B_out[i, :] = M[i, :] Hinv, four output columns per thread.
template <bool BF16>
__global__ void k_apply_inverse(const float* __restrict__ M, int64_t n, int R, const float* __restrict__ Hinv,
                                void* __restrict__ Bout, int64_t ldo) {
    extern __shared__ float hs[];  // R x R
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) hs[k] = Hinv[k];
    __syncthreads();
    const int per_row = R / 4;
    const int64_t total = n * per_row;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / per_row;
        const int c = 4 * (int)(t % per_row);
        float4 acc = f4_zero();
        const float* m = M + i * R;
        for (int k = 0; k < R; ++k) {
            const float mk = m[k];
            const float4 h = *reinterpret_cast<const float4*>(hs + k * R + c);
            acc = f4_fmas(h, mk, acc);
        }
        if (BF16) {
            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(Bout) + i * ldo + c;
            o[0] = __float2bfloat16_rn(acc.x);
            o[1] = __float2bfloat16_rn(acc.y);
            o[2] = __float2bfloat16_rn(acc.z);
            o[3] = __float2bfloat16_rn(acc.w);
        } else {
            *reinterpret_cast<float4*>(static_cast<float*>(Bout) + i * ldo + c) = acc;
        }
    }
}

struct AlsWs {
    float* M;
    double* G;
    double* L;
    double* LT;
    double* dinv;
    float* Hinv;
    int* fail;
};

template <typename C>
AlsWs layout_als(C& c, int64_t n, int R) {
    AlsWs w;
    w.M = c.template take<float>((size_t)std::max<int64_t>(n, 1) * R);
    w.G = c.template take<double>((size_t)R * (R + 1) / 2);
    w.L = c.template take<double>((size_t)R * R);
    w.LT = c.template take<double>((size_t)R * R);
    w.dinv = c.template take<double>((size_t)R);
    w.Hinv = c.template take<float>((size_t)R * R);
    w.fail = c.template take<int>(1);
    return w;
}

struct NullCarver {
    Sizer s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

}  // namespace

}  // namespace symgpu

using namespace symgpu;

extern "C" size_t sym_cp_als_workspace_bytes(sym_tensor X, int rank) {
    if (!X || rank < 4 || rank > 128) return 0;
    NullCarver c;
    layout_als(c, X->n, rank);
    return c.s.used;
}

extern "C" sym_status sym_cp_als_step(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, void* B_out,
                                      int64_t ldo, double ridge, int* info, void* ws, size_t ws_bytes,
                                      sym_stream_t stream) {
    // M lives in the workspace with row stride = rank; validate B and B_out as factors
    sym_status st = validate_mttkrp_args(X, B, bdt, rank, ldb, static_cast<float*>(ws), rank);
    if (st != SYM_OK) return st;
    if (!B_out || ldo < rank || ldo % 4 != 0 || !aligned(B_out, bdt == SYM_BF16 ? 8 : 16)) return SYM_E_INVALID;
    if (!(ridge >= 0.0)) return SYM_E_INVALID;
    if (!ws || !aligned(ws, 256)) return SYM_E_INVALID;
    if (ws_bytes < sym_cp_als_workspace_bytes(X, rank)) return SYM_E_NOMEM;
    cudaStream_t s = as_stream(stream);
    const bool bf16 = bdt == SYM_BF16;
    Carver c(ws, ws_bytes);
    AlsWs w = layout_als(c, X->n, rank);
    st = mttkrp_core(X, B, bf16, rank, ldb, w.M, rank, s);
    if (st != SYM_OK) return st;
    st = gram_launch(X->n, B, bf16, rank, ldb, w.G, s);
    if (st != SYM_OK) return st;
    const size_t lsmem = sizeof(double) * (size_t)rank * rank;
    SYM_TRY(raise_smem_limit(k_cholesky, lsmem));
    {
        SYM_PROF("cp_als_cholesky", s);
        k_cholesky<<<1, 1024, lsmem, s>>>(w.G, rank, X->order - 1, ridge, w.L, w.LT, w.dinv, w.fail, info);
        SYM_CHECK_LAUNCH();
    }
    {
        const size_t ismem = lsmem + sizeof(double) * INV_WARPS * (size_t)rank;  // <= 136 KB at rank 128
        SYM_TRY(raise_smem_limit(k_inverse_columns, ismem));
        SYM_PROF("cp_als_inverse", s);
        k_inverse_columns<<<(rank + INV_WARPS - 1) / INV_WARPS, INV_WARPS * 32, ismem, s>>>(w.L, w.LT, w.dinv, rank,
                                                                                          w.fail, w.Hinv);
        SYM_CHECK_LAUNCH();
    }
    if (X->n == 0) return SYM_OK;
    const size_t asmem = sizeof(float) * (size_t)rank * rank;
    const int64_t work = X->n * (rank / 4);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, (work + 255) / 256));
    SYM_PROF("cp_als_apply", s);
    if (bf16) {
        SYM_TRY(raise_smem_limit(k_apply_inverse<true>, asmem));
        k_apply_inverse<true><<<grid, 256, asmem, s>>>(w.M, X->n, rank, w.Hinv, B_out, ldo);
    } else {
        SYM_TRY(raise_smem_limit(k_apply_inverse<false>, asmem));
        k_apply_inverse<false><<<grid, 256, asmem, s>>>(w.M, X->n, rank, w.Hinv, B_out, ldo);
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}
