// One symmetric CP-ALS update of the shared factor (the decomposition the
// symmetric MTTKRP serves, Sec. 5.2.6: one factor B for every mode):
//   M     = MTTKRP(X, B)                                  (symmetric kernels)
//   H     = (B^T B) raised elementwise to N-1, + ridge I   (FP64)
//   B_new = M H^{-1}
// H is R x R (R <= 128): one CTA factorises it (Cholesky, FP64), inverts the
// triangular factor and forms H^{-1} = L^{-T} L^{-1}; the n x R product with
// M runs in FP32 with H^{-1} staged in shared memory.  A non-positive pivot is
// reported in *info (1-based column) and leaves B_new = 0.
#include <algorithm>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

__device__ __forceinline__ int tri_index(int r, int s, int R) {  // r <= s
    return r * R - r * (r - 1) / 2 + (s - r);
}

// H = G^(o(N-1)) + ridge I; L = chol(H); Linv = L^{-1}; Hinv = Linv^T Linv.
__global__ void k_chol_inverse(const double* __restrict__ G, int R, int power, double ridge,
                               double* __restrict__ Linv, float* __restrict__ Hinv, int* __restrict__ info_out) {
    extern __shared__ double L[];  // R x R, lower triangle used
    __shared__ int s_fail;
    __shared__ double s_d;
    if (threadIdx.x == 0) s_fail = 0;
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) {
        const int r = k / R, c = k % R;
        const double g = G[r <= c ? tri_index(r, c, R) : tri_index(c, r, R)];
        double h = 1.0;
        for (int q = 0; q < power; ++q) h *= g;
        L[k] = h + (r == c ? ridge : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < R; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j * R + j];
            for (int k = 0; k < j; ++k) d -= L[j * R + k] * L[j * R + k];
            if (!(d > 0.0)) {
                s_fail = j + 1;
            } else {
                s_d = sqrt(d);
                L[j * R + j] = s_d;
            }
        }
        __syncthreads();
        if (s_fail) break;
        for (int i = j + 1 + threadIdx.x; i < R; i += blockDim.x) {
            double t = L[i * R + j];
            for (int k = 0; k < j; ++k) t -= L[i * R + k] * L[j * R + k];
            L[i * R + j] = t / s_d;
        }
        __syncthreads();
    }
    const int fail = s_fail;
    if (threadIdx.x == 0 && info_out) *info_out = fail;
    if (fail) {
        for (int k = threadIdx.x; k < R * R; k += blockDim.x) Hinv[k] = 0.f;
        return;
    }
    // column c of L^{-1} by forward substitution (one thread per column)
    for (int c = threadIdx.x; c < R; c += blockDim.x) {
        for (int i = 0; i < R; ++i) {
            if (i < c) {
                Linv[i * R + c] = 0.0;
                continue;
            }
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) t -= L[i * R + k] * Linv[k * R + c];
            Linv[i * R + c] = t / L[i * R + i];
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) {
        const int r = k / R, c = k % R;
        double t = 0.0;
        for (int q = max(r, c); q < R; ++q) t += Linv[q * R + r] * Linv[q * R + c];
        Hinv[k] = (float)t;
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
    double* Linv;
    float* Hinv;
};

template <typename C>
AlsWs layout_als(C& c, int64_t n, int R) {
    AlsWs w;
    w.M = c.template take<float>((size_t)std::max<int64_t>(n, 1) * R);
    w.G = c.template take<double>((size_t)R * (R + 1) / 2);
    w.Linv = c.template take<double>((size_t)R * R);
    w.Hinv = c.template take<float>((size_t)R * R);
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
    SYM_CUDA(cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    {
        SYM_PROF("cp_als_factorise", s);
        k_chol_inverse<<<1, 128, lsmem, s>>>(w.G, rank, X->order - 1, ridge, w.Linv, w.Hinv, info);
        SYM_CHECK_LAUNCH();
    }
    if (X->n == 0) return SYM_OK;
    const size_t asmem = sizeof(float) * (size_t)rank * rank;
    const int64_t work = X->n * (rank / 4);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 4, (work + 255) / 256));
    SYM_PROF("cp_als_apply", s);
    if (bf16) {
        SYM_CUDA(cudaFuncSetAttribute(k_apply_inverse<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asmem));
        k_apply_inverse<true><<<grid, 256, asmem, s>>>(w.M, X->n, rank, w.Hinv, B_out, ldo);
    } else {
        SYM_CUDA(cudaFuncSetAttribute(k_apply_inverse<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asmem));
        k_apply_inverse<false><<<grid, 256, asmem, s>>>(w.M, X->n, rank, w.Hinv, B_out, ldo);
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}
