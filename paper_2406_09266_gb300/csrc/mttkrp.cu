// sym_mttkrp: the C entry point of the symmetric MTTKRP, and the FP64 CP-fit
// residual that rides along with it.
//
// CP-fit residual (the symmetric CPD that MTTKRP serves, Sec. 5.2.6): with unit
// weights, Mcp = sum_r b_r (x) ... (x) b_r and
//   ||X - Mcp||^2 = ||X||^2 - 2 <X, Mcp> + ||Mcp||^2,
//   <X, Mcp>      = sum_{i,r} B[i,r] * M[i,r]        (M = the MTTKRP output),
//   ||Mcp||^2     = sum_{r,s} G[r,s]^N,  G = B^T B.
// The three terms nearly cancel when the fit is good, so they are formed in
// FP64: Gram products are split exactly into two floats (p = a*b rounded,
// e = fma(a, b, -p)), accumulated as a double-float pair over a 32-row tile,
// then summed across tiles in FP64; <B, M> widens both factors to FP64 (the
// product of two floats is exact in FP64).  ||X||^2 was summed in FP64 when the
// tensor was created.
#include <algorithm>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

constexpr int GRAM_ROWS = 32;
constexpr int GRAM_PPT = 16;  // (r, s) pairs per thread

template <bool BF16>
__device__ __forceinline__ float load_b(const void* B, int64_t i, int64_t ldb, int r) {
    if constexpr (BF16) {
        const unsigned short* b = static_cast<const unsigned short*>(B);
        return __uint_as_float(((unsigned)b[i * ldb + r]) << 16);
    } else {
        return static_cast<const float*>(B)[i * ldb + r];
    }
}

// G[r,s] += sum_i B[i,r] B[i,s] over this CTA's rows.
template <bool BF16>
__global__ void k_gram(const void* __restrict__ B, int64_t n, int64_t ldb, int R, double* __restrict__ G,
                       int64_t rows_per_cta) {
    extern __shared__ float tile[];  // GRAM_ROWS x R
    const int pairs = R * R;
    double acc[GRAM_PPT];
#pragma unroll
    for (int k = 0; k < GRAM_PPT; ++k) acc[k] = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int64_t t0 = r0; t0 < r1; t0 += GRAM_ROWS) {
        const int rows = (int)((r1 - t0) < GRAM_ROWS ? (r1 - t0) : GRAM_ROWS);
        __syncthreads();
        for (int k = threadIdx.x; k < GRAM_ROWS * R; k += blockDim.x) {
            int i = k / R, r = k % R;
            tile[k] = (i < rows) ? load_b<BF16>(B, t0 + i, ldb, r) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GRAM_PPT; ++k) {
            const int pr = threadIdx.x + k * blockDim.x;
            if (pr >= pairs) break;
            const int r = pr / R, s = pr % R;
            float hi = 0.f, lo = 0.f;
            for (int i = 0; i < rows; ++i) {
                const float a = tile[i * R + r], b = tile[i * R + s];
                const float p = a * b;
                const float e = fmaf(a, b, -p);  // a*b == p + e exactly
                const float t = hi + p;           // two-sum of hi and p
                const float bp = t - hi;
                const float err = (hi - (t - bp)) + (p - bp);
                hi = t;
                lo += err + e;
            }
            acc[k] += (double)hi + (double)lo;
        }
    }
#pragma unroll
    for (int k = 0; k < GRAM_PPT; ++k) {
        const int pr = threadIdx.x + k * blockDim.x;
        if (pr < pairs) atomicAdd(&G[pr], acc[k]);
    }
}

// xm += sum_{i,r} B[i,r] M[i,r] in FP64 (exact products).
template <bool BF16>
__global__ void k_dot_bm(const void* __restrict__ B, int64_t ldb, const float* __restrict__ M, int64_t ldm,
                         int64_t n, int R, double* __restrict__ out) {
    double acc = 0.0;
    const int64_t total = n * R;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / R;
        const int r = (int)(k % R);
        acc += (double)load_b<BF16>(B, i, ldb, r) * (double)M[i * ldm + r];
    }
    acc = warp_sum(acc);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(out, t);
    }
}

__global__ void k_residual_final(const double* __restrict__ G, int R, int order, const double* __restrict__ xm,
                                 double normsq, double* __restrict__ residual) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < R * R; k += blockDim.x) {
        double g = G[k], p = 1.0;
        for (int q = 0; q < order; ++q) p *= g;
        acc += p;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm += sh[w];
        *residual = normsq - 2.0 * (*xm) + mm;
    }
}

struct ResidualWs {
    double* G;
    double* xm;
};

template <typename C>
ResidualWs layout_residual(C& c, int R) {
    ResidualWs w;
    w.G = c.template take<double>((size_t)R * R);
    w.xm = c.template take<double>(1);
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

sym_status residual_launch(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, const float* M,
                           int64_t ldm, double* residual, void* ws, size_t ws_bytes, cudaStream_t s) {
    Carver c(ws, ws_bytes);
    ResidualWs w = layout_residual(c, R);
    if (!w.G || !w.xm) return SYM_E_NOMEM;
    SYM_CUDA(cudaMemsetAsync(ws, 0, c.used, s));
    const int sms = sm_count();
    const int threads = std::max(128, std::min(1024, ((R * R + GRAM_PPT - 1) / GRAM_PPT + 31) / 32 * 32));
    const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>(2 * sms, (X->n + GRAM_ROWS - 1) / GRAM_ROWS));
    int64_t rows_per_cta = (X->n + ctas - 1) / ctas;
    rows_per_cta = (rows_per_cta + GRAM_ROWS - 1) / GRAM_ROWS * GRAM_ROWS;
    const unsigned grid = (unsigned)((X->n + rows_per_cta - 1) / rows_per_cta);
    const size_t smem = sizeof(float) * GRAM_ROWS * R;
    {
        SYM_PROF("cpfit_gram", s);
        if (bf16)
            k_gram<true><<<grid, threads, smem, s>>>(B, X->n, ldb, R, w.G, rows_per_cta);
        else
            k_gram<false><<<grid, threads, smem, s>>>(B, X->n, ldb, R, w.G, rows_per_cta);
        SYM_CHECK_LAUNCH();
    }
    const unsigned g2 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * sms, (X->n * R + 255) / 256));
    {
        SYM_PROF("cpfit_dot", s);
        if (bf16)
            k_dot_bm<true><<<g2, 256, 0, s>>>(B, ldb, M, ldm, X->n, R, w.xm);
        else
            k_dot_bm<false><<<g2, 256, 0, s>>>(B, ldb, M, ldm, X->n, R, w.xm);
        SYM_CHECK_LAUNCH();
    }
    k_residual_final<<<1, 256, 0, s>>>(w.G, R, X->order, w.xm, X->info.normsq, residual);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

size_t residual_ws_bytes(int R) {
    NullCarver c;
    layout_residual(c, R);
    return c.s.used;
}

sym_status validate_mttkrp_args(const sym_tensor_s* X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                const float* M, int64_t ldm) {
    if (!X || !B || !M) return SYM_E_INVALID;
    if (bdt != SYM_F32 && bdt != SYM_BF16) return SYM_E_INVALID;
    if (rank < 4 || rank > 128 || rank % 4 != 0) return SYM_E_INVALID;
    if (ldb < rank || ldm < rank || ldb % 4 != 0 || ldm % 4 != 0) return SYM_E_INVALID;
    if (!aligned(B, bdt == SYM_BF16 ? 8 : 16) || !aligned(M, 16)) return SYM_E_INVALID;
    return SYM_OK;
}

sym_status mttkrp_core(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M, int64_t ldm,
                       int chunk, bool factorised, cudaStream_t s) {
    if (ldm == R)
        SYM_CUDA(cudaMemsetAsync(M, 0, sizeof(float) * (size_t)X->n * R, s));
    else
        SYM_CUDA(cudaMemset2DAsync(M, sizeof(float) * ldm, 0, sizeof(float) * R, X->n, s));
    if (X->nnz == 0) return SYM_OK;
    switch (X->order) {
        case 2: return launch_mttkrp_order<2>(X, B, bf16, R, ldb, M, ldm, chunk, factorised, s);
        case 3: return launch_mttkrp_order<3>(X, B, bf16, R, ldb, M, ldm, chunk, factorised, s);
        case 4: return launch_mttkrp_order<4>(X, B, bf16, R, ldb, M, ldm, chunk, factorised, s);
        case 5: return launch_mttkrp_order<5>(X, B, bf16, R, ldb, M, ldm, chunk, factorised, s);
        default: return SYM_E_UNSUPPORTED;
    }
}

int default_chunk(const sym_tensor_s* X) {
    if (X->chunk > 0) return X->chunk;
    return 256;
}

}  // namespace symgpu

using namespace symgpu;

extern "C" size_t sym_mttkrp_workspace_bytes(sym_tensor X, int rank, sym_dtype bdt, int want_residual) {
    (void)X;
    (void)bdt;
    if (!want_residual || rank <= 0) return 0;
    return residual_ws_bytes(rank);
}

extern "C" sym_status sym_mttkrp(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                                 int64_t ldm, double* residual, void* ws, size_t ws_bytes, sym_stream_t stream) {
    sym_status st = validate_mttkrp_args(X, B, bdt, rank, ldb, M, ldm);
    if (st != SYM_OK) return st;
    if (residual) {
        if (!ws || !aligned(ws, 256)) return SYM_E_INVALID;
        if (ws_bytes < residual_ws_bytes(rank)) return SYM_E_NOMEM;
    }
    cudaStream_t s = as_stream(stream);
    const bool bf16 = bdt == SYM_BF16;
    const int chunk = default_chunk(X);
    st = mttkrp_core(X, B, bf16, rank, ldb, M, ldm, chunk > 0 ? chunk : 256, X->chunk >= 0, s);
    if (st != SYM_OK) return st;
    if (residual) return residual_launch(X, B, bf16, rank, ldb, M, ldm, residual, ws, ws_bytes, s);
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_set_chunk(sym_tensor X, int entries_per_warp) {
    if (!X) return SYM_E_INVALID;
    // > 0: entries per warp (multiple of 32); 0: default; -1: unfactorised per-entry kernel
    if (entries_per_warp > 0 && entries_per_warp % 32 != 0) return SYM_E_INVALID;
    if (entries_per_warp < -1) return SYM_E_INVALID;
    X->chunk = entries_per_warp;
    return SYM_OK;
}
