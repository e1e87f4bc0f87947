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
#include <cstdio>
#include <string>
#include <vector>

#include "common.cuh"
#include "mttkrp.cuh"
#include "tensor.cuh"

namespace symgpu {

namespace {

constexpr int GRAM_ROWS = 32;
constexpr int GRAM_THREADS = 544;          // >= 528 blocks of 4 x 4 pairs in the upper block triangle of R = 128
constexpr int GRAM_ROWS_PER_CTA = 128;     // rows of B per CTA (4 tiles)
static_assert(GRAM_THREADS >= 32 * 33 / 2, "one CTA must cover every block of the largest rank");

template <bool BF16>
__device__ __forceinline__ float load_b(const void* B, int64_t i, int64_t ldb, int r) {
    if constexpr (BF16) {
        const unsigned short* b = static_cast<const unsigned short*>(B);
        return __uint_as_float(((unsigned)b[i * ldb + r]) << 16);
    } else {
        return static_cast<const float*>(B)[i * ldb + r];
    }
}

// Triangular index p = r*R - r*(r-1)/2 + (s - r) of the pair (r, s), r <= s.
__device__ __forceinline__ void tri_pair(int p, int R, int* r_out, int* s_out) {
    const double t = 2.0 * R + 1.0;
    int r = (int)((t - sqrt(t * t - 8.0 * p)) * 0.5);
    if (r < 0) r = 0;
    if (r > R - 1) r = R - 1;
    auto start = [R](int q) { return q * R - q * (q - 1) / 2; };
    while (r > 0 && start(r) > p) --r;
    while (r + 1 < R && start(r + 1) <= p) ++r;
    *r_out = r;
    *s_out = r + (p - start(r));
}

// G[r,s] += sum_i B[i,r] B[i,s] over this CTA's rows, for r <= s only (G is
// symmetric); G is stored as the packed upper triangle.  Thread t owns one
// 4 x 4 block (r in [4 bi, 4 bi + 4), s in [4 bj, 4 bj + 4)) of the upper block
// triangle bi <= bj, so each staged row costs it two 16-byte shared loads for
// 16 products.  Per 32-row tile every product is split exactly into two floats
// and accumulated as a double-float pair; the tile sums are added in FP64.
template <bool BF16>
__global__ void __launch_bounds__(GRAM_THREADS) k_gram(const void* __restrict__ B, int64_t n, int64_t ldb, int R,
                                                       double* __restrict__ G, int64_t rows_per_cta) {
    extern __shared__ float tile[];  // GRAM_ROWS x R
    const int RB = R / 4;
    const int nblk = RB * (RB + 1) / 2;
    int bi = 0, bj = 0;
    const bool active = (int)threadIdx.x < nblk;
    if (active) tri_pair((int)threadIdx.x, RB, &bi, &bj);
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = min(n, r0 + rows_per_cta);
    for (int64_t t0 = r0; t0 < r1; t0 += GRAM_ROWS) {
        const int rows = (int)((r1 - t0) < GRAM_ROWS ? (r1 - t0) : GRAM_ROWS);
        __syncthreads();
        for (int k = threadIdx.x; k < GRAM_ROWS * R; k += blockDim.x) {
            const int i = k / R, r = k % R;
            tile[k] = (i < rows) ? load_b<BF16>(B, t0 + i, ldb, r) : 0.f;
        }
        __syncthreads();
        if (!active) continue;
        float hi[16], lo[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) hi[k] = lo[k] = 0.f;
        for (int i = 0; i < rows; ++i) {
            const float4 a4 = *reinterpret_cast<const float4*>(tile + i * R + 4 * bi);
            const float4 b4 = *reinterpret_cast<const float4*>(tile + i * R + 4 * bj);
            const float a[4] = {a4.x, a4.y, a4.z, a4.w}, b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int k = 4 * u + v;
                    const float p = a[u] * b[v];
                    const float e = fmaf(a[u], b[v], -p);  // a*b == p + e exactly
                    const float t = hi[k] + p;             // two-sum of hi and p
                    const float bp = t - hi[k];
                    const float err = (hi[k] - (t - bp)) + (p - bp);
                    hi[k] = t;
                    lo[k] += err + e;
                }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[k] += (double)hi[k] + (double)lo[k];
    }
    if (!active) return;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = 4 * bi + u, sidx = 4 * bj + v;
            if (r > sidx) continue;  // lower half of a diagonal block
            atomicAdd(&G[r * R - r * (r - 1) / 2 + (sidx - r)], acc[4 * u + v]);
        }
}

// CTA size of k_gram: one thread per 4 x 4 block of the upper block triangle.
int gram_threads(int R) {
    const int RB = R / 4;
    return std::max(32, (RB * (RB + 1) / 2 + 31) / 32 * 32);
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
    const int pairs = R * (R + 1) / 2;
    for (int k = threadIdx.x; k < pairs; k += blockDim.x) {
        int r, s;
        tri_pair(k, R, &r, &s);
        double g = G[k], p = 1.0;
        for (int q = 0; q < order; ++q) p *= g;
        acc += (r == s) ? p : 2.0 * p;  // off-diagonal pairs stand for (r,s) and (s,r)
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
    w.G = c.template take<double>((size_t)R * (R + 1) / 2);
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
    return residual_launch_gram(X, B, bf16, R, ldb, M, ldm, residual, ws, ws_bytes, nullptr, nullptr, s);
}

sym_status residual_launch_gram(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, const float* M,
                                int64_t ldm, double* residual, void* ws, size_t ws_bytes, const double* G_in,
                                double* G_out, cudaStream_t s) {
    Carver c(ws, ws_bytes);
    ResidualWs w = layout_residual(c, R);
    if (!w.G || !w.xm) return SYM_E_NOMEM;
    SYM_CUDA(cudaMemsetAsync(ws, 0, c.used, s));
    const int sms = sm_count();
    const int threads = gram_threads(R);
    const int64_t rows_per_cta = GRAM_ROWS_PER_CTA;
    const unsigned grid = (unsigned)std::max<int64_t>(1, (X->n + rows_per_cta - 1) / rows_per_cta);
    const size_t smem = sizeof(float) * GRAM_ROWS * R;
    const double* G = G_in;
    if (!G) {  // G = B^T B, into the caller's buffer or the workspace
        double* Gw = G_out ? G_out : w.G;
        if (G_out) SYM_CUDA(cudaMemsetAsync(G_out, 0, sizeof(double) * (size_t)R * (R + 1) / 2, s));
        SYM_PROF("cpfit_gram", s);
        if (bf16)
            k_gram<true><<<grid, threads, smem, s>>>(B, X->n, ldb, R, Gw, rows_per_cta);
        else
            k_gram<false><<<grid, threads, smem, s>>>(B, X->n, ldb, R, Gw, rows_per_cta);
        SYM_CHECK_LAUNCH();
        G = Gw;
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
    k_residual_final<<<1, 256, 0, s>>>(G, R, X->order, w.xm, X->info.normsq, residual);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

// G (packed upper triangle, FP64) = B^T B, exact products and FP64 sums.
sym_status gram_launch(int64_t n, const void* B, bool bf16, int R, int64_t ldb, double* G, cudaStream_t s) {
    SYM_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * (size_t)R * (R + 1) / 2, s));
    if (n == 0) return SYM_OK;
    const int threads = gram_threads(R);
    const int64_t rows_per_cta = GRAM_ROWS_PER_CTA;
    const unsigned grid = (unsigned)std::max<int64_t>(1, (n + rows_per_cta - 1) / rows_per_cta);
    const size_t smem = sizeof(float) * GRAM_ROWS * R;
    SYM_PROF("gram", s);
    if (bf16)
        k_gram<true><<<grid, threads, smem, s>>>(B, n, ldb, R, G, rows_per_cta);
    else
        k_gram<false><<<grid, threads, smem, s>>>(B, n, ldb, R, G, rows_per_cta);
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

thread_local const SideLaunch* t_side_launch = nullptr;

const SideLaunch* side_launch_for_device(int device) {
    struct PerThread {
        SideLaunch sl[16] = {};
        bool tried[16] = {};
        ~PerThread() {
            for (auto& x : sl) {
                if (x.fork) cudaEventDestroy(x.fork);
                if (x.join) cudaEventDestroy(x.join);
                if (x.stream) cudaStreamDestroy(x.stream);
            }
        }
    };
    thread_local PerThread pt;
    if (device < 0 || device >= 16) return nullptr;
    SideLaunch& x = pt.sl[device];
    if (!pt.tried[device]) {
        pt.tried[device] = true;
        if (cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;  // (left partly created; no overlap on this device for this thread)
        }
    }
    return (x.stream && x.fork && x.join) ? &x : nullptr;
}

namespace {
// Sets the calling thread's side launch for the duration of one public call.
struct SideScope {
    const SideLaunch* prev;
    explicit SideScope(bool on) : prev(t_side_launch) {
        t_side_launch = on ? side_launch_for_device(current_device()) : nullptr;
    }
    ~SideScope() { t_side_launch = prev; }
};
}  // namespace

sym_status mttkrp_core_cfg(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                           int64_t ldm, const sym_mttkrp_cfg& cfg, cudaStream_t s) {
    if (ldm == R)
        SYM_CUDA(cudaMemsetAsync(M, 0, sizeof(float) * (size_t)X->n * R, s));
    else
        SYM_CUDA(cudaMemset2DAsync(M, sizeof(float) * ldm, 0, sizeof(float) * R, X->n, s));
    if (X->nnz == 0) return SYM_OK;
    switch (X->order) {
        case 2: return launch_mttkrp_order<2>(X, B, bf16, R, ldb, M, ldm, cfg, s);
        case 3: return launch_mttkrp_order<3>(X, B, bf16, R, ldb, M, ldm, cfg, s);
        case 4: return launch_mttkrp_order<4>(X, B, bf16, R, ldb, M, ldm, cfg, s);
        case 5: return launch_mttkrp_order<5>(X, B, bf16, R, ldb, M, ldm, cfg, s);
        default: return SYM_E_UNSUPPORTED;
    }
}

sym_status mttkrp_core(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M, int64_t ldm,
                       cudaStream_t s) {
    return mttkrp_core_cfg(X, B, bf16, R, ldb, M, ldm, X->cfg, s);
}

// The tensor restricted to canonical entries [first, first + count): the
// strict stream precedes the diagonal stream in the same arrays, so the part is
// one contiguous slice whose first max(0, min(nnz_strict, first + count) - first)
// entries are strict.  The leaf index describes the whole strict stream and is
// dropped.
sym_tensor_s tensor_part(const sym_tensor_s* X, int64_t first, int64_t count) {
    sym_tensor_s P = *X;
    P.klo = X->klo + first;
    P.khi = X->khi ? X->khi + first : nullptr;
    P.val = X->val + first;
    P.nnz = count;
    P.nnz_strict = std::max<int64_t>(0, std::min<int64_t>(X->nnz_strict, first + count) - first);
    P.rklo = nullptr;
    P.rkhi = nullptr;
    P.rval = nullptr;
    return P;
}

sym_status validate_mttkrp_cfg(const sym_mttkrp_cfg* c) {
    if (!c) return SYM_E_INVALID;
    if (c->strict_kernel < 0 || c->strict_kernel > 4) return SYM_E_INVALID;
    if (c->entries_per_warp < 0 || c->entries_per_warp % 32 != 0 || c->entries_per_warp > (1 << 24))
        return SYM_E_INVALID;
    if (c->entries_per_warp == 0 && c->strict_kernel != SYM_MTTKRP_PIPELINED) return SYM_E_INVALID;
    if (c->threads_per_cta < 64 || c->threads_per_cta > 512 || c->threads_per_cta % 32) return SYM_E_INVALID;
    if (c->ctas_per_sm < 1 || c->ctas_per_sm > 8) return SYM_E_INVALID;
    if (c->strict_smem_kb < 0 || c->strict_smem_kb > 220 || c->diag_smem_kb < 0 || c->diag_smem_kb > 220)
        return SYM_E_INVALID;
    if (c->b_share_pct < 0 || c->b_share_pct > 100) return SYM_E_INVALID;
    if (c->leaf_index != 0 && c->leaf_index != 1) return SYM_E_INVALID;
    const bool depth_field = c->strict_kernel == SYM_MTTKRP_LANE;
    if (depth_field ? (c->vec_per_lane != 1 && c->vec_per_lane != 2 && c->vec_per_lane != 4)
                    : (c->vec_per_lane != 1 && c->vec_per_lane != 2))
        return SYM_E_INVALID;
    if ((c->stream_hint != 0 && c->stream_hint != 1) || (c->l1_pref != 0 && c->l1_pref != 1)) return SYM_E_INVALID;
    if (c->root_combine != 0 && c->root_combine != 1) return SYM_E_INVALID;
    return SYM_OK;
}

namespace {

std::string tune_key(const sym_tensor_s* X, int rank, sym_dtype bdt) {
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, current_device()) == cudaSuccess) name = prop.name;
    for (auto& ch : name)
        if (ch == ' ') ch = '_';
    char buf[320];
    snprintf(buf, sizeof(buf), "mttkrp3|%s|N%d|n%lld|nnz%lld|strict%lld|R%d|%s|leaf%d", name.c_str(), X->order,
             (long long)X->n, (long long)X->nnz, (long long)X->nnz_strict, rank, bdt == SYM_BF16 ? "bf16" : "f32",
             X->rklo ? 1 : 0);
    return buf;
}

bool tune_lookup(const char* path, const std::string& key, sym_mttkrp_cfg* cfg, float* ms) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[640];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[400];
        sym_mttkrp_cfg c;
        float t;
        if (sscanf(line, "%399s %d %d %d %d %d %d %d %d %d %d %d %d %f", k, &c.strict_kernel, &c.entries_per_warp,
                   &c.threads_per_cta, &c.ctas_per_sm, &c.strict_smem_kb, &c.diag_smem_kb, &c.b_share_pct,
                   &c.leaf_index, &c.vec_per_lane, &c.stream_hint, &c.l1_pref, &c.root_combine, &t) == 14 &&
            key == k && validate_mttkrp_cfg(&c) == SYM_OK) {
            *cfg = c;
            *ms = t;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void tune_store(const char* path, const std::string& key, const sym_mttkrp_cfg& c, float ms) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %d %d %.6f\n", key.c_str(), c.strict_kernel, c.entries_per_warp,
            c.threads_per_cta, c.ctas_per_sm, c.strict_smem_kb, c.diag_smem_kb, c.b_share_pct, c.leaf_index,
            c.vec_per_lane, c.stream_hint, c.l1_pref, c.root_combine, ms);
    fclose(f);
}

}  // namespace

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
    {
        SideScope side(true);  // the diagonal stream's kernel beside the strict one
        st = mttkrp_core(X, B, bf16, rank, ldb, M, ldm, s);
    }
    if (st != SYM_OK) return st;
    if (residual) return residual_launch(X, B, bf16, rank, ldb, M, ldm, residual, ws, ws_bytes, s);
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_range(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                                       int64_t ldm, int64_t first, int64_t count, int accumulate,
                                       sym_stream_t stream) {
    sym_status st = validate_mttkrp_args(X, B, bdt, rank, ldb, M, ldm);
    if (st != SYM_OK) return st;
    if (first < 0 || count < 0 || first > X->nnz || count > X->nnz - first) return SYM_E_INVALID;
    if (accumulate != 0 && accumulate != 1) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    if (!accumulate) {
        if (ldm == rank)
            SYM_CUDA(cudaMemsetAsync(M, 0, sizeof(float) * (size_t)X->n * rank, s));
        else
            SYM_CUDA(cudaMemset2DAsync(M, sizeof(float) * ldm, 0, sizeof(float) * rank, X->n, s));
    }
    if (count == 0) return SYM_OK;
    const sym_tensor_s P = tensor_part(X, first, count);
    const bool bf16 = bdt == SYM_BF16;
    switch (X->order) {
        case 2: return launch_mttkrp_order<2>(&P, B, bf16, rank, ldb, M, ldm, X->cfg, s);
        case 3: return launch_mttkrp_order<3>(&P, B, bf16, rank, ldb, M, ldm, X->cfg, s);
        case 4: return launch_mttkrp_order<4>(&P, B, bf16, rank, ldb, M, ldm, X->cfg, s);
        case 5: return launch_mttkrp_order<5>(&P, B, bf16, rank, ldb, M, ldm, X->cfg, s);
        default: return SYM_E_UNSUPPORTED;
    }
}

extern "C" sym_status sym_mttkrp_default_config(sym_mttkrp_cfg* out) {
    if (!out) return SYM_E_INVALID;
    *out = sym_mttkrp_cfg{SYM_MTTKRP_PLAIN, 256, 256, 2, 0, 96, 0, 1, 1, 0, 0, 1};
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_set_config(sym_tensor X, const sym_mttkrp_cfg* cfg) {
    if (!X) return SYM_E_INVALID;
    sym_status st = validate_mttkrp_cfg(cfg);
    if (st != SYM_OK) return st;
    X->cfg = *cfg;
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_get_config(sym_tensor X, sym_mttkrp_cfg* out) {
    if (!X || !out) return SYM_E_INVALID;
    *out = X->cfg;
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_set_chunk(sym_tensor X, int entries_per_warp) {
    if (!X) return SYM_E_INVALID;
    sym_mttkrp_cfg c;
    sym_mttkrp_default_config(&c);
    if (entries_per_warp > 0) {
        if (entries_per_warp % 32 != 0) return SYM_E_INVALID;
        c.strict_kernel = SYM_MTTKRP_PLAIN;
        c.entries_per_warp = entries_per_warp;
    } else if (entries_per_warp == -1) {
        c.strict_kernel = SYM_MTTKRP_UNFACTORISED;
    } else if (entries_per_warp != 0) {
        return SYM_E_INVALID;
    }
    X->cfg = c;
    return SYM_OK;
}

extern "C" sym_status sym_mttkrp_autotune(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                          float* M, int64_t ldm, const char* cache_path, sym_stream_t stream,
                                          sym_mttkrp_cfg* best, float* best_ms) {
    return sym_mttkrp_autotune_cold(X, B, bdt, rank, ldb, M, ldm, nullptr, 0, cache_path, stream, best, best_ms);
}

extern "C" sym_status sym_mttkrp_autotune_cold(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                               float* M, int64_t ldm, void* flush, size_t flush_bytes,
                                               const char* cache_path, sym_stream_t stream, sym_mttkrp_cfg* best,
                                               float* best_ms) {
    sym_status st = validate_mttkrp_args(X, B, bdt, rank, ldb, M, ldm);
    if (st != SYM_OK) return st;
    if ((flush == nullptr) != (flush_bytes == 0)) return SYM_E_INVALID;
    const std::string key = tune_key(X, rank, bdt) + (flush ? "|cold" : "|warm");
    sym_mttkrp_cfg found;
    float found_ms = 0.f;
    if (tune_lookup(cache_path, key, &found, &found_ms)) {
        X->cfg = found;
        if (best) *best = found;
        if (best_ms) *best_ms = found_ms;
        return SYM_OK;
    }
    cudaStream_t s = as_stream(stream);
    const bool bf16 = bdt == SYM_BF16;
    std::vector<sym_mttkrp_cfg> cands;
    for (int leaf : {0, 1}) {
        if (leaf && !X->rklo) continue;
        for (int chunk : {128, 256, 512})
            for (int sh : {0, 1})
                for (int l1 : {0, 1}) cands.push_back({SYM_MTTKRP_PLAIN, chunk, 256, 2, 0, 0, 0, leaf, 1, sh, l1, 1});
    }
    if (rank >= 8)
        for (int chunk : {256, 512}) cands.push_back({SYM_MTTKRP_PLAIN, chunk, 256, 2, 0, 0, 0, 0, 2, 0, 0, 1});
    for (int chunk : {128, 256, 512})
        for (int thr : {128, 256}) cands.push_back({SYM_MTTKRP_STAGED, chunk, thr, 2, 0, 0, 0, 0, 1, 0, 0, 1});
    for (int chunk : {128, 256}) cands.push_back({SYM_MTTKRP_PIPELINED, chunk, 256, 2, 0, 0, 0, 0, 1, 0, 0, 1});
    for (int depth : {1, 4, 2}) {  // lane shapes: one or four leaf rows in flight, or 8 columns per lane
        // (8 columns per lane measured slower than 4 below rank 64: too few lanes per entry)
        if ((depth == 4 && rank < 16) || (depth == 2 && rank < 64)) continue;
        for (int chunk : {128, 256, 512}) {
            cands.push_back({SYM_MTTKRP_LANE, chunk, 256, 2, 0, 0, 0, 0, depth, 1, 0, 1});  // one pass
            if (!X->rklo) continue;
            for (int rc : {2, 4})  // two passes, unfactorised root pass of 64 rc entries per warp
                cands.push_back({SYM_MTTKRP_LANE, chunk, 256, rc, 0, 0, 0, 1, depth, 1, 0, 1});
            cands.push_back({SYM_MTTKRP_LANE, chunk, 256, 2, 1, 0, 0, 1, depth, 1, 0, 1});  // factorised root pass
        }
    }
    cands.push_back({SYM_MTTKRP_PIPELINED, 0, 512, 2, 0, 0, 0, 0, 1, 0, 0, 1});
    cands.push_back({SYM_MTTKRP_PIPELINED, 0, 512, 2, 96, 0, 50, 0, 1, 0, 0, 1});
    cands.push_back({SYM_MTTKRP_UNFACTORISED, 256, 256, 2, 0, 0, 0, 0, 1, 0, 0, 1});
    {  // the plain and lane kernels also without the combined root flush
        const size_t base = cands.size();
        for (size_t k = 0; k < base; ++k)
            if (cands[k].strict_kernel == SYM_MTTKRP_PLAIN || cands[k].strict_kernel == SYM_MTTKRP_LANE) {
                sym_mttkrp_cfg c = cands[k];
                c.root_combine = 0;
                cands.push_back(c);
            }
    }
    cudaEvent_t e0, e1;
    SYM_CUDA(cudaEventCreate(&e0));
    SYM_CUDA(cudaEventCreate(&e1));
    SideScope side(true);  // candidates timed as sym_mttkrp runs them
    auto time_cfg = [&](const sym_mttkrp_cfg& c, float* out) -> bool {
        if (mttkrp_core_cfg(X, B, bf16, rank, ldb, M, ldm, c, s) != SYM_OK) return false;  // warm-up
        float tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            // cold: the caller's buffer (larger than L2) is rewritten before each timed run
            if (flush && cudaMemsetAsync(flush, rep + 1, flush_bytes, s) != cudaSuccess) return false;
            cudaEventRecord(e0, s);
            if (mttkrp_core_cfg(X, B, bf16, rank, ldb, M, ldm, c, s) != SYM_OK) return false;
            cudaEventRecord(e1, s);
            float t = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return false;
            tot += t;
        }
        *out = tot / 3;
        return true;
    };
    // strict-stream kernel first (diagonal stream at the default), then the diagonal option
    sym_mttkrp_cfg bc;
    sym_mttkrp_default_config(&bc);
    float bt = 1e30f;
    bool any = false;
    for (auto c : cands) {
        c.diag_smem_kb = bc.diag_smem_kb;
        float t;
        if (time_cfg(c, &t) && t < bt) {
            bt = t;
            bc = c;
            any = true;
        }
    }
    if (any && X->nnz > X->nnz_strict) {
        for (int kb : {0, 48, 96}) {
            sym_mttkrp_cfg c = bc;
            c.diag_smem_kb = kb;
            float t;
            if (time_cfg(c, &t) && t < bt) {
                bt = t;
                bc = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!any) return SYM_E_CUDA;
    X->cfg = bc;
    if (best) *best = bc;
    if (best_ms) *best_ms = bt;
    tune_store(cache_path, key, bc, bt);
    return SYM_OK;
}
