// SSYMV and SYPRD over the upper triangle of a symmetric matrix (Sec. 3.1
// figure "spmv_code": an off-diagonal canonical read feeds y[i] and y[j]; a
// diagonal read feeds y[i] once), with the row partial kept in registers
// (workspace transformation, Sec. 4.2.8: the example there is this kernel) and
// SYPRD fused into the same pass (Sec. 3.2.2: off-diagonal terms weighted 2).
// Also: the Bellman-Ford relaxation over the same storage (Sec. 5.2.2) and the
// full-CSR (both triangles) baseline.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "spmv.cuh"

namespace symgpu {

int spmv_lanes(int64_t n, int64_t nnz) {
    double avg = n > 0 ? (double)nnz / (double)n : 1.0;
    int L = 2;
    while (L < 32 && L < avg) L <<= 1;
    return L;
}

namespace {

constexpr int SV_THREADS = 256;

__device__ __forceinline__ float group_sum(float v, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One group of L lanes per row; rows [row0, row_end) are dealt to groups in order.
template <int L, bool SYPRD>
__global__ void __launch_bounds__(SV_THREADS) k_ssymv(int64_t row0, int64_t row_end, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ val,
                                                      const float* __restrict__ x, float* __restrict__ y,
                                                      double* __restrict__ partials, int64_t ncols = INT64_MAX,
                                                      int64_t nnz = INT64_MAX) {
    constexpr int GPC = SV_THREADS / L;
    const int lane = threadIdx.x & 31;
    const int s = lane % L;
    const int64_t i = row0 + (int64_t)blockIdx.x * GPC + threadIdx.x / L;
    const int64_t n = row_end;
    float rowsum = 0.f, syp = 0.f;
    if (i < n) {
        const float xi = x[i];
        const int p1 = rowptr[i + 1];
        for (int p = rowptr[i] + s; p < p1; p += L) {
            if (!SYM_INDEX_OK(p, nnz)) break;  // bounds-checked build: a row pointer past the entries
            const int j = col[p];
            if (!SYM_INDEX_OK(j, ncols)) continue;  // bounds-checked build: a column outside the matrix
            const float a = val[p];
            const float t = a * x[j];
            rowsum += t;
            if (j != i) {
                atomicAdd(&y[j], a * xi);
                if (SYPRD) syp += 2.f * t;
            } else if (SYPRD) {
                syp += t;
            }
        }
        if (SYPRD) syp *= xi;
    }
    rowsum = group_sum(rowsum, L);
    if (i < n && s == 0 && rowsum != 0.f) atomicAdd(&y[i], rowsum);
    if (SYPRD) {
        __shared__ float sh[SV_THREADS / 32];
        float w = warp_sum(syp);
        if (lane == 0) sh[threadIdx.x >> 5] = w;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int k = 0; k < SV_THREADS / 32; ++k) t += sh[k];
            partials[blockIdx.x] = (double)t;
        }
    }
}

// Cross-block SYPRD sum in FP64, fixed order (deterministic).
__global__ void k_sum_partials(const double* __restrict__ partials, int64_t count, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) acc += partials[k];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

template <int L>
sym_status launch_ssymv_l(const sym_csr_upper* A, const float* x, float* y, double* syprd, double* partials,
                          cudaStream_t s, int64_t row0 = 0, int64_t row_end = -1) {
    constexpr int GPC = SV_THREADS / L;
    if (row_end < 0) row_end = A->n;
    const unsigned grid = (unsigned)std::max<int64_t>(1, (row_end - row0 + GPC - 1) / GPC);
    SYM_PROF("ssymv", s);
    if (syprd)
        k_ssymv<L, true><<<grid, SV_THREADS, 0, s>>>(row0, row_end, A->rowptr, A->col, A->val, x, y, partials, A->n,
                                                     A->nnz);
    else
        k_ssymv<L, false><<<grid, SV_THREADS, 0, s>>>(row0, row_end, A->rowptr, A->col, A->val, x, y, partials, A->n,
                                                      A->nnz);
    SYM_CHECK_LAUNCH();
    if (syprd) {
        k_sum_partials<<<1, 1024, 0, s>>>(partials, grid, syprd);
        SYM_CHECK_LAUNCH();
    }
    return SYM_OK;
}

int64_t ssymv_ctas(const sym_csr_upper* A) {
    const int L = spmv_lanes(A->n, A->nnz);
    const int64_t gpc = SV_THREADS / L;
    return std::max<int64_t>(1, (A->n + gpc - 1) / gpc);
}

// ---------------------------------------------------------------- validation

__global__ void k_check_upper(int64_t n, int64_t nnz, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, unsigned long long* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    if (i == 0 && p0 != 0) ok = false;
    if (i == n - 1 && p1 != nnz) ok = false;
    if (p1 < p0) ok = false;
    for (int p = p0; ok && p < p1; ++p) {
        const int j = col[p];
        if (j < i || j >= n) ok = false;
        if (p > p0 && j <= col[p - 1]) ok = false;
    }
    if (!ok) atomicAdd(bad, 1ull);
}

// ---------------------------------------------------------------- Bellman-Ford

__device__ __forceinline__ void atomic_min_float(float* addr, float v) {
    // Order-preserving on IEEE bit patterns: signed compare for v >= 0,
    // unsigned max for negative v (larger pattern = more negative value).
    if (v >= 0.f)
        atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else
        atomicMax(reinterpret_cast<unsigned*>(addr), __float_as_uint(v));
}

template <int L>
__global__ void __launch_bounds__(SV_THREADS) k_bellman(int64_t n, const int32_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col,
                                                        const float* __restrict__ val, const float* __restrict__ d,
                                                        float* __restrict__ y) {
    constexpr int GPC = SV_THREADS / L;
    const int s = (threadIdx.x & 31) % L;
    const int64_t i = (int64_t)blockIdx.x * GPC + threadIdx.x / L;
    if (i >= n) return;
    const float di = d[i];
    float best = INFINITY;
    const int p1 = rowptr[i + 1];
    for (int p = rowptr[i] + s; p < p1; p += L) {
        const int j = col[p];
        const float a = val[p];
        best = fminf(best, a + d[j]);
        if (j != i) atomic_min_float(&y[j], a + di);
    }
    if (best < INFINITY) atomic_min_float(&y[i], best);
}

// ---------------------------------------------------------------- full CSR

template <int L>
__global__ void __launch_bounds__(SV_THREADS) k_spmv_full(int64_t n, const int32_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ col,
                                                          const float* __restrict__ val, const float* __restrict__ x,
                                                          float* __restrict__ y) {
    constexpr int GPC = SV_THREADS / L;
    const int s = (threadIdx.x & 31) % L;
    const int64_t i = (int64_t)blockIdx.x * GPC + threadIdx.x / L;
    float acc = 0.f;
    if (i < n)
        for (int p = rowptr[i] + s; p < rowptr[i + 1]; p += L) acc += val[p] * x[col[p]];
    acc = group_sum(acc, L);
    if (i < n && s == 0) y[i] = acc;
}

// strict-upper entry p of row i -> key (col << bits) | row, payload p
__global__ void k_lower_keys(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             int bits, uint64_t* __restrict__ keys, uint32_t* __restrict__ pay,
                             const uint32_t* __restrict__ slot, unsigned* __restrict__ lower_cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = slot[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        const int j = col[p];
        if (j == i) continue;
        keys[k] = ((uint64_t)j << bits) | (uint64_t)i;
        pay[k] = (uint32_t)p;
        atomicAdd(&lower_cnt[j], 1u);
        ++k;
    }
}

__global__ void k_strict_count(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               uint32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = 0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) c += (col[p] != i);
    cnt[i] = c;
}

__global__ void k_full_rowlen(int64_t n, const int32_t* __restrict__ rowptr, const unsigned* __restrict__ lower_cnt,
                              int64_t* __restrict__ len) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    len[i] = (i < n) ? (int64_t)lower_cnt[i] + (rowptr[i + 1] - rowptr[i]) : 0;
}

__global__ void k_fill_lower(int64_t m, int bits, const uint64_t* __restrict__ keys, const uint32_t* __restrict__ pay,
                             const float* __restrict__ val, const int64_t* __restrict__ full_ptr,
                             const int64_t* __restrict__ lower_start, int32_t* __restrict__ fcol,
                             float* __restrict__ fval) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const uint64_t key = keys[k];
    const int64_t j = (int64_t)(key >> bits);                  // full row
    const int32_t i = (int32_t)(key & ((1ull << bits) - 1));  // full column
    const int64_t dst = full_ptr[j] + (k - lower_start[j]);
    fcol[dst] = i;
    fval[dst] = val[pay[k]];
}

__global__ void k_fill_upper(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const float* __restrict__ val, const int64_t* __restrict__ full_ptr,
                             const unsigned* __restrict__ lower_cnt, int32_t* __restrict__ frow,
                             int32_t* __restrict__ fcol, float* __restrict__ fval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    frow[i] = (int32_t)full_ptr[i];
    if (i == n) return;
    const int64_t base = full_ptr[i] + lower_cnt[i];
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        fcol[base + (p - rowptr[i])] = col[p];
        fval[base + (p - rowptr[i])] = val[p];
    }
}

__global__ void k_lower_start(int64_t n, const unsigned* __restrict__ lower_cnt, int64_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = lower_cnt[i];
}

int bits_of(int64_t n) {
    int b = 1;
    while ((1ll << b) < n) ++b;
    return b;
}

template <typename C>
void layout_expand_ws(C& c, int64_t n, int64_t nnz, uint64_t** k0, uint32_t** p0, uint64_t** k1, uint32_t** p1,
                      uint32_t** slot, unsigned** lcnt, int64_t** len, int64_t** fptr, int64_t** lstart,
                      void** radix, void** scan) {
    size_t m = nnz > 0 ? (size_t)nnz : 1;
    *k0 = c.template take<uint64_t>(m);
    *p0 = c.template take<uint32_t>(m);
    *k1 = c.template take<uint64_t>(m);
    *p1 = c.template take<uint32_t>(m);
    *slot = c.template take<uint32_t>((size_t)n + 1);
    *lcnt = c.template take<unsigned>((size_t)n + 1);
    *len = c.template take<int64_t>((size_t)n + 1);
    *fptr = c.template take<int64_t>((size_t)n + 1);
    *lstart = c.template take<int64_t>((size_t)n + 1);
    *radix = c.template take<char>(radix_ws_bytes((int64_t)m, 1));
    *scan = c.template take<char>(scan_ws_bytes((int64_t)std::max<int64_t>(m, n + 1)));
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
void layout_full(C& c, int64_t n, int64_t full_nnz, int32_t** rp, int32_t** col, float** val) {
    *rp = c.template take<int32_t>((size_t)n + 1);
    *col = c.template take<int32_t>((size_t)std::max<int64_t>(full_nnz, 1));
    *val = c.template take<float>((size_t)std::max<int64_t>(full_nnz, 1));
}

}  // namespace

sym_status ssymv_launch(const sym_csr_upper* A, const float* x, float* y, double* syprd, double* partials,
                        cudaStream_t s) {
    if (A->n == 0) {
        if (syprd) SYM_CUDA(cudaMemsetAsync(syprd, 0, sizeof(double), s));
        return SYM_OK;
    }
    if (ssymv_single_launch(A)) return ssymv_cluster_launch(A, x, y, syprd, s);
    SYM_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)A->n, s));
    switch (spmv_lanes(A->n, A->nnz)) {
        case 2: return launch_ssymv_l<2>(A, x, y, syprd, partials, s);
        case 4: return launch_ssymv_l<4>(A, x, y, syprd, partials, s);
        case 8: return launch_ssymv_l<8>(A, x, y, syprd, partials, s);
        case 16: return launch_ssymv_l<16>(A, x, y, syprd, partials, s);
        default: return launch_ssymv_l<32>(A, x, y, syprd, partials, s);
    }
}

size_t ssymv_partials_bytes(const sym_csr_upper* A) { return align_up(sizeof(double) * ssymv_ctas(A), 256); }

// Rows [r0, r1) only, multi-block form, y not cleared.
sym_status ssymv_rows_launch(const sym_csr_upper* A, const float* x, float* y, double* syprd, double* partials,
                             int64_t r0, int64_t r1, cudaStream_t s) {
    if (r1 <= r0) {
        if (syprd) SYM_CUDA(cudaMemsetAsync(syprd, 0, sizeof(double), s));
        return SYM_OK;
    }
    switch (spmv_lanes(A->n, A->nnz)) {
        case 2: return launch_ssymv_l<2>(A, x, y, syprd, partials, s, r0, r1);
        case 4: return launch_ssymv_l<4>(A, x, y, syprd, partials, s, r0, r1);
        case 8: return launch_ssymv_l<8>(A, x, y, syprd, partials, s, r0, r1);
        case 16: return launch_ssymv_l<16>(A, x, y, syprd, partials, s, r0, r1);
        default: return launch_ssymv_l<32>(A, x, y, syprd, partials, s, r0, r1);
    }
}

sym_status validate_csr(const sym_csr_upper* A) {
    if (!A || A->n < 0 || A->nnz < 0 || A->n > 0x7fffffffLL || A->nnz > 0x7fffffffLL) return SYM_E_INVALID;
    if (A->n > 0 && !A->rowptr) return SYM_E_INVALID;
    if (A->nnz > 0 && (!A->col || !A->val)) return SYM_E_INVALID;
    return SYM_OK;
}

}  // namespace symgpu

using namespace symgpu;

extern "C" size_t sym_spmv_workspace_bytes(const sym_csr_upper* A) {
    if (validate_csr(A) != SYM_OK) return 0;
    return ssymv_partials_bytes(A);
}

extern "C" sym_status sym_spmv(const sym_csr_upper* A, const float* x, float* y, double* syprd, void* ws,
                               size_t ws_bytes, sym_stream_t stream) {
    sym_status st = validate_csr(A);
    if (st != SYM_OK) return st;
    if (A->n > 0 && (!x || !y)) return SYM_E_INVALID;
    if (syprd) {
        if (!ws || !aligned(ws, 256)) return SYM_E_INVALID;
        if (ws_bytes < ssymv_partials_bytes(A)) return SYM_E_NOMEM;
    }
    return ssymv_launch(A, x, y, syprd, static_cast<double*>(ws), as_stream(stream));
}

extern "C" sym_status sym_spmv_rows(const sym_csr_upper* A, const float* x, float* y, double* syprd,
                                    int64_t row_begin, int64_t row_end, int accumulate, void* ws, size_t ws_bytes,
                                    sym_stream_t stream) {
    sym_status st = validate_csr(A);
    if (st != SYM_OK) return st;
    if (row_begin < 0 || row_end < row_begin || row_end > A->n) return SYM_E_INVALID;
    if (accumulate != 0 && accumulate != 1) return SYM_E_INVALID;
    if (A->n > 0 && (!x || !y)) return SYM_E_INVALID;
    if (syprd) {
        if (!ws || !aligned(ws, 256)) return SYM_E_INVALID;
        if (ws_bytes < ssymv_partials_bytes(A)) return SYM_E_NOMEM;
    }
    cudaStream_t s = as_stream(stream);
    if (!accumulate && A->n > 0) SYM_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * (size_t)A->n, s));
    return ssymv_rows_launch(A, x, y, syprd, static_cast<double*>(ws), row_begin, row_end, s);
}

extern "C" sym_status sym_csr_upper_check(const sym_csr_upper* A, int64_t* bad, sym_stream_t stream) {
    sym_status st = validate_csr(A);
    if (st != SYM_OK || !bad) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    SYM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int64_t), s));
    if (A->n == 0) return SYM_OK;
    k_check_upper<<<(unsigned)((A->n + 255) / 256), 256, 0, s>>>(A->n, A->nnz, A->rowptr, A->col,
                                                                  reinterpret_cast<unsigned long long*>(bad));
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" sym_status sym_bellman_step(const sym_csr_upper* A, const float* d, float* y, sym_stream_t stream) {
    sym_status st = validate_csr(A);
    if (st != SYM_OK) return st;
    if (A->n == 0) return SYM_OK;
    if (!d || !y) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    SYM_CUDA(cudaMemcpyAsync(y, d, sizeof(float) * (size_t)A->n, cudaMemcpyDeviceToDevice, s));
    const int L = spmv_lanes(A->n, A->nnz);
    const int64_t gpc = SV_THREADS / L;
    const unsigned grid = (unsigned)((A->n + gpc - 1) / gpc);
    switch (L) {
        case 2: k_bellman<2><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, d, y); break;
        case 4: k_bellman<4><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, d, y); break;
        case 8: k_bellman<8><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, d, y); break;
        case 16: k_bellman<16><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, d, y); break;
        default: k_bellman<32><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, d, y); break;
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

extern "C" size_t sym_csr_expand_bytes(const sym_csr_upper* A, size_t* ws_bytes) {
    if (validate_csr(A) != SYM_OK) return 0;
    NullCarver w;
    uint64_t *k0, *k1;
    uint32_t *p0, *p1, *slot;
    unsigned* lcnt;
    int64_t *len, *fptr, *lstart;
    void *radix, *scan;
    layout_expand_ws(w, A->n, A->nnz, &k0, &p0, &k1, &p1, &slot, &lcnt, &len, &fptr, &lstart, &radix, &scan);
    if (ws_bytes) *ws_bytes = w.s.used;
    NullCarver a;
    int32_t *rp, *col;
    float* val;
    layout_full(a, A->n, 2 * A->nnz, &rp, &col, &val);  // upper bound: 2 nnz
    return a.s.used;
}

extern "C" sym_status sym_csr_expand_upper(const sym_csr_upper* A, void* arena, size_t arena_bytes, void* ws,
                                           size_t ws_bytes, sym_stream_t stream, sym_csr_full* out) {
    sym_status st = validate_csr(A);
    if (st != SYM_OK || !out || !arena || !ws) return SYM_E_INVALID;
    size_t need_w = 0;
    size_t need_a = sym_csr_expand_bytes(A, &need_w);
    if (arena_bytes < need_a || ws_bytes < need_w) return SYM_E_NOMEM;
    cudaStream_t s = as_stream(stream);
    const int64_t n = A->n;
    Carver W(ws, ws_bytes);
    uint64_t *k0, *k1;
    uint32_t *p0, *p1, *slot;
    unsigned* lcnt;
    int64_t *len, *fptr, *lstart;
    void *radix, *scan;
    layout_expand_ws(W, n, A->nnz, &k0, &p0, &k1, &p1, &slot, &lcnt, &len, &fptr, &lstart, &radix, &scan);
    Carver Ar(arena, arena_bytes);
    int32_t *frow, *fcol;
    float* fval;
    layout_full(Ar, n, 2 * A->nnz, &frow, &fcol, &fval);
    if (n == 0) {
        SYM_CUDA(cudaMemsetAsync(frow, 0, sizeof(int32_t), s));
        *out = sym_csr_full{0, 0, frow, fcol, fval};
        return SYM_OK;
    }
    const unsigned g = (unsigned)((n + 256) / 256);
    SYM_CUDA(cudaMemsetAsync(lcnt, 0, sizeof(unsigned) * (size_t)(n + 1), s));
    // slots of each row's strict entries in the key array
    k_strict_count<<<g, 256, 0, s>>>(n, A->rowptr, A->col, slot);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_u32(slot, slot, n, scan, s);
    if (st != SYM_OK) return st;
    int64_t m = 0;
    {
        uint32_t last_slot = 0, last_cnt = 0;
        // strict count = slot[n-1] + count of row n-1
        SYM_CUDA(cudaMemcpyAsync(&last_slot, slot + (n - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        SYM_CUDA(cudaStreamSynchronize(s));
        int32_t rp[2];
        SYM_CUDA(cudaMemcpy(rp, A->rowptr + (n - 1), sizeof(rp), cudaMemcpyDeviceToHost));
        std::vector<int32_t> c(rp[1] - rp[0]);
        if (!c.empty()) SYM_CUDA(cudaMemcpy(c.data(), A->col + rp[0], sizeof(int32_t) * c.size(), cudaMemcpyDeviceToHost));
        for (int32_t j : c) last_cnt += (j != (int32_t)(n - 1));
        m = (int64_t)last_slot + last_cnt;
    }
    k_lower_keys<<<g, 256, 0, s>>>(n, A->rowptr, A->col, bits_of(n), k0, p0, slot, lcnt);
    SYM_CHECK_LAUNCH();
    uint64_t *sk, *sh;
    uint32_t* sp;
    st = radix_sort_pairs(1, k0, nullptr, p0, k1, nullptr, p1, m, 2 * bits_of(n), radix, s, &sk, &sh, &sp);
    if (st != SYM_OK) return st;
    k_full_rowlen<<<g, 256, 0, s>>>(n, A->rowptr, lcnt, len);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_i64(len, fptr, n + 1, scan, s);
    if (st != SYM_OK) return st;
    k_lower_start<<<g, 256, 0, s>>>(n, lcnt, lstart);
    SYM_CHECK_LAUNCH();
    st = exclusive_scan_i64(lstart, lstart, n, scan, s);
    if (st != SYM_OK) return st;
    if (m > 0) {
        k_fill_lower<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, bits_of(n), sk, sp, A->val, fptr, lstart, fcol,
                                                                 fval);
        SYM_CHECK_LAUNCH();
    }
    k_fill_upper<<<g, 256, 0, s>>>(n, A->rowptr, A->col, A->val, fptr, lcnt, frow, fcol, fval);
    SYM_CHECK_LAUNCH();
    SYM_CUDA(cudaStreamSynchronize(s));
    *out = sym_csr_full{n, A->nnz + m, frow, fcol, fval};
    return SYM_OK;
}

extern "C" sym_status sym_spmv_full(const sym_csr_full* A, const float* x, float* y, sym_stream_t stream) {
    if (!A || A->n < 0) return SYM_E_INVALID;
    if (A->n == 0) return SYM_OK;
    if (!x || !y || !A->rowptr) return SYM_E_INVALID;
    cudaStream_t s = as_stream(stream);
    const int L = spmv_lanes(A->n, A->nnz);
    const int64_t gpc = SV_THREADS / L;
    const unsigned grid = (unsigned)((A->n + gpc - 1) / gpc);
    SYM_PROF("spmv_full", s);
    switch (L) {
        case 2: k_spmv_full<2><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, x, y); break;
        case 4: k_spmv_full<4><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, x, y); break;
        case 8: k_spmv_full<8><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, x, y); break;
        case 16: k_spmv_full<16><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, x, y); break;
        default: k_spmv_full<32><<<grid, SV_THREADS, 0, s>>>(A->n, A->rowptr, A->col, A->val, x, y); break;
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}
