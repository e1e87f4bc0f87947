// Shared helpers of the symgpu library (device utilities, status plumbing).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "symgpu.h"

namespace symgpu {

// Records the CUDA error for sym_last_cuda_error() and maps it to SYM_E_CUDA.
sym_status cuda_status(cudaError_t e);

#define SYM_CUDA(call)                                   \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return symgpu::cuda_status(_e); \
    } while (0)

#define SYM_CHECK_LAUNCH() SYM_CUDA(cudaGetLastError())

#define SYM_TRY(call)                          \
    do {                                       \
        sym_status _st = (call);               \
        if (_st != SYM_OK) return _st;         \
    } while (0)

inline cudaStream_t as_stream(sym_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over a caller-given device region (never calls cudaMalloc).
struct Carver {
    char* base;
    size_t cap;
    size_t used = 0;
    Carver(void* p, size_t c) : base(static_cast<char*>(p)), cap(c) {}
    template <typename T>
    T* take(size_t count) {
        size_t off = align_up(used, 256);
        size_t need = off + align_up(count * sizeof(T), 256);
        if (need > cap) return nullptr;
        used = need;
        return reinterpret_cast<T*>(base + off);
    }
};
// Size-only twin of Carver for the *_bytes queries.
struct Sizer {
    size_t used = 0;
    template <typename T>
    void take(size_t count) { used = align_up(used, 256) + align_up(count * sizeof(T), 256); }
};

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int sm_count();
// Raises a kernel's dynamic shared-memory limit on the current device to at
// least `bytes` and never lowers it, so that launches of one kernel with
// different sizes from several host threads cannot undercut one another.
sym_status raise_smem_limit(const void* func, size_t bytes);
template <typename K>
inline sym_status raise_smem_limit(K* kernel, size_t bytes) {
    return raise_smem_limit(reinterpret_cast<const void*>(kernel), bytes);
}
int current_device();

// Records an event pair around a kernel launch when profiling is enabled.
struct ProfScope {
    const char* name;
    cudaStream_t stream;
    void* start;
    ProfScope(const char* n, cudaStream_t s);
    ~ProfScope();
};
#define SYM_PROF(name, stream) symgpu::ProfScope _sym_prof_scope(name, stream)

// ---------------------------------------------------------------- bounds-checked build
//
// Compiled with -DSYM_BOUNDS_CHECK (the separate libsymgpu_bc.so), the kernels
// of the hot path check every gathered or scattered index against the extent
// of its array before the access; an index outside it skips the access and adds
// one to a caller-given device counter (sym_bounds_check_attach), never a trap.
// Device code cannot share one global across translation units without
// relocatable device code, so every translation unit holds its own copy of the
// counter's address and registers a setter that sym_bounds_check_attach calls.
// In the normal build SYM_INDEX_OK is the constant true and nothing is emitted.
void bc_register_setter(sym_status (*set)(unsigned long long*));
#ifdef SYM_BOUNDS_CHECK
static __device__ unsigned long long* g_bc_counter = nullptr;
namespace {
inline sym_status bc_set_counter_here(unsigned long long* p) {
    return cuda_status(cudaMemcpyToSymbol(g_bc_counter, &p, sizeof(p)));
}
struct BcRegistrar {
    BcRegistrar() { bc_register_setter(&bc_set_counter_here); }
};
static BcRegistrar g_bc_registrar;
}  // namespace
__device__ __forceinline__ bool bc_index_ok(int64_t i, int64_t n) {
    if (i >= 0 && i < n) return true;
    unsigned long long* c = g_bc_counter;
    if (c) atomicAdd(c, 1ull);
    return false;
}
#define SYM_INDEX_OK(i, n) symgpu::bc_index_ok((int64_t)(i), (int64_t)(n))
#else
#define SYM_INDEX_OK(i, n) true
#endif

// ---------------------------------------------------------------- device utils

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 f4_mul(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 f4_scale(float4 a, float s) {
    return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
// a + b * c
__device__ __forceinline__ float4 f4_fma(float4 b, float4 c, float4 a) {
    return make_float4(fmaf(b.x, c.x, a.x), fmaf(b.y, c.y, a.y), fmaf(b.z, c.z, a.z), fmaf(b.w, c.w, a.w));
}
// a + b * s
__device__ __forceinline__ float4 f4_fmas(float4 b, float s, float4 a) {
    return make_float4(fmaf(b.x, s, a.x), fmaf(b.y, s, a.y), fmaf(b.z, s, a.z), fmaf(b.w, s, a.w));
}

// Vector reduction into global memory (16 bytes, no return value).
__device__ __forceinline__ void red_add_f4(float* p, float4 v) {
    atomicAdd(reinterpret_cast<float4*>(p), v);
}

// Loads 4 consecutive factor entries as floats (FP32 or BF16 storage).
template <bool BF16>
__device__ __forceinline__ float4 load_row4(const void* B, int64_t row, int64_t ldb, int col) {
    if constexpr (BF16) {
        const __nv_bfloat16* b = static_cast<const __nv_bfloat16*>(B) + row * ldb + col;
        uint2 u = __ldg(reinterpret_cast<const uint2*>(b));
        float4 r;
        r.x = __uint_as_float(u.x << 16);
        r.y = __uint_as_float(u.x & 0xffff0000u);
        r.z = __uint_as_float(u.y << 16);
        r.w = __uint_as_float(u.y & 0xffff0000u);
        return r;
    } else {
        const float* b = static_cast<const float*>(B) + row * ldb + col;
        return __ldg(reinterpret_cast<const float4*>(b));
    }
}

// ---------------------------------------------------------------- host primitives

// Exclusive prefix sum of `n` values (in may equal out).  Scratch from scan_ws_bytes.
size_t scan_ws_bytes(int64_t n);
sym_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s);
sym_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, cudaStream_t s);

// LSD radix sort of (key, payload) pairs on the low `bits` bits of the key.
// KW = 1: 64-bit keys; KW = 2: 128-bit keys stored as (lo, hi) word arrays.
// Results land in (keys_out, pay_out).  Scratch from radix_ws_bytes.
size_t radix_ws_bytes(int64_t n, int kw);
sym_status radix_sort_pairs(int kw, uint64_t* klo, uint64_t* khi, uint32_t* pay, uint64_t* klo_alt,
                            uint64_t* khi_alt, uint32_t* pay_alt, int64_t n, int bits, void* ws,
                            cudaStream_t s, uint64_t** klo_out, uint64_t** khi_out, uint32_t** pay_out);

}  // namespace symgpu
