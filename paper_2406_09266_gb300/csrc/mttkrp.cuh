// Symmetric MTTKRP kernels (Sec. 4.3 "MTTKRP Demonstration", Sec. 5.2.6):
//   M[i, r] = sum over the full tensor X[i, k, l, ..] B[k, r] B[l, r] ...
// read from the canonical triangle only.
//
// STRICT stream (all indices distinct, Sec. 4.2.9 diagonal splitting): each
// entry c_1 < ... < c_N with value v stands for N! full-tensor entries, and
// the N!/N = (N-1)! of them that start with c_p all add the same term
// v * prod_{q != p} B[c_q] to row c_p (distributive assignment grouping,
// Sec. 4.2.7: the factor 2 of the 3-way split loop nest).  The kernels walk the
// sorted entries as a CSF tree (Sec. 2.2) and factorise the sums level by
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
// contiguous range and keeps its fiber state in registers across batches.
#pragma once

#include <algorithm>
#include <atomic>
#include <cstdlib>

#include "common.cuh"
#include "tensor.cuh"

namespace symgpu {

constexpr int MT_THREADS = 256;

template <int N, int KW>
__device__ __forceinline__ void decode_entry(uint64_t lo, uint64_t hi, int bits, int32_t* c) {
    unpack_key<N, KW>(KeyWords{lo, hi}, bits, c);
}

// Bounds-checked build: every coordinate of a decoded entry against the tensor's
// dimension n (a violation is counted and the entry skipped); true otherwise.
template <int N>
__device__ __forceinline__ bool coords_in_range(const int32_t* c, int64_t n) {
#ifdef SYM_BOUNDS_CHECK
    bool ok = true;
#pragma unroll
    for (int q = 0; q < N; ++q) ok = SYM_INDEX_OK(c[q], n) && ok;
    return ok;
#else
    (void)c;
    (void)n;
    return true;
#endif
}

__device__ __forceinline__ float f4_get(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Output rows below H accumulate in a shared-memory copy of M (flushed once per
// CTA); the other rows take one 16-byte vector reduction in global memory.
// The four shared-memory adds of a lane start at a lane-dependent column so
// that the lanes of a group hit different banks.
struct RowSink {
    float* smem;  // H x R floats
    int H;
    int R;
    float* M;
    int64_t ldm;
    __device__ __forceinline__ void add(int64_t row, int col, float4 v) const {
        if (row < H) {
            float* p = smem + row * R + col;
            // lanes l, l+8, l+16, l+24 share a bank group of four; their rotations differ
            const int lane = threadIdx.x & 31;
            const int rot = lane + (lane >> 3);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = (k + rot) & 3;
                atomicAdd(p + j, f4_get(v, j));
            }
        } else {
            red_add_f4(M + row * ldm + col, v);
        }
    }
};

__device__ __forceinline__ void sink_zero(float* smem, int count) {
    float4* s4 = reinterpret_cast<float4*>(smem);
    for (int k = threadIdx.x; k < count / 4; k += blockDim.x) s4[k] = f4_zero();
}

__device__ __forceinline__ void sink_flush(const float* smem, int H, int R, float* M, int64_t ldm) {
    const float4* s4 = reinterpret_cast<const float4*>(smem);
    const int per_row = R / 4;
    for (int k = threadIdx.x; k < H * per_row; k += blockDim.x) {
        const float4 v = s4[k];
        if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
            red_add_f4(M + (int64_t)(k / per_row) * ldm + 4 * (k % per_row), v);
    }
}

// Factor rows below HB come from a shared-memory copy of B (loaded once per CTA,
// BF16 widened to FP32), the others from global memory.
template <bool BF16>
struct RowSource {
    const float* smem;  // HB x R floats
    int HB;
    int R;
    const void* B;
    int64_t ldb;
    __device__ __forceinline__ float4 get(int64_t row, int col) const {
        if (row < HB) return *reinterpret_cast<const float4*>(smem + row * R + col);
        return load_row4<BF16>(B, row, ldb, col);
    }
};

template <bool BF16>
__device__ __forceinline__ void source_fill(float* smem, int HB, int R, const void* B, int64_t ldb) {
    const int per_row = R / 4;
    for (int k = threadIdx.x; k < HB * per_row; k += blockDim.x) {
        const int row = k / per_row, c4 = 4 * (k % per_row);
        *reinterpret_cast<float4*>(smem + row * R + c4) = load_row4<BF16>(B, row, ldb, c4);
    }
}

// Range of the strict stream owned by the calling warp: fixed chunks of
// `chunk` entries (chunk > 0), or, for chunk == 0, CTA c owns the contiguous
// slice [nnz*c/G, nnz*(c+1)/G) and each warp a contiguous part of it.
__device__ __forceinline__ void warp_range(int64_t nnz, int64_t chunk, int64_t* start, int64_t* end) {
    if (chunk > 0) {
        const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        *start = warp * chunk;
        *end = min(*start + chunk, nnz);
    } else {
        const int nw = blockDim.x >> 5, wi = threadIdx.x >> 5;
        const int64_t c0 = nnz * blockIdx.x / gridDim.x, c1 = nnz * (blockIdx.x + 1) / gridDim.x;
        *start = c0 + (c1 - c0) * wi / nw;
        *end = c0 + (c1 - c0) * (wi + 1) / nw;
    }
}

// Final root flush of a CTA's lane groups, combined in shared memory.  Under a
// skewed distribution a few root fibers hold a large share of the entries
// (Zipf(1.2): the hottest root 22 % of the 3-way stream), so every warp in
// their span ends inside them and would reduce its root sum into the same
// output row.  Instead the groups' (root, R-float sum) pairs are merged by a
// pairwise tree in shared memory: at distance d, group g (a multiple of 2d)
// absorbs group g + d when both hold the same root (or g holds none), and
// otherwise group g + d reduces its own sum into its row.  Every sum is added
// exactly once; a CTA whose groups all end in one root issues one reduction.
// Every thread of the CTA must call this (it holds barriers); `valid` is false
// for a group with nothing to flush.
// Its shared memory is dynamic (root_flush_smem bytes, given at launch only
// when the flush is combined), so a kernel launched without it keeps the whole
// unified L1 / shared memory as L1.
template <int L>
constexpr size_t root_flush_smem() {
    return sizeof(float4) * MT_THREADS + sizeof(int32_t) * (MT_THREADS / L);
}

template <int L>
__device__ __forceinline__ void cta_root_flush(int32_t root, float4 v, bool valid, bool on, float* M, int64_t ldm,
                                               int col, float w) {
    extern __shared__ __align__(16) unsigned char root_flush_dyn[];
    float4* s_vec = reinterpret_cast<float4*>(root_flush_dyn);                       // MT_THREADS
    int32_t* s_root = reinterpret_cast<int32_t*>(root_flush_dyn + sizeof(float4) * MT_THREADS);  // MT_THREADS / L
    const int gid = (int)threadIdx.x / L, sl = (int)threadIdx.x % L;
    const int ng = (int)blockDim.x / L;
    int32_t rg = valid ? root : -1;
    float4 acc = valid ? v : f4_zero();
    if (sl == 0) s_root[gid] = rg;
    s_vec[threadIdx.x] = acc;
    __syncthreads();
    for (int d = 1; d < ng; d <<= 1) {
        const bool lead = (gid % (2 * d)) == 0 && gid + d < ng;
        if (lead) {
            const int32_t rp = s_root[gid + d];
            const float4 vp = s_vec[(gid + d) * L + sl];
            if (rp >= 0) {
                if (rp == rg) {
                    acc.x += vp.x;
                    acc.y += vp.y;
                    acc.z += vp.z;
                    acc.w += vp.w;
                } else if (rg < 0) {
                    rg = rp;
                    acc = vp;
                } else if (on) {
                    red_add_f4(M + (int64_t)rp * ldm + col, f4_scale(vp, w));
                }
            }
        }
        __syncthreads();
        if (lead) {
            if (sl == 0) s_root[gid] = rg;
            s_vec[threadIdx.x] = acc;
        }
        __syncthreads();
    }
    if (gid == 0 && rg >= 0 && on) red_add_f4(M + (int64_t)rg * ldm + col, f4_scale(acc, w));
}

// CSF-factorised strict-stream kernel, no shared memory, one entry at a time
// per lane group (the simplest form).
//   MODE 0: every position (fiber flushes for c_1..c_{N-1}, a reduction per
//           entry for the leaf c_N);
//   MODE 1: the same without the leaf reductions (the leaf index covers them);
//   MODE 2: run over the leaf index (tuples reversed, c_N first) and flush the
//           root level only: row c_N receives (N-1)! * sum over its subtree of
//           v * prod_{q<N} B[c_q], accumulated in registers.
template <int N, int KW, int L, bool BF16, int MODE>
__global__ void __launch_bounds__(MT_THREADS, (N <= 3 && KW == 1 && L > 1) ? 5 : 1) k_mttkrp_strict(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk, int stream_hint, int64_t nrows = INT64_MAX, int combine = 1) {
    static_assert(N >= 2 && N <= 5, "order");
    constexpr int LV = N - 1;  // fiber levels above the leaf
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    int64_t start, end;
    warp_range(nnz, chunk, &start, &end);
    // a warp past the end still reaches the CTA's final root flush (a barrier)

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
            if (stream_hint) {  // evict-first: the stream is read once
                mlo = __ldcs(klo + e);
                if (KW == 2) mhi = __ldcs(khi + e);
                mv = __ldcs(val + e);
            } else {
                mlo = klo[e];
                if (KW == 2) mhi = khi[e];
                mv = val[e];
            }
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
            if (!coords_in_range<N>(c, nrows)) continue;
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
                            if (MODE != 2 || q == 0) {
                                float4 out = (q > 0) ? f4_mul(P[q - 1], T[q]) : T[q];
                                if (on) red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
                            }
                            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
                            T[q] = f4_zero();
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < LV; ++q) {
                    if (q >= d) {
                        cur[q] = c[q];
                        // the root row's own factor is not needed when only the root is flushed
                        Brow[q] = (on && (MODE != 2 || q > 0)) ? load_row4<BF16>(B, c[q], ldb, col) : f4_zero();
                        if (MODE != 2) P[q] = (q > 0) ? f4_mul(P[q - 1], Brow[q]) : Brow[q];
                    }
                }
                have = true;
            }
            const float4 bl = on ? load_row4<BF16>(B, c[N - 1], ldb, col) : f4_zero();
            T[LV - 1] = f4_fmas(bl, v, T[LV - 1]);
            if (MODE == 0 && on) red_add_f4(M + (int64_t)c[N - 1] * ldm + col, f4_scale(P[LV - 1], w * v));
        }
    }
    if (have && on) {
#pragma unroll
        for (int q = LV - 1; q >= 1; --q) {
            if (MODE != 2) {
                const float4 out = f4_mul(P[q - 1], T[q]);
                red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
            }
            T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
        }
    }
    if (combine)  // uniform over the grid: every thread of the CTA reaches the barriers or none does
        cta_root_flush<L>(cur[0], T[0], have, on, M, ldm, col, w);
    else if (have && on)
        red_add_f4(M + (int64_t)cur[0] * ldm + col, f4_scale(T[0], w));
}

// The plain kernel with VPL float4 column groups per lane (L = R / (4 VPL) lanes
// per entry; group v of a lane at columns 4 l + 4 L v, so each vector access of
// the L lanes covers 16 L contiguous bytes of the row), so one warp instruction
// serves more entries and the per-entry
// scalar work (shuffles, key decode, fiber tests, addressing) is spread over
// fewer lanes.  Every position is handled in this one pass.
template <int N, int KW, int L, int VPL, bool BF16>
__global__ void __launch_bounds__(MT_THREADS) k_mttkrp_strict_wide(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk) {
    constexpr int LV = N - 1;
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col0 = 4 * (lane % L);  // column group v of this lane starts at col0 + 4 L v
    int64_t start, end;
    warp_range(nnz, chunk, &start, &end);
    if (start >= end || col0 >= R) {
        // lanes without columns still take part in the shuffles below
        if (start >= end) return;
    }
    int32_t cur[LV];
    float4 Brow[LV][VPL], P[LV][VPL], T[LV][VPL];
#pragma unroll
    for (int q = 0; q < LV; ++q) {
        cur[q] = -1;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            Brow[q][v] = f4_zero();
            P[q][v] = f4_zero();
            T[q][v] = f4_zero();
        }
    }
    bool have = false;
    bool on[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) on[v] = col0 + 4 * L * v < R;
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
            const float x = __shfl_sync(0xffffffffu, mv, src);
            if (b0 + src >= end || !on[0]) continue;
            int32_t c[N];
            decode_entry<N, KW>(lo, hi, bits, c);
            int d = LV;
#pragma unroll
            for (int q = LV - 1; q >= 0; --q)
                if (!have || c[q] != cur[q]) d = q;
            if (d < LV) {
                if (have) {
#pragma unroll
                    for (int q = LV - 1; q >= 0; --q) {
                        if (q >= d) {
#pragma unroll
                            for (int v = 0; v < VPL; ++v) {
                                float4 out = (q > 0) ? f4_mul(P[q - 1][v], T[q][v]) : T[q][v];
                                if (on[v]) red_add_f4(M + (int64_t)cur[q] * ldm + col0 + 4 * L * v, f4_scale(out, w));
                                if (q > 0) T[q - 1][v] = f4_fma(Brow[q][v], T[q][v], T[q - 1][v]);
                                T[q][v] = f4_zero();
                            }
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < LV; ++q) {
                    if (q >= d) {
                        cur[q] = c[q];
#pragma unroll
                        for (int v = 0; v < VPL; ++v) {
                            Brow[q][v] = on[v] ? load_row4<BF16>(B, c[q], ldb, col0 + 4 * L * v) : f4_zero();
                            P[q][v] = (q > 0) ? f4_mul(P[q - 1][v], Brow[q][v]) : Brow[q][v];
                        }
                    }
                }
                have = true;
            }
            float4 bl[VPL];
#pragma unroll
            for (int v = 0; v < VPL; ++v) bl[v] = on[v] ? load_row4<BF16>(B, c[N - 1], ldb, col0 + 4 * L * v) : f4_zero();
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                T[LV - 1][v] = f4_fmas(bl[v], x, T[LV - 1][v]);
                if (on[v]) red_add_f4(M + (int64_t)c[N - 1] * ldm + col0 + 4 * L * v, f4_scale(P[LV - 1][v], w * x));
            }
        }
    }
    if (have) {
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                float4 out = (q > 0) ? f4_mul(P[q - 1][v], T[q][v]) : T[q][v];
                if (on[v]) red_add_f4(M + (int64_t)cur[q] * ldm + col0 + 4 * L * v, f4_scale(out, w));
                if (q > 0) T[q - 1][v] = f4_fma(Brow[q][v], T[q][v], T[q - 1][v]);
            }
        }
    }
}

// ---------------------------------------------------------------- staged leaf rows

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Bytes of one staged leaf row slice held by one lane (4 columns).
template <bool BF16>
constexpr int stage_lane_bytes() { return BF16 ? 8 : 16; }

// The plain kernel with the leaf factor rows of the NEXT batch of 32 entries
// copied into a per-warp shared-memory double buffer (cp.async) while the
// current batch is processed, so a warp keeps up to 32 row copies in flight
// without holding them in registers.  Each lane copies, and later reads, only
// its own 4 columns of each row, so no synchronisation beyond the cp.async
// group wait is needed.
template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(512) k_mttkrp_strict_staged(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk) {
    extern __shared__ float4 stage_mem[];
    constexpr int LV = N - 1;
    constexpr int LB = stage_lane_bytes<BF16>();
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int s_lane = lane % L;
    const int col = 4 * s_lane;
    const bool on = col < R;
    // per warp: 2 buffers x 32 slots x L lane slices of LB bytes
    char* wbuf = reinterpret_cast<char*>(stage_mem) + (size_t)(threadIdx.x >> 5) * (2 * 32 * L * LB);
    int64_t start, end;
    warp_range(nnz, chunk, &start, &end);
    if (start >= end) return;

    // loads the keys of the batch starting at b0 (lane e holds entry b0+e) and
    // issues the copies of its leaf rows into buffer `buf`
    auto fetch = [&](int64_t b0, int buf, uint64_t& mlo, uint64_t& mhi, float& mv) {
        const int64_t e = b0 + lane;
        mlo = 0;
        mhi = 0;
        mv = 0.f;
        int32_t leaf = 0;
        if (e < end) {
            mlo = klo[e];
            if (KW == 2) mhi = khi[e];
            mv = val[e];
            int32_t c[N];
            decode_entry<N, KW>(mlo, mhi, bits, c);
            leaf = c[N - 1];
        }
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            const int slot = g * L + t;
            const int32_t row = __shfl_sync(0xffffffffu, leaf, slot);
            if (on && b0 + slot < end) {
                char* dst = wbuf + ((size_t)(buf * 32 + slot) * L + s_lane) * LB;
                if (BF16)
                    cp_async_8(dst, static_cast<const char*>(B) + ((int64_t)row * ldb + col) * 2);
                else
                    cp_async_16(dst, static_cast<const char*>(B) + ((int64_t)row * ldb + col) * 4);
            }
        }
        cp_async_commit();
    };

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
    uint64_t mlo, mhi;
    float mv;
    fetch(start, 0, mlo, mhi, mv);
    int buf = 0;
    for (int64_t b0 = start; b0 < end; b0 += 32, buf ^= 1) {
        uint64_t nlo = 0, nhi = 0;
        float nv = 0.f;
        if (b0 + 32 < end)
            fetch(b0 + 32, buf ^ 1, nlo, nhi, nv);
        else
            cp_async_commit();  // keep one group per batch so the wait below always targets this batch
        cp_async_wait_prev();
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            const int src = g * L + t;
            const uint64_t lo = __shfl_sync(0xffffffffu, mlo, src);
            const uint64_t hi = (KW == 2) ? __shfl_sync(0xffffffffu, mhi, src) : 0ull;
            const float v = __shfl_sync(0xffffffffu, mv, src);
            if (b0 + src >= end || !on) continue;
            int32_t c[N];
            decode_entry<N, KW>(lo, hi, bits, c);
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
                            red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
                            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
                            T[q] = f4_zero();
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < LV; ++q) {
                    if (q >= d) {
                        cur[q] = c[q];
                        Brow[q] = load_row4<BF16>(B, c[q], ldb, col);
                        P[q] = (q > 0) ? f4_mul(P[q - 1], Brow[q]) : Brow[q];
                    }
                }
                have = true;
            }
            const char* sp = wbuf + ((size_t)(buf * 32 + src) * L + s_lane) * LB;
            float4 bl;
            if (BF16) {
                const uint2 u = *reinterpret_cast<const uint2*>(sp);
                bl = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                                 __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
            } else {
                bl = *reinterpret_cast<const float4*>(sp);
            }
            T[LV - 1] = f4_fmas(bl, v, T[LV - 1]);
            red_add_f4(M + (int64_t)c[N - 1] * ldm + col, f4_scale(P[LV - 1], w * v));
        }
        mlo = nlo;
        mhi = nhi;
        mv = nv;
    }
    if (have && on) {
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
            float4 out = (q > 0) ? f4_mul(P[q - 1], T[q]) : T[q];
            red_add_f4(M + (int64_t)cur[q] * ldm + col, f4_scale(out, w));
            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Same computation with a one-deep software pipeline (the next entry's leaf
// factor row is requested before the current entry is processed), a choice of
// chunked or persistent work ranges, and optional shared-memory hot rows for M
// (H rows) and B (HB rows).
template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(512) k_mttkrp_strict_pipe(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk, int H, int HB) {
    extern __shared__ float4 sink_mem[];
    constexpr int LV = N - 1;
    float* sm_m = reinterpret_cast<float*>(sink_mem);
    float* sm_b = sm_m + (size_t)H * R;
    const RowSink sink{sm_m, H, R, M, ldm};
    const RowSource<BF16> src_b{sm_b, HB, R, B, ldb};
    if (H + HB > 0) {
        sink_zero(sm_m, H * R);
        source_fill<BF16>(sm_b, HB, R, B, ldb);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int g = lane / L;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    int64_t start, end;
    warp_range(nnz, chunk, &start, &end);

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
        // entries of this group in this batch: b0 + g*L + t, valid while t < nval
        const int64_t left = end - (b0 + g * L);
        const int nval = left <= 0 ? 0 : (left >= L ? L : (int)left);
        int32_t cn[N];
        float vn = 0.f;
        float4 bn = f4_zero();
        {
            const uint64_t lo = __shfl_sync(0xffffffffu, mlo, g * L);
            const uint64_t hi = (KW == 2) ? __shfl_sync(0xffffffffu, mhi, g * L) : 0ull;
            vn = __shfl_sync(0xffffffffu, mv, g * L);
            decode_entry<N, KW>(lo, hi, bits, cn);
            if (nval > 0 && on) bn = src_b.get(cn[N - 1], col);
        }
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            int32_t c[N];
#pragma unroll
            for (int q = 0; q < N; ++q) c[q] = cn[q];
            const float v = vn;
            const float4 bl = bn;
            if (t + 1 < L) {  // issue the next entry's leaf gather first
                const int srcl = g * L + t + 1;
                const uint64_t lo = __shfl_sync(0xffffffffu, mlo, srcl);
                const uint64_t hi = (KW == 2) ? __shfl_sync(0xffffffffu, mhi, srcl) : 0ull;
                vn = __shfl_sync(0xffffffffu, mv, srcl);
                decode_entry<N, KW>(lo, hi, bits, cn);
                if (t + 1 < nval && on) bn = src_b.get(cn[N - 1], col);
            }
            if (t >= nval || !on) continue;
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
                            sink.add(cur[q], col, f4_scale(out, w));
                            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
                            T[q] = f4_zero();
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < LV; ++q) {
                    if (q >= d) {
                        cur[q] = c[q];
                        Brow[q] = src_b.get(c[q], col);
                        P[q] = (q > 0) ? f4_mul(P[q - 1], Brow[q]) : Brow[q];
                    }
                }
                have = true;
            }
            T[LV - 1] = f4_fmas(bl, v, T[LV - 1]);
            sink.add(c[N - 1], col, f4_scale(P[LV - 1], w * v));
        }
    }
    if (have && on) {
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
            float4 out = (q > 0) ? f4_mul(P[q - 1], T[q]) : T[q];
            sink.add(cur[q], col, f4_scale(out, w));
            if (q > 0) T[q - 1] = f4_fma(Brow[q], T[q], T[q - 1]);
        }
    }
    if (H > 0) {
        __syncthreads();
        sink_flush(sm_m, H, R, M, ldm);
    }
}

// Strict-stream kernel with lane-parallel decoding (SYM_MTTKRP_LANE).
//
// The other strict kernels have all L lanes of a group shuffle, decode and
// compare every entry's key; that scalar work, repeated by every lane, is most
// of their instructions.  Here the group's lanes decode L consecutive entries
// in parallel, one each, and each finds the first fiber level at which its
// entry differs from the entry before it (the previous lane's, or for the
// group's first lane the last entry of the group's previous batch).  The group
// then steps through its L entries with one broadcast of a packed word (leaf
// row << 3 | first changed level) and one of the value per entry; coordinates
// of the upper levels are broadcast only when a fiber changes.
//
// Work: warp w takes entries [w chunk, (w + 1) chunk); its G = 32 / L groups
// split that range into G contiguous parts.  The positions it updates:
//   MODE 0: every position (leaf reductions per entry, fiber flushes above);
//   MODE 1: all but the leaf (the leaf's rows are left to a root-only pass);
//   MODE 2: the root only, over the leaf index (tuples reversed and sorted, so
//           the root is the LARGEST index of each tuple).
// MODE 1 over the canonical stream plus a root-only pass over the leaf index
// cover every position exactly once with no per-entry reduction.  D leaf rows
// are requested before the D entries are processed, and each batch's keys one
// batch ahead.  Each lane owns V float4 column groups (columns 4 l + 4 L u,
// u < V, for lane l of the group: each gather / reduction instruction of the
// group covers 16 L contiguous bytes of the row), so a wider V spreads the
// per-entry scalar work (broadcasts, address arithmetic, loop control) over
// more columns and lets a warp hold 32 / L entries at once with L = R / (4 V).
template <int N, int KW, int L, bool BF16, int MODE, int D, int V>
__global__ void __launch_bounds__(256, V == 1 ? (D == 1 ? 4 : 3) : 3) k_mttkrp_lane(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk, int stream_hint, int64_t nrows = INT64_MAX, int combine = 1) {
    static_assert(N >= 2 && N <= 5, "order");
    static_assert(D >= 1 && D <= L && L % D == 0, "prefetch depth divides the lanes per entry");
    static_assert(V == 1 || V == 2, "column groups per lane");
    constexpr int LV = N - 1;
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int g = lane / L, sl = lane % L;
    const int col = 4 * sl;  // column group u of this lane starts at col + 4 L u
    bool on[V];
#pragma unroll
    for (int u = 0; u < V; ++u) on[u] = col + 4 * L * u < R;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // a warp past the end runs no batch but still reaches the CTA's final root flush (a barrier)
    const int64_t ws = min(warp * chunk, nnz);
    const int64_t we = min(ws + chunk, nnz);
    const int64_t sub = (we - ws + G - 1) / G;
    const int64_t gs = min(ws + g * sub, we), ge = min(gs + sub, we);
    const int nb = (int)((sub + L - 1) / L);  // batches: the same count for every group of the warp

    int32_t cur[LV], lastc[LV];
    float4 Brow[LV][V], P[LV][V], T[LV][V];
#pragma unroll
    for (int q = 0; q < LV; ++q) {
        cur[q] = -1;
        lastc[q] = -1;
#pragma unroll
        for (int u = 0; u < V; ++u) {
            Brow[q][u] = f4_zero();
            P[q][u] = f4_zero();
            T[q][u] = f4_zero();
        }
    }
    bool have = false;
    // flush the open fibers at levels >= max(dt, qmin) (deepest first), each into its row with its prefix product
    auto flush = [&](int dt, int qmin) {
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
            if (q >= dt && q >= qmin) {
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    if (on[u] && (MODE != 2 || q == 0)) {
                        const float4 out = (q > 0) ? f4_mul(P[q - 1][u], T[q][u]) : T[q][u];
                        red_add_f4(M + (int64_t)cur[q] * ldm + col + 4 * L * u, f4_scale(out, w));
                    }
                    if (q > 0) T[q - 1][u] = f4_fma(Brow[q][u], T[q][u], T[q - 1][u]);
                    T[q][u] = f4_zero();
                }
            }
        }
    };
    // the next batch's keys are requested one batch ahead, so the stream's DRAM latency overlaps the work
    auto fetch = [&](int bb, uint64_t& flo, uint64_t& fhi, float& fv) {
        const int64_t fe = gs + (int64_t)bb * L + sl;
        flo = 0;
        fhi = 0;
        fv = 0.f;
        if (bb < nb && fe < ge) {
            if (stream_hint) {
                flo = __ldcs(klo + fe);
                if (KW == 2) fhi = __ldcs(khi + fe);
                fv = __ldcs(val + fe);
            } else {
                flo = klo[fe];
                if (KW == 2) fhi = khi[fe];
                fv = val[fe];
            }
        }
    };
    uint64_t nlo, nhi;
    float nv;
    fetch(0, nlo, nhi, nv);
    for (int b = 0; b < nb; ++b) {
        // ---- lane-parallel decode: this lane's entry and its first changed level
        const uint64_t lo = nlo, hi = nhi;
        const float v = nv;
        fetch(b + 1, nlo, nhi, nv);
        int32_t c[N];
        decode_entry<N, KW>(lo, hi, bits, c);
        int d = LV;
#pragma unroll
        for (int q = LV - 1; q >= 0; --q) {
            const int32_t up = __shfl_up_sync(0xffffffffu, c[q], 1, L);
            const int32_t prev = sl == 0 ? lastc[q] : up;
            if (c[q] != prev) d = q;
        }
        if (b == 0 && sl == 0) d = 0;  // the group's first entry opens every level
        // level 7 marks an entry the bounds-checked build drops (an index outside [0, n))
        const bool valid = gs + (int64_t)b * L + sl < ge;
        const bool inr = !valid || coords_in_range<N>(c, nrows);
        const uint32_t packed = inr ? (((uint32_t)c[N - 1] << 3) | (uint32_t)d) : 7u;
#pragma unroll
        for (int q = 0; q < LV; ++q) lastc[q] = __shfl_sync(0xffffffffu, c[q], g * L + L - 1);
        // entries of this batch that belong to the group (group-uniform)
        const int nvalid = (int)min((int64_t)L, max((int64_t)0, ge - (gs + (int64_t)b * L)));

        // ---- the group steps through its L entries, D at a time
#pragma unroll 1
        for (int t0 = 0; t0 < L; t0 += D) {
            uint32_t pk[D];
            float vt[D];
            float4 bl[D][V];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                pk[k] = __shfl_sync(0xffffffffu, packed, g * L + t0 + k);
                vt[k] = __shfl_sync(0xffffffffu, v, g * L + t0 + k);
                const bool ok = (t0 + k < nvalid) && (pk[k] & 7u) != 7u;
#pragma unroll
                for (int u = 0; u < V; ++u)
                    bl[k][u] = (ok && on[u]) ? load_row4<BF16>(B, (int64_t)(pk[k] >> 3), ldb, col + 4 * L * u)
                                             : f4_zero();
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (t0 + k >= nvalid) continue;  // group-uniform
                const int dt = (int)(pk[k] & 7u);
                if (dt == 7) continue;  // dropped by the bounds check
                if (dt < LV) {
                    if (have) flush(dt, 0);
#pragma unroll
                    for (int q = 0; q < LV; ++q) {
                        if (q >= dt) {
                            cur[q] = __shfl_sync(gmask, c[q], t0 + k, L);
#pragma unroll
                            for (int u = 0; u < V; ++u) {
                                Brow[q][u] = (on[u] && (MODE != 2 || q > 0))
                                                 ? load_row4<BF16>(B, cur[q], ldb, col + 4 * L * u)
                                                 : f4_zero();
                                if (MODE != 2) P[q][u] = (q > 0) ? f4_mul(P[q - 1][u], Brow[q][u]) : Brow[q][u];
                            }
                        }
                    }
                    have = true;
                }
#pragma unroll
                for (int u = 0; u < V; ++u) {
                    T[LV - 1][u] = f4_fmas(bl[k][u], vt[k], T[LV - 1][u]);
                    if (MODE == 0 && on[u])
                        red_add_f4(M + (int64_t)(pk[k] >> 3) * ldm + col + 4 * L * u,
                                   f4_scale(P[LV - 1][u], w * vt[k]));
                }
            }
        }
    }
    // levels below the root as usual; the root through the CTA's combined flush
    if (have) flush(0, 1);
#pragma unroll
    for (int u = 0; u < V; ++u) {
        if (combine) {  // uniform over the grid
            if (u > 0) __syncthreads();  // the previous column group's shared slots are read
            cta_root_flush<L>(cur[0], T[0][u], have, on[u], M, ldm, col + 4 * L * u, w);
        } else if (have && on[u]) {
            red_add_f4(M + (int64_t)cur[0] * ldm + col + 4 * L * u, f4_scale(T[0][u], w));
        }
    }
}

// Root-only pass over the leaf index, unfactorised below the root (the second
// pass of the two-pass schedule).  Over the leaf index (tuples reversed and
// sorted) the root c_1 of each entry is the largest index of the canonical
// tuple; row c_1 receives (N-1)! times the sum over its root fiber of
// v prod_{q>1} B[c_q], accumulated in registers and reduced once per fiber.
// Below the root no fiber is tracked: every entry multiplies its N - 1 rows
// directly (the rows are the smallest indices of their tuples, the hottest rows
// under a skewed distribution, so they come from L1).  Lanes decode one entry
// each; the group then steps through them with one broadcast per row offset,
// one for the value and one for the root change.
template <int N, int KW, int L, bool BF16, int V>
__global__ void __launch_bounds__(256, V == 1 ? 4 : 3) k_mttkrp_rootpass(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t nnz,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, float w,
    int64_t chunk, int stream_hint, int64_t nrows = INT64_MAX) {
    static_assert(N >= 2 && N <= 5, "order");
    constexpr int G = 32 / L;
    const int lane = threadIdx.x & 31;
    const int g = lane / L, sl = lane % L;
    const int col = 4 * sl;  // column group u of this lane starts at col + 4 L u
    bool on[V];
#pragma unroll
    for (int u = 0; u < V; ++u) on[u] = col + 4 * L * u < R;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t ws = warp * chunk;
    if (ws >= nnz) return;
    const int64_t we = min(ws + chunk, nnz);
    const int64_t sub = (we - ws + G - 1) / G;
    const int64_t gs = min(ws + g * sub, we), ge = min(gs + sub, we);
    const int nb = (int)((sub + L - 1) / L);

    auto fetch = [&](int bb, uint64_t& flo, uint64_t& fhi, float& fv) {
        const int64_t fe = gs + (int64_t)bb * L + sl;
        flo = 0;
        fhi = 0;
        fv = 0.f;
        if (bb < nb && fe < ge) {
            if (stream_hint) {
                flo = __ldcs(klo + fe);
                if (KW == 2) fhi = __ldcs(khi + fe);
                fv = __ldcs(val + fe);
            } else {
                flo = klo[fe];
                if (KW == 2) fhi = khi[fe];
                fv = val[fe];
            }
        }
    };
    int32_t root = -1, lastroot = -1;
    float4 acc[V];
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] = f4_zero();
    auto flush_root = [&]() {
#pragma unroll
        for (int u = 0; u < V; ++u)
            if (on[u]) red_add_f4(M + (int64_t)root * ldm + col + 4 * L * u, f4_scale(acc[u], w));
    };
    uint64_t nlo, nhi;
    float nv;
    fetch(0, nlo, nhi, nv);
    for (int b = 0; b < nb; ++b) {
        const uint64_t lo = nlo, hi = nhi;
        const float v = nv;
        fetch(b + 1, nlo, nhi, nv);
        int32_t c[N];
        decode_entry<N, KW>(lo, hi, bits, c);
        const int32_t up = __shfl_up_sync(0xffffffffu, c[0], 1, L);
        const int32_t prev = sl == 0 ? lastroot : up;
        int32_t newroot = (c[0] != prev || (b == 0 && sl == 0)) ? c[0] : -1;  // -1: same root as before
        if (!coords_in_range<N>(c, nrows) && gs + (int64_t)b * L + sl < ge) newroot = -2;  // dropped entry
        lastroot = __shfl_sync(0xffffffffu, c[0], g * L + L - 1);
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
            const int src = g * L + t;
            const int32_t nr = __shfl_sync(0xffffffffu, newroot, src);
            const float vt = __shfl_sync(0xffffffffu, v, src);
            int32_t r[N - 1];
#pragma unroll
            for (int q = 1; q < N; ++q) r[q - 1] = __shfl_sync(0xffffffffu, c[q], src);
            // Past the group's last entry the lanes skip the work but stay in the loop: every lane of the
            // warp must reach each full-warp shuffle above, whatever its group's entry count.
            if (gs + (int64_t)b * L + t >= ge || nr == -2) continue;
            if (nr >= 0) {  // a new root fiber starts at this entry
                if (root >= 0) flush_root();
                root = nr;
#pragma unroll
                for (int u = 0; u < V; ++u) acc[u] = f4_zero();
            }
#pragma unroll
            for (int u = 0; u < V; ++u) {
                if (on[u]) {
                    float4 prod = load_row4<BF16>(B, r[0], ldb, col + 4 * L * u);
#pragma unroll
                    for (int q = 1; q < N - 1; ++q) prod = f4_mul(prod, load_row4<BF16>(B, r[q], ldb, col + 4 * L * u));
                    acc[u] = f4_fmas(prod, vt, acc[u]);
                }
            }
        }
    }
    if (root >= 0) flush_root();
}

// One entry per lane group, any equality pattern (the diagonal stream; with
// all-distinct entries it is the unfactorised per-entry form).  Grid-stride
// over entries; optional shared-memory hot rows as above.
template <int N, int KW, int L, bool BF16>
__global__ void __launch_bounds__(512) k_mttkrp_entries(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const float* __restrict__ val, int64_t cnt,
    int bits, const void* __restrict__ B, int64_t ldb, int R, float* __restrict__ M, int64_t ldm, int H, int HB,
    int64_t nrows = INT64_MAX) {
    extern __shared__ float4 sink_mem[];
    float* sm_m = reinterpret_cast<float*>(sink_mem);
    float* sm_b = sm_m + (size_t)H * R;
    const RowSink sink{sm_m, H, R, M, ldm};
    const RowSource<BF16> src_b{sm_b, HB, R, B, ldb};
    if (H + HB > 0) {
        sink_zero(sm_m, H * R);
        source_fill<BF16>(sm_b, HB, R, B, ldb);
        __syncthreads();
    }
    constexpr int GPW = 32 / L;
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane % L);
    const bool on = col < R;
    const int64_t group = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW + lane / L;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x >> 5) * GPW;
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    for (int64_t e = group; e < cnt && on; e += ngroups) {
        int32_t c[N];
        decode_entry<N, KW>(klo[e], KW == 2 ? khi[e] : 0ull, bits, c);
        if (!coords_in_range<N>(c, nrows)) continue;
        const float v = val[e];
        float4 b[N];
#pragma unroll
        for (int q = 0; q < N; ++q) b[q] = src_b.get(c[q], col);
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
            sink.add(c[p], col, f4_scale(f4_mul(pre[p], suf[p + 1]), W * v));
        }
    }
    if (H > 0) {
        __syncthreads();
        sink_flush(sm_m, H, R, M, ldm);
    }
}

// ---------------------------------------------------------------- launch

// A second stream for the diagonal stream's kernel, so it runs beside the
// strict stream's kernel instead of after it (the two add into M with
// atomics, so their order does not matter).  Set for the calling host thread
// by the public MTTKRP entry points; null elsewhere (the serving runtime
// overlaps whole requests instead).
struct SideLaunch {
    cudaStream_t stream;
    cudaEvent_t fork, join;
};
extern thread_local const SideLaunch* t_side_launch;
const SideLaunch* side_launch_for_device(int device);  // per host thread and device; null on failure

// Smallest shared-memory carveout (percent of the SM's maximum) that holds
// `smem` bytes of shared memory for as many CTAs of MT_THREADS threads as an
// SM can run (plus the 1 KB the hardware reserves per CTA); the rest of the
// unified L1 / shared memory stays L1.  0 when the kernel takes none.
inline int l1_carveout_pct(size_t smem) {
    if (smem == 0) return 0;
    static std::atomic<int> smem_sm{0};  // every device of the process is a GB300
    if (smem_sm.load() <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, current_device()) != cudaSuccess ||
            v <= 0)
            return (int)cudaSharedmemCarveoutDefault;
        smem_sm.store(v);
    }
    const size_t need = (size_t)(2048 / MT_THREADS) * (smem + 1024);
    return (int)std::min<size_t>(100, (need * 100 + (size_t)smem_sm.load() - 1) / (size_t)smem_sm.load());
}

// Hot-row sizing within a shared-memory budget: rows of M (H) and of B (HB).
struct SinkPlan {
    int H;
    int HB;
    size_t bytes;
};
inline SinkPlan plan_sink(int64_t n, int R, int kb, int b_share_pct) {
    if (kb <= 0) return SinkPlan{0, 0, 0};
    const size_t row = (size_t)R * sizeof(float);
    const size_t budget = (size_t)kb * 1024;
    int HB = (int)std::min<int64_t>(n, (int64_t)(budget * (size_t)b_share_pct / 100 / row));
    int H = (int)std::min<int64_t>(n, (int64_t)((budget - (size_t)HB * row) / row));
    return SinkPlan{H, HB, (size_t)(H + HB) * row};
}

// Lane-kernel shapes selected by vec_per_lane: 1 = one float4 column group per
// lane, one leaf row in flight; 4 = the same with four leaf rows requested
// together; 2 = two column groups per lane (half the lanes per entry).
template <int N, int KW, int L, bool BF16, int MODE>
sym_status launch_lane_m(int shape, int64_t cnt, const uint64_t* klo, const uint64_t* khi, const float* val, int bits,
                         const void* B, int64_t ldb, int R, float* M, int64_t ldm, float w, int64_t chunk,
                         int stream_hint, const char* name, cudaStream_t s, int64_t nrows, int combine) {
    const int64_t warps = (cnt + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    constexpr int LH = L >= 2 ? L / 2 : 1;
    const size_t rf = combine ? root_flush_smem<L>() : 0, rfh = combine ? root_flush_smem<LH>() : 0;
    SYM_PROF(name, s);
    if (shape == 4 && L >= 4)
        k_mttkrp_lane<N, KW, L, BF16, MODE, (L >= 4 ? 4 : 1), 1><<<grid, 256, rf, s>>>(
            klo, khi, val, cnt, bits, B, ldb, R, M, ldm, w, chunk, stream_hint, nrows, combine);
    else if (shape == 2 && L >= 2)
        k_mttkrp_lane<N, KW, LH, BF16, MODE, 1, 2><<<grid, 256, rfh, s>>>(klo, khi, val, cnt, bits, B, ldb, R, M, ldm,
                                                                        w, chunk, stream_hint, nrows, combine);
    else
        k_mttkrp_lane<N, KW, L, BF16, MODE, 1, 1><<<grid, 256, rf, s>>>(klo, khi, val, cnt, bits, B, ldb, R, M, ldm, w,
                                                                      chunk, stream_hint, nrows, combine);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

template <int N, int KW, int L, bool BF16>
sym_status launch_rootpass(int shape, int64_t cnt, const uint64_t* klo, const uint64_t* khi, const float* val,
                           int bits, const void* B, int64_t ldb, int R, float* M, int64_t ldm, float w, int64_t chunk,
                           int stream_hint, cudaStream_t s, int64_t nrows) {
    const int64_t warps = (cnt + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
    constexpr int LH = L >= 2 ? L / 2 : 1;
    SYM_PROF("mttkrp_strict_leaf", s);
    if (shape == 2 && L >= 2)
        k_mttkrp_rootpass<N, KW, LH, BF16, 2><<<grid, 256, 0, s>>>(klo, khi, val, cnt, bits, B, ldb, R, M, ldm, w,
                                                                   chunk, stream_hint, nrows);
    else
        k_mttkrp_rootpass<N, KW, L, BF16, 1><<<grid, 256, 0, s>>>(klo, khi, val, cnt, bits, B, ldb, R, M, ldm, w,
                                                                  chunk, stream_hint, nrows);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

template <int N, int KW, int L, bool BF16>
sym_status launch_mttkrp_shape(const sym_tensor_s* X, const void* B, int R, int64_t ldb, float* M, int64_t ldm,
                               const sym_mttkrp_cfg& cfg, cudaStream_t s) {
    const int64_t ns = X->nnz_strict, nd = X->nnz - X->nnz_strict;
    const int fact[6] = {1, 1, 2, 6, 24, 120};
    const int sms = sm_count();
    const int threads = std::max(64, std::min(512, (int)cfg.threads_per_cta)) / 32 * 32;
    const SideLaunch* side = (ns > 0 && nd > 0) ? t_side_launch : nullptr;
    cudaStream_t ds = s;  // the diagonal stream's kernel
    if (side) {
        SYM_CUDA(cudaEventRecord(side->fork, s));
        SYM_CUDA(cudaStreamWaitEvent(side->stream, side->fork, 0));
        ds = side->stream;
    }
    if (ns > 0) {
        if (cfg.strict_kernel == SYM_MTTKRP_PLAIN) {
            const int64_t chunk = cfg.entries_per_warp > 0 ? cfg.entries_per_warp : 256;
            const int64_t warps = (ns + chunk - 1) / chunk;
            const unsigned grid = (unsigned)((warps * 32 + MT_THREADS - 1) / MT_THREADS);
            const bool leaf_pass = cfg.leaf_index != 0 && X->rklo != nullptr;
            constexpr int L2 = L / 2;   // lanes per entry with 8 columns per lane
            // carveout preference: as much of the unified L1 / shared memory as L1 as leaves room for the
            // combined root flush's shared memory in every CTA an SM can hold, or the driver default
            const size_t rf_smem = cfg.root_combine ? root_flush_smem<L>() : 0;
            SYM_CUDA(cudaFuncSetAttribute(k_mttkrp_strict<N, KW, L, BF16, 0>,
                                          cudaFuncAttributePreferredSharedMemoryCarveout,
                                          cfg.l1_pref ? l1_carveout_pct(rf_smem) : (int)cudaSharedmemCarveoutDefault));
            if (!leaf_pass && cfg.vec_per_lane == 2 && L2 >= 1) {
                SYM_PROF("mttkrp_strict", s);
                k_mttkrp_strict_wide<N, KW, (L2 >= 1 ? L2 : 1), 2, BF16><<<grid, MT_THREADS, 0, s>>>(
                    X->klo, X->khi, X->val, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1], chunk);
            } else if (!leaf_pass) {
                SYM_PROF("mttkrp_strict", s);
                k_mttkrp_strict<N, KW, L, BF16, 0><<<grid, MT_THREADS, rf_smem, s>>>(
                    X->klo, X->khi, X->val, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1], chunk,
                    cfg.stream_hint, X->n, cfg.root_combine);
            } else {
                {
                    SYM_PROF("mttkrp_strict", s);
                    k_mttkrp_strict<N, KW, L, BF16, 1><<<grid, MT_THREADS, rf_smem, s>>>(
                        X->klo, X->khi, X->val, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1], chunk,
                        cfg.stream_hint, X->n, cfg.root_combine);
                }
                SYM_CHECK_LAUNCH();
                SYM_PROF("mttkrp_strict_leaf", s);
                k_mttkrp_strict<N, KW, L, BF16, 2><<<grid, MT_THREADS, rf_smem, s>>>(
                    X->rklo, X->rkhi, X->rval, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1], chunk,
                    cfg.stream_hint, X->n, cfg.root_combine);
            }
        } else if (cfg.strict_kernel == SYM_MTTKRP_PIPELINED) {
            const SinkPlan sp = plan_sink(X->n, R, cfg.strict_smem_kb, cfg.b_share_pct);
            if (sp.bytes > 48 * 1024)
                SYM_TRY(raise_smem_limit(k_mttkrp_strict_pipe<N, KW, L, BF16>, sp.bytes));
            unsigned grid;
            if (cfg.entries_per_warp > 0) {
                const int64_t warps = (ns + cfg.entries_per_warp - 1) / cfg.entries_per_warp;
                grid = (unsigned)((warps * 32 + threads - 1) / threads);
            } else {
                grid = (unsigned)std::max<int64_t>(
                    1, std::min<int64_t>((int64_t)sms * std::max(1, (int)cfg.ctas_per_sm), (ns + 255) / 256));
            }
            SYM_PROF("mttkrp_strict", s);
            k_mttkrp_strict_pipe<N, KW, L, BF16><<<grid, threads, sp.bytes, s>>>(
                X->klo, X->khi, X->val, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1],
                std::max<int64_t>(0, cfg.entries_per_warp), sp.H, sp.HB);
        } else if (cfg.strict_kernel == SYM_MTTKRP_LANE && X->n <= (1 << 29)) {  // leaf row << 3 fits 32 bits
            // leaf_index = 1 with a leaf index: the canonical stream for every position but the leaf, then
            // the leaf index for its root; otherwise one pass over the canonical stream
            const bool two = cfg.leaf_index != 0 && X->rklo != nullptr;
            const int64_t chunk = cfg.entries_per_warp > 0 ? cfg.entries_per_warp : 256;
            sym_status ls = two ? launch_lane_m<N, KW, L, BF16, 1>(cfg.vec_per_lane, ns, X->klo, X->khi, X->val,
                                                                   X->bits, B, ldb, R, M, ldm, (float)fact[N - 1],
                                                                   chunk, cfg.stream_hint, "mttkrp_strict", s, X->n, cfg.root_combine)
                                : launch_lane_m<N, KW, L, BF16, 0>(cfg.vec_per_lane, ns, X->klo, X->khi, X->val,
                                                                   X->bits, B, ldb, R, M, ldm, (float)fact[N - 1],
                                                                   chunk, cfg.stream_hint, "mttkrp_strict", s, X->n, cfg.root_combine);
            if (ls == SYM_OK && two) {
                if (cfg.strict_smem_kb == 0) {  // root pass unfactorised below the root
                    const int64_t rchunk = cfg.ctas_per_sm > 0 ? 64LL * cfg.ctas_per_sm : 256;
                    ls = launch_rootpass<N, KW, L, BF16>(cfg.vec_per_lane, ns, X->rklo, X->rkhi, X->rval, X->bits, B,
                                                         ldb, R, M, ldm, (float)fact[N - 1], rchunk, cfg.stream_hint,
                                                         s, X->n);
                } else {
                    ls = launch_lane_m<N, KW, L, BF16, 2>(cfg.vec_per_lane, ns, X->rklo, X->rkhi, X->rval, X->bits,
                                                          B, ldb, R, M, ldm, (float)fact[N - 1], chunk,
                                                          cfg.stream_hint, "mttkrp_strict_leaf", s, X->n, cfg.root_combine);
                }
            }
            if (ls != SYM_OK) return ls;
        } else if (cfg.strict_kernel == SYM_MTTKRP_STAGED) {
            const int64_t chunk = cfg.entries_per_warp > 0 ? cfg.entries_per_warp : 256;
            const size_t per_warp = (size_t)2 * 32 * L * stage_lane_bytes<BF16>();
            int st_threads = threads;
            while (st_threads > 64 && per_warp * (st_threads / 32) > 96 * 1024) st_threads /= 2;
            const size_t smem = per_warp * (st_threads / 32);
            if (smem > 48 * 1024)
                SYM_TRY(raise_smem_limit(k_mttkrp_strict_staged<N, KW, L, BF16>, smem));
            const int64_t warps = (ns + chunk - 1) / chunk;
            const unsigned grid = (unsigned)((warps * 32 + st_threads - 1) / st_threads);
            SYM_PROF("mttkrp_strict", s);
            k_mttkrp_strict_staged<N, KW, L, BF16><<<grid, st_threads, smem, s>>>(
                X->klo, X->khi, X->val, ns, X->bits, B, ldb, R, M, ldm, (float)fact[N - 1], chunk);
        } else {
            const int64_t gpc = (threads / 32) * (32 / L);
            const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((ns + gpc - 1) / gpc,
                                                                                     (int64_t)sms * 16));
            SYM_PROF("mttkrp_strict", s);
            k_mttkrp_entries<N, KW, L, BF16><<<grid, threads, 0, s>>>(X->klo, X->khi, X->val, ns, X->bits, B, ldb, R,
                                                                      M, ldm, 0, 0, X->n);
        }
        SYM_CHECK_LAUNCH();
    }
    if (nd > 0) {
        const uint64_t* dlo = X->klo + ns;
        const uint64_t* dhi = X->khi ? X->khi + ns : nullptr;
        const SinkPlan sp = plan_sink(X->n, R, cfg.diag_smem_kb, cfg.b_share_pct);
        if (sp.bytes > 48 * 1024)
            SYM_TRY(raise_smem_limit(k_mttkrp_entries<N, KW, L, BF16>, sp.bytes));
        const int dthreads = sp.bytes > 0 ? 512 : 256;
        const int64_t gpc = (dthreads / 32) * (32 / L);
        const int64_t cap = sp.bytes > 0 ? (int64_t)sms * (sp.bytes > 100 * 1024 ? 1 : 2) : (int64_t)sms * 16;
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nd + gpc - 1) / gpc, cap));
        {
            SYM_PROF("mttkrp_diag", ds);
            k_mttkrp_entries<N, KW, L, BF16><<<grid, dthreads, sp.bytes, ds>>>(dlo, dhi, X->val + ns, nd, X->bits, B,
                                                                               ldb, R, M, ldm, sp.H, sp.HB, X->n);
            SYM_CHECK_LAUNCH();
        }
        if (side) {
            SYM_CUDA(cudaEventRecord(side->join, ds));
            SYM_CUDA(cudaStreamWaitEvent(s, side->join, 0));
        }
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
                            const sym_mttkrp_cfg& cfg, cudaStream_t s) {
    switch (lanes_for_rank(R)) {
        case 1: return launch_mttkrp_shape<N, KW, 1, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        case 2: return launch_mttkrp_shape<N, KW, 2, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        case 4: return launch_mttkrp_shape<N, KW, 4, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        case 8: return launch_mttkrp_shape<N, KW, 8, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        case 16: return launch_mttkrp_shape<N, KW, 16, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        case 32: return launch_mttkrp_shape<N, KW, 32, BF16>(X, B, R, ldb, M, ldm, cfg, s);
        default: return SYM_E_UNSUPPORTED;
    }
}

template <int N>
sym_status launch_mttkrp_impl(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                              int64_t ldm, const sym_mttkrp_cfg& cfg, cudaStream_t s) {
    if (X->kw == 1)
        return bf16 ? launch_mttkrp_kw<N, 1, true>(X, B, R, ldb, M, ldm, cfg, s)
                    : launch_mttkrp_kw<N, 1, false>(X, B, R, ldb, M, ldm, cfg, s);
    return bf16 ? launch_mttkrp_kw<N, 2, true>(X, B, R, ldb, M, ldm, cfg, s)
                : launch_mttkrp_kw<N, 2, false>(X, B, R, ldb, M, ldm, cfg, s);
}

template <int N>
sym_status launch_mttkrp_order(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M,
                               int64_t ldm, const sym_mttkrp_cfg& cfg, cudaStream_t s);

// Entry points shared with the serving runtime (defined in mttkrp.cu).
sym_status mttkrp_core(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, float* M, int64_t ldm,
                       cudaStream_t s);
sym_status residual_launch(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, const float* M,
                           int64_t ldm, double* residual, void* ws, size_t ws_bytes, cudaStream_t s);
// The same with the Gram matrix B^T B (packed upper triangle, FP64) taken from G_in when given (not
// recomputed), else computed into G_out when given (kept for later calls), else into the workspace.
sym_status residual_launch_gram(const sym_tensor_s* X, const void* B, bool bf16, int R, int64_t ldb, const float* M,
                                int64_t ldm, double* residual, void* ws, size_t ws_bytes, const double* G_in,
                                double* G_out, cudaStream_t s);
size_t residual_ws_bytes(int R);
// G (packed upper triangle r <= s, FP64, overwritten) = B^T B.
sym_status gram_launch(int64_t n, const void* B, bool bf16, int R, int64_t ldb, double* G, cudaStream_t s);
sym_status validate_mttkrp_args(const sym_tensor_s* X, const void* B, sym_dtype bdt, int rank, int64_t ldb,
                                const float* M, int64_t ldm);
sym_status validate_mttkrp_cfg(const sym_mttkrp_cfg* c);

}  // namespace symgpu
