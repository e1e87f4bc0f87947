// Banded batched SSYMV + SYPRD.
//
// Each instance b (n_b rows) is cut into nb = ceil(n_b / W) bands of W rows.
// Its canonical (upper) entries a_ij, j >= i, fall into blocks (I, J) with
// I = i / W <= J = j / W.  A block needs x and y of bands I and J only: the
// row part y[i] += a_ij x_j reads x_J and writes y_I, the mirrored part
// y[j] += a_ij x_i (Sec. 3.1: the one stored entry applied for both of its
// distinct permutations) reads x_I and writes y_J.  With both bands in shared
// memory the random 4-byte gathers and reductions of the CSR kernel, each of
// which costs a 32-byte L2 sector, become shared-memory accesses; y_J is then
// reduced into global memory once per block, coalesced, 16 bytes per lane.
//
// Work unit = one row band (b, I); its CTA keeps x_I / y_I for the whole
// unit and x_J / y_J per block (both double-buffered).  The plan stores the
// unit's entries block by block (row-major inside a block, the CSR order) as a
// packed 4-byte in-band (row, col) pair plus the value: the same canonical
// entries and the same 8 bytes per entry as the CSR's col + val, without the
// row pointers.  Units are assigned to persistent CTAs at plan time (largest
// first, to the least-loaded CTA) and flattened into one task per non-empty
// block.  In each CTA one producer warp walks its task list (itself
// bulk-copied into shared memory), stages the x bands and streams the entries
// through a ring of chunk slots with bulk asynchronous copies (cp.async.bulk,
// full / empty mbarrier pair per slot); the other warps consume.
//
// SYPRD (Sec. 3.2.2, off-diagonal terms twice): each consumer thread carries
// its terms in an FP32 two-sum pair (error-free addition: the pair holds the
// exact sum of the rounded chunk sums), converts it to FP64 at the end of the
// unit; one FP64 partial per unit, summed per instance in a fixed order by the
// batch finaliser.
#include <algorithm>
#include <atomic>
#include <functional>
#include <thread>
#include <new>
#include <queue>
#include <utility>
#include <vector>

#include "spmv_band.cuh"

namespace symgpu {

namespace {

// ---------------------------------------------------------------- PTX: mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 32-bit shared-window accesses (explicit state space: no generic-address checks).
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void reds_add_f32(uint32_t a, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;\n" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the async proxy (the bulk copies).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `parity` to complete; gives up after `limit_ns`
// (2 s in normal runs).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Global -> shared bulk copy; bytes a multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------------- device helpers

// g[0..w) += s[0..w) (or = when `plain`), then s[0..w) = 0.  s is placed in
// shared memory with the same 16-byte phase as g (the y buffers carry a lead
// of 0..3 floats), so the aligned body moves as 16-byte vectors on both
// sides: one shared load, one global vector reduction (skipped when all four
// are zero) and one shared store per 4 elements.  Thread t touches the same
// elements in every pass, so no barrier is needed before the zeroing.
__device__ __forceinline__ void band_flush(float* g, float* s, int w, bool plain, int t, int nt) {
    const int head = min(w, (int)(((16u - ((uint32_t)reinterpret_cast<uintptr_t>(g) & 15u)) & 15u) >> 2));
    for (int k = t; k < head; k += nt) {
        if (plain) {
            g[k] = s[k];
        } else if (s[k] != 0.f) {
            atomicAdd(g + k, s[k]);
        }
        s[k] = 0.f;
    }
    const int nv = (w - head) >> 2;
    float4* sv = reinterpret_cast<float4*>(s + head);
    float4* gv = reinterpret_cast<float4*>(g + head);
    for (int v = t; v < nv; v += nt) {
        const float4 q = sv[v];
        if (plain) {
            gv[v] = q;
        } else if (q.x != 0.f || q.y != 0.f || q.z != 0.f || q.w != 0.f) {
            red_add_f4(reinterpret_cast<float*>(gv + v), q);
        }
        sv[v] = f4_zero();
    }
    for (int k = head + 4 * nv + t; k < w; k += nt) {
        if (plain) {
            g[k] = s[k];
        } else if (s[k] != 0.f) {
            atomicAdd(g + k, s[k]);
        }
        s[k] = 0.f;
    }
}

// Offset (0..3 floats) that gives a shared buffer the 16-byte phase of g.
__device__ __forceinline__ int phase_of(const float* g) {
    return (int)(((uint32_t)reinterpret_cast<uintptr_t>(g) >> 2) & 3u);
}

// A thread's 4 consecutive entries of a block (one 16-byte vector of each
// stream), sorted by (row, col).  MODE 0: diagonal block (I, I), both indices
// in band I; 1: block (I, J) with band J staged; 2: block (I, J) with x_J / y_J
// in global memory (blocks too sparse to stage).  Branch-free: the row part
// is summed over runs of equal rows in registers and reduced once per run
// (predicated on the run's last entry), the mirrored part once per entry.
// Padding entries (only at the end of a block) contribute nothing.
template <int MODE, bool SYPRD>
__device__ __forceinline__ void band_vec4(uint4 pk, float4 av, const float* xI, float* yI, const float* xJ,
                                          float* yJ, float& sp, int wI = 0x7fffffff, int wJ = 0x7fffffff) {
    const uint32_t k[4] = {pk.x, pk.y, pk.z, pk.w};
    const float a[4] = {av.x, av.y, av.z, av.w};
    bool v[4];
    int r[4], c[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[e] = k[e] != BAND_PAD;
        r[e] = v[e] ? (int)(k[e] >> 16) : (e > 0 ? r[e - 1] : 0);
        c[e] = v[e] ? (int)(k[e] & 0xffffu) : 0;
#ifdef SYM_BOUNDS_CHECK
        if (v[e] && (!SYM_INDEX_OK(r[e], wI) || !SYM_INDEX_OK(c[e], MODE == 0 ? wI : wJ))) {
            v[e] = false;  // an in-band pair outside its band: dropped
            r[e] = 0;
            c[e] = 0;
        }
#endif
    }
    float t[4], xr[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        xr[e] = xI[r[e]];
        const float xc = MODE == 0 ? xI[c[e]] : (MODE == 1 ? xJ[c[e]] : __ldg(xJ + c[e]));
        t[e] = v[e] ? a[e] * xc : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool off_diag = MODE != 0 || c[e] != r[e];
        if (v[e] && off_diag) atomicAdd(MODE == 0 ? &yI[c[e]] : &yJ[c[e]], a[e] * xr[e]);
        if (SYPRD) sp = fmaf(off_diag ? 2.f * t[e] : t[e], xr[e], sp);
    }
    float run = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        run = (e > 0 && r[e] == r[e - 1]) ? run + t[e] : t[e];
        // a trailing pad repeats the last row, so the run of the last entry
        // ends at e = 3 (every run holds at least one real entry: e = 0 is one)
        const bool end = e == 3 || r[e + 1 < 4 ? e + 1 : 3] != r[e];
        if (end) atomicAdd(&yI[r[e]], run);
    }
}

// One lane's entries of a chunk of bank groups: groups cw, cw + NC, ... (one
// entry per lane each; the group's rows, and its columns, are spread over the
// 32 banks where the block allows it).  MODE as for band_vec4; shared-memory
// operands are 32-bit shared-window addresses (xI, yI: band I; xJ, yJ: band J
// in modes 0 and 1), band J in global memory in mode 2 (gxJ, gyJ).  The row
// part and the mirrored part are one reduction each; padding contributes nothing.
template <int MODE, bool SYPRD, int EPL>
__device__ __forceinline__ void band_groups(uint32_t gi, uint32_t gv, int m, int first, int stride, uint32_t xI,
                                            uint32_t yI, uint32_t xJ, uint32_t yJ, const float* gxJ, float* gyJ,
                                            float& sp, int wI = 0x7fffffff, int wJ = 0x7fffffff) {
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
        const int e = first + q * stride;
        if (e >= m) break;
        const uint32_t k = lds_u32(gi + 4u * (uint32_t)e);
        if (k == BAND_PAD) break;  // padding only trails a block's last group
        const float a = lds_f32(gv + 4u * (uint32_t)e);
        const uint32_t r4 = (k >> 16) << 2, c4 = (k & 0xffffu) << 2;
        if (!SYM_INDEX_OK(k >> 16, wI) || !SYM_INDEX_OK(k & 0xffffu, MODE == 0 ? wI : wJ)) continue;
        const float xr = lds_f32(xI + r4);
        const float xc = MODE == 2 ? __ldg(gxJ + (c4 >> 2)) : lds_f32((MODE == 0 ? xI : xJ) + c4);
        const float t = a * xc;
        reds_add_f32(yI + r4, t);
        const bool off_diag = MODE != 0 || c4 != r4;
        if (MODE == 2) {
            atomicAdd(gyJ + (c4 >> 2), a * xr);
        } else if (off_diag) {
            reds_add_f32((MODE == 0 ? yI : yJ) + c4, a * xr);
        }
        if (SYPRD) sp = fmaf(off_diag ? 2.f * t : t, xr, sp);
    }
}

// (hi, lo) += v exactly (two-sum, no branch): hi + lo carries every bit of the
// accumulated float sums.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

// What the producer tells the consumers about one ring slot (48 bytes, read
// as three 16-byte vectors).
struct __align__(16) ChunkMeta {
    int64_t base;  // instance's first global row
    int64_t slot;  // SYPRD partial slot of the unit
    int32_t flags; // task flags | CM_* chunk flags
    int32_t m;     // entries in the chunk (multiple of 4)
    int32_t I, J, wI, wJ;
    int32_t leadI, leadJ;  // offset of band I / J inside its staged x buffer
};
constexpr int CM_FIRST_SEG = 1 << 4, CM_LAST_SEG = 1 << 5, CM_END = 1 << 6;
constexpr int TASKS_PER_BUF = 32;  // task records per shared-memory task buffer (two buffers)

// Stages x[src .. src+len) into buf (shared) for the consumers: one bulk copy
// of the 16-byte-aligned superset when x is 16-byte aligned (the copy starts
// `lead` floats before src and never reads past x_end), the few floats it
// cannot cover with plain loads; completion on `bar` (one arrival + bytes).
// Returns lead.
__device__ __forceinline__ int stage_x(float* buf, const float* src, int len, const float* x_end, bool x16,
                                       uint64_t* bar) {
    if (!x16) {
        for (int t = 0; t < len; ++t) buf[t] = src[t];
        mbar_expect_tx(bar, 0);
        return 0;
    }
    const int lead = (int)(((uint32_t)reinterpret_cast<uintptr_t>(src) & 15u) >> 2);
    const float* s0 = src - lead;
    const int tot = lead + len;
    int nvec = tot >> 2;
    if ((tot & 3) && s0 + 4 * (nvec + 1) <= x_end) ++nvec;  // the last vector stays inside x
    for (int t = 4 * nvec; t < tot; ++t) buf[t] = s0[t];
    mbar_expect_tx(bar, (uint32_t)nvec * 16u);
    if (nvec > 0) bulk_g2s(buf, s0, (uint32_t)nvec * 16u, bar);
    return lead;
}

// Copies tasks [t, t + cnt) into a task buffer (completion on bar).
__device__ __forceinline__ void fetch_tasks(BandTask* buf, const BandTask* tasks, int t, int cnt, uint64_t* bar) {
    const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(BandTask);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(buf, tasks + t, bytes, bar);
}

// Warp-specialised persistent kernel.  Warp 0 (one lane) is the producer: it
// walks the CTA's task list, stages x of band I / J into double buffers and
// streams the entries into a ring of `S` chunk slots.  Warps 2.. consume:
// each takes EPL entries per lane of every chunk (bank groups, or 16-byte
// vectors of 4 row-major entries) and never waits for the other consumers:
// it releases a chunk, an x band or a y band with one mbarrier arrival.
// Warp 1 flushes: once every consumer has released a y band it reduces the
// band into global memory, zeroes it and hands it back (y_I with the row
// band's SYPRD partial).  Every wait is bounded (wait_ns, 2 s in normal
// runs); on a timeout the kernel records bit 0 of *err and stops, and the
// producer still waits (bounded) for every copy it issued before it exits.
// skip_chunk >= 0 is a test hook: CTA 0 withholds that chunk of its stream.
template <bool SYPRD, int EPL>
__global__ void __launch_bounds__(1024, 1) k_ssymv_band(const BandTask* __restrict__ tasks,
                                                        const int32_t* __restrict__ cta_ptr,
                                                        const uint32_t* __restrict__ eidx,
                                                        const float* __restrict__ evals, const float* __restrict__ x,
                                                        int64_t x_rows, float* __restrict__ y,
                                                        double* __restrict__ partials, int W, int S,
                                                        unsigned* __restrict__ err, uint64_t wait_ns,
                                                        int64_t skip_chunk) {
    extern __shared__ __align__(128) unsigned char band_smem[];
    __shared__ double s_red[2][32];  // per y_I buffer: one SYPRD partial per consumer warp
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NC = (int)(blockDim.x >> 5) - 2;  // consumer warps (warp 0 produces, warp 1 flushes)
    const int NV = NC * 32;                     // 16-byte vectors per chunk per step (row-major blocks)
    const int CH = NV * EPL;                    // entries per chunk
    const int WB = W + 4;                       // staged x band with its alignment lead
    float* xIb = reinterpret_cast<float*>(band_smem);  // [2][WB]
    float* xJb = xIb + 2 * WB;                          // [2][WB]
    float* yIb = xJb + 2 * WB;                          // [2][WB] (y band with its 16-byte phase lead)
    float* yJb = yIb + 2 * WB;                          // [2][WB]
    uint32_t* ring_i = reinterpret_cast<uint32_t*>(yJb + 2 * WB);
    float* ring_v = reinterpret_cast<float*>(ring_i + (size_t)S * CH);
    BandTask* tbuf = reinterpret_cast<BandTask*>(ring_v + (size_t)S * CH);  // [2][TASKS_PER_BUF]
    ChunkMeta* meta = reinterpret_cast<ChunkMeta*>(tbuf + 2 * TASKS_PER_BUF);
    uint64_t* full = reinterpret_cast<uint64_t*>(meta + S);
    uint64_t* empty = full + S;
    uint64_t* xI_full = empty + S;  // [2]
    uint64_t* xI_empty = xI_full + 2;
    uint64_t* xJ_full = xI_empty + 2;
    uint64_t* xJ_empty = xJ_full + 2;
    uint64_t* t_full = xJ_empty + 2;
    uint64_t* yJ_done = t_full + 2;  // [2] consumers finished a block with this y_J buffer
    uint64_t* yJ_free = yJ_done + 2; // [2] the flusher reduced and zeroed it
    uint64_t* yI_done = yJ_free + 2; // [2] the same for y_I at the end of a row band
    uint64_t* yI_free = yI_done + 2;
    const int t_begin = cta_ptr[blockIdx.x], t_end = cta_ptr[blockIdx.x + 1];
    for (int k = tid; k < 4 * WB; k += blockDim.x) yIb[k] = 0.f;  // y_I and y_J buffers start at zero
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], NC);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&xI_full[k], 1);
            mbar_init(&xJ_full[k], 1);
            mbar_init(&xI_empty[k], NC);
            mbar_init(&xJ_empty[k], NC);
            mbar_init(&t_full[k], 1);
            mbar_init(&yJ_done[k], NC);
            mbar_init(&yJ_free[k], 1);
            mbar_init(&yI_done[k], NC);
            mbar_init(&yI_free[k], 1);
        }
        mbar_init_fence();
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        const bool x16 = ((uintptr_t)x & 15u) == 0;
        const float* x_end = x + x_rows;
        const int ntask = t_end - t_begin;
        const int nbatch = (ntask + TASKS_PER_BUF - 1) / TASKS_PER_BUF;
        for (int b = 0; b < 2 && b < nbatch; ++b)
            fetch_tasks(tbuf + b * TASKS_PER_BUF, tasks, t_begin + b * TASKS_PER_BUF,
                        min(TASKS_PER_BUF, ntask - b * TASKS_PER_BUF), &t_full[b]);
        int64_t k = 0;  // chunks issued
        int pslot = 0;        // ring slot of chunk k (k % S)
        uint32_t pphase = 0;  // (k / S) & 1
        int ucnt = 0, scnt = 0;
        int leadI = 0;
        bool ok = true;
        for (int t = 0; t < ntask && ok; ++t) {
            const int b = t / TASKS_PER_BUF, ti = t % TASKS_PER_BUF;
            if (ti == 0 && !(ok = mbar_wait_bounded(&t_full[b & 1], (uint32_t)((b >> 1) & 1), wait_ns))) break;
            const BandTask T = tbuf[(b & 1) * TASKS_PER_BUF + ti];
            if ((ti == TASKS_PER_BUF - 1 || t == ntask - 1) && b + 2 < nbatch)  // buffer read out: refill it
                fetch_tasks(tbuf + (b & 1) * TASKS_PER_BUF, tasks, t_begin + (b + 2) * TASKS_PER_BUF,
                            min(TASKS_PER_BUF, ntask - (b + 2) * TASKS_PER_BUF), &t_full[b & 1]);
            const int mode = T.flags >> TASK_MODE_SHIFT;
            if (T.flags & TASK_FIRST) {
                const int bI = ucnt & 1;
                if (ucnt >= 2 && !(ok = mbar_wait_bounded(&xI_empty[bI], (uint32_t)(((ucnt >> 1) - 1) & 1), wait_ns)))
                    break;
                leadI = stage_x(xIb + bI * WB, x + T.base + (int64_t)T.I * W, T.wI, x_end, x16, &xI_full[bI]);
                ++ucnt;
            }
            int leadJ = 0;
            if (mode == 1) {
                const int bJ = scnt & 1;
                if (scnt >= 2 && !(ok = mbar_wait_bounded(&xJ_empty[bJ], (uint32_t)(((scnt >> 1) - 1) & 1), wait_ns)))
                    break;
                leadJ = stage_x(xJb + bJ * WB, x + T.base + (int64_t)T.J * W, T.wJ, x_end, x16, &xJ_full[bJ]);
                ++scnt;
            }
            for (int o = 0; o < T.cnt; o += CH, ++k) {
                const int slot = pslot;
                if (k >= S && !(ok = mbar_wait_bounded(&empty[slot], pphase ^ 1u, wait_ns))) break;  // previous use drained
                const int m = min(CH, T.cnt - o);
                if (blockIdx.x == 0 && k == skip_chunk) {
                    // test hook: this chunk is never delivered (no arrival, no copy), so the
                    // consumers' bounded wait on it runs out; nothing is left in flight
                    if (++pslot == S) {
                        pslot = 0;
                        pphase ^= 1u;
                    }
                    continue;
                }
                ChunkMeta& cm = meta[slot];
                cm.base = T.base;
                cm.slot = T.slot;
                cm.m = m;
                cm.I = T.I;
                cm.J = T.J;
                cm.wI = T.wI;
                cm.wJ = T.wJ;
                cm.leadI = leadI;
                cm.leadJ = leadJ;
                cm.flags = (T.flags & ~(TASK_FIRST | TASK_LAST)) | (o == 0 ? CM_FIRST_SEG : 0) |
                           (o + CH >= T.cnt ? CM_LAST_SEG : 0) | (o == 0 ? (T.flags & TASK_FIRST) : 0) |
                           (o + CH >= T.cnt ? (T.flags & TASK_LAST) : 0);
                const uint32_t bytes = (uint32_t)m * 4u;
                mbar_expect_tx(&full[slot], 2u * bytes);
                bulk_g2s(ring_i + (size_t)slot * CH, eidx + T.start + o, bytes, &full[slot]);
                bulk_g2s(ring_v + (size_t)slot * CH, evals + T.start + o, bytes, &full[slot]);
                if (++pslot == S) {
                    pslot = 0;
                    pphase ^= 1u;
                }
            }
        }
        if (ok) {
            const int slot = pslot;
            if (k < S || (ok = mbar_wait_bounded(&empty[slot], pphase ^ 1u, wait_ns))) {
                meta[slot].flags = CM_END;
                mbar_arrive(&full[slot]);
                ++k;
            }
        }
        if (!ok) atomicOr(err, 1u);
        // Every copy issued into this CTA's shared memory lands before the
        // producer thread (and so the CTA) exits.
        for (int64_t j = k > S ? k - S : 0; j < k; ++j) mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1), wait_ns);
        for (int b = 0; b < 2; ++b) {
            const int ui = ucnt - 1 - ((ucnt - 1 - b) & 1);  // last use of x_I buffer b
            if (ui >= 0) mbar_wait_bounded(&xI_full[b], (uint32_t)((ui >> 1) & 1), wait_ns);
            const int si = scnt - 1 - ((scnt - 1 - b) & 1);
            if (si >= 0) mbar_wait_bounded(&xJ_full[b], (uint32_t)((si >> 1) & 1), wait_ns);
            const int bi = nbatch - 1 - ((nbatch - 1 - b) & 1);  // last batch in task buffer b
            if (bi >= 0) mbar_wait_bounded(&t_full[b], (uint32_t)((bi >> 1) & 1), wait_ns);
        }
        return;
    }

    if (warp == 1) {
        // ------------------------------------------------------------ flusher
        // Walks the same task list: when every consumer warp is done with a
        // y band it reduces the band into global memory (16-byte vectors),
        // zeroes it and hands it back; at a row band's end it also sums the
        // consumer warps' SYPRD partials into the unit's FP64 slot.
        int ucnt = 0, scnt = 0;
        for (int t = t_begin; t < t_end; ++t) {
            const BandTask T = tasks[t];
            if ((T.flags >> TASK_MODE_SHIFT) == 1) {
                const int b = scnt & 1;
                if (!mbar_wait_bounded(&yJ_done[b], (uint32_t)((scnt >> 1) & 1), wait_ns)) {
                    if (lane == 0) atomicOr(err, 1u);
                    return;
                }
                float* g = y + T.base + (int64_t)T.J * W;
                band_flush(g, yJb + b * WB + phase_of(g), T.wJ, false, lane, 32);
                __syncwarp();
                if (lane == 0) mbar_arrive(&yJ_free[b]);
                ++scnt;
            }
            if (T.flags & TASK_LAST) {
                const int b = ucnt & 1;
                if (!mbar_wait_bounded(&yI_done[b], (uint32_t)((ucnt >> 1) & 1), wait_ns)) {
                    if (lane == 0) atomicOr(err, 1u);
                    return;
                }
                float* g = y + T.base + (int64_t)T.I * W;
                band_flush(g, yIb + b * WB + phase_of(g), T.wI, (T.flags & TASK_SINGLE) != 0, lane, 32);
                if (SYPRD && lane == 0) {
                    double tot = 0.0;
                    for (int q = 0; q < NC; ++q) tot += s_red[b][q];  // fixed order
                    partials[T.slot] = tot;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&yI_free[b]);
                ++ucnt;
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int cw = warp - 2;
    int ucnt = 0, scnt = 0;
    int bI = 0, bJ = 0;
    float s_hi = 0.f, s_lo = 0.f;
    int slot = 0;         // ring slot of the next chunk
    uint32_t phase = 0;   // its phase parity
    for (;;) {
        if (!mbar_wait_bounded(&full[slot], phase, wait_ns)) {
            if (lane == 0) atomicOr(err, 1u);
            break;
        }
        ChunkMeta cm;
        {
            const int4* src = reinterpret_cast<const int4*>(meta + slot);  // 3 broadcast 16-byte loads
            int4* dst = reinterpret_cast<int4*>(&cm);
            dst[0] = src[0];
            dst[1] = src[1];
            dst[2] = src[2];
        }
        if (cm.flags & CM_END) break;
        const int mode = cm.flags >> TASK_MODE_SHIFT;
        if (cm.flags & TASK_FIRST) {
            bI = ucnt & 1;
            if (!mbar_wait_bounded(&xI_full[bI], (uint32_t)((ucnt >> 1) & 1), wait_ns) ||
                (ucnt >= 2 && !mbar_wait_bounded(&yI_free[bI], (uint32_t)(((ucnt >> 1) - 1) & 1), wait_ns))) {
                if (lane == 0) atomicOr(err, 1u);
                break;
            }
            ++ucnt;
        }
        if ((cm.flags & CM_FIRST_SEG) && mode == 1) {
            bJ = scnt & 1;
            if (!mbar_wait_bounded(&xJ_full[bJ], (uint32_t)((scnt >> 1) & 1), wait_ns) ||
                (scnt >= 2 && !mbar_wait_bounded(&yJ_free[bJ], (uint32_t)(((scnt >> 1) - 1) & 1), wait_ns))) {
                if (lane == 0) atomicOr(err, 1u);
                break;
            }
            ++scnt;
        }
        const float* xI = xIb + bI * WB + cm.leadI;
        float* yI = yIb + bI * WB + phase_of(y + cm.base + (int64_t)cm.I * W);
        const uint4* vi = reinterpret_cast<const uint4*>(ring_i + (size_t)slot * CH);
        const float4* vv = reinterpret_cast<const float4*>(ring_v + (size_t)slot * CH);
        float* yJ1 = yJb + bJ * WB + phase_of(y + cm.base + (int64_t)cm.J * W);  // staged y_J (mode 1)
        float sp = 0.f;
        if (cm.flags & TASK_GROUPED) {
            // groups of 32 entries: warp cw takes groups cw, cw + NC, ...; one entry per lane
            const uint32_t gi = smem_u32(ring_i + (size_t)slot * CH), gv = smem_u32(ring_v + (size_t)slot * CH);
            const int first = cw * BAND_GROUP + lane, stride = NC * BAND_GROUP;
            const uint32_t sxI = smem_u32(xI), syI = smem_u32(yI);
            if (mode == 0) {
                band_groups<0, SYPRD, EPL>(gi, gv, cm.m, first, stride, sxI, syI, sxI, syI, nullptr, nullptr, sp,
                                           cm.wI, cm.wJ);
            } else if (mode == 1) {
                band_groups<1, SYPRD, EPL>(gi, gv, cm.m, first, stride, sxI, syI,
                                           smem_u32(xJb + bJ * WB + cm.leadJ), smem_u32(yJ1), nullptr, nullptr, sp, cm.wI, cm.wJ);
            } else {
                const int64_t off = cm.base + (int64_t)cm.J * W;
                band_groups<2, SYPRD, EPL>(gi, gv, cm.m, first, stride, sxI, syI, 0u, 0u, x + off, y + off, sp,
                                           cm.wI, cm.wJ);
            }
        } else
#pragma unroll
        for (int v = 0; v < (EPL + 3) / 4; ++v) {
            const int e = v * NV + cw * 32 + lane;  // this lane's 16-byte vector of the chunk
            if (4 * e < cm.m) {
                const uint4 pk = vi[e];
                const float4 av = vv[e];
                if (mode == 0) {
                    band_vec4<0, SYPRD>(pk, av, xI, yI, xI, yI, sp, cm.wI, cm.wJ);
                } else if (mode == 1) {
                    band_vec4<1, SYPRD>(pk, av, xI, yI, xJb + bJ * WB + cm.leadJ, yJ1, sp, cm.wI, cm.wJ);
                } else {
                    const int64_t off = cm.base + (int64_t)cm.J * W;
                    band_vec4<2, SYPRD>(pk, av, xI, yI, x + off, y + off, sp, cm.wI, cm.wJ);
                }
            }
        }
        if (SYPRD) two_sum_add(s_hi, s_lo, sp);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot]);
        if (cm.flags & CM_LAST_SEG) {
            // this warp is done with the block: release x_J / y_J (and x_I / y_I at a row band's end)
            double w = 0.0;
            if (SYPRD && (cm.flags & TASK_LAST)) {
                w = warp_sum((double)s_hi + (double)s_lo);
                s_hi = s_lo = 0.f;
            }
            if (lane == 0) {
                if (mode == 1) {
                    mbar_arrive(&xJ_empty[bJ]);
                    mbar_arrive(&yJ_done[bJ]);
                }
                if (cm.flags & TASK_LAST) {
                    if (SYPRD) s_red[bI][cw] = w;
                    mbar_arrive(&xI_empty[bI]);
                    mbar_arrive(&yI_done[bI]);
                }
            }
        }
        if (++slot == S) {
            slot = 0;
            phase ^= 1u;
        }
    }
}

// ---------------------------------------------------------------- plan-time kernels (one warp per unit)

constexpr int PLAN_WARPS = 8;

__global__ void k_band_count(const BandUnit* __restrict__ units, int64_t nunits, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, int W, int32_t* __restrict__ cnt,
                             unsigned* __restrict__ err) {
    __shared__ int32_t hist[PLAN_WARPS][BAND_MAX_BANDS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * PLAN_WARPS + w;
    if (u >= nunits) return;
    const BandUnit U = units[u];
    int32_t* h = hist[w];
    for (int k = lane; k < U.nseg; k += 32) h[k] = 0;
    __syncwarp();
    const int64_t r0 = U.base + (int64_t)U.I * W;
    const int wI = min(W, U.n - U.I * W);
    for (int r = 0; r < wI; ++r) {
        const int64_t p1 = rowptr[r0 + r + 1];
        for (int64_t q = rowptr[r0 + r] + lane; q < p1; q += 32) {
            const int64_t c = (int64_t)col[q] - U.base;  // column inside the instance
            if (c < (int64_t)U.I * W + r) {
                atomicOr(err, 2u);  // below the diagonal
            } else if (c >= U.n) {
                atomicOr(err, 4u);  // outside the instance
            } else {
                atomicAdd(&h[(int)(c / W) - U.I], 1);
            }
        }
    }
    __syncwarp();
    for (int k = lane; k < U.nseg; k += 32) cnt[U.seg0 + k] = h[k];
}

// Writes each unit's entries block by block; inside a block in CSR order
// (stable multi-split of every row by column band), then pads each block.
__global__ void k_band_scatter(const BandUnit* __restrict__ units, int64_t nunits, const BandSeg* __restrict__ segs,
                               const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const float* __restrict__ val, int W, uint32_t* __restrict__ eidx,
                               float* __restrict__ evals) {
    __shared__ int32_t fill[PLAN_WARPS][BAND_MAX_BANDS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * PLAN_WARPS + w;
    if (u >= nunits) return;
    const BandUnit U = units[u];
    int32_t* f = fill[w];
    for (int k = lane; k < U.nseg; k += 32) f[k] = 0;
    __syncwarp();
    const int64_t r0 = U.base + (int64_t)U.I * W;
    const int wI = min(W, U.n - U.I * W);
    for (int r = 0; r < wI; ++r) {
        const int64_t p0 = rowptr[r0 + r], p1 = rowptr[r0 + r + 1];
        for (int64_t q0 = p0; q0 < p1; q0 += 32) {
            const int64_t q = q0 + lane;
            int rel = -1;
            int64_t c = 0;
            if (q < p1) {
                c = (int64_t)col[q] - U.base;
                if (c >= (int64_t)U.I * W + r && c < U.n) rel = (int)(c / W) - U.I;
            }
            const unsigned m = __match_any_sync(0xffffffffu, rel);
            const int rank = __popc(m & lanemask_lt());
            if (rel >= 0) {
                const BandSeg g = segs[U.seg0 + rel];
                const int64_t pos = g.start + f[rel] + rank;
                eidx[pos] = ((uint32_t)r << 16) | (uint32_t)(c - (int64_t)(U.I + rel) * W);
                evals[pos] = val[q];
            }
            __syncwarp();
            if (rel >= 0 && rank == 0) f[rel] += __popc(m);
            __syncwarp();
        }
    }
    for (int k = 0; k < U.nseg; ++k) {
        const BandSeg g = segs[U.seg0 + k];
        for (int e = f[k] + lane; e < g.cnt; e += 32) {
            eidx[g.start + e] = BAND_PAD;
            evals[g.start + e] = 0.f;
        }
    }
}

// ---------------------------------------------------------------- plan-time bank grouping (host)

// Rewrites one block (n_in entries in row-major order, trailing pads) as
// groups of 32 whose rows, and whose columns, fall in distinct banks (mod 32)
// where possible.  Greedy per group: row banks with the most entries left
// first, each taking the column bank with the most entries left that the
// group has not used `cap` times; when a group cannot be filled, cap grows
// for the rest of the block (so every group but the last is full).
// Output: n_out = ceil(E / 32) * 32 entries, the last group padded.
void group_block(const uint32_t* ki, const float* kv, int64_t n_in, uint32_t* out_k, float* out_v, int64_t n_out,
                 std::vector<int64_t>& idx) {
    int32_t cnt[1024] = {0};
    int64_t E = 0;
    for (int64_t e = 0; e < n_in; ++e) {
        const uint32_t k = ki[e];
        if (k == BAND_PAD) continue;
        ++cnt[((k >> 16) & 31u) << 5 | (k & 31u)];
        ++E;
    }
    int64_t head[1024];
    int64_t acc = 0;
    for (int b = 0; b < 1024; ++b) {
        head[b] = acc;
        acc += cnt[b];
    }
    idx.resize((size_t)E);
    {
        int64_t fillp[1024];
        std::copy(head, head + 1024, fillp);
        for (int64_t e = 0; e < n_in; ++e) {
            const uint32_t k = ki[e];
            if (k != BAND_PAD) idx[(size_t)fillp[((k >> 16) & 31u) << 5 | (k & 31u)]++] = e;
        }
    }
    int32_t rowrem[32] = {0}, colrem[32] = {0};
    uint32_t avail[32] = {0};
    for (int i = 0; i < 32; ++i)
        for (int j = 0; j < 32; ++j)
            if (cnt[i * 32 + j]) {
                rowrem[i] += cnt[i * 32 + j];
                colrem[j] += cnt[i * 32 + j];
                avail[i] |= 1u << j;
            }
    int cap = 1;
    int64_t outpos = 0, left = E;
    while (left > 0) {
        const int target = (int)std::min<int64_t>(BAND_GROUP, left);
        int ro[32], co[32];
        for (int a = 0; a < 32; ++a) ro[a] = co[a] = a;
        std::stable_sort(ro, ro + 32, [&](int a, int b) { return rowrem[a] > rowrem[b]; });
        std::stable_sort(co, co + 32, [&](int a, int b) { return colrem[a] > colrem[b]; });
        int usedR[32] = {0}, usedC[32] = {0};
        uint32_t fullC = 0;
        int picks[BAND_GROUP];
        int np = 0;
        for (int pass = 0; pass < cap && np < target; ++pass)
            for (int a = 0; a < 32 && np < target; ++a) {
                const int i = ro[a];
                if (usedR[i] != pass) continue;
                const uint32_t cand = avail[i] & ~fullC;
                if (!cand) continue;
                for (int b2 = 0; b2 < 32; ++b2) {
                    const int j = co[b2];
                    if (!((cand >> j) & 1u)) continue;
                    const int b = i * 32 + j;
                    picks[np++] = b;
                    if (--cnt[b] == 0) avail[i] &= ~(1u << j);
                    --rowrem[i];
                    --colrem[j];
                    ++usedR[i];
                    if (++usedC[j] == cap) fullC |= 1u << j;
                    break;
                }
            }
        if (np < target) {  // cannot fill this group at this cap: undo, relax
            for (int q = 0; q < np; ++q) {
                const int b = picks[q], i = b >> 5, j = b & 31;
                ++cnt[b];
                avail[i] |= 1u << j;
                ++rowrem[i];
                ++colrem[j];
            }
            ++cap;
            continue;
        }
        for (int q = 0; q < np; ++q) {
            const int64_t e = idx[(size_t)head[picks[q]]++];
            out_k[outpos] = ki[e];
            out_v[outpos] = kv[e];
            ++outpos;
        }
        left -= np;
    }
    for (; outpos < n_out; ++outpos) {
        out_k[outpos] = BAND_PAD;
        out_v[outpos] = 0.f;
    }
}

// Regroups every block of the plan (device arrays, row-major layout given by
// `segs` and the real entry counts `cnt`) into bank groups; rewrites segs.
sym_status band_regroup(BandPlan& P, std::vector<BandSeg>& segs, const std::vector<int32_t>& cnt, int64_t n_in,
                        int64_t cap, cudaStream_t s) {
    const size_t nsegs = segs.size();
    std::vector<BandSeg> out(segs);
    int64_t total = 0;
    for (size_t q = 0; q < nsegs; ++q) {
        const int64_t c32 = ((int64_t)cnt[q] + BAND_GROUP - 1) / BAND_GROUP * BAND_GROUP;
        out[q].start = total;
        out[q].cnt = (int32_t)c32;
        total += c32;
    }
    if (total > cap) return SYM_E_NOMEM;
    std::vector<uint32_t> hi, ho;
    std::vector<float> hv, hw;
    try {
        hi.resize((size_t)n_in);
        hv.resize((size_t)n_in);
        ho.resize((size_t)total);
        hw.resize((size_t)total);
    } catch (...) {
        return SYM_E_NOMEM;
    }
    SYM_CUDA(cudaMemcpyAsync(hi.data(), P.eidx, sizeof(uint32_t) * (size_t)n_in, cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaMemcpyAsync(hv.data(), P.evals, sizeof(float) * (size_t)n_in, cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    std::atomic<int64_t> next{0};
    auto work = [&]() {
        std::vector<int64_t> idx;
        for (;;) {
            const int64_t q = next.fetch_add(1);
            if (q >= (int64_t)nsegs) break;
            const BandSeg& a = segs[(size_t)q];
            const BandSeg& b = out[(size_t)q];
            group_block(hi.data() + a.start, hv.data() + a.start, a.cnt, ho.data() + b.start, hw.data() + b.start,
                        b.cnt, idx);
        }
    };
    const unsigned hw_threads = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    try {
        for (unsigned t = 1; t < hw_threads; ++t) pool.emplace_back(work);
    } catch (...) {
        // fewer threads: the calling thread still does all remaining work
    }
    work();
    for (auto& t : pool) t.join();
    SYM_CUDA(cudaMemcpyAsync(P.eidx, ho.data(), sizeof(uint32_t) * (size_t)total, cudaMemcpyHostToDevice, s));
    SYM_CUDA(cudaMemcpyAsync(P.evals, hw.data(), sizeof(float) * (size_t)total, cudaMemcpyHostToDevice, s));
    SYM_CUDA(cudaStreamSynchronize(s));  // the host buffers die here
    segs.swap(out);
    P.nentries = total;
    return SYM_OK;
}

int plan_grid(const sym_tile_cfg* cfg) { return sm_count() * cfg->ctas_per_sm; }

int band_epl(const sym_tile_cfg* cfg) { return cfg->band_chunk > 0 ? cfg->band_chunk : 4; }

void count_units(const int64_t* hro, int64_t count, const sym_tile_cfg* cfg, int64_t* nunits, int64_t* nsegs) {
    *nunits = 0;
    *nsegs = 0;
    for (int64_t b = 0; b < count; ++b) {
        const int nb = band_count(hro[b + 1] - hro[b], cfg);
        *nunits += nb;
        *nsegs += (int64_t)nb * (nb + 1) / 2;
    }
}

template <typename C>
void band_layout(C& c, BandPlan& P, int64_t nunits, int64_t nsegs, int64_t cap, int grid, int32_t** counts) {
    P.units = c.template take<BandUnit>((size_t)std::max<int64_t>(nunits, 1));
    P.segs = c.template take<BandSeg>((size_t)std::max<int64_t>(nsegs, 1));
    P.tasks = c.template take<BandTask>((size_t)std::max<int64_t>(nsegs, 1));
    P.cta_ptr = c.template take<int32_t>((size_t)grid + 1);
    *counts = c.template take<int32_t>((size_t)std::max<int64_t>(nsegs, 1));
    P.eidx = c.template take<uint32_t>((size_t)std::max<int64_t>(cap, 4));
    P.evals = c.template take<float>((size_t)std::max<int64_t>(cap, 4));
    P.err = c.template take<unsigned>(1);
}

struct SizerCarver {
    Sizer& s;
    template <typename T>
    T* take(size_t n) {
        s.take<T>(n);
        return nullptr;
    }
};

template <bool SYPRD, int EPL>
sym_status launch_band_v(const BandPlan& P, const float* x, float* y, double* partials, cudaStream_t s) {
    SYM_TRY(raise_smem_limit(k_ssymv_band<SYPRD, EPL>, P.smem));
    k_ssymv_band<SYPRD, EPL><<<P.grid, P.threads, P.smem, s>>>(P.tasks, P.cta_ptr, P.eidx, P.evals, x, P.x_rows, y,
                                                                partials, P.W, P.stages, P.err, P.wait_ns,
                                                                P.skip_chunk);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

template <bool SYPRD>
sym_status launch_band(const BandPlan& P, const float* x, float* y, double* partials, cudaStream_t s) {
    switch (P.epl) {
        case 1: return launch_band_v<SYPRD, 1>(P, x, y, partials, s);
        case 2: return launch_band_v<SYPRD, 2>(P, x, y, partials, s);
        case 4: return launch_band_v<SYPRD, 4>(P, x, y, partials, s);
        case 8: return launch_band_v<SYPRD, 8>(P, x, y, partials, s);
        case 16: return launch_band_v<SYPRD, 16>(P, x, y, partials, s);
        default: return SYM_E_INVALID;
    }
}

}  // namespace

int band_count(int64_t n, const sym_tile_cfg* cfg) {
    if (!cfg || cfg->band_rows <= 0 || n <= 0) return 0;
    const int64_t nb = (n + cfg->band_rows - 1) / cfg->band_rows;
    return nb <= cfg->band_max ? (int)nb : 0;
}

size_t band_smem(const sym_tile_cfg* cfg, int* stages) {
    *stages = 0;
    if (!cfg || cfg->band_rows <= 0 || cfg->ctas_per_sm < 1 || cfg->threads_per_cta < 96) return 0;
    const int epl = band_epl(cfg);
    if (epl != 1 && epl != 2 && epl != 4 && epl != 8 && epl != 16) return 0;
    int optin = 0, per_sm = 0;
    const int dev = current_device();
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        // no device (CPU-only host): GB300 figures, so sizes can still be queried
        optin = 232448;
        per_sm = 233472;
    }
    const int64_t budget =
        std::min<int64_t>(optin, per_sm / cfg->ctas_per_sm - 1024) - (int64_t)sizeof(double) * 64 - 64;
    // x_I, x_J double buffers (W + 4 floats each), y_I, y_J double buffers,
    // two task buffers, the x / task barriers; then per ring slot the chunk,
    // its ChunkMeta and its two barriers
    const int64_t fixed = 4LL * (8LL * cfg->band_rows + 32) + 2LL * TASKS_PER_BUF * (int64_t)sizeof(BandTask) + 18 * 8;
    const int64_t chunk = 32LL * epl * (cfg->threads_per_cta / 32 - 2);  // entries
    const int64_t per_stage = chunk * 8 + (int64_t)sizeof(ChunkMeta) + 16;
    const int64_t st = std::min<int64_t>(16, (budget - fixed) / per_stage);
    if (st < 2) return 0;
    *stages = (int)st;
    return (size_t)(fixed + st * per_stage);
}

void band_size(Sizer& s, const sym_csr_batch* A, const int64_t* hro, const sym_tile_cfg* cfg) {
    int64_t nunits, nsegs;
    count_units(hro, A->count, cfg, &nunits, &nsegs);
    if (nunits == 0) return;
    BandPlan P;
    int32_t* counts;
    SizerCarver c{s};
    band_layout(c, P, nunits, nsegs, A->total_nnz + 31 * nsegs, plan_grid(cfg), &counts);
}

sym_status band_build(BandPlan& P, Carver& c, const sym_csr_batch* A, const int64_t* hro, const sym_tile_cfg* cfg,
                      const std::vector<int64_t>& slot_of, cudaStream_t s) {
    P = BandPlan();
    int64_t nunits, nsegs;
    count_units(hro, A->count, cfg, &nunits, &nsegs);
    if (nunits == 0) return SYM_OK;
    if (nsegs > 0x3fffffffLL || nunits > 0x3fffffffLL) return SYM_E_UNSUPPORTED;
    const int W = cfg->band_rows;
    P.W = W;
    P.threads = cfg->threads_per_cta;
    P.epl = band_epl(cfg);
    P.order = cfg->band_order;
    P.smem = band_smem(cfg, &P.stages);
    if (P.stages < 2) return SYM_E_INVALID;
    P.grid = plan_grid(cfg);
    P.nunits = nunits;
    P.nsegs = nsegs;
    P.x_rows = A->total_rows;
    const int64_t cap = A->total_nnz + 31 * nsegs;
    int32_t* counts = nullptr;
    band_layout(c, P, nunits, nsegs, cap, P.grid, &counts);
    if (!P.err) return SYM_E_NOMEM;

    std::vector<BandUnit> units;
    std::vector<int32_t> cnt;
    std::vector<BandSeg> segs;
    try {
        units.reserve((size_t)nunits);
        cnt.resize((size_t)nsegs);
        segs.resize((size_t)nsegs);
    } catch (...) {
        return SYM_E_NOMEM;
    }
    int64_t seg = 0;
    for (int64_t b = 0; b < A->count; ++b) {
        const int64_t n = hro[b + 1] - hro[b];
        const int nb = band_count(n, cfg);
        for (int I = 0; I < nb; ++I) {
            units.push_back(BandUnit{hro[b], slot_of[(size_t)b] + I, (int32_t)n, I, (int32_t)seg, nb - I});
            seg += nb - I;
        }
    }
    SYM_CUDA(cudaMemcpyAsync(P.units, units.data(), sizeof(BandUnit) * units.size(), cudaMemcpyHostToDevice, s));
    SYM_CUDA(cudaMemsetAsync(P.err, 0, sizeof(unsigned), s));
    const unsigned pg = (unsigned)((nunits + PLAN_WARPS - 1) / PLAN_WARPS);
    k_band_count<<<pg, 32 * PLAN_WARPS, 0, s>>>(P.units, nunits, A->rowptr, A->col, W, counts, P.err);
    SYM_CHECK_LAUNCH();
    unsigned herr = 0;
    SYM_CUDA(cudaMemcpyAsync(cnt.data(), counts, sizeof(int32_t) * cnt.size(), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaMemcpyAsync(&herr, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    SYM_CUDA(cudaStreamSynchronize(s));
    if (herr & 2u) return SYM_E_NONCANONICAL;
    if (herr & 4u) return SYM_E_RANGE;

    // Block layout (row-major, padded to 4 entries) and staging decision.
    int64_t start = 0;
    for (int64_t k = 0; k < nunits; ++k) {
        const BandUnit& U = units[(size_t)k];
        for (int q = 0; q < U.nseg; ++q) {
            const int64_t sgi = U.seg0 + q;
            const int J = U.I + q;
            const int wJ = std::min<int>(W, U.n - J * W);
            const int64_t c4 = ((int64_t)cnt[(size_t)sgi] + 3) & ~3LL;
            const bool staged = q == 0 || 8 * c4 >= wJ;
            segs[(size_t)sgi] = BandSeg{start, (int32_t)c4, J | (staged ? BAND_STAGED : 0)};
            start += c4;
        }
    }
    if (start > cap) return SYM_E_NOMEM;
    P.nentries = start;
    SYM_CUDA(cudaMemcpyAsync(P.segs, segs.data(), sizeof(BandSeg) * segs.size(), cudaMemcpyHostToDevice, s));
    k_band_scatter<<<pg, 32 * PLAN_WARPS, 0, s>>>(P.units, nunits, P.segs, A->rowptr, A->col, A->val, W, P.eidx,
                                                  P.evals);
    SYM_CHECK_LAUNCH();
    SYM_CUDA(cudaStreamSynchronize(s));  // segs (host) is rewritten below
    if (P.order == 1) {
        const sym_status gs = band_regroup(P, segs, cnt, start, cap, s);
        if (gs != SYM_OK) return gs;
    }

    // Unit cost (entries + staged floats), then largest unit first, each to the
    // least-loaded CTA; units without entries are left out.
    std::vector<double> cost((size_t)nunits, 0.0);
    for (int64_t k = 0; k < nunits; ++k) {
        const BandUnit& U = units[(size_t)k];
        const int wI = std::min<int>(W, U.n - U.I * W);
        bool any = false;
        for (int q = 0; q < U.nseg; ++q) {
            const BandSeg& g = segs[(size_t)(U.seg0 + q)];
            if (g.cnt == 0) continue;
            any = true;
            cost[(size_t)k] += (double)g.cnt + (q > 0 && (g.code & BAND_STAGED) ? std::min<int>(W, U.n - (U.I + q) * W) : 0);
        }
        if (any) cost[(size_t)k] += wI;
    }
    std::vector<int64_t> order;
    order.reserve((size_t)nunits);
    for (int64_t k = 0; k < nunits; ++k)
        if (cost[(size_t)k] > 0) order.push_back(k);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[(size_t)a] > cost[(size_t)b]; });
    std::vector<std::vector<int32_t>> lists((size_t)P.grid);
    using Load = std::pair<double, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int g = 0; g < P.grid; ++g) heap.push(Load{0.0, g});
    for (int64_t k : order) {
        Load l = heap.top();
        heap.pop();
        lists[(size_t)l.second].push_back((int32_t)k);
        l.first += cost[(size_t)k];
        heap.push(l);
    }
    // One task per non-empty block, unit by unit.
    std::vector<BandTask> tasks;
    std::vector<int32_t> cta_ptr((size_t)P.grid + 1, 0);
    try {
        tasks.reserve((size_t)nsegs);
    } catch (...) {
        return SYM_E_NOMEM;
    }
    for (int g = 0; g < P.grid; ++g) {
        cta_ptr[(size_t)g] = (int32_t)tasks.size();
        for (int32_t k : lists[(size_t)g]) {
            const BandUnit& U = units[(size_t)k];
            const int nb = (U.n + W - 1) / W;
            const int wI = std::min<int>(W, U.n - U.I * W);
            const size_t first = tasks.size();
            for (int q = 0; q < U.nseg; ++q) {
                const BandSeg& g2 = segs[(size_t)(U.seg0 + q)];
                if (g2.cnt == 0) continue;
                const int J = U.I + q;
                const int mode = q == 0 ? 0 : ((g2.code & BAND_STAGED) ? 1 : 2);
                const int flags = (mode << TASK_MODE_SHIFT) | (nb == 1 ? TASK_SINGLE : 0) |
                                  (P.order == 1 ? TASK_GROUPED : 0);
                tasks.push_back(BandTask{g2.start, U.base, U.slot, g2.cnt, flags, U.I, J, wI,
                                         std::min<int>(W, U.n - J * W)});
            }
            tasks[first].flags |= TASK_FIRST;
            tasks.back().flags |= TASK_LAST;
        }
    }
    cta_ptr[(size_t)P.grid] = (int32_t)tasks.size();
    P.ntasks = (int64_t)tasks.size();
    SYM_CUDA(cudaMemcpyAsync(P.cta_ptr, cta_ptr.data(), sizeof(int32_t) * cta_ptr.size(), cudaMemcpyHostToDevice, s));
    if (!tasks.empty())
        SYM_CUDA(cudaMemcpyAsync(P.tasks, tasks.data(), sizeof(BandTask) * tasks.size(), cudaMemcpyHostToDevice, s));
    SYM_CUDA(cudaStreamSynchronize(s));  // the host vectors above die here
    return SYM_OK;
}

sym_status band_enqueue(const BandPlan& P, const float* x, float* y, double* partials, bool syprd, cudaStream_t s) {
    if (P.ntasks == 0) return SYM_OK;
    SYM_PROF("ssymv_band", s);
    return syprd ? launch_band<true>(P, x, y, partials, s) : launch_band<false>(P, x, y, partials, s);
}

}  // namespace symgpu
