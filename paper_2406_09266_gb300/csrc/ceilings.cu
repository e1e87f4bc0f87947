// Measured ceilings of the operations the symmetric kernels are made of.
//
// The symmetric MTTKRP reads its tensor stream once (a few bytes per entry), so
// DRAM bandwidth is not what bounds it: each canonical entry gathers factor rows
// and adds into output rows that sit in L2 (or in shared memory for hot rows).
// These kernels time those primitive operations alone on the running GPU, so a
// kernel's throughput can be stated as a fraction of the ceiling that binds it:
//   FMA          FP32 fused multiply-add issue (FLOP/s);
//   ROW_GATHER   random rows of R floats read from an L2-resident table (rows/s);
//   ROW_RED      random rows of R floats reduced with 16-byte vector `red` (rows/s);
//   GATHER_RED   one random gather plus one random reduction per entry (entries/s),
//                the per-entry pattern of a leaf update in global memory;
//   SMEM_F32     a row of R floats added with float atomics into a shared-memory
//                table of `rows` rows (rows/s), the hot-row sink of the MTTKRP;
//   SMEM_U32     the same with 32-bit integer atomics (reference point);
//   HBM_COPY     streaming copy of half the buffer onto the other half (bytes/s).
// A lane group of R/4 lanes handles one row, each lane 4 consecutive floats, as
// in the MTTKRP kernels.  Row numbers come from a counter-based 32-bit mixer
// (the MurmurHash3 finaliser), so no index array is streamed.
#include <algorithm>

#include "common.cuh"

namespace symgpu {
namespace {

constexpr int CEIL_THREADS = 256;

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Uniform row in [0, n) from a 32-bit hash (multiply-high).
__device__ __forceinline__ int64_t pick_row(uint32_t h, int64_t n) {
    return (int64_t)(((uint64_t)h * (uint64_t)n) >> 32);
}

__global__ void __launch_bounds__(CEIL_THREADS) k_ceil_fma(float* out, int64_t iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3f * (float)threadIdx.x + (float)k;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.0f) out[blockIdx.x & 1023] = s;  // keeps the chains alive; never true for these inputs
}

// MODE 0 gather, 1 reduction, 2 gather + reduction.
template <int L, int MODE>
__global__ void __launch_bounds__(CEIL_THREADS) k_ceil_rows(const float* __restrict__ Bt, float* __restrict__ Mt,
                                                          int64_t n, int R, int64_t iters, float* out) {
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane % L);
    const int64_t group = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / L) + lane / L;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x >> 5) * (32 / L);
    float4 acc = f4_zero();
    const float4 one = make_float4(1.f, 1.f, 1.f, 1.f);
    for (int64_t it = 0; it < iters; ++it) {
        const uint32_t h = fmix32((uint32_t)(it * ngroups + group) * 2u + 1u);
        if (MODE != 1) {
            const int64_t r = pick_row(h, n);
            const float4 v = __ldg(reinterpret_cast<const float4*>(Bt + r * R + col));
            acc = make_float4(acc.x + v.x, acc.y + v.y, acc.z + v.z, acc.w + v.w);
        }
        if (MODE != 0) {
            const int64_t r = pick_row(MODE == 2 ? fmix32(h) : h, n);
            red_add_f4(Mt + r * R + col, one);
        }
    }
    if (MODE != 1 && acc.x == -1.0f) out[0] = acc.y + acc.z + acc.w;  // keeps the loads alive
}

// Row adds into a shared-memory table of H rows.  U32: integer atomics.  The
// lane's four adds start at a rotated column so the 32 lanes of a warp (two
// rows at R = 64) meet 32 distinct banks.
template <int L, bool U32>
__global__ void __launch_bounds__(CEIL_THREADS) k_ceil_smem(int H, int R, int64_t iters, float* out) {
    extern __shared__ float4 ceil_smem[];
    float* tab = reinterpret_cast<float*>(ceil_smem);
    for (int k = threadIdx.x; k < H * R; k += blockDim.x) tab[k] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int col = 4 * (lane % L);
    const int rot = lane + (lane >> 3);
    const int64_t group = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / L) + lane / L;
    const int64_t ngroups = ((int64_t)gridDim.x * blockDim.x >> 5) * (32 / L);
    for (int64_t it = 0; it < iters; ++it) {
        const uint32_t h = fmix32((uint32_t)(it * ngroups + group) * 2u + 1u);
        const int64_t row = pick_row(h, H);
        if (row < 0 || row >= H || col + 3 >= R) {  // cannot happen: recorded instead of accessed
            atomicOr(reinterpret_cast<unsigned*>(out) + 1023, 1u);
            continue;
        }
        float* p = tab + row * R + col;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = (k + rot) & 3;
            if (U32)
                atomicAdd(reinterpret_cast<unsigned*>(p + j), 1u);
            else
                atomicAdd(p + j, 1.0f);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && tab[0] == -1.0f) out[blockIdx.x & 1023] = tab[1];
}

// ---------------------------------------------------------------- bulk-copy (TMA engine) row operations

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Lane 0 of each warp moves CEIL_BULK rows per iteration with single-instruction
// bulk copies: BULK_GATHER copies random rows of B (R floats each) into the
// warp's shared buffer (completion counted on an mbarrier; the wait is bounded
// and records a timeout instead of hanging); BULK_RED reduces the warp's shared
// buffer into random rows of M (cp.reduce.async.bulk .add.f32), waiting for the
// reads of the previous group before the next one.  Rows/s = CEIL_BULK x
// iterations x warps / time.
constexpr int CEIL_BULK = 8;

template <bool RED>
__global__ void __launch_bounds__(CEIL_THREADS) k_ceil_bulk(const float* __restrict__ Bt, float* __restrict__ Mt,
                                                          int64_t n, int R, int64_t iters, float* out) {
    extern __shared__ __align__(128) unsigned char bulk_smem[];
    __shared__ __align__(8) uint64_t bar[CEIL_THREADS / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t row_bytes = (uint32_t)R * 4u;
    float* buf = reinterpret_cast<float*>(bulk_smem) + (size_t)warp * CEIL_BULK * R;
    for (int k = lane; k < CEIL_BULK * R; k += 32) buf[k] = 1.0f;
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar[warp])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the buffer is visible to the bulk copies
    __syncwarp();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    uint32_t phase = 0;
    for (int64_t it = 0; it < iters; ++it) {
        if (lane == 0) {
            if (!RED)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(&bar[warp])),
                             "r"(row_bytes * CEIL_BULK)
                             : "memory");
#pragma unroll
            for (int k = 0; k < CEIL_BULK; ++k) {
                const uint32_t h = fmix32((uint32_t)((it * nw + gw) * CEIL_BULK + k) * 2u + 1u);
                const int64_t r = pick_row(h, n);
                if (RED)
                    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;\n" ::"l"(
                                     Mt + r * R),
                                 "r"(smem_addr(buf + k * R)), "r"(row_bytes)
                                 : "memory");
                else
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                            smem_addr(buf + k * R)),
                        "l"(Bt + r * R), "r"(row_bytes), "r"(smem_addr(&bar[warp]))
                        : "memory");
            }
            if (RED) {
                asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
                asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
            }
        }
        if (!RED) {
            // bounded wait for this iteration's rows (records a timeout, never hangs): lane 0 waits and the
            // warp follows its verdict, so every lane leaves the loop together; on a timeout lane 0 waits once
            // more, bounded, for the copies still in flight, then the warp stops
            uint32_t ok = 0;
            if (lane == 0) {
                for (int spin = 0; spin < (1 << 22) && !ok; ++spin)
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, "
                        "1, 0, p;\n}\n"
                        : "=r"(ok)
                        : "r"(smem_addr(&bar[warp])), "r"(phase)
                        : "memory");
                if (!ok) {
                    atomicOr(reinterpret_cast<unsigned*>(out) + 1023, 2u);
                    uint32_t late = 0;
                    for (int spin = 0; spin < (1 << 22) && !late; ++spin)
                        asm volatile(
                            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 "
                            "%0, 1, 0, p;\n}\n"
                            : "=r"(late)
                            : "r"(smem_addr(&bar[warp])), "r"(phase)
                            : "memory");
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            // the other lanes observe the completed phase too before reading the rows
            if (lane != 0) {
                uint32_t seen = 0;
                for (int spin = 0; spin < 64 && !seen; ++spin)
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 "
                        "%0, 1, 0, p;\n}\n"
                        : "=r"(seen)
                        : "r"(smem_addr(&bar[warp])), "r"(phase)
                        : "memory");
            }
            phase ^= 1u;
            acc += buf[lane % R];
            __syncwarp();  // every lane has read before the next copies overwrite the buffer
        }
    }
    if (RED && lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    if (acc == -1.0f) out[0] = acc;
}

__global__ void k_ceil_copy(const float4* __restrict__ a, float4* __restrict__ b, int64_t n4) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += (int64_t)gridDim.x * blockDim.x)
        b[k] = __ldcs(a + k);
}

template <int L>
sym_status launch_rows(int kind, float* buf, int64_t n, int R, int64_t iters, unsigned grid, size_t smem, int H,
                       cudaStream_t s) {
    const bool on_chip = kind == SYM_CEIL_SMEM_F32 || kind == SYM_CEIL_SMEM_U32;
    float* Bt = buf;
    float* Mt = on_chip ? buf : buf + n * R;
    float* out = on_chip ? buf : buf + 2 * n * R;
    switch (kind) {
        case SYM_CEIL_ROW_GATHER:
            k_ceil_rows<L, 0><<<grid, CEIL_THREADS, 0, s>>>(Bt, Mt, n, R, iters, out);
            break;
        case SYM_CEIL_ROW_RED:
            k_ceil_rows<L, 1><<<grid, CEIL_THREADS, 0, s>>>(Bt, Mt, n, R, iters, out);
            break;
        case SYM_CEIL_GATHER_RED:
            k_ceil_rows<L, 2><<<grid, CEIL_THREADS, 0, s>>>(Bt, Mt, n, R, iters, out);
            break;
        case SYM_CEIL_SMEM_F32:
            SYM_TRY(raise_smem_limit(k_ceil_smem<L, false>, smem));
            k_ceil_smem<L, false><<<grid, CEIL_THREADS, smem, s>>>(H, R, iters, out);
            break;
        case SYM_CEIL_SMEM_U32:
            SYM_TRY(raise_smem_limit(k_ceil_smem<L, true>, smem));
            k_ceil_smem<L, true><<<grid, CEIL_THREADS, smem, s>>>(H, R, iters, out);
            break;
        case SYM_CEIL_BULK_GATHER:
            SYM_TRY(raise_smem_limit(k_ceil_bulk<false>, smem));
            k_ceil_bulk<false><<<grid, CEIL_THREADS, smem, s>>>(Bt, Mt, n, R, iters, out);
            break;
        case SYM_CEIL_BULK_RED:
            SYM_TRY(raise_smem_limit(k_ceil_bulk<true>, smem));
            k_ceil_bulk<true><<<grid, CEIL_THREADS, smem, s>>>(Bt, Mt, n, R, iters, out);
            break;
        default:
            return SYM_E_INVALID;
    }
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

bool bulk_kind(int kind) { return kind == SYM_CEIL_BULK_GATHER || kind == SYM_CEIL_BULK_RED; }
bool row_kind(int kind) { return (kind >= SYM_CEIL_ROW_GATHER && kind <= SYM_CEIL_SMEM_U32) || bulk_kind(kind); }
bool smem_kind(int kind) { return kind == SYM_CEIL_SMEM_F32 || kind == SYM_CEIL_SMEM_U32; }

}  // namespace
}  // namespace symgpu

using namespace symgpu;

extern "C" size_t sym_ceiling_bytes(int kind, int64_t rows, int rank) {
    if (kind == SYM_CEIL_FMA) return 4096;
    if (kind == SYM_CEIL_HBM_COPY) return rows > 0 ? (size_t)rows * 16 * 2 : 0;
    if (smem_kind(kind)) return rows > 0 ? 4096 : 0;
    if (!row_kind(kind) || rows <= 0 || rank < 4 || rank > 128 || rank % 4) return 0;
    return (size_t)2 * rows * rank * sizeof(float) + 4096;
}

extern "C" sym_status sym_ceiling_run(int kind, void* buf, size_t buf_bytes, int64_t rows, int rank, int64_t ops,
                                      int reps, sym_stream_t stream, double* rate, float* ms) {
    if (!buf || !rate || !ms || reps < 1 || reps > 1000 || ops < 0) return SYM_E_INVALID;
    if (!aligned(buf, 256)) return SYM_E_INVALID;
    const size_t need = sym_ceiling_bytes(kind, rows, rank);
    if (need == 0) return SYM_E_INVALID;
    if (buf_bytes < need) return SYM_E_NOMEM;
    cudaStream_t s = as_stream(stream);
    const int sms = sm_count();
    int lanes = 1;
    while (4 * lanes < rank) lanes <<= 1;
    if (row_kind(kind) && 4 * lanes != rank) return SYM_E_INVALID;  // one full lane group per row
    size_t smem = 0;
    if (smem_kind(kind)) {
        smem = (size_t)rows * rank * sizeof(float);
        if (rows < 1 || smem > 200 * 1024) return SYM_E_INVALID;
    }
    if (bulk_kind(kind)) smem = (size_t)(CEIL_THREADS / 32) * CEIL_BULK * rank * sizeof(float);
    // Launch shape: 8 CTAs of 256 threads per SM (row kinds: as resident as
    // shared memory allows), each group doing iters row operations.
    int ctas_per_sm = 8;
    if (smem_kind(kind)) ctas_per_sm = std::max<int>(1, std::min<int>(8, (int)((220 * 1024) / std::max<size_t>(smem, 1))));
    const unsigned grid = (unsigned)(sms * ctas_per_sm);
    if (bulk_kind(kind)) ctas_per_sm = std::max<int>(1, std::min<int>(8, (int)((200 * 1024) / smem)));
    const unsigned grid_b = (unsigned)(sms * ctas_per_sm);
    const int64_t groups = bulk_kind(kind) ? (int64_t)grid_b * (CEIL_THREADS / 32) * CEIL_BULK
                                           : (int64_t)grid * (CEIL_THREADS / 32) * (row_kind(kind) ? (32 / lanes) : 1);
    const int64_t iters = std::max<int64_t>(1, ops / std::max<int64_t>(groups, 1));
    float* fb = static_cast<float*>(buf);

    auto launch = [&]() -> sym_status {
        if (kind == SYM_CEIL_FMA) {
            k_ceil_fma<<<grid, CEIL_THREADS, 0, s>>>(fb, iters, 0.999f, 1e-3f);
            SYM_CHECK_LAUNCH();
            return SYM_OK;
        }
        if (kind == SYM_CEIL_HBM_COPY) {
            const int64_t n4 = rows;  // float4 elements per half
            k_ceil_copy<<<(unsigned)(sms * 8), 512, 0, s>>>(reinterpret_cast<const float4*>(buf),
                                                           reinterpret_cast<float4*>(buf) + n4, n4);
            SYM_CHECK_LAUNCH();
            return SYM_OK;
        }
        if (bulk_kind(kind)) return launch_rows<1>(kind, fb, rows, rank, iters, grid_b, smem, (int)rows, s);
        switch (lanes) {
            case 1: return launch_rows<1>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            case 2: return launch_rows<2>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            case 4: return launch_rows<4>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            case 8: return launch_rows<8>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            case 16: return launch_rows<16>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            case 32: return launch_rows<32>(kind, fb, rows, rank, iters, grid, smem, (int)rows, s);
            default: return SYM_E_INVALID;
        }
    };
    if (row_kind(kind) && !smem_kind(kind)) {
        if (bulk_kind(kind) && !aligned(buf, 16)) return SYM_E_INVALID;
        SYM_CUDA(cudaMemsetAsync(buf, 0, (size_t)2 * rows * rank * sizeof(float) + 4096, s));
    }
    SYM_TRY(launch());  // warm-up (and L2 fill for the row kinds)
    cudaEvent_t e0, e1;
    SYM_CUDA(cudaEventCreate(&e0));
    SYM_CUDA(cudaEventCreate(&e1));
    sym_status st = SYM_OK;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == SYM_OK; ++r) st = launch();
    cudaEventRecord(e1, s);
    float t = 0.f;
    if (st == SYM_OK) {
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            st = cuda_status(cudaGetLastError());
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SYM_OK) return st;
    *ms = t / reps;
    const double sec = (double)*ms * 1e-3;
    double work;
    if (kind == SYM_CEIL_FMA)
        work = 2.0 * 8.0 * (double)iters * grid * CEIL_THREADS;
    else if (kind == SYM_CEIL_HBM_COPY)
        work = 2.0 * 16.0 * (double)rows;
    else
        work = (double)iters * groups;
    *rate = sec > 0 ? work / sec : 0.0;
    return SYM_OK;
}
