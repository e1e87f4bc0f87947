// Device-wide exclusive scan and LSD radix sort (keys of 64 or 128 bits with a
// 32-bit payload).  Used by tensor canonicalisation (lexicographic order of the
// canonical coordinates) and by the expanded-tensor baseline.
#include "common.cuh"

namespace symgpu {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-level exclusive scan of one tile; writes the tile total to sums[blockIdx].
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const T* __restrict__ in, T* __restrict__ out,
                                                             int64_t n, T* __restrict__ sums) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        v[k] = (i < n) ? in[i] : T(0);
        run += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = warp_incl_scan(run);
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        T t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : T(0);
        T ti = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == SCAN_THREADS / 32 - 1 && sums) sums[blockIdx.x] = ti;
    }
    __syncthreads();
    T off = warp_tot[w] + incl - run;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, int64_t n, const T* __restrict__ offs) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const T add = offs[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x) {
        int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

template <typename T>
sym_status scan_impl(const T* in, T* out, int64_t n, void* ws, cudaStream_t s) {
    if (n <= 0) return SYM_OK;
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_tiles<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, (T*)nullptr);
        SYM_CHECK_LAUNCH();
        return SYM_OK;
    }
    T* sums = static_cast<T*>(ws);
    char* rest = static_cast<char*>(ws) + align_up(tiles * sizeof(T), 256);
    k_scan_tiles<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    SYM_CHECK_LAUNCH();
    sym_status st = scan_impl<T>(sums, sums, tiles, rest, s);
    if (st != SYM_OK) return st;
    k_scan_add<T><<<(unsigned)tiles, 256, 0, s>>>(out, n, sums);
    SYM_CHECK_LAUNCH();
    return SYM_OK;
}

// Two-level exclusive scan for the radix count arrays: per-tile exclusive
// prefixes in `out` and the exclusive scan of the tile totals in `sums`, so a
// consumer reads out[i] + sums[i / SCAN_TILE] and no pass adds the tile
// offsets back into `out`.  Needs at most SCAN_TILE tiles (false otherwise).
bool scan_two_level_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums, cudaStream_t s) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (n <= 0 || tiles > SCAN_TILE) return false;
    k_scan_tiles<uint32_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    k_scan_tiles<uint32_t><<<1, SCAN_THREADS, 0, s>>>(sums, sums, tiles, (uint32_t*)nullptr);
    return true;
}

__device__ __forceinline__ uint32_t count_offset(const uint32_t* offsets, const uint32_t* tile_sums, int64_t i) {
    return offsets[i] + (tile_sums ? tile_sums[i / SCAN_TILE] : 0u);
}

// ---------------------------------------------------------------- radix sort

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int RS_WARPS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_ROUNDS = 8;                      // items per lane
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 2048 items per CTA

template <int KW>
__device__ __forceinline__ unsigned digit_of(const uint64_t* klo, const uint64_t* khi, int64_t i, int shift) {
    if constexpr (KW == 2) {
        uint64_t w = (shift < 64) ? klo[i] : khi[i];
        return (unsigned)((w >> (shift & 63)) & (RADIX - 1));
    } else {
        return (unsigned)((klo[i] >> shift) & (RADIX - 1));
    }
}

template <int KW>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint64_t* __restrict__ klo,
                                                           const uint64_t* __restrict__ khi, int64_t n,
                                                           int shift, uint32_t* __restrict__ counts,
                                                           int64_t ntiles) {
    __shared__ uint32_t h[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    // every key of the thread is requested before the first count is taken
    unsigned dg[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = base + (int64_t)r * RS_THREADS + threadIdx.x;
        dg[r] = i < n ? digit_of<KW>(klo, khi, i, shift) : 0xffffu;
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r)
        if (dg[r] != 0xffffu) atomicAdd(&h[dg[r]], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) counts[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter: warp w owns tile items [w*256, w*256+256) in 8 rounds of 32;
// ranks within a round come from __match_any_sync, across rounds from a
// running per-(warp, digit) counter, across warps from a per-digit scan.
template <int KW>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(
    const uint64_t* __restrict__ klo, const uint64_t* __restrict__ khi, const uint32_t* __restrict__ pay,
    uint64_t* __restrict__ olo, uint64_t* __restrict__ ohi, uint32_t* __restrict__ opay, int64_t n, int shift,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ tile_sums, int64_t ntiles) {
    __shared__ uint32_t cnt[RS_WARPS][RADIX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < RS_WARPS * RADIX; t += RS_THREADS) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ROUNDS);
    uint64_t lo[RS_ROUNDS];
    uint64_t hi[RS_ROUNDS];
    uint32_t pl[RS_ROUNDS];
    unsigned dg[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            lo[r] = klo[i];
            hi[r] = (KW == 2) ? khi[i] : 0;
            pl[r] = pay[i];
            uint64_t word = (KW == 2 && shift >= 64) ? hi[r] : lo[r];
            dg[r] = (unsigned)((word >> (shift & 63)) & (RADIX - 1));
            atomicAdd(&cnt[w][dg[r]], 1u);
        } else {
            dg[r] = 0xffffu;  // sentinel group, never written
        }
    }
    __syncthreads();
    // per digit: exclusive offsets across warps, seeded with the global offset
    for (int d = threadIdx.x; d < RADIX; d += RS_THREADS) {
        uint32_t run = count_offset(offsets, tile_sums, (int64_t)d * ntiles + blockIdx.x);
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned ltmask = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
        unsigned rank = __popc(peers & ltmask);
        if (dg[r] != 0xffffu) {
            uint32_t pos = cnt[w][dg[r]] + rank;
            olo[pos] = lo[r];
            if (KW == 2) ohi[pos] = hi[r];
            opay[pos] = pl[r];
        }
        __syncwarp();
        if (dg[r] != 0xffffu && rank == 0) cnt[w][dg[r]] += __popc(peers);
        __syncwarp();
    }
}

// Stable scatter of 64-bit keys through shared memory: the same ranks as
// k_radix_scatter place the tile in digit order in shared memory first, then
// consecutive threads write consecutive output positions of each digit's run
// (coalesced stores instead of one scattered 8-byte store per item).
#ifndef SYM_RS_MIN_BLOCKS
#define SYM_RS_MIN_BLOCKS 1  // CTAs per SM the staged scatter is compiled for (register budget)
#endif
__global__ void __launch_bounds__(RS_THREADS, SYM_RS_MIN_BLOCKS) k_radix_scatter_staged(const uint64_t* __restrict__ klo,
                                                                     const uint32_t* __restrict__ pay,
                                                                     uint64_t* __restrict__ olo,
                                                                     uint32_t* __restrict__ opay, int64_t n, int shift,
                                                                     const uint32_t* __restrict__ offsets,
                                                                     const uint32_t* __restrict__ tile_sums,
                                                                     int64_t ntiles) {
    static_assert(RS_THREADS == RADIX, "one thread per digit in the tile scan");
    __shared__ uint32_t cnt[RS_WARPS][RADIX];
    __shared__ uint32_t gbase[RADIX];  // output position of the digit's run in this tile, minus its start in the tile
    __shared__ uint32_t wsum[RS_WARPS];
    __shared__ uint64_t s_lo[RS_TILE];
    __shared__ uint32_t s_pl[RS_TILE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // this thread's digit offset, requested first so its latency overlaps the tile's loads
    const uint32_t goff = count_offset(offsets, tile_sums, (int64_t)threadIdx.x * ntiles + blockIdx.x);
    for (int t = threadIdx.x; t < RS_WARPS * RADIX; t += RS_THREADS) (&cnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int64_t wbase = tbase + (int64_t)w * (32 * RS_ROUNDS);
    uint64_t lo[RS_ROUNDS];
    uint32_t pl[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = wbase + r * 32 + lane;
        lo[r] = 0;
        pl[r] = 0;
        if (i < n) {
            lo[r] = klo[i];
            pl[r] = pay[i];
        }
    }
    // Per-warp multisplit without atomics: in each round the lanes holding one
    // digit find each other (match), the first of them advances the warp's count
    // of that digit and hands the old count to the others; an item's offset in
    // its warp's run of the digit is that count plus its rank among the lanes
    // (input order, so the sort stays stable).
    // (offsets are below 256, the warp's item count: four to a register)
    const unsigned ltmask = lanemask_lt();
    uint32_t off[RS_ROUNDS / 4] = {};
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t i = wbase + r * 32 + lane;
        const unsigned dg = i < n ? (unsigned)((lo[r] >> shift) & (RADIX - 1)) : 0xffffu;  // 0xffff: no item
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && dg != 0xffffu) {
            base = cnt[w][dg];
            cnt[w][dg] = base + (uint32_t)__popc(peers);
        }
        const uint32_t o = __shfl_sync(0xffffffffu, base, leader) + (uint32_t)__popc(peers & ltmask);
        off[r / 4] |= (o & 0xffu) << (8 * (r % 4));
        __syncwarp();  // the count update is seen by the next round's leaders
    }
    __syncthreads();
    // Thread d: the digit's count in the tile, its start in the tile (exclusive
    // scan over digits), and the per-warp starts within its run.
    {
        const int d = threadIdx.x;
        uint32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) tot += cnt[ww][d];
        const uint32_t incl = warp_incl_scan(tot);
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t start = incl - tot;
        for (int k = 0; k < w; ++k) start += wsum[k];
        gbase[d] = goff - start;
        uint32_t run = start;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            const uint32_t c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        if (wbase + r * 32 + lane < n) {
            const unsigned dg = (unsigned)((lo[r] >> shift) & (RADIX - 1));
            const uint32_t p = cnt[w][dg] + ((off[r / 4] >> (8 * (r % 4))) & 0xffu);
            s_lo[p] = lo[r];
            s_pl[p] = pl[r];
        }
    }
    __syncthreads();
    const int m = n - tbase < RS_TILE ? (int)(n - tbase) : RS_TILE;
    for (int j = threadIdx.x; j < m; j += RS_THREADS) {
        const uint64_t k = s_lo[j];
        const uint32_t pos = gbase[(unsigned)((k >> shift) & (RADIX - 1))] + (uint32_t)j;
        olo[pos] = k;
        opay[pos] = s_pl[j];
    }
}

}  // namespace

size_t scan_ws_bytes(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        total += align_up(m * sizeof(int64_t), 256);
    }
    return total + 256;
}

sym_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, ws, s);
}
sym_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, void* ws, cudaStream_t s) {
    return scan_impl<uint32_t>(in, out, n, ws, s);
}

size_t radix_ws_bytes(int64_t n, int kw) {
    (void)kw;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t nc = ntiles * RADIX;
    return 2 * align_up(nc * sizeof(uint32_t), 256) + scan_ws_bytes(nc);
}

sym_status radix_sort_pairs(int kw, uint64_t* klo, uint64_t* khi, uint32_t* pay, uint64_t* klo_alt,
                            uint64_t* khi_alt, uint32_t* pay_alt, int64_t n, int bits, void* ws,
                            cudaStream_t s, uint64_t** klo_out, uint64_t** khi_out, uint32_t** pay_out) {
    *klo_out = klo;
    *khi_out = khi;
    *pay_out = pay;
    if (n <= 1 || bits <= 0) return SYM_OK;
    if (n > 0xffffffffLL) return SYM_E_UNSUPPORTED;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t nc = ntiles * RADIX;
    uint32_t* counts = static_cast<uint32_t*>(ws);
    uint32_t* offs = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + align_up(nc * sizeof(uint32_t), 256));
    void* sws = static_cast<char*>(ws) + 2 * align_up(nc * sizeof(uint32_t), 256);
    uint64_t *a_lo = klo, *a_hi = khi, *b_lo = klo_alt, *b_hi = khi_alt;
    uint32_t *a_p = pay, *b_p = pay_alt;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        if (kw == 2) {
            k_radix_hist<2><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(a_lo, a_hi, n, shift, counts, ntiles);
        } else {
            k_radix_hist<1><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(a_lo, a_hi, n, shift, counts, ntiles);
        }
        SYM_CHECK_LAUNCH();
        // digit offsets: two-level (tile prefixes + scanned tile sums, read together by the scatter) when the
        // count array has at most SCAN_TILE tiles, else a full scan
        const uint32_t* tsums = static_cast<const uint32_t*>(sws);
        if (scan_two_level_u32(counts, offs, nc, static_cast<uint32_t*>(sws), s)) {
            SYM_CHECK_LAUNCH();
        } else {
            tsums = nullptr;
            sym_status st = exclusive_scan_u32(counts, offs, nc, sws, s);
            if (st != SYM_OK) return st;
        }
        if (kw == 2) {
            k_radix_scatter<2><<<(unsigned)ntiles, RS_THREADS, 0, s>>>(a_lo, a_hi, a_p, b_lo, b_hi, b_p, n, shift,
                                                                      offs, tsums, ntiles);
        } else {
            k_radix_scatter_staged<<<(unsigned)ntiles, RS_THREADS, 0, s>>>(a_lo, a_p, b_lo, b_p, n, shift, offs,
                                                                         tsums, ntiles);
        }
        SYM_CHECK_LAUNCH();
        uint64_t* t = a_lo; a_lo = b_lo; b_lo = t;
        t = a_hi; a_hi = b_hi; b_hi = t;
        uint32_t* tp = a_p; a_p = b_p; b_p = tp;
    }
    *klo_out = a_lo;
    *khi_out = a_hi;
    *pay_out = a_p;
    return SYM_OK;
}

}  // namespace symgpu
