// Banded batched SSYMV + SYPRD: plan layout and the calls the batch plan
// (spmv_batch.cu) makes into spmv_band.cu.
#pragma once

#include <vector>

#include "common.cuh"

namespace symgpu {

// One row band I of one instance: the CTA that owns it keeps x and y of band I
// in shared memory while it streams the blocks (I, J), J = I .. nb-1.
struct BandUnit {
    int64_t base;  // global row of the instance's first row
    int64_t slot;  // SYPRD partial slot (slots of one instance are contiguous)
    int32_t n;     // rows of the instance
    int32_t I;     // row band
    int32_t seg0;  // first block record of this row band
    int32_t nseg;  // blocks (I, I) .. (I, nb-1)
};

// One block (I, J): its entries are eidx/evals[start, start + cnt), cnt a
// multiple of 4 (the tail is padded with BAND_PAD entries).
struct BandSeg {
    int64_t start;
    int32_t cnt;
    int32_t code;  // J | BAND_STAGED when band J of x / y is staged in shared memory
};

// One non-empty block (I, J) in a CTA's work list (48 bytes, 16-byte multiple).
struct BandTask {
    int64_t start;  // first entry in eidx / evals (multiple of 4)
    int64_t base;   // instance's first global row
    int64_t slot;   // SYPRD partial slot of row band I
    int32_t cnt;    // entries, a multiple of 4, > 0
    int32_t flags;  // block kind << TASK_MODE_SHIFT | TASK_FIRST | TASK_LAST | TASK_SINGLE
    int32_t I, J;   // row band, column band
    int32_t wI, wJ; // rows in band I / J
};
static_assert(sizeof(BandTask) == 48, "BandTask is copied in 16-byte units");

constexpr uint32_t BAND_PAD = 0xffffffffu;  // padding entry (in-band indices are < 65536)
constexpr int32_t BAND_STAGED = 1 << 30;
constexpr int BAND_MAX_BANDS = 64;
// Block kinds: 0 = diagonal block (I, I); 1 = band J staged in shared memory;
// 2 = band J read / reduced in global memory (blocks too sparse to stage).
constexpr int TASK_FIRST = 1, TASK_LAST = 2, TASK_SINGLE = 4, TASK_GROUPED = 8, TASK_MODE_SHIFT = 8;
constexpr int BAND_GROUP = 32;  // entries per bank group (one per lane)

struct BandPlan {
    int W = 0;          // rows per band
    int threads = 0;    // CTA size: one producer warp + consumer warps
    int epl = 4;        // entries per consumer lane per chunk
    int order = 0;      // 0: row-major blocks; 1: bank-grouped blocks
    int stages = 0;     // chunk slots in the ring
    int grid = 0;       // persistent CTAs (static task lists)
    size_t smem = 0;    // dynamic shared memory per CTA
    int64_t nunits = 0, nsegs = 0, ntasks = 0, nentries = 0;
    int64_t x_rows = 0;            // rows of x (bounds of the staging copies)
    BandUnit* units = nullptr;     // [device] plan-time: row bands
    BandSeg* segs = nullptr;       // [device] plan-time: blocks
    BandTask* tasks = nullptr;     // [device] per CTA, in processing order
    int32_t* cta_ptr = nullptr;    // [device] grid + 1 offsets into tasks
    uint32_t* eidx = nullptr;      // [device] packed (row - I W) << 16 | (col - J W)
    float* evals = nullptr;        // [device]
    unsigned* err = nullptr;       // [device] bit 0: a bounded wait ran out; bits 1, 2: bad column (plan time)
    uint64_t wait_ns = 2000000000ull;  // limit of every bounded wait in the kernel
    int64_t skip_chunk = -1;       // test hook: chunk of CTA 0 that is never delivered (-1: none)
};

// Instances on the banded path and their band counts (0 = tile path).
int band_count(int64_t n, const sym_tile_cfg* cfg);
// Shared memory the banded kernel needs per CTA for this config, and the
// stage count it gets (0 stages = the config does not fit).
size_t band_smem(const sym_tile_cfg* cfg, int* stages);
// Arena bytes of the banded part of a plan (an upper bound: assumes all
// total_nnz entries are banded, each block padded by up to 31 entries).
void band_size(Sizer& s, const sym_csr_batch* A, const int64_t* host_row_off, const sym_tile_cfg* cfg);
// Builds the banded part: counts the blocks on the device, lays them out on
// the host, reorders the entries on the device.  `slot_of` gives the first
// SYPRD slot of each instance.  Synchronises `s`.
sym_status band_build(BandPlan& P, Carver& c, const sym_csr_batch* A, const int64_t* host_row_off,
                      const sym_tile_cfg* cfg, const std::vector<int64_t>& slot_of, cudaStream_t s);
// Enqueues the banded kernel (y must already be zeroed).
sym_status band_enqueue(const BandPlan& P, const float* x, float* y, double* partials, bool syprd,
                        cudaStream_t s);

}  // namespace symgpu
