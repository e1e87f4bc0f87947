/*
 * symgpu.h — C ABI of the GB300 symmetric sparse kernels (SySTeC hot path).
 *
 * The paper: "SySTeC: A Symmetric Sparse Tensor Compiler", arXiv 2406.09266.
 * A fully symmetric tensor X (Sec. 2.1, Def. "Symmetry") is stored by its
 * canonical triangle only: coordinates with i_1 <= i_2 <= ... <= i_N (Sec. 2.1,
 * Def. "Canonical", upper triangle).  Each stored entry stands for every
 * DISTINCT permutation of its indices (Sec. 3.1: n!/m! assignments when m
 * indices are equal; Sec. 4.1, unique symmetry group S_P|E), and the kernels
 * apply it once per such permutation.
 *
 * Conventions for every call:
 *   - Indices are 0-based.  Dense matrices are row-major with an explicit row
 *     stride (ld*) in elements.
 *   - Pointers marked [device] are CUDA device pointers; [host] are host
 *     pointers.  All device memory is owned by the caller (the library calls
 *     cudaMalloc/cudaFree only in sym_devloop_create / sym_devloop_destroy, for
 *     the request loop's own ring and counters): handles and scratch are carved
 *     out of caller-given arenas and workspaces whose sizes come from the *_bytes
 *     queries.  Arenas and workspaces must be 256-byte aligned.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Compute calls are asynchronous on that stream unless documented otherwise.
 *   - Every call returns a sym_status.  Argument errors are detected on the host
 *     before anything is enqueued and leave outputs untouched.  No C++
 *     exception and no abort crosses this boundary.
 *   - Handles are thread-compatible: concurrent calls on one handle need
 *     external synchronisation; distinct handles are independent.
 */
#ifndef SYMGPU_H
#define SYMGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Every entry point below is exported from libsymgpu.so even when the library
 * is compiled with hidden default visibility. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

#define SYMGPU_VERSION 1

typedef void* sym_stream_t; /* cudaStream_t */

typedef enum {
    SYM_OK = 0,
    SYM_E_INVALID = -1,      /* bad argument (null pointer, size, alignment, unsupported shape) */
    SYM_E_NONCANONICAL = -2, /* input claimed canonical is not (CSR column below the diagonal, unsorted) */
    SYM_E_RANGE = -3,        /* an index outside [0, n) */
    SYM_E_DUPLICATE = -4,    /* two stored entries with the same index multiset */
    SYM_E_NOMEM = -5,        /* arena or workspace smaller than the *_bytes query */
    SYM_E_BUDGET = -6,       /* request larger than the serving HBM budget */
    SYM_E_TIMEOUT = -7,      /* a bounded wait ran out */
    SYM_E_CUDA = -8,         /* a CUDA runtime call failed (see sym_last_cuda_error) */
    SYM_E_BADREQ = -9,       /* malformed serving request */
    SYM_E_UNSUPPORTED = -10, /* valid but not implemented here (e.g. order > 5) */
    SYM_E_NOTFOUND = -11,    /* unknown ticket */
    SYM_PENDING = 1          /* serving request not finished yet */
} sym_status;

typedef enum { SYM_F32 = 0, SYM_BF16 = 1 } sym_dtype;

typedef enum {
    SYM_DUP_ERROR = 0,      /* any repeated index multiset is an error */
    SYM_DUP_KEEP_EQUAL = 1  /* keep the first copy; copies must carry bit-identical values */
} sym_dup_policy;

const char* sym_status_string(sym_status s);
/* Last CUDA error code seen by the library in this thread (cudaError_t as int). */
int sym_last_cuda_error(void);
int sym_version(void);

/* Optional per-kernel timing: when enabled, the library records a CUDA event
 * pair on the launching stream around each of its kernel launches.
 * sym_profile_read synchronises on the recorded events and returns, per kernel
 * name, the launch count and the summed event time. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} sym_profile_entry;
sym_status sym_profile_enable(int on);
/* Returns the number of entries written (at most max_entries). */
int sym_profile_read(sym_profile_entry* out, int max_entries);
sym_status sym_profile_reset(void);

/* Bounds-checked build (no paper counterpart: a checking aid in place of a
 * memory checker).  libsymgpu_bc.so is this library compiled with
 * -DSYM_BOUNDS_CHECK: the kernels of the hot path (canonical-stream MTTKRP,
 * SSYMV / SYPRD in the multi-block, one-launch and banded forms) check every
 * gathered or scattered index against the extent of its array, skip an access
 * outside it and add one to *counter; they never trap.  sym_bounds_check_enabled
 * returns 1 in that library and 0 here; sym_bounds_check_attach sets the
 * counter [device, 8-byte aligned, caller-owned; NULL detaches] for every
 * kernel of the library (SYM_E_UNSUPPORTED in the normal build).  Synchronous. */
int sym_bounds_check_enabled(void);
sym_status sym_bounds_check_attach(unsigned long long* counter);

/* Measured ceilings of the operations the kernels are made of (no paper
 * counterpart: the denominators of the roofline fractions the benchmarks
 * report).  Each kind times one kernel of the primitive operation alone:
 *   SYM_CEIL_FMA         FP32 fused multiply-add issue; *rate in FLOP/s.
 *   SYM_CEIL_ROW_GATHER  random rows of `rank` floats read from a table of
 *                        `rows` rows (L2-resident when it fits); rows/s.
 *   SYM_CEIL_ROW_RED     random rows reduced with 16-byte vector `red`; rows/s.
 *   SYM_CEIL_GATHER_RED  one random gather and one random reduction; entries/s.
 *   SYM_CEIL_SMEM_F32    a row added with float atomics into a shared-memory
 *                        table of `rows` rows (rows * rank * 4 <= 200 KiB); rows/s.
 *   SYM_CEIL_SMEM_U32    the same with 32-bit integer atomics; rows/s.
 *   SYM_CEIL_HBM_COPY    streaming copy of `rows` 16-byte elements; bytes/s
 *                        (read + write).
 *   SYM_CEIL_BULK_GATHER random rows read with one bulk copy (cp.async.bulk)
 *                        per row into shared memory; rows/s.
 *   SYM_CEIL_BULK_RED    random rows reduced from shared memory with one bulk
 *                        reduction (cp.reduce.async.bulk .add.f32) per row; rows/s.
 * `ops` row operations (FMA: about ops / 2^11 FLOP per thread) per launch,
 * `reps` timed launches after one warm-up.  buf [device, 256-byte aligned,
 * >= sym_ceiling_bytes] is scratch, overwritten.  Synchronous; *ms = mean time
 * of one launch.  Row kinds need rank in 4..128 with rank / 4 a power of two. */
typedef enum {
    SYM_CEIL_FMA = 0,
    SYM_CEIL_ROW_GATHER = 1,
    SYM_CEIL_ROW_RED = 2,
    SYM_CEIL_GATHER_RED = 3,
    SYM_CEIL_SMEM_F32 = 4,
    SYM_CEIL_SMEM_U32 = 5,
    SYM_CEIL_HBM_COPY = 6,
    SYM_CEIL_BULK_GATHER = 7,
    SYM_CEIL_BULK_RED = 8
} sym_ceiling_kind;
/* Bytes of scratch for sym_ceiling_run (0 = invalid arguments). */
size_t sym_ceiling_bytes(int kind, int64_t rows, int rank);
sym_status sym_ceiling_run(int kind, void* buf, size_t buf_bytes, int64_t rows, int rank, int64_t ops, int reps,
                           sym_stream_t stream, double* rate, float* ms);

/* ===================================================================== */
/* SSYMV / SYPRD over an upper-triangle CSR (Sec. 3.1 figure "spmv_code",  */
/* Sec. 5.2.1 SSYMV y[i] = A[i,j] x[j], Sec. 5.2.3 SYPRD y = x[i]A[i,j]x[j]) */
/* ===================================================================== */

/* Upper triangle of a symmetric n x n matrix in CSR: row i holds columns
 * j >= i, strictly increasing.  All arrays [device]; rowptr has n+1 entries. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const float* val;
} sym_csr_upper;

/* Workspace for sym_spmv when SYPRD is requested (per-block FP64 partials). */
size_t sym_spmv_workspace_bytes(const sym_csr_upper* A);

/* y = A x with A symmetric (both triangles), reading each stored entry once:
 * an off-diagonal entry a_ij (i < j) adds a x_j to y_i and a x_i to y_j; a
 * diagonal entry adds a x_i to y_i once.  y [device, n floats] is overwritten.
 * If syprd [device, 1 double] is not NULL it receives x^T A x, with the
 * off-diagonal terms weighted 2 (invisible output symmetry, Sec. 3.2.2), per-
 * block partials formed in FP32 and the cross-block sum in FP64.  x, y: n
 * floats [device], 16-byte aligned not required.  ws may be NULL when syprd is
 * NULL.  The CSR is trusted (use sym_csr_upper_check to validate).
 * Matrices with n <= 8192 whose x, a partial y, rowptr, 1/8 of the entries
 * and the exchange inbox fit in 160 KiB of shared memory per CTA run as one
 * launch of one 8-CTA thread-block cluster (a partial y per CTA in shared
 * memory, exchanged by bulk copies between the CTAs and summed in a fixed
 * order; FP32 SYPRD partials per warp, FP64 across warps and CTAs; column
 * indices outside [0, n) are skipped; if the exchange does not complete within
 * about 2 s, y and SYPRD are set to NaN); larger ones as a memset, the SSYMV
 * kernel and the FP64 finaliser. */
sym_status sym_spmv(const sym_csr_upper* A, const float* x, float* y, double* syprd, void* ws,
                    size_t ws_bytes, sym_stream_t stream);

/* Row partition of SSYMV / SYPRD (the natural shard of the product over
 * several devices: row ranges, then one sum of y and of SYPRD; Sec. 3.1 with
 * the rows split).  Adds the contribution of the stored entries of rows
 * [row_begin, row_end) -- y[i] += a x[j] and, for j > i, y[j] += a x[i] -- into
 * y (accumulate = 1) or into zeros (accumulate = 0; all n entries of y are
 * cleared first).  syprd [device, nullable] receives those rows' share of
 * x^T A x, sum_i x[i] (2 sum_{j>i} a_ij x[j] + a_ii x[i]), FP32 per block and
 * FP64 across blocks.  Summing y and syprd over any partition of [0, n) into row
 * ranges gives sym_spmv's results (up to rounding).  Always the multi-block
 * form.  ws [device] >= sym_spmv_workspace_bytes(A) when syprd is given. */
sym_status sym_spmv_rows(const sym_csr_upper* A, const float* x, float* y, double* syprd, int64_t row_begin,
                         int64_t row_end, int accumulate, void* ws, size_t ws_bytes, sym_stream_t stream);

/* 1 when sym_spmv / sym_spmv_noalloc run A as the one-launch cluster form, 0
 * otherwise (also for an invalid descriptor).  Host-only: reads the descriptor
 * fields n and nnz, touches no device memory. */
int sym_spmv_single_launch(const sym_csr_upper* A);

/* Test hook of the one-launch form's bounded inbox wait (no paper
 * counterpart): runs A as the cluster form with the wait limited to
 * wait_limit_ns (<= 0: the normal 2 s); for skip_to in 0..7 no CTA pushes its
 * partial y (or its SYPRD partial) into CTA skip_to's inbox, so that CTA's
 * wait runs out with no copy in flight towards it and it writes NaN to its
 * rows of y (CTA 0 also to syprd); the other rows are exact.  skip_to = -1: a
 * normal run.  SYM_E_UNSUPPORTED when A does not take the one-launch form. */
sym_status sym_spmv_cluster_bounded(const sym_csr_upper* A, const float* x, float* y, double* syprd,
                                    int64_t wait_limit_ns, int skip_to, sym_stream_t stream);

/* Allocation-free variant of sym_spmv (the paper has no counterpart: it is a
 * service to callers that cannot allocate).  For callers that cannot hand the
 * library any device memory: hosts whose pool allocator owns the whole device,
 * code that must keep working once device memory is exhausted, or loops that
 * must not call cudaMalloc because it can synchronise the device.  It computes
 * exactly what sym_spmv computes; the per-block FP64 SYPRD partials live in a
 * 256 KiB array compiled into the library, which every GPU that loads the
 * library keeps until the process exits.  Limit, for calls with syprd only:
 * at most 32,768 partial slots (sym_spmv_workspace_bytes(A) <= 256 KiB; always
 * true for n <= 262,144 rows), otherwise SYM_E_UNSUPPORTED (use sym_spmv with a
 * workspace); calls without syprd have no size limit.  The first call with
 * syprd on a device looks up the array's device address (make it before any
 * stream capture); the address is kept, so do not call this again on a device
 * after cudaDeviceReset.  Calls share the array, so calls whose work overlaps
 * on the GPU race and must be serialised by the caller.  Allocates nothing. */
sym_status sym_spmv_noalloc(const sym_csr_upper* A, const float* x, float* y, double* syprd, sym_stream_t stream);

/* Validates an upper CSR on the device; *bad [device, 1 int64] receives the
 * number of offending rows (0 = valid).  ws >= sym_spmv_workspace_bytes(A). */
sym_status sym_csr_upper_check(const sym_csr_upper* A, int64_t* bad, sym_stream_t stream);

/* Bellman-Ford relaxation over the same storage (Sec. 5.2.2):
 * y[i] = min(d[i], min over stored (i,j) and (j,i) of a + d[other]).  y, d: n floats. */
sym_status sym_bellman_step(const sym_csr_upper* A, const float* d, float* y, sym_stream_t stream);

/* Baseline: the same product from a full (both-triangle) CSR built by
 * sym_csr_expand_upper; plain row-per-warp SpMV. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const float* val;
} sym_csr_full;
/* Bytes of the full CSR (rowptr + col + val) and of the build workspace. */
size_t sym_csr_expand_bytes(const sym_csr_upper* A, size_t* ws_bytes);
/* Writes the full CSR of A into arena [device] (rowptr | col | val, each
 * 256-byte aligned) and fills *out.  Synchronises `stream`. */
sym_status sym_csr_expand_upper(const sym_csr_upper* A, void* arena, size_t arena_bytes, void* ws,
                                size_t ws_bytes, sym_stream_t stream, sym_csr_full* out);
sym_status sym_spmv_full(const sym_csr_full* A, const float* x, float* y, sym_stream_t stream);

/* ===================================================================== */
/* Batched SSYMV + SYPRD: many independent matrices in one persistent launch */
/* ===================================================================== */

/* Instance b owns global rows [row_off[b], row_off[b+1]) of x and y; rowptr is
 * global (nnz offsets, int64, total_rows+1 entries); col holds GLOBAL column
 * indices, each inside its own instance's row range and >= its row.  All
 * arrays [device]. */
typedef struct {
    int64_t count;
    int64_t total_rows;
    int64_t total_nnz;
    const int64_t* row_off;
    const int64_t* rowptr;
    const int32_t* col;
    const float* val;
} sym_csr_batch;

/* Work decomposition of the persistent kernel. */
typedef struct {
    int32_t rows_per_tile;    /* rows in one work tile (tiles never straddle instances) */
    int32_t lanes_per_row;    /* 1..32, power of two: lanes cooperating on one row */
    int32_t threads_per_cta;  /* 128..1024, multiple of 32 */
    int32_t ctas_per_sm;      /* persistent CTAs per SM */
    int32_t local_smem_kb;    /* instances whose n floats fit in this much shared memory are processed whole
                                 by one CTA with y (and x, when 2n floats fit) on chip; 0 = all on tiles */
    int32_t tile_order;       /* 0: tiles in instance order; 1: interleaved across instances, so CTAs that run
                                 together reduce into different instances' y */
    int32_t x_smem_kb;        /* > 0: each tile copies the first x_smem_kb*256 floats of its x window
                                 (x[row0 ..]) into shared memory and gathers from there; rows_per_tile must
                                 not exceed that many floats */
    int32_t band_rows;        /* > 0 (multiple of 4, 256..16384): banded path.  Instance b is cut into
                                 nb = ceil(n_b / band_rows) bands of rows; the upper triangle falls into
                                 blocks (I, J), I <= J < nb.  The plan keeps a reordered copy of those
                                 instances' canonical entries (4-byte packed in-band (row, col) + value,
                                 block by block, row-major inside a block) and one CTA works through one
                                 row band I at a time with x and y of bands I and J in shared memory: the
                                 mirrored updates y[j] += a x_i (Sec. 3.1) become shared-memory adds and
                                 each band of y is reduced into global memory once per block, with
                                 16-byte vector reductions.  One producer warp streams the entries with
                                 bulk asynchronous copies (cp.async.bulk + mbarrier) several chunks ahead
                                 and stages the x bands, one warp reduces the finished y bands into
                                 global memory, the other warps consume.  threads_per_cta (96..1024: one
                                 producer warp + one flusher warp + consumer warps) and ctas_per_sm (1 or 2)
                                 shape the banded kernel; the band buffers (32 * band_rows bytes) and at
                                 least two chunks must fit in one CTA's shared memory (SYM_E_INVALID
                                 otherwise: band_rows up to ~5,600 on GB300).  Instances with
                                 nb > band_max stay on the tile path (lanes_per_row, rows_per_tile,
                                 x_smem_kb apply to those).  local_smem_kb must be 0. */
    int32_t band_max;         /* banded path only: largest band count per instance (1..64) */
    int32_t band_chunk;       /* banded path only: entries per consumer lane per streamed chunk (a chunk is
                                 this times 32 x the consumer warps): 4, 8, 16 (0 = 4), or 1, 2 with
                                 band_order 1.  Smaller chunks leave room for more of them in flight. */
    int32_t band_order;       /* banded path only: order of the entries inside a block.  0: row-major (each
                                 lane takes 4 consecutive entries; runs of one row are summed in registers).
                                 1: bank groups: the plan regroups each block into groups of 32 entries whose
                                 rows, and whose columns, fall in distinct shared-memory banks where the
                                 block allows it (a greedy matching per group on the host, relaxed to 2, 3,
                                 ... entries per bank only for the groups it cannot fill otherwise); a warp
                                 takes one group at a time, one entry per lane, so its x gathers and y
                                 reductions meet no bank conflicts.  Padding: at most 31 entries per block. */
} sym_tile_cfg;

/* A plan: the tile list and the FP64 partial buffers, carved from `arena`. */
typedef struct sym_batch_plan_s* sym_batch_plan;
/* host_row_off: [host] copy of row_off (count+1 entries), used to size tiles. */
size_t sym_spmv_batch_plan_bytes(const sym_csr_batch* A, const int64_t* host_row_off, const sym_tile_cfg* cfg);
sym_status sym_spmv_batch_plan_create(const sym_csr_batch* A, const int64_t* host_row_off,
                                      const sym_tile_cfg* cfg, void* arena, size_t arena_bytes,
                                      sym_stream_t stream, sym_batch_plan* out);
/* y = A_b x_b for every instance; syprd [device, count doubles] (nullable)
 * receives x_b^T A_b x_b (FP64 cross-tile sums).  One persistent launch plus
 * the reset and finalise steps, all on `stream`. */
sym_status sym_spmv_batch_run(sym_batch_plan plan, const float* x, float* y, double* syprd,
                              sym_stream_t stream);
/* Captures sym_spmv_batch_run into a CUDA graph (fixed pointers) and replays
 * it with sym_spmv_batch_graph_launch.  The graph lives in the plan. */
sym_status sym_spmv_batch_capture(sym_batch_plan plan, const float* x, float* y, double* syprd,
                                  sym_stream_t stream);
sym_status sym_spmv_batch_graph_launch(sym_batch_plan plan, sym_stream_t stream);
/* Device-side status of the plan's banded kernel: SYM_E_TIMEOUT when one of
 * its bounded waits on a bulk copy gave up (the kernel then left the rest of
 * its work undone and y / syprd are incomplete), SYM_OK otherwise.  The flag is
 * sticky for the plan's lifetime.  Synchronises the device (the plan may have
 * run on any stream), then reads one word. */
sym_status sym_spmv_batch_check(sym_batch_plan plan);
/* Clears the plan's device status word (enqueued on `stream`). */
sym_status sym_spmv_batch_clear_status(sym_batch_plan plan, sym_stream_t stream);
/* Test hook of the bounded waits (no paper counterpart): sym_spmv_batch_run
 * with every bounded wait of the banded kernel limited to wait_limit_ns (<= 0:
 * the normal 2 s) and, for skip_chunk >= 0, chunk `skip_chunk` of the first
 * CTA's entry stream withheld (never announced, never copied), so that the
 * consumers' wait on it runs out without any copy left in flight.  The kernel
 * then sets bit 0 of the status word (sym_spmv_batch_check reports
 * SYM_E_TIMEOUT), leaves the rest of its work undone and returns; y and syprd
 * are incomplete.  The plan itself is not changed. */
sym_status sym_spmv_batch_run_bounded(sym_batch_plan plan, const float* x, float* y, double* syprd,
                                      int64_t wait_limit_ns, int64_t skip_chunk, sym_stream_t stream);
sym_status sym_spmv_batch_plan_destroy(sym_batch_plan plan);

/* Autotuner: times candidate sym_tile_cfg shapes on this batch (each as a
 * plan built in `arena`, so arena must hold the largest candidate plan:
 * sym_spmv_batch_plan_bytes with rows_per_tile = 1 bounds them all), keeps the
 * fastest, and records it in the text cache file `cache_path` (nullable) keyed
 * by device name and batch shape.  A cache hit skips the timing.  Synchronous. */
sym_status sym_autotune_spmv_batch(const sym_csr_batch* A, const int64_t* host_row_off, const float* x,
                                   float* y, double* syprd, void* arena, size_t arena_bytes,
                                   const char* cache_path, sym_stream_t stream, sym_tile_cfg* best,
                                   float* best_ms);

/* ===================================================================== */
/* Fully symmetric sparse tensors of order 2..5                            */
/* ===================================================================== */

typedef struct sym_tensor_s* sym_tensor;

/* Sizes for sym_tensor_create: *arena_bytes stays owned by the tensor,
 * *ws_bytes is scratch needed only during the call. */
sym_status sym_tensor_create_bytes(int order, int64_t n, int64_t nnz, size_t* arena_bytes,
                                   size_t* ws_bytes);

/* Canonicalises a coordinate list into the tensor's device layout (Sec. 2.1
 * canonical triangle; Sec. 4.2.9 diagonal splitting):
 *   1. every coordinate tuple is sorted ascending and range checked;
 *   2. entries are sorted lexicographically (radix sort of packed keys);
 *   3. repeated multisets follow `dup` (never summed);
 *   4. entries are split, order preserved, into the STRICT stream (all
 *      indices distinct) and the DIAGONAL stream (some index repeated);
 *   5. exact counts are taken (per equality pattern, full-tensor nonzeros,
 *      fibers) and ||X||^2 over the full tensor is summed in FP64.
 * idx [device, or page-locked host memory the device can address (cudaHostAlloc
 * / cudaHostRegister): order rows of nnz int32, row q at idx + q*ld_idx, any
 * position order per tuple.  It is read once, by the packing kernel, so a
 * host coordinate list crosses the host link inside that kernel instead of in
 * a separate copy; pageable host memory is refused with SYM_E_INVALID].
 * val [device, or page-locked host memory]: nnz floats, read out of order after
 * the sort; host values are copied into the workspace on a stream of the call's
 * own while the keys are packed and sorted, so the copy overlaps the sort.
 * Order 2..5, 1 <= n < 2^31, order * ceil(log2 n) <= 128.  Synchronises
 * `stream` (it reads back counts).  On error no tensor is created. */
sym_status sym_tensor_create(int order, int64_t n, int64_t nnz, const int32_t* idx, int64_t ld_idx,
                             const float* val, sym_dup_policy dup, void* arena, size_t arena_bytes,
                             void* ws, size_t ws_bytes, sym_stream_t stream, sym_tensor* out);

typedef struct {
    int32_t order;
    int32_t key_bits;          /* bits per index in the packed keys */
    int64_t n;
    int64_t nnz;               /* canonical entries kept */
    int64_t nnz_strict;
    int64_t nnz_diag;
    int64_t duplicates_dropped;
    int64_t counts_by_pattern[16]; /* bit q of the pattern: c_q == c_{q+1} */
    int64_t expanded_nnz;      /* sum over entries of the distinct-permutation count */
    int64_t root_fibers;       /* distinct c_1 */
    int64_t l2_fibers;         /* distinct (c_1, c_2) */
    double normsq;             /* ||X||^2 of the full tensor, FP64 */
    size_t arena_used;
} sym_tensor_info_t;

sym_status sym_tensor_info(sym_tensor X, sym_tensor_info_t* out);

/* Writes the canonical entries [device]: first the strict stream, then the
 * diagonal stream, each in lexicographic order.  cidx has order rows of
 * ld_out int32 (ld_out >= nnz), cval nnz floats. */
sym_status sym_tensor_export(sym_tensor X, int32_t* cidx, int64_t ld_out, float* cval, sym_stream_t stream);

sym_status sym_tensor_destroy(sym_tensor X);

/* Leaf index (orders >= 3): the strict stream a second time, each tuple
 * reversed (c_N first) and sorted, so that the MTTKRP can treat the last
 * position as the root of a second CSF traversal and accumulate its rows in
 * registers instead of reducing into M once per entry.  It costs one more copy
 * of the strict stream (arena) and a sort (workspace).  Synchronises `stream`. */
sym_status sym_tensor_leaf_index_bytes(sym_tensor X, size_t* arena_bytes, size_t* ws_bytes);
sym_status sym_tensor_add_leaf_index(sym_tensor X, void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                                     sym_stream_t stream);

/* Relocatable image of a tensor (no paper counterpart: the residency
 * mechanism of the serving runtime).  sym_tensor_save writes the tensor's
 * canonical arrays (and its leaf index, if it has one) with a header into
 * `host` [host, >= sym_tensor_image_bytes(X) bytes; pinned memory makes the
 * copies asynchronous], enqueued on `stream`: the image is complete once the
 * stream has reached that point.  sym_tensor_load rebuilds a tensor from an
 * image into `arena` [device, 256-byte aligned, >= sym_tensor_load_bytes(host)]
 * with copies enqueued on `stream`; the handle is returned at once and is
 * usable by work enqueued after the copies on the same stream (or on streams
 * that wait for it).  The image must stay unchanged until those copies have
 * completed.  A loaded tensor computes exactly what the saved one did. */
size_t sym_tensor_image_bytes(sym_tensor X);
sym_status sym_tensor_save(sym_tensor X, void* host, size_t host_bytes, sym_stream_t stream);
size_t sym_tensor_load_bytes(const void* host);
/* The tensor_info of the tensor an image holds (read from the host header). */
sym_status sym_tensor_image_info(const void* host, sym_tensor_info_t* out);
sym_status sym_tensor_load(const void* host, void* arena, size_t arena_bytes, sym_stream_t stream, sym_tensor* out);

/* Order-2 tensors: the canonical entries as an upper-triangle CSR (row i holds
 * columns j >= i, ascending).  rowptr: n+1 int64, col: nnz int32, val: nnz
 * floats, all [device]; ws >= sym_tensor_upper_csr_ws_bytes(X). */
size_t sym_tensor_upper_csr_ws_bytes(sym_tensor X);
sym_status sym_tensor_upper_csr(sym_tensor X, int64_t* rowptr, int32_t* col, float* val, void* ws, size_t ws_bytes,
                                sym_stream_t stream);

/* Counter-based SplitMix64 coordinate generator for large on-device pools:
 * draw q of entry e is word e*order+q of the stream with `seed`; index =
 * high 32 bits * n >> 32; value = the entry's multiset hash mapped to a 24-bit
 * uniform in [-1, 1) (equal multisets get equal values, so the keep-equal
 * duplicate policy merges repeats).  idx: order rows of ld_idx int32 [device]. */
sym_status sym_gen_coords(int order, int64_t n, int64_t count, uint64_t seed, int32_t* idx, int64_t ld_idx,
                          float* val, sym_stream_t stream);

/* Counter-based generator of batched symmetric matrices: instance b (global
 * rows [row_off[b], row_off[b+1]), n_b rows) receives draws
 * [draw_off[b], draw_off[b+1]); draw d is word d of the SplitMix64 stream with
 * `seed`, u = (word >> 11) * 2^-53, slot s = floor(u * n_b(n_b+1)/2) of the
 * row-major upper triangle, mapped to (i, j), i <= j, written as GLOBAL indices
 * idx[0][d], idx[1][d] with value = the pair's multiset hash in [-1, 1)
 * (repeats carry equal values).  row_off, draw_off: count+1 int64 [device]. */
sym_status sym_gen_batch_coords(int64_t count, const int64_t* row_off, const int64_t* draw_off, int64_t total_draws,
                                uint64_t seed, int32_t* idx, int64_t ld_idx, float* val, sym_stream_t stream);

/* ===================================================================== */
/* Symmetric MTTKRP (Sec. 4.3, Sec. 5.2.6):                                */
/*   M[i, r] = sum over the full tensor X[i, k, l, ..] B[k, r] B[l, r] ..  */
/* with one shared factor B (the symmetric CPD update).                     */
/* ===================================================================== */

/* Workspace for sym_mttkrp (needed when residual != NULL; 0 otherwise). */
size_t sym_mttkrp_workspace_bytes(sym_tensor X, int rank, sym_dtype bdt, int want_residual);

/* M [device, n x rank floats, row stride ldm, overwritten] = MTTKRP of X with
 * B [device, n x rank, row stride ldb, FP32 or BF16 per bdt; BF16 values are
 * widened to FP32 on load and all accumulation is FP32].
 * The strict stream applies weight (N-1)! per position; the diagonal stream
 * applies per-run integer weights (N-1)!/((m_t-1)! prod_{s!=t} m_s!).
 * rank: 4..128, multiple of 4; ldb, ldm multiples of 4 (8 for BF16 ldb is not
 * required); B and M 16-byte aligned.
 * residual [device, 1 double] (nullable): the CP-fit residual
 * ||X - sum_r b_r^(x)N||^2 = ||X||^2 - 2<X,Mcp> + ||Mcp||^2 with unit weights,
 * evaluated in FP64 (exact FP32 products, double-float partials, FP64 sums). */
sym_status sym_mttkrp(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                      int64_t ldm, double* residual, void* ws, size_t ws_bytes, sym_stream_t stream);

/* Entry partition of the MTTKRP (the natural shard over several devices:
 * contiguous ranges of canonical entries with the factor replicated, then one
 * sum of the partial outputs).  Adds the contribution of canonical entries
 * [first, first + count) -- in the order sym_tensor_export writes them: the
 * strict stream, then the diagonal stream -- into M (accumulate = 1) or into
 * zeros (accumulate = 0).  Summing M over any partition of [0, nnz) gives
 * sym_mttkrp's M (up to rounding).  Uses the tensor's kernel configuration but
 * always walks the canonical stream (a leaf index covers the whole tensor and is
 * not used for a part).  Arguments as for sym_mttkrp. */
sym_status sym_mttkrp_range(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                            int64_t ldm, int64_t first, int64_t count, int accumulate, sym_stream_t stream);

/* Kernel configuration of one tensor's MTTKRP calls (all variants compute the
 * same result; they differ in speed).  The autotuner below picks one. */
typedef enum {
    SYM_MTTKRP_PLAIN = 0,        /* CSF-factorised, chunked warps, reductions to global memory */
    SYM_MTTKRP_PIPELINED = 1,    /* the same with the next leaf gather issued early; chunked or persistent;
                                    optional shared-memory hot rows */
    SYM_MTTKRP_UNFACTORISED = 2, /* one entry per lane group, every position updated separately */
    SYM_MTTKRP_STAGED = 3,       /* the plain kernel with the next batch's leaf factor rows copied into a
                                    shared-memory double buffer (cp.async) while the current batch runs */
    SYM_MTTKRP_LANE = 4          /* chunked warps whose lanes decode one entry each and find its first changed
                                    fiber level, the group then stepping through the entries with one broadcast
                                    per entry; with leaf_index = 1 and a leaf index, two passes with no
                                    per-entry reduction: the canonical stream for every position but the leaf,
                                    then the leaf index for its root (the largest index of each tuple),
                                    unfactorised below the root when strict_smem_kb = 0 */
} sym_mttkrp_kernel;
typedef struct {
    int32_t strict_kernel;     /* sym_mttkrp_kernel for the strict stream */
    int32_t entries_per_warp;  /* work chunk per warp, a multiple of 32; 0 = persistent contiguous slices
                                  (pipelined kernel only) */
    int32_t threads_per_cta;   /* pipelined / unfactorised / staged kernels: 64..512 */
    int32_t ctas_per_sm;       /* persistent grids: CTAs per SM; lane kernel: entries per warp of the
                                  unfactorised root pass / 64 */
    int32_t strict_smem_kb;    /* pipelined kernel: shared memory per CTA for hot (low-index) rows, 0 = none;
                                  lane kernel: 0 = unfactorised root pass, 1 = factorised root pass */
    int32_t diag_smem_kb;      /* diagonal stream: the same, 0 = none */
    int32_t b_share_pct;       /* share of that shared memory holding rows of B (the rest holds rows of M) */
    int32_t leaf_index;        /* plain kernel: 1 = take the leaf position from the tensor's leaf index (see
                                  sym_tensor_add_leaf_index) instead of one reduction per entry (also for the
                                  lane kernel; ignored without a leaf index) */
    int32_t vec_per_lane;      /* plain kernel: float4 column groups per lane, 1 or 2 (2 needs rank >= 8);
                                  lane kernel: its shape, 1 = 4 columns per lane, 4 = the same with four leaf
                                  gathers issued together per lane group (needs rank >= 16), 2 = 8 columns per
                                  lane (ranks below 8 run shape 1) */
    int32_t stream_hint;       /* plain kernel: 1 = read the canonical stream with evict-first loads so it does not
                                  displace factor rows from L1 / L2 */
    int32_t l1_pref;           /* plain kernel: 1 = ask for the largest L1 (no shared-memory carveout) */
    int32_t root_combine;      /* plain and lane kernels: 1 = a CTA merges its lane groups' final root sums in
                                  shared memory and reduces each root once (pays off when a few roots hold a
                                  large share of the entries), 0 = one reduction per lane group */
} sym_mttkrp_cfg;
sym_status sym_mttkrp_default_config(sym_mttkrp_cfg* out);
sym_status sym_mttkrp_set_config(sym_tensor X, const sym_mttkrp_cfg* cfg);
sym_status sym_mttkrp_get_config(sym_tensor X, sym_mttkrp_cfg* out);
/* Shorthand: > 0 selects the plain kernel with that many entries per warp,
 * 0 restores the default configuration, -1 selects the unfactorised kernel. */
sym_status sym_mttkrp_set_chunk(sym_tensor X, int entries_per_warp);
/* Times candidate configurations on this tensor with these operands (M is
 * overwritten), stores the fastest in the tensor and appends it to the text
 * cache `cache_path` (nullable) keyed by device and problem shape; a cache hit
 * skips the timing.  Synchronous. */
sym_status sym_mttkrp_autotune(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                               int64_t ldm, const char* cache_path, sym_stream_t stream, sym_mttkrp_cfg* best,
                               float* best_ms);
/* The same with every timed run preceded by a rewrite of flush [device,
 * flush_bytes, caller-owned scratch, overwritten; make it larger than L2], so
 * the candidates are compared with cold caches, as a caller that runs other
 * work between calls sees them (a small tensor that fits in L2 otherwise
 * favours configurations that re-read it).  flush NULL with flush_bytes 0 is
 * sym_mttkrp_autotune; cache entries of the two are kept apart. */
sym_status sym_mttkrp_autotune_cold(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                                    int64_t ldm, void* flush, size_t flush_bytes, const char* cache_path,
                                    sym_stream_t stream, sym_mttkrp_cfg* best, float* best_ms);

/* One symmetric CP-ALS update of the shared factor (the decomposition the
 * symmetric MTTKRP serves, Sec. 5.2.6):
 *   B_out = M H^{-1},  M = MTTKRP(X, B),  H = (B^T B)^{o(N-1)} + ridge I
 * (o(N-1): elementwise power).  H is formed, Cholesky-factorised and inverted
 * in FP64; the n x R product runs in FP32 and is stored in B's dtype.
 * info [device, 1 int] (nullable) receives 0, or the 1-based column of a
 * non-positive pivot (then B_out = 0).  B_out must not alias B.  ws >=
 * sym_cp_als_workspace_bytes (it holds M, G, L, L^T, H^{-1} and a status word). */
size_t sym_cp_als_workspace_bytes(sym_tensor X, int rank);
sym_status sym_cp_als_step(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, void* B_out,
                           int64_t ldo, double ridge, int* info, void* ws, size_t ws_bytes, sym_stream_t stream);

/* Mode-1 TTM of a fully symmetric 3-way tensor with visible output symmetry
 * (Sec. 4.2, the symmetrised TTM listing and the output-symmetry listings;
 * Sec. 5.2.5):
 *   C[j, l, r] = sum_k A[k, j, l] B[k, r]      (paper: C[i, j, l] = A[k, j, l] * B[k, i])
 * C is symmetric in (j, l); only the canonical triangle j <= l is computed,
 * each canonical entry of A is read once and makes one update per distinct
 * index value (3 for a strict entry: half of its 6 assignments).
 * Layout of C (device, float32, caller-owned, 16-byte aligned, overwritten),
 * rank index fastest, `rank` floats per output position:
 *   SYM_TTM_PACKED: positions (j, l), j <= l, at p = j n - j (j - 1) / 2 + (l - j);
 *   SYM_TTM_FULL:   n x n positions at j n + l; the lower triangle is filled by a
 *                   replication pass after the canonical computation.
 * sym_ttm_output_elems gives the float count (-1 for bad arguments).
 * B: n x rank (row stride ldb), FP32 or BF16; rank 4..128, multiple of 4.
 * Order other than 3, or n > 2^21 (whose output could not be stored):
 * SYM_E_UNSUPPORTED.  Results are accumulated with floating-point atomics:
 * not bitwise reproducible run to run. */
typedef enum { SYM_TTM_PACKED = 0, SYM_TTM_FULL = 1 } sym_ttm_layout;
/* Schedule of the TTM kernels (nullable in sym_ttm: defaults).
 * entries_per_warp: consecutive canonical entries per warp chunk (multiple of 32);
 * ctas_per_sm: 0 = one chunk per warp over a full grid; 1..8 = persistent grid
 *   of that many CTAs per SM, warp w taking chunks w, w + W, ... so the GPU
 *   walks the sorted stream front to back (output rows stay in L2);
 * leaf_index: -1 = use the tensor's leaf index when it has one, 0 = never,
 *   1 = always (SYM_E_INVALID without one).  With it the k = a updates of
 *   strict entries become per-fiber sums in a second pass. */
typedef struct {
    int32_t entries_per_warp;
    int32_t ctas_per_sm;
    int32_t leaf_index;
} sym_ttm_cfg;
sym_status sym_ttm_default_config(sym_ttm_cfg* out);
int64_t sym_ttm_output_elems(int64_t n, int rank, sym_ttm_layout layout);
sym_status sym_ttm(sym_tensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C, sym_ttm_layout layout,
                   const sym_ttm_cfg* cfg, sym_stream_t stream);

/* ===================================================================== */
/* Baseline: MTTKRP over the fully expanded (non-symmetric) tensor          */
/* ===================================================================== */

typedef struct sym_expanded_s* sym_expanded;
/* Sizes for the expanded tensor (all distinct permutations of every entry). */
sym_status sym_expanded_bytes(sym_tensor X, size_t* arena_bytes, size_t* ws_bytes);
/* Writes every distinct permutation of every canonical entry, sorted
 * lexicographically (mode-1 major).  Synchronises `stream`. */
sym_status sym_expanded_create(sym_tensor X, void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                               sym_stream_t stream, sym_expanded* out);
sym_status sym_expanded_info(sym_expanded E, int64_t* nnz);
sym_status sym_expanded_export(sym_expanded E, int32_t* eidx, int64_t ld_out, float* evals, sym_stream_t stream);
/* Plain mode-1 MTTKRP over the expanded tensor: no symmetry used, no atomics
 * except at chunk seams (entries are sorted by mode 1). */
sym_status sym_mttkrp_expanded(sym_expanded E, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* M,
                               int64_t ldm, sym_stream_t stream);
/* Plain mode-1 TTM over the expanded 3-way tensor (no symmetry used): every
 * output position of the full n x n x rank layout (SYM_TTM_FULL) is computed,
 * each (c_1, c_2) fiber summed in registers.  Order other than 3:
 * SYM_E_UNSUPPORTED. */
sym_status sym_ttm_expanded(sym_expanded E, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C,
                            sym_stream_t stream);
sym_status sym_expanded_destroy(sym_expanded E);

/* ===================================================================== */
/* Partially symmetric tensors (Sec. 2.1, Def. "Partial Symmetry")         */
/* ===================================================================== */

/* The `order` modes (1..5) are split into `nparts` consecutive parts of sizes
 * part[0..nparts) (summing to order); the indices of part p range over
 * [0, dim[p]).  The tensor is unchanged by any permutation that moves positions
 * only inside their part, so its canonical triangle keeps the indices
 * non-decreasing inside every part (Sec. 2.1, Def. "Canonical") and one stored
 * entry stands for every distinct arrangement obtained by permuting inside
 * parts (prod over parts of s_p! / prod m!).  One part of size `order` is full
 * symmetry; parts of size 1 are modes without symmetry. */
typedef struct sym_ptensor_s* sym_ptensor;

typedef struct {
    int32_t order;
    int32_t nparts;
    int32_t key_bits;            /* sum over modes of ceil(log2 dim) (<= 128) */
    int64_t nnz;                 /* canonical entries kept */
    int64_t expanded_nnz;        /* full-tensor nonzeros: sum of the arrangements (exact) */
    int64_t duplicates_dropped;  /* SYM_DUP_KEEP_EQUAL copies removed */
    double normsq;               /* ||X||^2 over the full tensor (FP64) */
} sym_ptensor_info_t;

/* Arena (kept by the handle) and workspace (create only) bytes.  part, dim [host]. */
sym_status sym_ptensor_create_bytes(int order, int nparts, const int32_t* part, const int64_t* dim, int64_t nnz,
                                    size_t* arena_bytes, size_t* ws_bytes);
/* Canonicalises the coordinate list idx [device, order arrays of nnz int32 at
 * stride ld_idx] / val [device, nnz floats] on the device: sort inside every
 * part, check each index against its part's dimension (SYM_E_RANGE), sort
 * entries lexicographically, resolve repeated tuples by `dup`
 * (SYM_E_DUPLICATE).  Any inside-part permutation of a stored tuple gives the
 * same tensor.  Synchronises `stream`. */
sym_status sym_ptensor_create(int order, int nparts, const int32_t* part, const int64_t* dim, int64_t nnz,
                              const int32_t* idx, int64_t ld_idx, const float* val, sym_dup_policy dup, void* arena,
                              size_t arena_bytes, void* ws, size_t ws_bytes, sym_stream_t stream, sym_ptensor* out);
sym_status sym_ptensor_info(sym_ptensor X, sym_ptensor_info_t* out);
/* Canonical entries in lexicographic order: cidx [device, order arrays at
 * stride ld_out >= nnz], cval [device, nnz]. */
sym_status sym_ptensor_export(sym_ptensor X, int32_t* cidx, int64_t ld_out, float* cval, sym_stream_t stream);
/* MTTKRP for the factor of part out_part: with f the first mode of that part,
 * M[i, r] = sum over the full tensor's nonzeros x with x_f = i of
 * X[x] * prod_{q != f} F_{part of q}[x_q, r] (Sec. 5.2.6 with one factor per
 * part; any mode of the part gives the same M).  factors [host array of
 * nparts device pointers]: part p's factor, dim[p] x rank, row stride ldf[p]
 * [host] (multiple of 4), FP32 or BF16 (16- / 8-byte aligned rows).  M
 * [device, dim[out_part] x rank, row stride ldm, 16-byte aligned] is
 * overwritten.  rank: 4..128, multiple of 4.  Per canonical entry and per
 * distinct index value u of the output part, one 16-byte-per-lane reduction:
 * M[u] += v W_u prod(F_P rows of the part's other positions)
 * prod_{Q != P} E(c_Q) prod(F_Q rows), W_u and E the integer arrangement
 * counts.  FP32 accumulation with floating-point atomics. */
sym_status sym_pmttkrp(sym_ptensor X, const void* const* factors, const int64_t* ldf, sym_dtype dtype, int rank,
                       int out_part, float* M, int64_t ldm, sym_stream_t stream);
/* Baseline: the same tensor with its symmetry expanded away — every inside-
 * part arrangement of every canonical entry stored (info.expanded_nnz
 * entries), as a tensor with `order` parts of size 1 (no symmetry left);
 * sym_pmttkrp on it with the first mode of a part as out_part gives that
 * part's MTTKRP without exploiting symmetry.  The expansion runs on the
 * device (arrangement counts, scan, next-permutation inside parts) and is
 * then canonicalised like any input.  Synchronises `stream`. */
sym_status sym_ptensor_expand_bytes(sym_ptensor X, size_t* arena_bytes, size_t* ws_bytes);
sym_status sym_ptensor_expand(sym_ptensor X, void* arena, size_t arena_bytes, void* ws, size_t ws_bytes,
                              sym_stream_t stream, sym_ptensor* out);
/* Mode-1 TTM of a partially symmetric order-3 tensor (Sec. 2.1, Def.
 * "Partial Symmetry", with the TTM of Sec. 4.2 and Sec. 5.2.5):
 *   C[j, l, r] = sum_k A[k, j, l] B[k, r]
 * over the full tensor, i.e. every canonical entry applied once for each of
 * its distinct inside-part arrangements.  B [device]: dim(part of mode 1) x
 * rank, row stride ldb, FP32 or BF16 (widened on load); rank 4..128, multiple
 * of 4.  C [device, float32, 16-byte aligned, overwritten], rank index fastest:
 *   SYM_TTM_FULL:   d2 x d3 positions at j d3 + l (d_q = range of mode q);
 *   SYM_TTM_PACKED: only when modes 2 and 3 are in one part (C symmetric in
 *                   (j, l)): positions j <= l at j d - j (j - 1) / 2 + (l - j).
 * sym_pttm_output_elems gives the float count (-1: order other than 3, bad
 * rank, or PACKED without the output symmetry).  Other orders:
 * SYM_E_UNSUPPORTED.  Floating-point atomics: not bitwise reproducible. */
int64_t sym_pttm_output_elems(sym_ptensor X, int rank, int layout);
sym_status sym_pttm(sym_ptensor X, const void* B, sym_dtype bdt, int rank, int64_t ldb, float* C, int layout,
                    sym_stream_t stream);

sym_status sym_ptensor_destroy(sym_ptensor X);

/* ===================================================================== */
/* Serving: continuous batching of MTTKRP requests                          */
/* ===================================================================== */

typedef struct sym_server_s* sym_server;

typedef struct {
    sym_tensor X;        /* a resident tensor */
    const void* B;       /* [device] factor, n x rank, row stride ldb */
    sym_dtype bdt;
    int32_t rank;
    int64_t ldb;
    float* M;            /* [device] output, n x rank, row stride ldm; caller keeps it alive until done */
    int64_t ldm;
    int32_t want_residual; /* 0: none; 1: the FP64 CP-fit residual; 2: the same, and B (same pointer, rank, ldb,
                              type and n) is unchanged since an earlier request to this server, so the Gram
                              matrix B^T B the server computed then may be reused (it keeps the 512 most recent) */
    uint64_t user_tag;
} sym_request;

typedef struct {
    sym_status status;   /* SYM_OK, an error, or SYM_PENDING */
    double residual;     /* CP-fit residual when requested */
    uint64_t user_tag;
    uint64_t t_submit_ns; /* host steady clock */
    uint64_t t_admit_ns;
    uint64_t t_done_ns;
} sym_result;

typedef struct {
    int32_t max_slots;         /* requests in flight at once (device streams) */
    int32_t max_rank;          /* largest rank accepted */
    size_t hbm_budget_bytes;   /* bound on the bytes touched by requests in flight */
    int32_t coalesce_small;    /* 1: the small requests admitted in one scheduler pass share one slot and run back
                                  to back on its stream with one completion event (up to 16 per group) */
    int64_t small_nnz;         /* "small": at most this many canonical entries (also picks high-priority slots) */
    int64_t wait_limit_ns;     /* bound used by sym_server_destroy's drain */
    size_t pool_bytes;         /* device pool for registered tensors (part of the arena and of the budget) */
    int64_t affinity_wait_ns;  /* a request whose registered tensor is not resident waits up to this long while
                                  requests for resident tensors are admitted first (0: first come, first served) */
} sym_server_cfg;

/* Device scratch the server needs (per-slot residual workspaces, then the
 * registered-tensor pool of cfg.pool_bytes). */
size_t sym_server_arena_bytes(const sym_server_cfg* cfg);
/* Starts the scheduler thread.  arena [device] holds per-slot scratch. */
sym_status sym_server_create(const sym_server_cfg* cfg, void* arena, size_t arena_bytes, int device,
                             sym_server* out);
/* Queues a request (non-blocking); *ticket identifies it.  The request is
 * validated on the host first: a bad one fails here with SYM_E_BADREQ or
 * SYM_E_BUDGET and gets no ticket. */
sym_status sym_batch_submit(sym_server S, const sym_request* req, uint64_t* ticket);
/* Registered tensors (residency managed by the server, no paper counterpart):
 * `image` [host] is a tensor image from sym_tensor_save that the caller keeps
 * unchanged for the server's lifetime.  The tensor is loaded into the pool when
 * a request needs it and dropped (least recently used first, never while a
 * request in flight uses it) when another one needs the room.  Requests whose
 * tensor is resident are admitted first; one that needs a load waits up to
 * cfg.affinity_wait_ns while others can run, so that the requests for its
 * tensor queued meanwhile share one load.  SYM_E_BUDGET if it could never fit
 * in the pool. */
sym_status sym_server_register(sym_server S, const void* image, uint64_t* id);
/* As sym_batch_submit for a registered tensor (req->X is ignored); the request
 * is validated on the host, and SYM_E_NOTFOUND names an unknown id. */
sym_status sym_batch_submit_registered(sym_server S, uint64_t id, const sym_request* req, uint64_t* ticket);
/* SYM_PENDING until the request finishes; then its result (once). */
sym_status sym_batch_poll(sym_server S, uint64_t ticket, sym_result* out);
/* Blocks up to timeout_ns for the result (SYM_E_TIMEOUT if it runs out). */
sym_status sym_batch_wait(sym_server S, uint64_t ticket, int64_t timeout_ns, sym_result* out);
typedef struct {
    int64_t submitted, admitted, completed, rejected;
    int64_t launches;          /* slot launches (a grouped launch counts once) */
    int64_t grouped_launches;  /* launches that ran two or more small requests */
    int64_t peak_inflight;     /* requests in flight at once */
    int64_t peak_bytes;        /* in-flight factor / output / tensor bytes plus resident pool bytes */
    int64_t loads;             /* registered tensors brought into the pool */
    int64_t evictions;         /* registered tensors dropped from the pool to make room */
    int64_t peak_resident_bytes, resident_bytes;
    int64_t gram_hits;         /* residuals that reused a cached Gram matrix (want_residual 2) */
} sym_server_stats;
sym_status sym_server_stats_get(sym_server S, sym_server_stats* out);
/* Drains queued and in-flight work (bounded by cfg.wait_limit_ns), stops the
 * scheduler thread and frees the server.  If the limit runs out it returns
 * SYM_E_TIMEOUT: queued requests are dropped, requests already on the device
 * keep running, and the handle must not be used again.  The server's own
 * streams, events and pinned buffers are then released by its scheduler thread
 * once the last in-flight request completes; the caller must keep the arena,
 * the tensors and every buffer of the in-flight requests alive until the device
 * has finished them (for instance until cudaDeviceSynchronize returns). */
sym_status sym_server_destroy(sym_server S);

/* ===================================================================== */
/* Serving: device-resident request loop (MTTKRP and SSYMV / SYPRD)          */
/* ===================================================================== */

/* One persistent kernel serves requests of any order, rank, factor type and
 * kind (symmetric MTTKRP, Sec. 4.3 / Sec. 5.2.6; SSYMV with optional SYPRD,
 * Sec. 3.1 / Sec. 5.2.1 / Sec. 5.2.3) on resident tensors and matrices.  A
 * request is published into a ring in mapped host memory; the kernel's CTAs
 * claim its chunks (output clearing first, then entry ranges), and the CTA that
 * finishes the last chunk writes a completion word back into mapped memory.  No
 * kernel is launched per request: the loop kernel runs while there is work and
 * leaves after cfg.idle_exit_ns without any (the next submission launches it
 * again).  MTTKRP runs in the per-entry form (every canonical entry updates the
 * rows of its distinct indices with their arrangement weights), so the loop
 * suits many small requests; the single calls stay faster for large ones.
 * Inputs (tensor, factor, CSR, x) must be complete on the device before their
 * submission; they are read through L2 only, so they may be rewritten between
 * requests.  Floating-point atomics: not bitwise reproducible. */
typedef struct sym_devloop_s* sym_devloop;

typedef struct {
    int32_t ring_slots;        /* requests published at once (power of two, 16..4096) */
    int32_t ctas;              /* CTAs of the loop kernel (0: two per SM) */
    size_t hbm_budget_bytes;   /* bound on the bytes touched by the published requests */
    int64_t idle_exit_ns;      /* the loop kernel leaves after this long without a published request (> 0) */
    int64_t wait_limit_ns;     /* bound of the kernel's internal waits and of sym_devloop_destroy's drain (> 0) */
} sym_devloop_cfg;

/* Allocates the ring, control and completion words (page-locked, mapped) and
 * the device counters, and calibrates the device clock against the host's
 * steady clock (result timestamps are host steady-clock nanoseconds).
 * Synchronous; SYM_E_INVALID for a bad cfg. */
sym_status sym_devloop_create(const sym_devloop_cfg* cfg, int device, sym_devloop* out);
/* M = MTTKRP(X, B) for a resident tensor (req->X; want_residual must be 0).
 * M [device, n x rank, row stride ldm] is overwritten (cleared by the loop);
 * argument rules as sym_mttkrp.  Requests are published in submission order
 * while a ring slot is free and the published requests' bytes (tensor arena,
 * factor, output) stay within the budget; the rest wait on the host and are
 * published by later calls (submit, poll, wait).  A request larger than the
 * whole budget fails with SYM_E_BUDGET; a malformed one with SYM_E_BADREQ.
 * The caller keeps every buffer alive until the request is done. */
sym_status sym_devloop_submit_mttkrp(sym_devloop L, const sym_request* req, uint64_t* ticket);
/* y = A x for an upper CSR (as sym_spmv; trusted, column indices outside
 * [0, n) skipped); y [device, n floats] overwritten; syprd [device, 1 double,
 * nullable] receives x^T A x (off-diagonal terms twice), FP32 per thread and
 * FP64 across threads and chunks. */
sym_status sym_devloop_submit_ssymv(sym_devloop L, const sym_csr_upper* A, const float* x, float* y,
                                    double* syprd, uint64_t user_tag, uint64_t* ticket);
/* SYM_PENDING until the request is done; then its result (once): status
 * SYM_OK, or SYM_E_TIMEOUT when an internal wait of the kernel ran out (its
 * outputs are then undefined, SYPRD NaN).  t_admit_ns is the publication time,
 * t_done_ns the kernel's completion time on the host clock.  Also retires
 * finished requests and publishes waiting ones. */
sym_status sym_devloop_poll(sym_devloop L, uint64_t ticket, sym_result* out);
/* Polls until the request is done or timeout_ns runs out (SYM_E_TIMEOUT). */
sym_status sym_devloop_wait(sym_devloop L, uint64_t ticket, int64_t timeout_ns, sym_result* out);
/* Test hook of the loop's bounded zero-chunk wait (no paper counterpart): with
 * hook = 1, requests submitted from now on have their zero chunks done but not
 * counted, so their compute chunks' wait runs out after cfg.wait_limit_ns and
 * they complete with SYM_E_TIMEOUT (outputs undefined, SYPRD NaN) while the
 * loop goes on serving; hook = 0 restores normal requests. */
sym_status sym_devloop_set_test_hook(sym_devloop L, int hook);
typedef struct {
    int64_t submitted, published, completed, rejected;
    int64_t launches;       /* launches of the loop kernel */
    int64_t peak_inflight;  /* published requests not yet retired, at most */
    int64_t peak_bytes;     /* their bytes, at most */
} sym_devloop_stats;
sym_status sym_devloop_stats_get(sym_devloop L, sym_devloop_stats* out);
/* Drains submitted work (bounded by cfg.wait_limit_ns), stops the loop kernel
 * and frees everything.  SYM_E_TIMEOUT if the drain ran out (requests still
 * waiting are dropped; the kernel finishes the chunks it holds and leaves). */
sym_status sym_devloop_destroy(sym_devloop L);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* SYMGPU_H */
