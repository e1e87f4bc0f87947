// Internal interface of the SSYMV/SYPRD kernels shared by the batched and the
// allocation-free entry points.
#pragma once

#include "common.cuh"

namespace symgpu {

// Lanes cooperating on one row, from the average row length.
int spmv_lanes(int64_t n, int64_t nnz);
// Checks the CSR descriptor fields on the host (not the arrays).
sym_status validate_csr(const sym_csr_upper* A);
// Bytes of FP64 per-block SYPRD partials for A.
size_t ssymv_partials_bytes(const sym_csr_upper* A);
// True when A is small enough for the one-launch cluster form.
bool ssymv_single_launch(const sym_csr_upper* A);
// The one-launch cluster form (no scratch; y need not be zeroed).
sym_status ssymv_cluster_launch(const sym_csr_upper* A, const float* x, float* y, double* syprd, cudaStream_t s);
// y = A x (and the SYPRD sum when syprd != NULL, partials = scratch doubles);
// small matrices take the one-launch cluster form.
sym_status ssymv_launch(const sym_csr_upper* A, const float* x, float* y, double* syprd, double* partials,
                        cudaStream_t s);

}  // namespace symgpu
