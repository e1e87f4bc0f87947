// Allocation-free SSYMV + SYPRD.
//
// sym_spmv needs a caller-provided workspace for its per-block FP64 SYPRD
// partials.  Some callers cannot provide one: a host application that hands
// the whole device memory to its own pool allocator and forbids allocations
// from libraries, code that must keep running after device memory is
// exhausted, or code that must not call cudaMalloc because it can synchronise
// the device in the middle of a latency-critical loop.  sym_spmv_noalloc runs
// the same kernels with the partials in a fixed array compiled into this
// library instead.
//
// The array is a file-scope __device__ object: every GPU that loads the library
// holds it (256 KiB) until the process exits.  Its host-side name is only a
// stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device that asks for SYPRD; make that first call before any stream
// capture.  The looked-up address is kept for the life of the process: after
// cudaDeviceReset the module may load at another address, so a process that
// resets a device must not call this entry point on it again.  All calls
// share the array: calls whose work overlaps on the GPU (other streams, other
// threads) race on it and must be serialised by the caller.  Nothing in it has
// to start at zero: each call writes every slot it later reads.  Only SYPRD
// uses the array, so the size limit applies only to calls that ask for it.
#include <mutex>

#include "common.cuh"
#include "spmv.cuh"

namespace {

constexpr int64_t kNoAllocSlots = 32768;  // FP64 partials: 256 KiB per device (one slot per 8+ rows)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_partials[kNoAllocSlots];

std::mutex g_noalloc_mu;
double* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the array on the current device (looked up once per device).
sym_status noalloc_partials(double** out) {
    int dev = 0;
    SYM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SYM_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return symgpu::cuda_status(e);
        g_noalloc_addr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_addr[dev];
    return SYM_OK;
}

}  // namespace

extern "C" sym_status sym_spmv_noalloc(const sym_csr_upper* A, const float* x, float* y, double* syprd,
                                       sym_stream_t stream) {
    using namespace symgpu;
    sym_status st = validate_csr(A);
    if (st != SYM_OK) return st;
    if (A->n > 0 && (!x || !y)) return SYM_E_INVALID;
    double* partials = nullptr;
    if (syprd) {
        // more partial slots than the fixed array holds: refused before anything is looked up or enqueued
        if (ssymv_partials_bytes(A) > sizeof(double) * (size_t)kNoAllocSlots) return SYM_E_UNSUPPORTED;
        st = noalloc_partials(&partials);
        if (st != SYM_OK) return st;
    }
    return ssymv_launch(A, x, y, syprd, partials, as_stream(stream));
}
