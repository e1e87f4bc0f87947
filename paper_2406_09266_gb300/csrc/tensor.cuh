// Device layout of a canonicalised symmetric tensor and its packed keys.
#pragma once

#include "common.cuh"

namespace symgpu {

struct KeyWords {
    uint64_t lo;
    uint64_t hi;
};

// key = sum_q c_q << (bits * (N-1-q)): c_1 is the most significant field, so
// integer order of keys is lexicographic order of the sorted tuples.
template <int N, int KW>
__host__ __device__ __forceinline__ KeyWords pack_key(const int32_t* c, int bits) {
    if constexpr (KW == 1) {
        uint64_t k = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) k = (k << bits) | (uint64_t)(uint32_t)c[q];
        return KeyWords{k, 0ull};
    } else {
        unsigned __int128 k = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) k = (k << bits) | (unsigned __int128)(uint32_t)c[q];
        return KeyWords{(uint64_t)k, (uint64_t)(k >> 64)};
    }
}

template <int N, int KW>
__host__ __device__ __forceinline__ void unpack_key(KeyWords w, int bits, int32_t* c) {
    if constexpr (KW == 1) {
        const uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1);
        uint64_t k = w.lo;
#pragma unroll
        for (int q = N - 1; q >= 0; --q) {
            c[q] = (int32_t)(k & mask);
            k >>= bits;
        }
    } else {
        const unsigned __int128 mask = (((unsigned __int128)1) << bits) - 1;
        unsigned __int128 k = ((unsigned __int128)w.hi << 64) | w.lo;
#pragma unroll
        for (int q = N - 1; q >= 0; --q) {
            c[q] = (int32_t)(uint64_t)(k & mask);
            k >>= bits;
        }
    }
}

}  // namespace symgpu

// Host-side handle.  Device arrays live in the caller's arena:
// entries [0, nnz_strict) are the strict stream, [nnz_strict, nnz) the
// diagonal stream, each in lexicographic order.
struct sym_tensor_s {
    int order;
    int bits;
    int kw;
    int64_t n;
    int64_t nnz;
    int64_t nnz_strict;
    uint64_t* klo;
    uint64_t* khi;
    float* val;
    uint64_t* rklo;  // leaf index: strict entries with reversed tuples (c_N first), sorted; null if absent
    uint64_t* rkhi;
    float* rval;
    sym_mttkrp_cfg cfg;  // MTTKRP kernel configuration
    int device;
    sym_tensor_info_t info;
};
