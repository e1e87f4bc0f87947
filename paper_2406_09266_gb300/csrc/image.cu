// Relocatable images of canonicalised tensors.
//
// A resident tensor (its canonical key / value arrays, and the leaf index when
// it has one) is saved into one host buffer: a fixed header followed by the
// arrays at 256-byte aligned offsets.  Loading copies the arrays back into any
// caller-given device arena and rebuilds the handle with pointers into it, so
// a serving runtime can drop a tensor from the device and bring it back
// without canonicalising it again.  The tensor is read-only once created, so
// the host image stays valid for as long as the caller keeps it.
#include <new>
#include <string.h>

#include "common.cuh"
#include "tensor.cuh"

namespace symgpu {
namespace {

constexpr uint64_t kImageMagic = 0x32474d4953594d53ull;  // "SMYSIMG2" read as little-endian bytes
constexpr size_t kHeaderBytes = 1024;

struct ImageHeader {
    uint64_t magic;
    int32_t order, bits, kw, has_leaf;
    int64_t n, nnz, nnz_strict;
    sym_mttkrp_cfg cfg;
    sym_tensor_info_t info;
};
static_assert(sizeof(ImageHeader) <= kHeaderBytes, "image header");

// Offsets (from the start of the arrays) of each array in both the host image
// and the device arena: the order and 256-byte alignment of a Carver.
struct ImageLayout {
    size_t lo, hi, val, rlo, rhi, rval, end;
};

ImageLayout image_layout(int64_t nnz, int64_t ns, int kw, bool leaf) {
    ImageLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = align_up(off, 256);
        off = o + align_up(bytes, 256);
        return o;
    };
    const size_t m = nnz > 0 ? (size_t)nnz : 1, ms = ns > 0 ? (size_t)ns : 1;
    L.lo = take(m * 8);
    L.hi = kw == 2 ? take(m * 8) : 0;
    L.val = take(m * 4);
    if (leaf) {
        L.rlo = take(ms * 8);
        L.rhi = kw == 2 ? take(ms * 8) : 0;
        L.rval = take(ms * 4);
    }
    L.end = off;
    return L;
}

}  // namespace
}  // namespace symgpu

using namespace symgpu;

extern "C" size_t sym_tensor_image_bytes(sym_tensor X) {
    if (!X) return 0;
    const ImageLayout L = image_layout(X->nnz, X->nnz_strict, X->kw, X->rklo != nullptr);
    return kHeaderBytes + L.end;
}

extern "C" sym_status sym_tensor_save(sym_tensor X, void* host, size_t host_bytes, sym_stream_t stream) {
    if (!X || !host) return SYM_E_INVALID;
    if (host_bytes < sym_tensor_image_bytes(X)) return SYM_E_NOMEM;
    const bool leaf = X->rklo != nullptr;
    const ImageLayout L = image_layout(X->nnz, X->nnz_strict, X->kw, leaf);
    ImageHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kImageMagic;
    h.order = X->order;
    h.bits = X->bits;
    h.kw = X->kw;
    h.has_leaf = leaf ? 1 : 0;
    h.n = X->n;
    h.nnz = X->nnz;
    h.nnz_strict = X->nnz_strict;
    h.cfg = X->cfg;
    h.info = X->info;
    char* base = static_cast<char*>(host);
    memset(base, 0, kHeaderBytes);
    memcpy(base, &h, sizeof(h));
    char* arr = base + kHeaderBytes;
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)X->nnz, ns = (size_t)X->nnz_strict;
    if (n > 0) {
        SYM_CUDA(cudaMemcpyAsync(arr + L.lo, X->klo, n * 8, cudaMemcpyDeviceToHost, s));
        if (X->kw == 2) SYM_CUDA(cudaMemcpyAsync(arr + L.hi, X->khi, n * 8, cudaMemcpyDeviceToHost, s));
        SYM_CUDA(cudaMemcpyAsync(arr + L.val, X->val, n * 4, cudaMemcpyDeviceToHost, s));
    }
    if (leaf && ns > 0) {
        SYM_CUDA(cudaMemcpyAsync(arr + L.rlo, X->rklo, ns * 8, cudaMemcpyDeviceToHost, s));
        if (X->kw == 2) SYM_CUDA(cudaMemcpyAsync(arr + L.rhi, X->rkhi, ns * 8, cudaMemcpyDeviceToHost, s));
        SYM_CUDA(cudaMemcpyAsync(arr + L.rval, X->rval, ns * 4, cudaMemcpyDeviceToHost, s));
    }
    return SYM_OK;
}

extern "C" size_t sym_tensor_load_bytes(const void* host) {
    if (!host) return 0;
    ImageHeader h;
    memcpy(&h, host, sizeof(h));
    if (h.magic != kImageMagic || h.order < 2 || h.order > 5 || (h.kw != 1 && h.kw != 2) || h.nnz < 0 ||
        h.nnz_strict < 0 || h.nnz_strict > h.nnz)
        return 0;
    return image_layout(h.nnz, h.nnz_strict, h.kw, h.has_leaf != 0).end;
}

extern "C" sym_status sym_tensor_load(const void* host, void* arena, size_t arena_bytes, sym_stream_t stream,
                                      sym_tensor* out) {
    if (!out) return SYM_E_INVALID;
    *out = nullptr;
    const size_t need = sym_tensor_load_bytes(host);
    if (need == 0) return SYM_E_INVALID;
    if (!arena || !aligned(arena, 256)) return SYM_E_INVALID;
    if (arena_bytes < need) return SYM_E_NOMEM;
    ImageHeader h;
    memcpy(&h, host, sizeof(h));
    const bool leaf = h.has_leaf != 0;
    const ImageLayout L = image_layout(h.nnz, h.nnz_strict, h.kw, leaf);
    const char* arr = static_cast<const char*>(host) + kHeaderBytes;
    char* dev = static_cast<char*>(arena);
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)h.nnz, ns = (size_t)h.nnz_strict;
    if (n > 0) {
        SYM_CUDA(cudaMemcpyAsync(dev + L.lo, arr + L.lo, n * 8, cudaMemcpyHostToDevice, s));
        if (h.kw == 2) SYM_CUDA(cudaMemcpyAsync(dev + L.hi, arr + L.hi, n * 8, cudaMemcpyHostToDevice, s));
        SYM_CUDA(cudaMemcpyAsync(dev + L.val, arr + L.val, n * 4, cudaMemcpyHostToDevice, s));
    }
    if (leaf && ns > 0) {
        SYM_CUDA(cudaMemcpyAsync(dev + L.rlo, arr + L.rlo, ns * 8, cudaMemcpyHostToDevice, s));
        if (h.kw == 2) SYM_CUDA(cudaMemcpyAsync(dev + L.rhi, arr + L.rhi, ns * 8, cudaMemcpyHostToDevice, s));
        SYM_CUDA(cudaMemcpyAsync(dev + L.rval, arr + L.rval, ns * 4, cudaMemcpyHostToDevice, s));
    }
    sym_tensor_s* t = new (std::nothrow) sym_tensor_s();
    if (!t) return SYM_E_NOMEM;
    t->order = h.order;
    t->bits = h.bits;
    t->kw = h.kw;
    t->n = h.n;
    t->nnz = h.nnz;
    t->nnz_strict = h.nnz_strict;
    t->klo = reinterpret_cast<uint64_t*>(dev + L.lo);
    t->khi = h.kw == 2 ? reinterpret_cast<uint64_t*>(dev + L.hi) : nullptr;
    t->val = reinterpret_cast<float*>(dev + L.val);
    t->rklo = leaf ? reinterpret_cast<uint64_t*>(dev + L.rlo) : nullptr;
    t->rkhi = (leaf && h.kw == 2) ? reinterpret_cast<uint64_t*>(dev + L.rhi) : nullptr;
    t->rval = leaf ? reinterpret_cast<float*>(dev + L.rval) : nullptr;
    t->cfg = h.cfg;
    t->device = current_device();
    t->info = h.info;
    t->info.arena_used = need;
    *out = t;
    return SYM_OK;
}

extern "C" sym_status sym_tensor_image_info(const void* host, sym_tensor_info_t* out) {
    if (!out || sym_tensor_load_bytes(host) == 0) return SYM_E_INVALID;
    ImageHeader h;
    memcpy(&h, host, sizeof(h));
    *out = h.info;
    return SYM_OK;
}
