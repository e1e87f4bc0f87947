// Batched SSYMV/SYPRD (placeholder entry points; implemented next).
#include "common.cuh"

extern "C" size_t sym_spmv_batch_plan_bytes(const sym_csr_batch*, const int64_t*, const sym_tile_cfg*) { return 0; }
extern "C" sym_status sym_spmv_batch_plan_create(const sym_csr_batch*, const int64_t*, const sym_tile_cfg*, void*,
                                                 size_t, sym_stream_t, sym_batch_plan* out) {
    if (out) *out = nullptr;
    return SYM_E_UNSUPPORTED;
}
extern "C" sym_status sym_spmv_batch_run(sym_batch_plan, const float*, float*, double*, sym_stream_t) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_spmv_batch_capture(sym_batch_plan, const float*, float*, double*, sym_stream_t) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_spmv_batch_graph_launch(sym_batch_plan, sym_stream_t) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_spmv_batch_plan_destroy(sym_batch_plan) { return SYM_OK; }
extern "C" sym_status sym_autotune_spmv_batch(const sym_csr_batch*, const int64_t*, const float*, float*, double*,
                                              void*, size_t, const char*, sym_stream_t, sym_tile_cfg*, float*) {
    return SYM_E_UNSUPPORTED;
}
