// Serving runtime (placeholder entry points; implemented next).
#include "common.cuh"

extern "C" size_t sym_server_arena_bytes(const sym_server_cfg*) { return 0; }
extern "C" sym_status sym_server_create(const sym_server_cfg*, void*, size_t, int, sym_server* out) {
    if (out) *out = nullptr;
    return SYM_E_UNSUPPORTED;
}
extern "C" sym_status sym_batch_submit(sym_server, const sym_request*, uint64_t*) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_batch_poll(sym_server, uint64_t, sym_result*) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_batch_wait(sym_server, uint64_t, int64_t, sym_result*) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_server_stats_get(sym_server, sym_server_stats*) { return SYM_E_UNSUPPORTED; }
extern "C" sym_status sym_server_destroy(sym_server) { return SYM_OK; }
