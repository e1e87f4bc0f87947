"""Python binding of libsymgpu (the C ABI in include/symgpu.h).

Argument marshalling only: PyTorch supplies device memory (arenas and
workspaces sized by the library's *_bytes queries) and streams; every step of
the symmetric kernels runs in libsymgpu's CUDA code.  There is no CPU fallback:
if the shared library is missing or cannot load, every call raises.

Names follow the C ABI: sym_tensor_create -> SymTensor, sym_mttkrp ->
SymTensor.mttkrp, sym_spmv -> spmv, sym_batch_submit/poll -> Server.submit/poll.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsymgpu.so")

SYM_OK, SYM_PENDING = 0, 1
STATUS = {0: "SYM_OK", -1: "SYM_E_INVALID", -2: "SYM_E_NONCANONICAL", -3: "SYM_E_RANGE", -4: "SYM_E_DUPLICATE",
          -5: "SYM_E_NOMEM", -6: "SYM_E_BUDGET", -7: "SYM_E_TIMEOUT", -8: "SYM_E_CUDA", -9: "SYM_E_BADREQ",
          -10: "SYM_E_UNSUPPORTED", -11: "SYM_E_NOTFOUND", 1: "SYM_PENDING"}
F32, BF16 = 0, 1
DUP_ERROR, DUP_KEEP_EQUAL = 0, 1
TTM_PACKED, TTM_FULL = 0, 1


class SymError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


# ------------------------------------------------------------------ C structs

class TtmCfg(C.Structure):
    _fields_ = [("entries_per_warp", C.c_int32), ("ctas_per_sm", C.c_int32), ("leaf_index", C.c_int32)]


class CsrUpper(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


CsrFull = CsrUpper


class CsrBatch(C.Structure):
    _fields_ = [("count", C.c_int64), ("total_rows", C.c_int64), ("total_nnz", C.c_int64),
                ("row_off", C.c_void_p), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class TileCfg(C.Structure):
    _fields_ = [("rows_per_tile", C.c_int32), ("lanes_per_row", C.c_int32), ("threads_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("local_smem_kb", C.c_int32), ("tile_order", C.c_int32),
                ("x_smem_kb", C.c_int32), ("band_rows", C.c_int32), ("band_max", C.c_int32),
                ("band_chunk", C.c_int32), ("band_order", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TensorInfo(C.Structure):
    _fields_ = [("order", C.c_int32), ("key_bits", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64),
                ("nnz_strict", C.c_int64), ("nnz_diag", C.c_int64), ("duplicates_dropped", C.c_int64),
                ("counts_by_pattern", C.c_int64 * 16), ("expanded_nnz", C.c_int64), ("root_fibers", C.c_int64),
                ("l2_fibers", C.c_int64), ("normsq", C.c_double), ("arena_used", C.c_size_t)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["counts_by_pattern"] = list(self.counts_by_pattern)
        return d


class PTensorInfo(C.Structure):
    _fields_ = [("order", C.c_int32), ("nparts", C.c_int32), ("key_bits", C.c_int32), ("nnz", C.c_int64),
                ("expanded_nnz", C.c_int64), ("duplicates_dropped", C.c_int64), ("normsq", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("X", C.c_void_p), ("B", C.c_void_p), ("bdt", C.c_int), ("rank", C.c_int32), ("ldb", C.c_int64),
                ("M", C.c_void_p), ("ldm", C.c_int64), ("want_residual", C.c_int32), ("user_tag", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("residual", C.c_double), ("user_tag", C.c_uint64),
                ("t_submit_ns", C.c_uint64), ("t_admit_ns", C.c_uint64), ("t_done_ns", C.c_uint64)]


class ServerCfg(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("max_rank", C.c_int32), ("hbm_budget_bytes", C.c_size_t),
                ("coalesce_small", C.c_int32), ("small_nnz", C.c_int64), ("wait_limit_ns", C.c_int64),
                ("pool_bytes", C.c_size_t), ("affinity_wait_ns", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("launches", C.c_int64), ("grouped_launches", C.c_int64),
                ("peak_inflight", C.c_int64), ("peak_bytes", C.c_int64), ("loads", C.c_int64),
                ("evictions", C.c_int64), ("peak_resident_bytes", C.c_int64), ("resident_bytes", C.c_int64),
                ("gram_hits", C.c_int64)]


class DevLoopCfg(C.Structure):
    _fields_ = [("ring_slots", C.c_int32), ("ctas", C.c_int32), ("hbm_budget_bytes", C.c_size_t),
                ("idle_exit_ns", C.c_int64), ("wait_limit_ns", C.c_int64)]


class DevLoopStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("published", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("launches", C.c_int64), ("peak_inflight", C.c_int64),
                ("peak_bytes", C.c_int64)]


class MttkrpCfg(C.Structure):
    _fields_ = [("strict_kernel", C.c_int32), ("entries_per_warp", C.c_int32), ("threads_per_cta", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("strict_smem_kb", C.c_int32), ("diag_smem_kb", C.c_int32),
                ("b_share_pct", C.c_int32), ("leaf_index", C.c_int32), ("vec_per_lane", C.c_int32),
                ("stream_hint", C.c_int32), ("l1_pref", C.c_int32), ("root_combine", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


MTTKRP_PLAIN, MTTKRP_PIPELINED, MTTKRP_UNFACTORISED, MTTKRP_STAGED, MTTKRP_LANE = 0, 1, 2, 3, 4


class ProfileEntry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double)]


# ------------------------------------------------------------------ loading

_lock = threading.Lock()
_lib = None

_SIGS = {
    "sym_status_string": ([C.c_int], C.c_char_p),
    "sym_last_cuda_error": ([], C.c_int),
    "sym_version": ([], C.c_int),
    "sym_profile_enable": ([C.c_int], C.c_int),
    "sym_profile_read": ([C.c_void_p, C.c_int], C.c_int),
    "sym_profile_reset": ([], C.c_int),
    "sym_bounds_check_enabled": ([], C.c_int),
    "sym_bounds_check_attach": ([C.c_void_p], C.c_int),
    "sym_ceiling_bytes": ([C.c_int, C.c_int64, C.c_int], C.c_size_t),
    "sym_ceiling_run": ([C.c_int, C.c_void_p, C.c_size_t, C.c_int64, C.c_int, C.c_int64, C.c_int, C.c_void_p,
                         C.c_void_p, C.c_void_p], C.c_int),
    "sym_spmv_workspace_bytes": ([C.c_void_p], C.c_size_t),
    "sym_spmv": ([C.c_void_p] * 5 + [C.c_size_t, C.c_void_p], C.c_int),
    "sym_spmv_noalloc": ([C.c_void_p] * 5, C.c_int),
    "sym_spmv_rows": ([C.c_void_p] * 4 + [C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_size_t, C.c_void_p],
                      C.c_int),
    "sym_spmv_single_launch": ([C.c_void_p], C.c_int),
    "sym_csr_upper_check": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_bellman_step": ([C.c_void_p] * 4, C.c_int),
    "sym_csr_expand_bytes": ([C.c_void_p, C.c_void_p], C.c_size_t),
    "sym_csr_expand_upper": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p,
                              C.c_void_p], C.c_int),
    "sym_spmv_full": ([C.c_void_p] * 4, C.c_int),
    "sym_spmv_batch_plan_bytes": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_size_t),
    "sym_spmv_batch_plan_create": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.c_void_p], C.c_int),
    "sym_spmv_batch_run": ([C.c_void_p] * 5, C.c_int),
    "sym_spmv_batch_capture": ([C.c_void_p] * 5, C.c_int),
    "sym_spmv_batch_graph_launch": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_spmv_batch_check": ([C.c_void_p], C.c_int),
    "sym_spmv_batch_clear_status": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_spmv_batch_run_bounded": ([C.c_void_p] * 4 + [C.c_int64, C.c_int64, C.c_void_p], C.c_int),
    "sym_spmv_cluster_bounded": ([C.c_void_p] * 4 + [C.c_int64, C.c_int, C.c_void_p], C.c_int),
    "sym_spmv_batch_plan_destroy": ([C.c_void_p], C.c_int),
    "sym_autotune_spmv_batch": ([C.c_void_p] * 6 + [C.c_size_t, C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p],
                                C.c_int),
    "sym_tensor_create_bytes": ([C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_create": ([C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                           C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_info": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_export": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_destroy": ([C.c_void_p], C.c_int),
    "sym_tensor_upper_csr_ws_bytes": ([C.c_void_p], C.c_size_t),
    "sym_tensor_image_bytes": ([C.c_void_p], C.c_size_t),
    "sym_tensor_save": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "sym_tensor_load_bytes": ([C.c_void_p], C.c_size_t),
    "sym_tensor_load": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_leaf_index_bytes": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_add_leaf_index": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p],
                                  C.c_int),
    "sym_tensor_upper_csr": ([C.c_void_p] * 5 + [C.c_size_t, C.c_void_p], C.c_int),
    "sym_gen_batch_coords": ([C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_int64,
                              C.c_void_p, C.c_void_p], C.c_int),
    "sym_gen_coords": ([C.c_int, C.c_int64, C.c_int64, C.c_uint64, C.c_void_p, C.c_int64, C.c_void_p,
                        C.c_void_p], C.c_int),
    "sym_mttkrp_workspace_bytes": ([C.c_void_p, C.c_int, C.c_int, C.c_int], C.c_size_t),
    "sym_mttkrp": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                    C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "sym_mttkrp_range": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int64,
                          C.c_int64, C.c_int, C.c_void_p], C.c_int),
    "sym_mttkrp_set_chunk": ([C.c_void_p, C.c_int], C.c_int),
    "sym_mttkrp_default_config": ([C.c_void_p], C.c_int),
    "sym_mttkrp_set_config": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_mttkrp_get_config": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_mttkrp_autotune": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_char_p,
                             C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_mttkrp_autotune_cold": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64,
                                  C.c_void_p, C.c_size_t, C.c_char_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_cp_als_workspace_bytes": ([C.c_void_p, C.c_int], C.c_size_t),
    "sym_cp_als_step": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_double,
                         C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p], C.c_int),
    "sym_ttm_output_elems": ([C.c_int64, C.c_int, C.c_int], C.c_int64),
    "sym_ttm_default_config": ([C.c_void_p], C.c_int),
    "sym_ttm": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p],
                C.c_int),
    "sym_ttm_expanded": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_expanded_bytes": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_expanded_create": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p,
                             C.c_void_p], C.c_int),
    "sym_expanded_info": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_expanded_export": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_mttkrp_expanded": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int64,
                             C.c_void_p], C.c_int),
    "sym_expanded_destroy": ([C.c_void_p], C.c_int),
    "sym_ptensor_create_bytes": ([C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
                                 C.c_int),
    "sym_ptensor_create": ([C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                            C.c_int, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p], C.c_int),
    "sym_ptensor_info": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_ptensor_export": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_pmttkrp": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64,
                     C.c_void_p], C.c_int),
    "sym_ptensor_expand_bytes": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_ptensor_expand": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p],
                           C.c_int),
    "sym_ptensor_destroy": ([C.c_void_p], C.c_int),
    "sym_pttm_output_elems": ([C.c_void_p, C.c_int, C.c_int], C.c_int64),
    "sym_pttm": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "sym_server_arena_bytes": ([C.c_void_p], C.c_size_t),
    "sym_server_create": ([C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p], C.c_int),
    "sym_batch_submit": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_batch_poll": ([C.c_void_p, C.c_uint64, C.c_void_p], C.c_int),
    "sym_server_register": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_batch_submit_registered": ([C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p], C.c_int),
    "sym_tensor_image_info": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_batch_wait": ([C.c_void_p, C.c_uint64, C.c_int64, C.c_void_p], C.c_int),
    "sym_server_stats_get": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_server_destroy": ([C.c_void_p], C.c_int),
    "sym_devloop_create": ([C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "sym_devloop_submit_mttkrp": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "sym_devloop_submit_ssymv": ([C.c_void_p] * 5 + [C.c_uint64, C.c_void_p], C.c_int),
    "sym_devloop_poll": ([C.c_void_p, C.c_uint64, C.c_void_p], C.c_int),
    "sym_devloop_wait": ([C.c_void_p, C.c_uint64, C.c_int64, C.c_void_p], C.c_int),
    "sym_devloop_stats_get": ([C.c_void_p, C.c_void_p], C.c_int),
    "sym_devloop_set_test_hook": ([C.c_void_p, C.c_int], C.c_int),
    "sym_devloop_destroy": ([C.c_void_p], C.c_int),
}


def exported_symbols():
    """Names the C ABI declares (include/symgpu.h) and this binding wires up."""
    return sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Loads libsymgpu.so; raises if it is missing (no fallback path exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libsymgpu.so is not built ({path}); run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes, f.restype = args, res
        _lib = L
        return L


def lib():
    return _lib if _lib is not None else load()


def check(code: int, what: str):
    if code != SYM_OK:
        raise SymError(code, what)


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _scratch(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _dtype_code(B: torch.Tensor) -> int:
    if B.dtype == torch.float32:
        return F32
    if B.dtype == torch.bfloat16:
        return BF16
    raise TypeError("factor must be float32 or bfloat16")


# ------------------------------------------------------------------ profiling

def profile_enable(on: bool = True):
    check(lib().sym_profile_enable(int(on)), "sym_profile_enable")


def profile_reset():
    check(lib().sym_profile_reset(), "sym_profile_reset")


def profile_read() -> dict:
    """{kernel name: (launches, total event ms)} since the last reset."""
    buf = (ProfileEntry * 64)()
    k = lib().sym_profile_read(buf, 64)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(k)}


# ------------------------------------------------------------------ SSYMV / SYPRD

CEILINGS = {"fma": 0, "row_gather": 1, "row_red": 2, "gather_red": 3, "smem_f32": 4, "smem_u32": 5, "hbm_copy": 6,
            "bulk_gather": 7, "bulk_red": 8}


def ceiling(kind: str, rows: int = 0, rank: int = 64, ops: int = 1 << 26, reps: int = 10, device=None,
            stream=None):
    """Times one primitive operation alone (sym_ceiling_run); returns (rate, ms per launch)."""
    k = CEILINGS[kind]
    nbytes = lib().sym_ceiling_bytes(k, rows, rank)
    if nbytes == 0:
        raise SymError(-1, "sym_ceiling_bytes")
    buf = _scratch(nbytes, device or torch.device("cuda", torch.cuda.current_device()))
    rate, ms = C.c_double(0), C.c_float(0)
    check(lib().sym_ceiling_run(k, _ptr(buf), nbytes, rows, rank, ops, reps, _stream(stream), C.byref(rate),
                                C.byref(ms)), "sym_ceiling_run")
    return rate.value, ms.value


def csr_upper(n, rowptr, col, val) -> CsrUpper:
    return CsrUpper(int(n), int(col.numel()), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())


def spmv_workspace(n, rowptr, col, val, device=None) -> torch.Tensor:
    A = csr_upper(n, rowptr, col, val)
    return _scratch(lib().sym_spmv_workspace_bytes(C.byref(A)), device or rowptr.device)


def spmv(n, rowptr, col, val, x, y=None, syprd=False, ws=None, stream=None):
    """y = A x for the symmetric A given by its upper-triangle CSR; optionally SYPRD x^T A x (FP64)."""
    A = csr_upper(n, rowptr, col, val)
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=x.device)
    s_out = torch.empty(1, dtype=torch.float64, device=x.device) if syprd else None
    if syprd and ws is None:
        ws = _scratch(lib().sym_spmv_workspace_bytes(C.byref(A)), x.device)
    check(lib().sym_spmv(C.byref(A), _ptr(x), _ptr(y), _ptr(s_out), _ptr(ws), ws.numel() if ws is not None else 0,
                         _stream(stream)), "sym_spmv")
    return (y, s_out) if syprd else y


def spmv_rows(n, rowptr, col, val, x, row_begin, row_end, y=None, syprd=False, accumulate=False, ws=None,
              stream=None):
    """One row-range part of y = A x (and of x^T A x): sym_spmv_rows."""
    A = csr_upper(n, rowptr, col, val)
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=x.device)
    s_out = torch.empty(1, dtype=torch.float64, device=x.device) if syprd else None
    if syprd and ws is None:
        ws = _scratch(lib().sym_spmv_workspace_bytes(C.byref(A)), x.device)
    check(lib().sym_spmv_rows(C.byref(A), _ptr(x), _ptr(y), _ptr(s_out), int(row_begin), int(row_end),
                              int(accumulate), _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream)),
          "sym_spmv_rows")
    return (y, s_out) if syprd else y


def spmv_cluster_bounded(n, rowptr, col, val, x, wait_limit_ns=0, skip_to=-1, stream=None):
    """Test hook of the one-launch form's inbox wait (sym_spmv_cluster_bounded); returns (y, syprd)."""
    A = csr_upper(n, rowptr, col, val)
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    s_out = torch.empty(1, dtype=torch.float64, device=x.device)
    check(lib().sym_spmv_cluster_bounded(C.byref(A), _ptr(x), _ptr(y), _ptr(s_out), int(wait_limit_ns), int(skip_to),
                                         _stream(stream)), "sym_spmv_cluster_bounded")
    return y, s_out


def spmv_single_launch(n, nnz) -> bool:
    """True when sym_spmv runs an n x n upper CSR with nnz entries as the one-launch cluster form (host-only)."""
    A = CsrUpper(int(n), int(nnz), 1, 1, 1)
    return bool(lib().sym_spmv_single_launch(C.byref(A)))


def spmv_noalloc(n, rowptr, col, val, x, y, syprd_out=None, stream=None):
    """sym_spmv_noalloc: the same product with no workspace (y and syprd_out preallocated by the caller)."""
    A = csr_upper(n, rowptr, col, val)
    check(lib().sym_spmv_noalloc(C.byref(A), _ptr(x), _ptr(y), _ptr(syprd_out), _stream(stream)), "sym_spmv_noalloc")
    return y


def csr_upper_check(n, rowptr, col, val, stream=None) -> int:
    A = csr_upper(n, rowptr, col, val)
    bad = torch.zeros(1, dtype=torch.int64, device=rowptr.device)
    check(lib().sym_csr_upper_check(C.byref(A), _ptr(bad), _stream(stream)), "sym_csr_upper_check")
    return int(bad.item())


def bellman_step(n, rowptr, col, val, d, y=None, stream=None):
    A = csr_upper(n, rowptr, col, val)
    if y is None:
        y = torch.empty_like(d)
    check(lib().sym_bellman_step(C.byref(A), _ptr(d), _ptr(y), _stream(stream)), "sym_bellman_step")
    return y


class FullCSR:
    """Both-triangle CSR built on the device from an upper CSR (the non-symmetric baseline)."""

    def __init__(self, n, rowptr, col, val, stream=None):
        A = csr_upper(n, rowptr, col, val)
        wsb = C.c_size_t(0)
        ab = lib().sym_csr_expand_bytes(C.byref(A), C.byref(wsb))
        self.arena = _scratch(ab, rowptr.device)
        ws = _scratch(wsb.value, rowptr.device)
        self.desc = CsrFull()
        check(lib().sym_csr_expand_upper(C.byref(A), _ptr(self.arena), self.arena.numel(), _ptr(ws), ws.numel(),
                                         _stream(stream), C.byref(self.desc)), "sym_csr_expand_upper")
        self.n, self.nnz = self.desc.n, self.desc.nnz

    def spmv(self, x, y=None, stream=None):
        if y is None:
            y = torch.empty_like(x)
        check(lib().sym_spmv_full(C.byref(self.desc), _ptr(x), _ptr(y), _stream(stream)), "sym_spmv_full")
        return y

    def arrays(self):
        """(rowptr, col, val) as torch views of the arena."""
        base = self.arena.data_ptr()
        n, nnz = self.n, self.nnz

        def view(ptr, count, dtype):
            off = ptr - base
            es = torch.tensor([], dtype=dtype).element_size()
            return self.arena[off: off + count * es].view(dtype)
        return (view(self.desc.rowptr, n + 1, torch.int32), view(self.desc.col, nnz, torch.int32),
                view(self.desc.val, nnz, torch.float32))


# ------------------------------------------------------------------ tensors

class SymTensor:
    """A canonicalised fully symmetric sparse tensor resident on the device."""

    def __init__(self, idx: torch.Tensor, val: torch.Tensor, n: int, dup: int = DUP_ERROR, stream=None,
                 ws: torch.Tensor | None = None):
        if idx.dim() != 2 or idx.dtype != torch.int32 or not (idx.is_cuda or idx.is_pinned()):
            raise TypeError("idx must be a (order, nnz) int32 CUDA tensor or pinned host tensor")
        if val.dtype != torch.float32 or not (val.is_cuda or val.is_pinned()):
            raise TypeError("val must be a float32 CUDA tensor or pinned host tensor")
        if not val.is_cuda and not val.is_contiguous():
            raise TypeError("a pinned host val must be contiguous")
        dev = val.device if val.is_cuda else (idx.device if idx.is_cuda else
                                              torch.device("cuda", torch.cuda.current_device()))
        order, nnz = idx.shape
        if idx.is_cuda:
            idx = idx.contiguous()
        elif not idx.is_contiguous():
            raise TypeError("a pinned host idx must be contiguous")
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_tensor_create_bytes(order, n, nnz, C.byref(ab), C.byref(wb)), "sym_tensor_create_bytes")
        self.arena = _scratch(ab.value, dev)
        if ws is None or ws.numel() < wb.value:
            ws = _scratch(wb.value, dev)
        h = C.c_void_p()
        check(lib().sym_tensor_create(order, n, nnz, _ptr(idx), max(nnz, 1),
                                      _ptr(val.contiguous() if val.is_cuda else val), dup, _ptr(self.arena),
                                      self.arena.numel(), _ptr(ws), ws.numel(), _stream(stream), C.byref(h)),
              "sym_tensor_create")
        self.handle = h
        self.order, self.n = order, n
        self.device = dev
        self._info = None

    def save_image(self, host: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Relocatable image of the tensor in (pinned) host memory (sym_tensor_save); synchronises the stream."""
        nb = lib().sym_tensor_image_bytes(self.handle)
        if host is None:
            host = torch.empty(nb, dtype=torch.uint8).pin_memory()
        check(lib().sym_tensor_save(self.handle, C.c_void_p(host.data_ptr()), host.numel(), _stream(stream)),
              "sym_tensor_save")
        (stream or torch.cuda.current_stream()).synchronize()
        return host

    @classmethod
    def from_image(cls, host: torch.Tensor, device=None, stream=None) -> "SymTensor":
        """A tensor rebuilt from an image (sym_tensor_load) into a fresh device arena."""
        dev = device or torch.device("cuda", torch.cuda.current_device())
        nb = lib().sym_tensor_load_bytes(C.c_void_p(host.data_ptr()))
        if nb == 0:
            raise SymError(-1, "sym_tensor_load_bytes")
        X = cls.__new__(cls)
        X.arena = _scratch(nb, dev)
        h = C.c_void_p()
        check(lib().sym_tensor_load(C.c_void_p(host.data_ptr()), _ptr(X.arena), X.arena.numel(), _stream(stream),
                                    C.byref(h)), "sym_tensor_load")
        X.handle = h
        X._info = None
        inf = X.info()
        X.order, X.n, X.device = inf["order"], inf["n"], dev
        return X

    @staticmethod
    def create_ws_bytes(order, n, nnz) -> int:
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_tensor_create_bytes(order, n, nnz, C.byref(ab), C.byref(wb)), "sym_tensor_create_bytes")
        return wb.value

    def info(self) -> dict:
        if self._info is None:
            inf = TensorInfo()
            check(lib().sym_tensor_info(self.handle, C.byref(inf)), "sym_tensor_info")
            self._info = inf.as_dict()
        return self._info

    @property
    def nnz(self) -> int:
        return self.info()["nnz"]

    def export(self, stream=None):
        """(cidx (order x nnz) int32, cval) on the device: strict stream, then diagonal stream."""
        nnz = self.nnz
        cidx = torch.empty((self.order, max(nnz, 1)), dtype=torch.int32, device=self.device)
        cval = torch.empty(max(nnz, 1), dtype=torch.float32, device=self.device)
        check(lib().sym_tensor_export(self.handle, _ptr(cidx), max(nnz, 1), _ptr(cval), _stream(stream)),
              "sym_tensor_export")
        return cidx[:, :nnz], cval[:nnz]

    def set_chunk(self, entries_per_warp: int):
        check(lib().sym_mttkrp_set_chunk(self.handle, entries_per_warp), "sym_mttkrp_set_chunk")

    def set_config(self, strict_kernel=MTTKRP_PLAIN, entries_per_warp=256, threads_per_cta=256, ctas_per_sm=2,
                   strict_smem_kb=0, diag_smem_kb=96, b_share_pct=0, leaf_index=1, vec_per_lane=1, stream_hint=0,
                   l1_pref=0, root_combine=1):
        cfg = MttkrpCfg(strict_kernel, entries_per_warp, threads_per_cta, ctas_per_sm, strict_smem_kb, diag_smem_kb,
                        b_share_pct, leaf_index, vec_per_lane, stream_hint, l1_pref, root_combine)
        check(lib().sym_mttkrp_set_config(self.handle, C.byref(cfg)), "sym_mttkrp_set_config")

    def add_leaf_index(self, stream=None):
        """Builds the leaf index (strict stream sorted by its last coordinate); MTTKRP then uses it."""
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_tensor_leaf_index_bytes(self.handle, C.byref(ab), C.byref(wb)), "sym_tensor_leaf_index_bytes")
        self.leaf_arena = _scratch(ab.value, self.device)
        ws = _scratch(wb.value, self.device)
        check(lib().sym_tensor_add_leaf_index(self.handle, _ptr(self.leaf_arena), self.leaf_arena.numel(), _ptr(ws),
                                              ws.numel(), _stream(stream)), "sym_tensor_add_leaf_index")
        self._info = None

    def get_config(self) -> dict:
        cfg = MttkrpCfg()
        check(lib().sym_mttkrp_get_config(self.handle, C.byref(cfg)), "sym_mttkrp_get_config")
        return cfg.as_dict()

    def autotune(self, B: torch.Tensor, M: torch.Tensor | None = None, cache_path: str | None = None, stream=None,
                 flush: torch.Tensor | None = None):
        """Times kernel configurations for these operands; keeps the fastest. Returns (config dict, ms).
        flush: a device buffer larger than L2, rewritten before every timed run (cold-cache comparison)."""
        rank = B.shape[1]
        if M is None:
            M = torch.empty((self.n, rank), dtype=torch.float32, device=B.device)
        best, ms = MttkrpCfg(), C.c_float(0)
        path = cache_path.encode() if cache_path else None
        if flush is None:
            check(lib().sym_mttkrp_autotune(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(M),
                                            M.stride(0), path, _stream(stream), C.byref(best), C.byref(ms)),
                  "sym_mttkrp_autotune")
        else:
            check(lib().sym_mttkrp_autotune_cold(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(M),
                                                 M.stride(0), _ptr(flush), flush.numel() * flush.element_size(),
                                                 path, _stream(stream), C.byref(best), C.byref(ms)),
                  "sym_mttkrp_autotune_cold")
        return best.as_dict(), ms.value

    def mttkrp_workspace(self, rank: int, bdt: int = F32, residual: bool = True) -> torch.Tensor:
        return _scratch(lib().sym_mttkrp_workspace_bytes(self.handle, rank, bdt, int(residual)), self.device)

    def mttkrp(self, B: torch.Tensor, M: torch.Tensor | None = None, residual: bool = False,
               ws: torch.Tensor | None = None, stream=None):
        """Symmetric MTTKRP M = X_(1) (B kr ... kr B); optional FP64 CP-fit residual (device scalar)."""
        rank = B.shape[1]
        bdt = _dtype_code(B)
        if M is None:
            M = torch.empty((self.n, rank), dtype=torch.float32, device=B.device)
        res = torch.empty(1, dtype=torch.float64, device=B.device) if residual else None
        if residual and ws is None:
            ws = self.mttkrp_workspace(rank, bdt, True)
        check(lib().sym_mttkrp(self.handle, _ptr(B), bdt, rank, B.stride(0), _ptr(M), M.stride(0), _ptr(res),
                               _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream)), "sym_mttkrp")
        return (M, res) if residual else M

    def mttkrp_range(self, B: torch.Tensor, first: int, count: int, M: torch.Tensor | None = None,
                     accumulate: bool = False, stream=None):
        """Contribution of canonical entries [first, first + count) to the MTTKRP (sym_mttkrp_range)."""
        rank = B.shape[1]
        if M is None:
            M = torch.empty((self.n, rank), dtype=torch.float32, device=B.device)
        check(lib().sym_mttkrp_range(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(M), M.stride(0),
                                     int(first), int(count), int(accumulate), _stream(stream)), "sym_mttkrp_range")
        return M

    def upper_csr(self, stream=None):
        """Order-2 tensors: (rowptr int64, col int32, val) of the canonical entries as an upper CSR."""
        if self.order != 2:
            raise ValueError("upper CSR needs an order-2 tensor")
        nnz = self.nnz
        rowptr = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
        val = torch.empty(max(nnz, 1), dtype=torch.float32, device=self.device)
        ws = _scratch(lib().sym_tensor_upper_csr_ws_bytes(self.handle), self.device)
        check(lib().sym_tensor_upper_csr(self.handle, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(ws), ws.numel(),
                                         _stream(stream)), "sym_tensor_upper_csr")
        return rowptr, col[:nnz], val[:nnz]

    def cp_als_step(self, B: torch.Tensor, B_out: torch.Tensor | None = None, ridge: float = 0.0, ws=None,
                    stream=None):
        """One symmetric CP-ALS update B_out = MTTKRP(X, B) ((B^T B)^{o(N-1)} + ridge I)^{-1}.

        Returns (B_out, info) with info a device int (0 = success, k = first non-positive pivot)."""
        rank = B.shape[1]
        if B_out is None:
            B_out = torch.empty_like(B)
        info = torch.zeros(1, dtype=torch.int32, device=B.device)
        if ws is None:
            ws = _scratch(lib().sym_cp_als_workspace_bytes(self.handle, rank), self.device)
        check(lib().sym_cp_als_step(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(B_out),
                                    B_out.stride(0), float(ridge), _ptr(info), _ptr(ws), ws.numel(), _stream(stream)),
              "sym_cp_als_step")
        return B_out, info

    def ttm(self, B: torch.Tensor, layout: str = "packed", C_out: torch.Tensor | None = None, cfg: dict | None = None,
            stream=None):
        """Mode-1 TTM C[j, l, :] = sum_k A[k, j, l] B[k, :] (order 3).

        layout "packed": the canonical triangle j <= l, shape (n (n + 1) / 2, R);
        layout "full": shape (n, n, R), the lower triangle filled by replication.
        cfg: fields of sym_ttm_cfg to override (entries_per_warp, ctas_per_sm, leaf_index)."""
        rank = B.shape[1]
        code = {"packed": TTM_PACKED, "full": TTM_FULL}[layout]
        elems = lib().sym_ttm_output_elems(self.n, rank, code)
        if elems < 0:
            raise SymError(-1, "sym_ttm_output_elems")
        if C_out is None:
            shape = (self.n * (self.n + 1) // 2, rank) if code == TTM_PACKED else (self.n, self.n, rank)
            C_out = torch.empty(shape, dtype=torch.float32, device=B.device)
        if C_out.numel() < elems or not C_out.is_contiguous():
            raise SymError(-1, "sym_ttm (output buffer)")
        tc = TtmCfg()
        check(lib().sym_ttm_default_config(C.byref(tc)), "sym_ttm_default_config")
        for k, v in (cfg or {}).items():
            setattr(tc, k, int(v))
        check(lib().sym_ttm(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(C_out), code,
                            C.byref(tc), _stream(stream)), "sym_ttm")
        return C_out

    def expanded(self, stream=None) -> "Expanded":
        return Expanded(self, stream)

    def close(self):
        if getattr(self, "handle", None):
            lib().sym_tensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gen_coords(order, n, count, seed, device="cuda", stream=None):
    """On-device counter-based coordinate pool (same definition as synth.coord_pool)."""
    idx = torch.empty((order, max(count, 1)), dtype=torch.int32, device=device)
    val = torch.empty(max(count, 1), dtype=torch.float32, device=device)
    check(lib().sym_gen_coords(order, n, count, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _ptr(idx), max(count, 1),
                               _ptr(val), _stream(stream)), "sym_gen_coords")
    return idx[:, :count], val[:count]


def gen_batch_coords(row_off: torch.Tensor, draw_off: torch.Tensor, seed: int, stream=None):
    """On-device draws for batched symmetric matrices (same definition as synth.batch_coords)."""
    total = int(draw_off[-1].item())
    idx = torch.empty((2, max(total, 1)), dtype=torch.int32, device=row_off.device)
    val = torch.empty(max(total, 1), dtype=torch.float32, device=row_off.device)
    check(lib().sym_gen_batch_coords(row_off.numel() - 1, _ptr(row_off), _ptr(draw_off), total,
                                     C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _ptr(idx), max(total, 1), _ptr(val),
                                     _stream(stream)), "sym_gen_batch_coords")
    return idx[:, :total], val[:total]


def make_batch(sizes, per_row: float, seed: int, device="cuda", stream=None):
    """Builds a BatchCSR on the device: counter-based draws, canonicalisation, upper CSR.

    Instance b has sizes[b] rows and round(per_row * sizes[b]) draws over its
    upper triangle; repeated positions merge (keep-equal), so rows hold on
    average slightly fewer than per_row entries.
    """
    import numpy as _np
    sizes = _np.asarray(sizes, dtype=_np.int64)
    row_off = _np.concatenate([[0], _np.cumsum(sizes)]).astype(_np.int64)
    draws = _np.rint(per_row * sizes).astype(_np.int64)
    draw_off = _np.concatenate([[0], _np.cumsum(draws)]).astype(_np.int64)
    ro = torch.from_numpy(row_off).to(device)
    do = torch.from_numpy(draw_off).to(device)
    idx, val = gen_batch_coords(ro, do, seed, stream)
    X = SymTensor(idx, val, int(row_off[-1]), dup=DUP_KEEP_EQUAL, stream=stream)
    del idx, val
    rowptr, col, v = X.upper_csr(stream)
    X.close()
    return BatchCSR(ro, rowptr, col.clone(), v.clone())


class Expanded:
    """The fully expanded (non-symmetric) tensor: every distinct permutation of every entry."""

    def __init__(self, X: SymTensor, stream=None):
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_expanded_bytes(X.handle, C.byref(ab), C.byref(wb)), "sym_expanded_bytes")
        self.arena = _scratch(ab.value, X.device)
        ws = _scratch(wb.value, X.device)
        h = C.c_void_p()
        check(lib().sym_expanded_create(X.handle, _ptr(self.arena), self.arena.numel(), _ptr(ws), ws.numel(),
                                        _stream(stream), C.byref(h)), "sym_expanded_create")
        del ws
        self.handle, self.order, self.n, self.device = h, X.order, X.n, X.device

    @property
    def nnz(self) -> int:
        v = C.c_int64(0)
        check(lib().sym_expanded_info(self.handle, C.byref(v)), "sym_expanded_info")
        return v.value

    def export(self, stream=None):
        nnz = self.nnz
        eidx = torch.empty((self.order, max(nnz, 1)), dtype=torch.int32, device=self.device)
        ev = torch.empty(max(nnz, 1), dtype=torch.float32, device=self.device)
        check(lib().sym_expanded_export(self.handle, _ptr(eidx), max(nnz, 1), _ptr(ev), _stream(stream)),
              "sym_expanded_export")
        return eidx[:, :nnz], ev[:nnz]

    def mttkrp(self, B, M=None, stream=None):
        rank = B.shape[1]
        if M is None:
            M = torch.empty((self.n, rank), dtype=torch.float32, device=B.device)
        check(lib().sym_mttkrp_expanded(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(M),
                                        M.stride(0), _stream(stream)), "sym_mttkrp_expanded")
        return M

    def ttm(self, B, C_out=None, stream=None):
        """Plain TTM over the expanded tensor (order 3): full (n, n, R) output."""
        rank = B.shape[1]
        if C_out is None:
            C_out = torch.empty((self.n, self.n, rank), dtype=torch.float32, device=B.device)
        check(lib().sym_ttm_expanded(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(C_out),
                                     _stream(stream)), "sym_ttm_expanded")
        return C_out

    def close(self):
        if getattr(self, "handle", None):
            lib().sym_expanded_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ partially symmetric tensors

class PTensor:
    """A partially symmetric sparse tensor (sym_ptensor_*): modes split into consecutive parts of sizes
    `parts`, part p's indices in [0, dims[p]); symmetric under permutations inside each part."""

    def __init__(self, idx: torch.Tensor, val: torch.Tensor, parts, dims, dup: int = DUP_ERROR, stream=None):
        if idx.dim() != 2 or idx.dtype != torch.int32 or not (idx.is_cuda or idx.is_pinned()):
            raise TypeError("idx must be a (order, nnz) int32 CUDA tensor or pinned host tensor")
        if val.dtype != torch.float32 or not (val.is_cuda or val.is_pinned()):
            raise TypeError("val must be a float32 CUDA tensor or pinned host tensor")
        if not val.is_cuda and not val.is_contiguous():
            raise TypeError("a pinned host val must be contiguous")
        dev = val.device if val.is_cuda else (idx.device if idx.is_cuda else
                                              torch.device("cuda", torch.cuda.current_device()))
        order, nnz = idx.shape
        if idx.is_cuda:
            idx = idx.contiguous()
        elif not idx.is_contiguous():
            raise TypeError("a pinned host idx must be contiguous")
        self._part = (C.c_int32 * len(parts))(*[int(p) for p in parts])
        self._dim = (C.c_int64 * len(dims))(*[int(d) for d in dims])
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_ptensor_create_bytes(order, len(parts), self._part, self._dim, nnz, C.byref(ab), C.byref(wb)),
              "sym_ptensor_create_bytes")
        self.arena = _scratch(ab.value, idx.device)
        ws = _scratch(wb.value, idx.device)
        h = C.c_void_p()
        check(lib().sym_ptensor_create(order, len(parts), self._part, self._dim, nnz, _ptr(idx), max(nnz, 1),
                                       _ptr(val.contiguous()), dup, _ptr(self.arena), self.arena.numel(), _ptr(ws),
                                       ws.numel(), _stream(stream), C.byref(h)), "sym_ptensor_create")
        self.handle = h
        self.order, self.parts, self.dims = order, tuple(int(p) for p in parts), tuple(int(d) for d in dims)
        self.device = idx.device

    def info(self) -> dict:
        inf = PTensorInfo()
        check(lib().sym_ptensor_info(self.handle, C.byref(inf)), "sym_ptensor_info")
        return inf.as_dict()

    @property
    def nnz(self) -> int:
        return self.info()["nnz"]

    def export(self, stream=None):
        """(cidx (order x nnz) int32, cval) on the device, lexicographic order."""
        nnz = self.nnz
        cidx = torch.empty((self.order, max(nnz, 1)), dtype=torch.int32, device=self.device)
        cval = torch.empty(max(nnz, 1), dtype=torch.float32, device=self.device)
        check(lib().sym_ptensor_export(self.handle, _ptr(cidx), max(nnz, 1), _ptr(cval), _stream(stream)),
              "sym_ptensor_export")
        return cidx[:, :nnz], cval[:nnz]

    def expand(self, stream=None) -> "PTensor":
        """The same tensor with every inside-part arrangement stored (one part per mode: no symmetry left)."""
        ab, wb = C.c_size_t(0), C.c_size_t(0)
        check(lib().sym_ptensor_expand_bytes(self.handle, C.byref(ab), C.byref(wb)), "sym_ptensor_expand_bytes")
        arena = _scratch(ab.value, self.device)
        ws = _scratch(wb.value, self.device)
        h = C.c_void_p()
        check(lib().sym_ptensor_expand(self.handle, _ptr(arena), arena.numel(), _ptr(ws), ws.numel(),
                                       _stream(stream), C.byref(h)), "sym_ptensor_expand")
        del ws
        E = PTensor.__new__(PTensor)
        E.handle, E.arena, E.device = h, arena, self.device
        E.order = self.order
        E.parts = (1,) * self.order
        E.dims = tuple(d for s_, d in zip(self.parts, self.dims) for _ in range(s_))
        return E

    def mttkrp(self, factors, out_part: int, M=None, stream=None):
        """MTTKRP for part out_part's factor; factors: one (dims[p], R) CUDA tensor per part, all FP32 or all BF16."""
        rank = factors[0].shape[1]
        dt = _dtype_code(factors[0])
        if any(_dtype_code(f) != dt or f.shape[1] != rank for f in factors):
            raise TypeError("factors must share dtype and rank")
        ptrs = (C.c_void_p * len(factors))(*[f.data_ptr() for f in factors])
        lds = (C.c_int64 * len(factors))(*[f.stride(0) for f in factors])
        if M is None:
            M = torch.empty((self.dims[out_part], rank), dtype=torch.float32, device=factors[0].device)
        check(lib().sym_pmttkrp(self.handle, ptrs, lds, dt, rank, out_part, _ptr(M), M.stride(0), _stream(stream)),
              "sym_pmttkrp")
        return M

    def ttm(self, B, layout: str = "full", C_out=None, stream=None):
        """Mode-1 TTM (order 3): C[j, l, :] = sum_k A[k, j, l] B[k, :]; 'packed' when modes 2, 3 share a part."""
        rank = B.shape[1]
        code = TTM_PACKED if layout == "packed" else TTM_FULL
        elems = lib().sym_pttm_output_elems(self.handle, rank, code)
        if elems < 0:
            raise SymError(-1, "sym_pttm_output_elems")
        if C_out is None:
            C_out = torch.empty(elems, dtype=torch.float32, device=B.device)
        check(lib().sym_pttm(self.handle, _ptr(B), _dtype_code(B), rank, B.stride(0), _ptr(C_out), code,
                             _stream(stream)), "sym_pttm")
        return C_out

    def close(self):
        if getattr(self, "handle", None):
            lib().sym_ptensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ batched SSYMV / SYPRD

class BatchCSR:
    """Concatenated upper CSRs of many independent symmetric matrices (device arrays)."""

    def __init__(self, row_off, rowptr, col, val):
        self.row_off, self.rowptr, self.col, self.val = row_off, rowptr, col, val
        self.host_row_off = row_off.cpu().numpy().astype("int64")
        self.desc = CsrBatch(len(self.host_row_off) - 1, int(self.host_row_off[-1]), int(col.numel()),
                             row_off.data_ptr(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())

    def _hro(self):
        return self.host_row_off.ctypes.data_as(C.c_void_p)


class BatchPlan:
    """Tile list + FP64 partial buffers for one batch and one tile shape (sym_spmv_batch_plan_*)."""

    def __init__(self, batch: BatchCSR, cfg: TileCfg, stream=None):
        self.batch, self.cfg = batch, cfg
        nb = lib().sym_spmv_batch_plan_bytes(C.byref(batch.desc), batch._hro(), C.byref(cfg))
        if nb == 0:
            raise SymError(-1, "sym_spmv_batch_plan_bytes")
        self.arena = _scratch(nb, batch.rowptr.device)
        h = C.c_void_p()
        check(lib().sym_spmv_batch_plan_create(C.byref(batch.desc), batch._hro(), C.byref(cfg), _ptr(self.arena),
                                               self.arena.numel(), _stream(stream), C.byref(h)),
              "sym_spmv_batch_plan_create")
        self.handle = h

    def run(self, x, y, syprd=None, stream=None):
        check(lib().sym_spmv_batch_run(self.handle, _ptr(x), _ptr(y), _ptr(syprd), _stream(stream)),
              "sym_spmv_batch_run")

    def capture(self, x, y, syprd=None, stream=None):
        check(lib().sym_spmv_batch_capture(self.handle, _ptr(x), _ptr(y), _ptr(syprd), _stream(stream)),
              "sym_spmv_batch_capture")

    def launch(self, stream=None):
        check(lib().sym_spmv_batch_graph_launch(self.handle, _stream(stream)), "sym_spmv_batch_graph_launch")

    def check(self):
        """Raises if the banded kernel gave up a bounded wait (synchronous)."""
        check(lib().sym_spmv_batch_check(self.handle), "sym_spmv_batch_check")

    def clear_status(self, stream=None):
        check(lib().sym_spmv_batch_clear_status(self.handle, _stream(stream)), "sym_spmv_batch_clear_status")

    def run_bounded(self, x, y, syprd=None, wait_limit_ns=0, skip_chunk=-1, stream=None):
        """Test hook: run with a short wait limit and optionally one chunk withheld (sym_spmv_batch_run_bounded)."""
        check(lib().sym_spmv_batch_run_bounded(self.handle, _ptr(x), _ptr(y), _ptr(syprd), int(wait_limit_ns),
                                               int(skip_chunk), _stream(stream)), "sym_spmv_batch_run_bounded")

    def close(self):
        if getattr(self, "handle", None):
            lib().sym_spmv_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_batch(batch: BatchCSR, x, y, syprd=None, cache_path=None, stream=None):
    """Times candidate tile shapes on this batch; returns (TileCfg, ms). Cached by device and shape."""
    # the largest candidate plans: one-row tiles, or the banded copy of the entries with the smallest bands
    nb = max(lib().sym_spmv_batch_plan_bytes(C.byref(batch.desc), batch._hro(), C.byref(c))
             for c in (TileCfg(16, 32, 256, 1, 0, 0, 0), TileCfg(256, 8, 256, 1, 0, 0, 0, 2048, 64)))
    arena = _scratch(nb, batch.rowptr.device)
    best = TileCfg()
    ms = C.c_float(0)
    check(lib().sym_autotune_spmv_batch(C.byref(batch.desc), batch._hro(), _ptr(x), _ptr(y), _ptr(syprd),
                                        _ptr(arena), arena.numel(),
                                        cache_path.encode() if cache_path else None, _stream(stream),
                                        C.byref(best), C.byref(ms)), "sym_autotune_spmv_batch")
    return best, ms.value


# ------------------------------------------------------------------ serving

class Server:
    """Continuous-batching MTTKRP server (sym_server_create / sym_batch_submit / sym_batch_poll)."""

    def __init__(self, max_slots=8, max_rank=64, hbm_budget_bytes=120 << 30, small_nnz=1_000_000,
                 wait_limit_s=30.0, device=None, coalesce_small=False, pool_bytes=0, affinity_wait_s=0.02):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.cfg = ServerCfg(max_slots, max_rank, hbm_budget_bytes, int(coalesce_small), small_nnz,
                             int(wait_limit_s * 1e9), int(pool_bytes), int(affinity_wait_s * 1e9))
        self.arena = _scratch(lib().sym_server_arena_bytes(C.byref(self.cfg)), dev)
        h = C.c_void_p()
        check(lib().sym_server_create(C.byref(self.cfg), _ptr(self.arena), self.arena.numel(), dev.index,
                                      C.byref(h)), "sym_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, X: SymTensor, B, M, residual=False, tag=0) -> int:
        """Queues M = MTTKRP(X, B).  residual: False, True (FP64 CP-fit residual), or 2 (the residual, with B
        unchanged since an earlier request to this server: its cached Gram matrix may be reused)."""
        req = Request(X.handle.value, B.data_ptr(), _dtype_code(B), B.shape[1], B.stride(0), M.data_ptr(),
                      M.stride(0), int(residual), tag)
        t = C.c_uint64(0)
        check(lib().sym_batch_submit(self.handle, C.byref(req), C.byref(t)), "sym_batch_submit")
        self._keep[t.value] = (X, B, M)
        return t.value

    def register(self, image: torch.Tensor) -> int:
        """Registers a tensor image (SymTensor.save_image); the server keeps it resident when needed."""
        tid = C.c_uint64(0)
        check(lib().sym_server_register(self.handle, C.c_void_p(image.data_ptr()), C.byref(tid)),
              "sym_server_register")
        self._keep[("image", tid.value)] = image
        return tid.value

    def submit_registered(self, tid: int, B, M, residual=False, tag=0) -> int:
        req = Request(None, B.data_ptr(), _dtype_code(B), B.shape[1], B.stride(0), M.data_ptr(), M.stride(0),
                      int(residual), tag)
        t = C.c_uint64(0)
        check(lib().sym_batch_submit_registered(self.handle, tid, C.byref(req), C.byref(t)),
              "sym_batch_submit_registered")
        self._keep[t.value] = (B, M)
        return t.value

    def poll(self, ticket: int):
        """None while pending; else a dict with status, residual and timestamps."""
        r = Result()
        code = lib().sym_batch_poll(self.handle, ticket, C.byref(r))
        if code == SYM_PENDING:
            return None
        check(code, "sym_batch_poll")
        self._keep.pop(ticket, None)
        return {"status": r.status, "residual": r.residual, "tag": r.user_tag, "t_submit_ns": r.t_submit_ns,
                "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns}

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = Result()
        check(lib().sym_batch_wait(self.handle, ticket, int(timeout_s * 1e9), C.byref(r)), "sym_batch_wait")
        self._keep.pop(ticket, None)
        return {"status": r.status, "residual": r.residual, "tag": r.user_tag, "t_submit_ns": r.t_submit_ns,
                "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns}

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().sym_server_stats_get(self.handle, C.byref(st)), "sym_server_stats_get")
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            code = lib().sym_server_destroy(self.handle)
            self.handle = None
            check(code, "sym_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(r):
    return {"status": r.status, "residual": r.residual, "tag": r.user_tag, "t_submit_ns": r.t_submit_ns,
            "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns}


class DevLoop:
    """Device-resident request loop (sym_devloop_*): one persistent kernel serves MTTKRP and SSYMV / SYPRD
    requests published into a ring in mapped host memory."""

    def __init__(self, ring_slots=1024, ctas=0, hbm_budget_bytes=120 << 30, idle_exit_s=0.002, wait_limit_s=10.0,
                 device=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.cfg = DevLoopCfg(ring_slots, ctas, hbm_budget_bytes, int(idle_exit_s * 1e9), int(wait_limit_s * 1e9))
        h = C.c_void_p()
        check(lib().sym_devloop_create(C.byref(self.cfg), dev.index, C.byref(h)), "sym_devloop_create")
        self.handle = h
        self._keep = {}

    def submit_mttkrp(self, X: "SymTensor", B, M, tag=0) -> int:
        """Queues M = MTTKRP(X, B) (M overwritten)."""
        req = Request(X.handle.value, B.data_ptr(), _dtype_code(B), B.shape[1], B.stride(0), M.data_ptr(),
                      M.stride(0), 0, tag)
        t = C.c_uint64(0)
        check(lib().sym_devloop_submit_mttkrp(self.handle, C.byref(req), C.byref(t)), "sym_devloop_submit_mttkrp")
        self._keep[t.value] = (X, B, M)
        return t.value

    def submit_ssymv(self, n, rowptr, col, val, x, y, syprd=None, tag=0) -> int:
        """Queues y = A x (and x^T A x into syprd, a 1-element float64 tensor, when given)."""
        A = csr_upper(n, rowptr, col, val)
        t = C.c_uint64(0)
        check(lib().sym_devloop_submit_ssymv(self.handle, C.byref(A), _ptr(x), _ptr(y), _ptr(syprd), tag,
                                             C.byref(t)), "sym_devloop_submit_ssymv")
        self._keep[t.value] = (rowptr, col, val, x, y, syprd)
        return t.value

    def poll(self, ticket: int):
        """None while pending; else a dict with status and timestamps."""
        r = Result()
        code = lib().sym_devloop_poll(self.handle, ticket, C.byref(r))
        if code == SYM_PENDING:
            return None
        check(code, "sym_devloop_poll")
        self._keep.pop(ticket, None)
        return _result_dict(r)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = Result()
        check(lib().sym_devloop_wait(self.handle, ticket, int(timeout_s * 1e9), C.byref(r)), "sym_devloop_wait")
        self._keep.pop(ticket, None)
        return _result_dict(r)

    def stats(self) -> dict:
        st = DevLoopStats()
        check(lib().sym_devloop_stats_get(self.handle, C.byref(st)), "sym_devloop_stats_get")
        return {f: getattr(st, f) for f, _ in DevLoopStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            code = lib().sym_devloop_destroy(self.handle)
            self.handle = None
            self._keep.clear()
            check(code, "sym_devloop_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
