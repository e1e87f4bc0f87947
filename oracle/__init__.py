"""Python view of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py.  The product package never imports it.

Each wrapper takes the user-level inputs (coordinate lists, upper CSR, dense
factors as float32/bfloat16-valued arrays), widens them to float64 and calls the
plain C definition.  See oracle.c for the paper passages each function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID, NONCANONICAL, RANGE, DUPLICATE, NOMEM = 0, -1, -2, -3, -4, -5


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} returned {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (portable flags; no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            i32p, f32p, f64p, i64p, u8p = (C.c_void_p,) * 5
            L.orc_canonicalize.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, C.c_int, i32p,
                                           f32p, C.POINTER(C.c_int64)]
            L.orc_check_canonical.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p]
            L.orc_distinct_perms.argtypes = [C.c_int, i32p]
            L.orc_distinct_perms.restype = C.c_int64
            L.orc_counts.argtypes = [C.c_int, C.c_int64, i32p, f32p, i64p, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double)]
            L.orc_mttkrp_enum.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, f64p,
                                          f64p, u8p]
            L.orc_mttkrp_enum_threads.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, f64p,
                                                  C.c_int]
            L.orc_mttkrp_runs.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, f64p]
            L.orc_check_upper_csr.argtypes = [C.c_int64, i32p, i32p]
            L.orc_ssymv_enum.argtypes = [C.c_int64, i32p, i32p, f32p, f64p, f64p, f64p]
            L.orc_syprd_enum.argtypes = [C.c_int64, i32p, i32p, f32p, f64p, f64p, f64p]
            L.orc_bellman_enum.argtypes = [C.c_int64, i32p, i32p, f32p, f64p, f64p]
            L.orc_cpfit.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, f64p, f64p,
                                    f64p]
            L.orc_expand.argtypes = [C.c_int, C.c_int64, i32p, f32p, C.c_int64, i32p, f32p,
                                     C.POINTER(C.c_int64)]
            L.orc_cp_als_step.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, C.c_double,
                                          f64p, C.POINTER(C.c_int)]
            L.orc_pcanonicalize.argtypes = [C.c_int, C.c_int, i32p, i64p, C.c_int64, i32p, f32p, C.c_int, i32p,
                                            f32p, C.POINTER(C.c_int64)]
            L.orc_pcounts.argtypes = [C.c_int, C.c_int, i32p, C.c_int64, i32p, f32p, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_double)]
            L.orc_pttm_enum.argtypes = [C.c_int, i32p, i64p, C.c_int64, i32p, f32p, f64p, C.c_int, f64p, f64p]
            L.orc_pmttkrp_enum.argtypes = [C.c_int, C.c_int, i32p, i64p, C.c_int64, i32p, f32p, f64p, C.c_int,
                                           C.c_int, f64p, f64p]
            L.orc_pexpand.argtypes = [C.c_int, C.c_int, i32p, C.c_int64, i32p, f32p, C.c_int64, i32p, f32p,
                                      C.POINTER(C.c_int64)]
            L.orc_ttm_enum.argtypes = [C.c_int, C.c_int64, C.c_int64, i32p, f32p, f64p, C.c_int, i32p, C.c_int64,
                                       f64p, f64p]
            for name in ("orc_pcanonicalize", "orc_pcounts", "orc_pmttkrp_enum", "orc_pexpand", "orc_ttm_enum", "orc_cp_als_step", "orc_canonicalize", "orc_check_canonical", "orc_counts", "orc_mttkrp_enum",
                         "orc_mttkrp_runs", "orc_check_upper_csr", "orc_ssymv_enum", "orc_syprd_enum",
                         "orc_bellman_enum", "orc_cpfit", "orc_expand"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _p(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


# ---------------------------------------------------------------- canonical form

def canonicalize(order, n, idx, val, dup_policy=0):
    """Returns (cidx (order x m) int32, cval float32), canonical and sorted."""
    idx = _c(idx, np.int32).reshape(order, -1)
    val = _c(val, np.float32)
    nnz = val.shape[0]
    cidx = np.zeros((order, max(nnz, 1)), dtype=np.int32)
    cval = np.zeros(max(nnz, 1), dtype=np.float32)
    m = C.c_int64(0)
    rc = lib().orc_canonicalize(order, n, nnz, _p(idx), _p(val), dup_policy, _p(cidx), _p(cval), C.byref(m))
    _check(rc, "canonicalize")
    m = m.value
    # the C routine compacts rows to stride m inside the nnz-wide buffer
    flat = cidx.reshape(-1)[: order * m].reshape(order, m) if m else np.zeros((order, 0), np.int32)
    return np.ascontiguousarray(flat), cval[:m].copy()


def check_canonical(order, n, cidx):
    cidx = _c(cidx, np.int32)
    return lib().orc_check_canonical(order, n, cidx.shape[1], _p(cidx))


def distinct_perms(c):
    c = _c(c, np.int32)
    return int(lib().orc_distinct_perms(len(c), _p(c)))


def counts(order, cidx, cval):
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    cnt = np.zeros(16, dtype=np.int64)
    ex, rf, l2 = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    ns = C.c_double(0)
    rc = lib().orc_counts(order, cval.shape[0], _p(cidx), _p(cval), _p(cnt), C.byref(ex), C.byref(rf),
                          C.byref(l2), C.byref(ns))
    _check(rc, "counts")
    return dict(by_pattern=cnt, expanded=ex.value, root_fibers=rf.value, l2_fibers=l2.value,
                normsq=ns.value)


# ---------------------------------------------------------------- MTTKRP

def mttkrp_enum(order, n, cidx, cval, B, want_abs=True, rows=None):
    """Definitional symmetric MTTKRP (distinct-permutation enumeration), FP64."""
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    R = B.shape[1]
    M = np.zeros((n, R), dtype=np.float64)
    Ma = np.zeros((n, R), dtype=np.float64) if want_abs else None
    mask = None
    if rows is not None:
        mask = np.zeros(n, dtype=np.uint8)
        mask[np.asarray(rows)] = 1
    rc = lib().orc_mttkrp_enum(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), R, _p(M), _p(Ma),
                               _p(mask))
    _check(rc, "mttkrp_enum")
    return (M, Ma) if want_abs else M


def mttkrp_enum_threads(order, n, cidx, cval, B, threads):
    """The definitional MTTKRP on `threads` host threads (contiguous entry ranges, private FP64 outputs
    summed in thread order): the multi-core timing baseline."""
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    M = np.zeros((n, B.shape[1]), dtype=np.float64)
    rc = lib().orc_mttkrp_enum_threads(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), B.shape[1], _p(M),
                                       int(threads))
    _check(rc, "mttkrp_enum_threads")
    return M


def mttkrp_runs(order, n, cidx, cval, B):
    """Per-run integer-weight symmetric MTTKRP, FP64."""
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    M = np.zeros((n, B.shape[1]), dtype=np.float64)
    rc = lib().orc_mttkrp_runs(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), B.shape[1], _p(M))
    _check(rc, "mttkrp_runs")
    return M


# ---------------------------------------------------------------- SSYMV / SYPRD

def check_upper_csr(n, rowptr, col):
    return lib().orc_check_upper_csr(n, _p(_c(rowptr, np.int32)), _p(_c(col, np.int32)))


def ssymv(n, rowptr, col, val, x):
    rowptr, col, val = _c(rowptr, np.int32), _c(col, np.int32), _c(val, np.float32)
    x = _c(x, np.float64)
    y = np.zeros(n, dtype=np.float64)
    ya = np.zeros(n, dtype=np.float64)
    _check(lib().orc_ssymv_enum(n, _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(ya)), "ssymv")
    return y, ya


def syprd(n, rowptr, col, val, x):
    rowptr, col, val = _c(rowptr, np.int32), _c(col, np.int32), _c(val, np.float32)
    x = _c(x, np.float64)
    s, sa = C.c_double(0), C.c_double(0)
    _check(lib().orc_syprd_enum(n, _p(rowptr), _p(col), _p(val), _p(x), C.byref(s), C.byref(sa)),
           "syprd")
    return s.value, sa.value


def bellman(n, rowptr, col, val, d):
    rowptr, col, val = _c(rowptr, np.int32), _c(col, np.int32), _c(val, np.float32)
    d = _c(d, np.float64)
    y = np.zeros(n, dtype=np.float64)
    _check(lib().orc_bellman_enum(n, _p(rowptr), _p(col), _p(val), _p(d), _p(y)), "bellman")
    return y


# ---------------------------------------------------------------- CP fit, expansion

def cpfit(order, n, cidx, cval, B):
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    res, ab = C.c_double(0), C.c_double(0)
    parts = np.zeros(3, dtype=np.float64)
    _check(lib().orc_cpfit(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), B.shape[1], C.byref(res),
                           C.byref(ab), _p(parts)), "cpfit")
    return res.value, ab.value, parts


def cp_als_step(order, n, cidx, cval, B, ridge=0.0):
    """One symmetric CP-ALS update B_new = M (B^T B)^{o(N-1)} + ridge I)^{-1}; returns (B_new, info)."""
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    out = np.zeros_like(B)
    info = C.c_int(0)
    _check(lib().orc_cp_als_step(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), B.shape[1], float(ridge),
                                 _p(out), C.byref(info)), "cp_als_step")
    return out, info.value


def ttm_enum(order, n, cidx, cval, B, want_abs=True, rows=None):
    """Definitional mode-1 TTM, FP64: C[j_2..j_N, r] = sum_k A[k, j_2..j_N] B[k, r].

    Returns the full dense output, shape (n,)*(order-1) + (R,) (and its |terms| sums); with `rows`
    only the slices C[j_2 = rows[s], ...], stacked in that order."""
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    R = B.shape[1]
    slot = None
    first = n
    if rows is not None:
        rows = np.asarray(rows)
        slot = np.full(n, -1, dtype=np.int32)
        slot[rows] = np.arange(rows.size, dtype=np.int32)
        first = rows.size
    shape = (first,) + (n,) * (order - 2) + (R,)
    Cm = np.zeros(shape, dtype=np.float64)
    Ca = np.zeros(shape, dtype=np.float64) if want_abs else None
    _check(lib().orc_ttm_enum(order, n, cval.shape[0], _p(cidx), _p(cval), _p(B), R, _p(slot), first, _p(Cm),
                              _p(Ca)), "ttm_enum")
    return (Cm, Ca) if want_abs else Cm


# ---------------------------------------------------------------- partial symmetry

def _parts(parts, dims=None):
    part = np.ascontiguousarray(parts, dtype=np.int32)
    dim = np.ascontiguousarray(dims if dims is not None else [1] * len(parts), dtype=np.int64)
    return part, dim, int(part.sum())


def pcanonicalize(parts, dims, idx, val, dup_policy=0):
    """Canonical form of a partially symmetric tensor: (cidx (order x m) int32, cval float32)."""
    part, dim, order = _parts(parts, dims)
    idx = _c(idx, np.int32).reshape(order, -1)
    val = _c(val, np.float32)
    nnz = val.shape[0]
    cidx = np.zeros((order, max(nnz, 1)), dtype=np.int32)
    cval = np.zeros(max(nnz, 1), dtype=np.float32)
    m = C.c_int64(0)
    _check(lib().orc_pcanonicalize(order, len(part), _p(part), _p(dim), nnz, _p(idx), _p(val), dup_policy, _p(cidx),
                                   _p(cval), C.byref(m)), "pcanonicalize")
    m = m.value
    flat = cidx.reshape(-1)[: order * m].reshape(order, m) if m else np.zeros((order, 0), np.int32)
    return np.ascontiguousarray(flat), cval[:m].copy()


def pcounts(parts, cidx, cval):
    part, _, order = _parts(parts)
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    ex, ns = C.c_int64(0), C.c_double(0)
    _check(lib().orc_pcounts(order, len(part), _p(part), cval.shape[0], _p(cidx), _p(cval), C.byref(ex),
                             C.byref(ns)), "pcounts")
    return dict(expanded=ex.value, normsq=ns.value)


def pmttkrp_enum(parts, dims, cidx, cval, factors, out_part, want_abs=True):
    """Definitional MTTKRP for part out_part's factor (factors: one dims[p] x R array per part), FP64."""
    part, dim, order = _parts(parts, dims)
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    R = np.asarray(factors[0]).shape[1]
    F = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.float64).reshape(-1) for f in factors]))
    M = np.zeros((int(dim[out_part]), R), dtype=np.float64)
    Ma = np.zeros_like(M) if want_abs else None
    _check(lib().orc_pmttkrp_enum(order, len(part), _p(part), _p(dim), cval.shape[0], _p(cidx), _p(cval), _p(F), R,
                                  out_part, _p(M), _p(Ma)), "pmttkrp_enum")
    return (M, Ma) if want_abs else M


def pttm_enum(parts, dims, cidx, cval, B, want_abs=True):
    """Definitional mode-1 TTM of a partially symmetric order-3 tensor, FP64: C (d2, d3, R) dense, with
    C[pi_2, pi_3, :] += v B[pi_1, :] for every inside-part arrangement pi of every canonical entry."""
    part, dim, order = _parts(parts, dims)
    if order != 3:
        raise ValueError("order-3 tensors only")
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    B = _c(B, np.float64)
    R = B.shape[1]
    dq = [int(dim[p]) for p in range(len(part)) for _ in range(int(part[p]))]
    Cm = np.zeros((dq[1], dq[2], R), dtype=np.float64)
    Ca = np.zeros_like(Cm) if want_abs else None
    _check(lib().orc_pttm_enum(len(part), _p(part), _p(dim), cval.shape[0], _p(cidx), _p(cval), _p(B), R, _p(Cm),
                               _p(Ca)), "pttm_enum")
    return (Cm, Ca) if want_abs else Cm


def pexpand(parts, cidx, cval):
    part, _, order = _parts(parts)
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    nnz = cval.shape[0]
    cnt = C.c_int64(0)
    lib().orc_pexpand(order, len(part), _p(part), nnz, _p(cidx), _p(cval), 0, None, None, C.byref(cnt))
    k = cnt.value
    eidx = np.zeros((order, max(k, 1)), dtype=np.int32)
    ev = np.zeros(max(k, 1), dtype=np.float32)
    _check(lib().orc_pexpand(order, len(part), _p(part), nnz, _p(cidx), _p(cval), max(k, 1), _p(eidx), _p(ev),
                             C.byref(cnt)), "pexpand")
    return eidx[:, :k].copy(), ev[:k].copy()


def expand(order, cidx, cval):
    cidx = _c(cidx, np.int32)
    cval = _c(cval, np.float32)
    nnz = cval.shape[0]
    cnt = C.c_int64(0)
    lib().orc_expand(order, nnz, _p(cidx), _p(cval), 0, None, None, C.byref(cnt))
    k = cnt.value
    eidx = np.zeros((order, max(k, 1)), dtype=np.int32)
    ev = np.zeros(max(k, 1), dtype=np.float32)
    _check(lib().orc_expand(order, nnz, _p(cidx), _p(cval), max(k, 1), _p(eidx), _p(ev), C.byref(cnt)),
           "expand")
    return eidx[:, :k].copy(), ev[:k].copy()


# ---------------------------------------------------------------- error metrics

def componentwise_error(got, ref, ref_abs):
    """max |got - ref| / sum|terms| over outputs; outputs with no terms must be exactly 0."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    ref_abs = np.asarray(ref_abs, dtype=np.float64)
    zero = ref_abs == 0
    if np.any(got[zero] != 0):
        return float("inf")
    nz = ~zero
    if not nz.any():
        return 0.0
    return float(np.max(np.abs(got[nz] - ref[nz]) / ref_abs[nz]))


def normwise_error(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    d = np.max(np.abs(np.asarray(got, dtype=np.float64) - ref))
    m = np.max(np.abs(ref))
    return float(d / m) if m > 0 else float(d)
