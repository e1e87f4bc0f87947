"""Primitive ceilings (sym_ceiling_run): argument checks on the host, and every kind timed once on the GPU.

The bench divides each kernel's algorithmic row operations by these rates, so a kind that silently did no
work (a rate far above the hardware's) would inflate every roofline fraction: the GPU test checks that the
rates are finite, positive and ordered as the hardware orders them.
"""
import ctypes
import math

import pytest

from tests.gpu_helpers import need_gpu


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_09266_gb300 import build
    return build.build()


def test_ceiling_sizes_on_the_host(libpath):
    import paper_2406_09266_gb300 as sg
    L = sg.load(libpath)
    assert L.sym_ceiling_bytes(0, 0, 0) == 4096                     # FMA: fixed scratch
    assert L.sym_ceiling_bytes(1, 1000, 64) == 2 * 1000 * 64 * 4 + 4096
    assert L.sym_ceiling_bytes(1, 1000, 6) == 0                     # rank not a multiple of 4
    assert L.sym_ceiling_bytes(1, 0, 64) == 0                       # no rows
    assert L.sym_ceiling_bytes(6, 1 << 20, 0) == (1 << 20) * 32     # copy: source and destination
    assert L.sym_ceiling_bytes(99, 1000, 64) == 0                   # unknown kind
    rate, ms = ctypes.c_double(0), ctypes.c_float(0)
    assert L.sym_ceiling_run(1, None, 0, 1000, 64, 1, 1, None, ctypes.byref(rate), ctypes.byref(ms)) == -1


@pytest.mark.gpu
def test_every_ceiling_kind_runs_and_orders():
    sg = need_gpu()
    rates = {}
    for kind, rows, rank in [("fma", 0, 64), ("row_gather", 20_000, 32), ("row_red", 20_000, 32),
                             ("gather_red", 20_000, 32), ("smem_f32", 256, 64), ("smem_u32", 256, 64),
                             ("hbm_copy", 1 << 24, 0), ("bulk_gather", 20_000, 32), ("bulk_red", 20_000, 32)]:
        rate, ms = sg.ceiling(kind, rows=rows, rank=rank, ops=1 << 22, reps=2)
        assert math.isfinite(rate) and rate > 0 and ms > 0, (kind, rate, ms)
        rates[kind] = rate
    assert rates["fma"] > 1e12                          # FLOP/s: tens of TFLOP/s on a GB300
    assert 1e11 < rates["hbm_copy"] < 1.5e13            # bytes/s: below HBM's nominal 8 TB/s (x ~1.9)
    # a gather and a reduction per row cost more than either alone
    assert rates["gather_red"] <= 1.05 * min(rates["row_gather"], rates["row_red"])
    # reductions are slower than gathers
    assert rates["row_red"] < rates["row_gather"]
