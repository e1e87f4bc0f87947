"""Host-side checks of the batched SSYMV plan sizes (no GPU): every banded shape the GPU tests
use is accepted, shapes whose bands do not fit in shared memory are rejected, and the banded
plan holds the reordered copy of the entries (8 bytes per entry plus block padding)."""
import ctypes

import numpy as np
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sg():
    from paper_2406_09266_gb300 import build
    build.build()
    import paper_2406_09266_gb300 as m
    m.load()
    return m


def plan_bytes(sg, sizes, nnz, cfg):
    ro = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    fake = 256  # non-null placeholders: the size query reads no device memory
    d = sg.CsrBatch(len(sizes), int(ro[-1]), nnz, fake, fake, fake, fake)
    return sg.lib().sym_spmv_batch_plan_bytes(ctypes.byref(d), ro.ctypes.data_as(ctypes.c_void_p),
                                              ctypes.byref(sg.TileCfg(*cfg)))


def test_gpu_test_band_shapes_are_valid(sg):
    from tests.test_gpu_batch import BAND_CFGS
    extra = [(256, 8, 256, 1, 0, 0, 0, 256, 64, 4, 0), (256, 8, 288, 1, 0, 0, 0, 4096, 64, 16, 0),
             (256, 8, 96, 2, 0, 0, 0, 512, 64, 8, 0), (256, 8, 512, 1, 0, 0, 0, 256, 64, 8, 0),
             (256, 8, 256, 1, 0, 0, 0, 256, 64, 4, 1), (256, 8, 288, 1, 0, 0, 0, 4096, 64, 16, 1)]
    for cfg in BAND_CFGS + extra:
        assert plan_bytes(sg, [4000, 4000], 100_000, cfg) > 0, cfg


def test_band_shapes_that_do_not_fit_are_rejected(sg):
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 1024, 1, 0, 0, 0, 8192, 64, 4)) == 0   # bands alone > 227 KB
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 4096, 64, 16)) == 0   # one 61 KB chunk only
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 4098, 64, 4)) == 0    # not a multiple of 4
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 224, 0, 0, 4096, 64, 4)) == 0  # with the local path
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 0, 0, 4)) == 0        # band_chunk without bands
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 4096, 64, 1, 0)) == 0  # 1 entry/lane: row-major
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 4096, 64, 3, 1)) == 0  # 3 entries per lane
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 1024, 1, 0, 0, 0, 5120, 64, 1, 1)) > 0  # 8 KB chunks, 8 stages
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 0, 0, 0, 1)) == 0     # band_order without bands
    assert plan_bytes(sg, [4000], 50_000, (256, 8, 512, 1, 0, 0, 0, 4096, 64, 4, 2)) == 0  # unknown order


def test_band_plan_holds_the_entry_copy(sg):
    nnz = 1_000_000
    tiles = plan_bytes(sg, [65536, 300], nnz, (256, 8, 512, 2, 0, 0, 0, 0, 0, 0))
    band = plan_bytes(sg, [65536, 300], nnz, (256, 8, 544, 1, 0, 0, 0, 4096, 64, 8, 1))
    assert band - tiles >= 8 * nnz + 8 * 31 * (16 * 17 // 2)   # every block may pad to a whole group of 32
    assert band - tiles < 8 * nnz + (4 << 20)
