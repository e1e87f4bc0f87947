"""Batched SSYMV/SYPRD (one persistent launch, CUDA-graph replay, autotuned tiles) vs the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu

pytestmark = pytest.mark.gpu


def make_small_batch(count, lo, hi, per_row, seed):
    sizes = synth.batch_sizes(count, lo, hi, seed)
    row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    draws = np.rint(per_row * sizes).astype(np.int64)
    draw_off = np.concatenate([[0], np.cumsum(draws)]).astype(np.int64)
    idx, val = synth.batch_coords(row_off, draw_off, seed)
    rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
    return sizes, row_off, draw_off, idx, val, rowptr, col, v


def oracle_batch(row_off, rowptr, col, val, x):
    ys, yas, ss, sas = [], [], [], []
    for b in range(len(row_off) - 1):
        r0, r1 = row_off[b], row_off[b + 1]
        rp = (rowptr[r0:r1 + 1] - rowptr[r0]).astype(np.int32)
        c = (col[rowptr[r0]:rowptr[r1]] - r0).astype(np.int32)
        v = val[rowptr[r0]:rowptr[r1]]
        xb = x[r0:r1].astype(np.float64)
        y, ya = oracle.ssymv(int(r1 - r0), rp, c, v, xb)
        s, sa = oracle.syprd(int(r1 - r0), rp, c, v, xb)
        ys.append(y); yas.append(ya); ss.append(s); sas.append(sa)
    return np.concatenate(ys), np.concatenate(yas), np.array(ss), np.array(sas)


def test_device_batch_generator_matches_host():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes, row_off, draw_off, idx, val, rowptr, col, v = make_small_batch(40, 8, 3000, 16, 3)
    gi, gv = sg.gen_batch_coords(dev(row_off), dev(draw_off), 3)
    assert np.array_equal(host(gi), idx)
    assert np.array_equal(host(gv).view(np.uint32), val.view(np.uint32))
    B = sg.make_batch(sizes, 16, 3)
    assert np.array_equal(host(B.rowptr), rowptr)
    assert np.array_equal(host(B.col), col)
    assert np.array_equal(host(B.val), v)
    assert torch.equal(B.row_off.cpu(), torch.from_numpy(row_off))


@pytest.mark.parametrize("cfg", [(16, 4, 256, 2, 0, 0, 0), (64, 16, 512, 2, 0, 1, 0), (1, 32, 128, 8, 0, 0, 0),
                                 (256, 8, 256, 4, 0, 1, 0), (64, 8, 512, 2, 224, 0, 0), (64, 16, 1024, 1, 224, 1, 0),
                                 (64, 4, 512, 2, 8, 0, 0), (2048, 8, 256, 4, 0, 0, 32), (256, 16, 512, 2, 0, 0, 1),
                                 (4096, 4, 1024, 1, 0, 0, 200)])
def test_batch_parity(cfg):
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes, row_off, draw_off, idx, val, rowptr, col, v = make_small_batch(97, 4, 4000, 16, 5)
    x = synth.vector_uniform(int(row_off[-1]), 5)
    batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
    plan = sg.BatchPlan(batch, sg.TileCfg(*cfg))
    xd = dev(x)
    y = torch.empty_like(xd)
    s = torch.empty(len(sizes), dtype=torch.float64, device="cuda")
    plan.run(xd, y, s)
    yr, ya, sr, sa = oracle_batch(row_off, rowptr, col, v, x)
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert np.max(np.abs(host(s) - sr) / np.maximum(sa, 1e-300)) <= TOL_F32
    # graph capture + replay gives the same answer (y re-zeroed inside the graph)
    y.fill_(123.0)
    plan.capture(xd, y, s)
    for _ in range(3):
        plan.launch()
    torch.cuda.synchronize()
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert np.max(np.abs(host(s) - sr) / np.maximum(sa, 1e-300)) <= TOL_F32


@pytest.mark.parametrize("local_kb", [0, 1, 224])
def test_batch_local_path_mixed(local_kb):
    """Instances on the shared-memory path (y and x on chip, y only) and on tiles in one batch."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes = np.array([100, 200, 40000, 300, 70000, 5, 0, 1000], np.int64)  # 1 KB holds 256 floats
    row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    draws = (sizes * 4).astype(np.int64)
    draw_off = np.concatenate([[0], np.cumsum(draws)]).astype(np.int64)
    idx, val = synth.batch_coords(row_off, draw_off, 21)
    rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
    x = synth.vector_uniform(int(row_off[-1]), 21)
    batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
    plan = sg.BatchPlan(batch, sg.TileCfg(64, 8, 512, 2, local_kb, 0, 0))
    y = torch.empty(int(row_off[-1]), device="cuda")
    s = torch.empty(len(sizes), dtype=torch.float64, device="cuda")
    plan.run(dev(x), y, s)
    yr, ya, sr, sa = oracle_batch(row_off, rowptr, col, v, x)
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    nz = sa > 0
    assert np.max(np.abs(host(s)[nz] - sr[nz]) / sa[nz]) <= TOL_F32
    assert np.all(host(s)[~nz] == 0.0)


def test_batch_with_empty_and_tiny_instances():
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes = np.array([1, 5, 1, 300, 2, 64], np.int64)
    row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    draws = np.array([0, 3, 1, 5000, 0, 700], np.int64)        # instances 0 and 4 have no entries
    draw_off = np.concatenate([[0], np.cumsum(draws)]).astype(np.int64)
    idx, val = synth.batch_coords(row_off, draw_off, 9)
    rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
    x = synth.vector_uniform(int(row_off[-1]), 9)
    batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
    plan = sg.BatchPlan(batch, sg.TileCfg(8, 4, 128, 2, 0, 1, 0))
    y = torch.empty(int(row_off[-1]), device="cuda")
    s = torch.empty(len(sizes), dtype=torch.float64, device="cuda")
    plan.run(dev(x), y, s)
    yr, ya, sr, sa = oracle_batch(row_off, rowptr, col, v, x)
    assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
    assert host(s)[0] == 0.0 and host(s)[4] == 0.0
    nz = sa > 0
    assert np.max(np.abs(host(s)[nz] - sr[nz]) / sa[nz]) <= TOL_F32


def test_autotune_picks_valid_cfg_and_caches(tmp_path):
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    sizes = synth.batch_sizes(64, 64, 8192, 11)
    batch = sg.make_batch(sizes, 16, 11)
    x = dev(synth.vector_uniform(int(batch.host_row_off[-1]), 11))
    y = torch.empty_like(x)
    s = torch.empty(len(sizes), dtype=torch.float64, device="cuda")
    cache = str(tmp_path / "tune.txt")
    cfg, ms = sg.autotune_batch(batch, x, y, s, cache_path=cache)
    assert cfg.lanes_per_row in (4, 8, 16, 32) and ms > 0
    assert len([ln for ln in open(cache).read().splitlines() if ln.strip()]) == 1
    cfg2, ms2 = sg.autotune_batch(batch, x, y, s, cache_path=cache)   # cache hit
    assert cfg2.as_dict() == cfg.as_dict() and abs(ms2 - ms) < 1e-3
    plan = sg.BatchPlan(batch, cfg)
    plan.run(x, y, s)
    ref = torch.empty_like(y)
    plan2 = sg.BatchPlan(batch, sg.TileCfg(64, 16, 256, 2, 0, 0, 0))
    s2 = torch.empty_like(s)
    plan2.run(x, ref, s2)
    torch.cuda.synchronize()
    assert float((y - ref).abs().max()) <= 1e-4 * float(ref.abs().max())
