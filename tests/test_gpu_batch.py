"""Batched SSYMV/SYPRD (one persistent launch, CUDA-graph replay, autotuned tiles) vs the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import TOL_F32, dev, host, need_gpu, torch

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


# ----------------------------------------------------------------------------- banded path

def run_plan(sg, row_off, rowptr, col, v, x, cfg, graph=False):
    torch = pytest.importorskip("torch")
    batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
    plan = sg.BatchPlan(batch, sg.TileCfg(*cfg))
    xd = dev(x)
    y = torch.full_like(xd, 77.0)
    s = torch.full((len(row_off) - 1,), 5.0, dtype=torch.float64, device="cuda")
    plan.run(xd, y, s)
    out = [(host(y), host(s))]
    if graph:
        y.fill_(123.0)
        plan.capture(xd, y, s)
        for _ in range(3):
            plan.launch()
        torch.cuda.synchronize()
        out.append((host(y), host(s)))
    plan.check()
    return out


def check_against_oracle(outs, row_off, rowptr, col, v, x):
    yr, ya, sr, sa = oracle_batch(row_off, rowptr, col, v, x)
    nz = sa > 0
    for yg, sgot in outs:
        assert oracle.componentwise_error(yg, yr, ya) <= TOL_F32
        assert np.max(np.abs(sgot[nz] - sr[nz]) / sa[nz], initial=0.0) <= TOL_F32
        assert np.all(sgot[~nz] == 0.0)


# (rows_per_tile, lanes, threads, ctas/SM, local, order, x_smem, band_rows, band_max, band_vec, band_order)
BAND_CFGS = [
    (256, 8, 512, 1, 0, 0, 0, 256, 64, 4, 0),     # up to 16 bands per instance, many blocks, multi-chunk blocks
    (256, 8, 256, 2, 0, 0, 0, 512, 4, 8, 0),      # instances beyond 4 bands stay on tiles (mixed plan)
    (256, 8, 1024, 1, 0, 0, 0, 4096, 64, 4, 0),   # 31 consumer warps, few bands; small instances in one band
    (64, 16, 128, 2, 0, 0, 0, 2048, 2, 16, 0),     # two CTAs per SM, 2-band cap, 16 entries per lane per chunk
    (256, 8, 288, 1, 0, 0, 0, 5120, 64, 8, 0),    # widest band: one band per instance (plain y stores)
    (256, 8, 512, 1, 0, 0, 0, 256, 64, 4, 1),     # bank-grouped blocks, many bands
    (256, 8, 1024, 1, 0, 0, 0, 4096, 64, 4, 1),   # bank-grouped, few bands
    (256, 8, 256, 2, 0, 0, 0, 512, 4, 8, 1),      # bank-grouped, mixed plan
    (256, 8, 1024, 1, 0, 0, 0, 5120, 64, 1, 1),   # bank-grouped, one entry per lane per chunk (many stages)
    (256, 8, 544, 1, 0, 0, 0, 2048, 64, 2, 1),    # bank-grouped, two entries per lane per chunk
]


@pytest.mark.parametrize("cfg", BAND_CFGS)
def test_batch_band_parity(cfg):
    """Banded path (x / y bands in shared memory, bulk-copied entry stream) vs the oracle, incl. graph replay."""
    sg = need_gpu()
    sizes, row_off, draw_off, idx, val, rowptr, col, v = make_small_batch(97, 4, 4000, 16, 5)
    x = synth.vector_uniform(int(row_off[-1]), 5)
    outs = run_plan(sg, row_off, rowptr, col, v, x, cfg, graph=True)
    check_against_oracle(outs, row_off, rowptr, col, v, x)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("per_row", [0.05, 0.6, 3.0])
def test_batch_band_sparse_blocks_direct_and_staged(per_row, order):
    """Sparse instances: blocks below the staging threshold reduce straight into global memory."""
    sg = need_gpu()
    sizes = np.array([3000, 1, 0, 2500, 777, 4096, 4097, 255, 256, 257], np.int64)
    row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    draws = np.rint(per_row * sizes).astype(np.int64)
    draw_off = np.concatenate([[0], np.cumsum(draws)]).astype(np.int64)
    idx, val = synth.batch_coords(row_off, draw_off, 31)
    rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
    x = synth.vector_uniform(int(row_off[-1]), 31)
    outs = run_plan(sg, row_off, rowptr, col, v, x, (256, 8, 512, 1, 0, 0, 0, 256, 64, 8 if order == 0 else 2, order))
    check_against_oracle(outs, row_off, rowptr, col, v, x)


def test_batch_band_dense_rows_and_diagonal_only():
    """One instance with a dense first row (one block spans many chunks; in bank groups its row bank
    forces groups with repeated banks), one diagonal-only instance."""
    sg = need_gpu()
    n0, n1 = 3000, 700
    rows, cols, vals = [], [], []
    rng = np.random.default_rng(4)
    for j in range(n0):                       # dense row 0 of instance 0
        rows.append(0); cols.append(j)
    for i in range(1, n0, 7):                 # a few more entries
        rows.append(i); cols.append(min(n0 - 1, i + 3))
    for i in range(n1):                       # instance 1: diagonal only
        rows.append(n0 + i); cols.append(n0 + i)
    rows, cols = np.array(rows, np.int64), np.array(cols, np.int64)
    o = np.lexsort((cols, rows))
    rows, cols = rows[o], cols[o]
    vals = rng.uniform(-1, 1, len(rows)).astype(np.float32)
    total = n0 + n1
    rowptr = np.zeros(total + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    row_off = np.array([0, n0, total], np.int64)
    x = synth.vector_uniform(total, 4)
    for cfg in [(256, 8, 256, 1, 0, 0, 0, 256, 64, 4, 0), (256, 8, 288, 1, 0, 0, 0, 4096, 64, 16, 0),
                (256, 8, 96, 2, 0, 0, 0, 512, 64, 8, 0), (256, 8, 256, 1, 0, 0, 0, 256, 64, 4, 1),
                (256, 8, 288, 1, 0, 0, 0, 4096, 64, 16, 1)]:
        outs = run_plan(sg, row_off, rowptr, cols.astype(np.int32), vals, x, cfg)
        check_against_oracle(outs, row_off, rowptr, cols.astype(np.int32), vals, x)


def test_batch_band_rejects_bad_columns():
    """A column below its row or outside its instance is caught when the banded plan is built."""
    sg = need_gpu()
    sizes = np.array([300, 200], np.int64)
    row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    draw_off = np.array([0, 1200, 2000], np.int64)
    idx, val = synth.batch_coords(row_off, draw_off, 8)
    rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
    cfg = sg.TileCfg(256, 8, 256, 1, 0, 0, 0, 256, 64, 4, 1)
    r = int(np.nonzero(np.diff(rowptr[:301]) > 0)[0][5])   # a non-empty row of instance 0 (row > 0)
    assert r >= 1
    for bad_col, code in [(r - 1, -2), (450, -3)]:   # below the diagonal; inside instance 1
        c2 = col.copy()
        c2[rowptr[r]] = bad_col
        batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(c2), dev(v))
        with pytest.raises(sg.SymError) as ei:
            sg.BatchPlan(batch, cfg)
        assert ei.value.code == code


@pytest.mark.parametrize("cfg", [(256, 8, 512, 1, 0, 0, 0, 256, 64, 4, 1), (256, 8, 1024, 1, 0, 0, 0, 4096, 64, 4, 0)])
def test_batch_band_tiny_empty_and_entryless(cfg):
    """Banded path on tiny, empty and entry-less instances, and on a batch with no entries at all."""
    sg = need_gpu()
    torch = pytest.importorskip("torch")
    for sizes, draws in [(np.array([1, 5, 1, 300, 2, 64, 0, 7], np.int64), np.array([0, 3, 1, 5000, 0, 700, 0, 0])),
                         (np.array([10, 20], np.int64), np.array([0, 0]))]:
        row_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        draw_off = np.concatenate([[0], np.cumsum(draws)]).astype(np.int64)
        idx, val = synth.batch_coords(row_off, draw_off, 13)
        rowptr, col, v = synth.batch_upper_csr_host(row_off, idx, val)
        x = synth.vector_uniform(int(row_off[-1]), 13)
        if col.size == 0:   # keep the device arrays non-empty; total_nnz = 0
            batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(np.zeros(1, np.int32))[:0],
                                dev(np.zeros(1, np.float32))[:0])
        else:
            batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
        plan = sg.BatchPlan(batch, sg.TileCfg(*cfg))
        y = torch.full((int(row_off[-1]),), 9.0, device="cuda")
        s = torch.full((len(sizes),), 9.0, dtype=torch.float64, device="cuda")
        plan.run(dev(x), y, s)
        plan.check()
        yr, ya, sr, sa = oracle_batch(row_off, rowptr, col, v, x)
        assert oracle.componentwise_error(host(y), yr, ya) <= TOL_F32
        nz = sa > 0
        assert np.all(host(s)[~nz] == 0.0)
        if nz.any():
            assert np.max(np.abs(host(s)[nz] - sr[nz]) / sa[nz]) <= TOL_F32


@pytest.mark.parametrize("order", [0, 1])
def test_batch_band_wait_runs_out_without_fault(order):
    """The banded kernel's bounded waits made to run out: the first CTA's first chunk is withheld (never
    announced, never copied) and every wait is limited to 1 ms.  The kernel returns, the plan's status word
    reports SYM_E_TIMEOUT, and after clearing it the next normal run is clean and matches the oracle."""
    sg = need_gpu()
    sizes, row_off, draw_off, idx, val, rowptr, col, v = make_small_batch(64, 4, 4000, 16, 9)
    x = synth.vector_uniform(int(row_off[-1]), 9)
    batch = sg.BatchCSR(dev(row_off), dev(rowptr), dev(col), dev(v))
    plan = sg.BatchPlan(batch, sg.TileCfg(256, 8, 512, 1, 0, 0, 0, 256, 64, 4, order))
    xd = dev(x)
    y = torch.zeros_like(xd)
    s = torch.zeros(len(row_off) - 1, dtype=torch.float64, device="cuda")
    plan.run_bounded(xd, y, s, wait_limit_ns=1_000_000, skip_chunk=0)
    torch.cuda.synchronize()
    with pytest.raises(sg.SymError) as e:
        plan.check()
    assert e.value.code == -7   # SYM_E_TIMEOUT
    plan.clear_status()
    plan.run(xd, y, s)
    plan.check()
    check_against_oracle([(host(y), host(s))], row_off, rowptr, col, v, x)
    # the hook with nothing withheld is a normal run
    plan.run_bounded(xd, y, s, wait_limit_ns=1_000_000)
    plan.check()
    check_against_oracle([(host(y), host(s))], row_off, rowptr, col, v, x)
