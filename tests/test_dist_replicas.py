"""The N-GPU bench path is N independent replicas (weak scaling, no data-path collective): the only
cross-rank steps are the barriers around the timed region and the max over ranks of the step time.
Checked here with world_size-2 gloo process groups on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, times, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    D = bench.Dist()
    D.barrier()
    ms = D.max(times[rank])          # the bench's step time: the slowest rank
    D.barrier()
    q.put((rank, D.ws, D.rank, ms))
    D.close()


@pytest.mark.timeout(120)
def test_two_replicas_barrier_and_max_over_ranks():
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.25, 3.5]
    ps = [ctx.Process(target=_worker, args=(r, port, times, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(90)
    assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 2 and g[3] == max(times) for g in got)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm's other ranks exit without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 3

    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_single_process_dist_is_a_no_op(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    D = bench.Dist()
    D.barrier()
    assert D.ws == 1 and D.max(2.5) == 2.5
    D.close()
