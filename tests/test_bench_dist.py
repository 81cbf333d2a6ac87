"""bench.py's multi-rank plumbing on CPU: two gloo ranks (the replicas path of --gpus N).

Each rank joins the process group the way bench.py does under torchrun, meets the others at
the barriers around the timed region, and takes the maximum of the per-rank times, which the
whole-job throughput divides by.  No GPU and no data-path collective are involved: the ranks
evolve independent replicas.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    t = 0.25 * (rank + 1)                  # this rank's "timed region" in seconds
    t_max = bench.max_over_ranks(ws, t)
    bench.barrier(ws)
    out.put((rank, t_max, ws * 10 / t_max))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_job_throughput():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; the job throughput counts both replicas
    assert [r for r, _, _ in res] == [0, 1]
    for _, t_max, value in res:
        assert t_max == pytest.approx(0.5)
        assert value == pytest.approx(2 * 10 / 0.5)


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    ws, r, local = bench.dist_init()
    assert (ws, r, local) == (1, 0, 0)
    assert bench.max_over_ranks(ws, 1.5) == 1.5
    bench.barrier(ws)
