"""Host logic of the multi-rank bench on CPU: two gloo ranks read their environment,
take the slowest rank's time and compute the whole-job rate the way bench.py does."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    my_ms = 100.0 * (r + 1)          # rank 1 is the slow one
    ms = bench.max_over_ranks(my_ms, dist, "cpu")
    rate = bench.aggregate_rate(1000, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, local, ms, rate))


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for r, (rank, w, local, ms, rate) in enumerate(got):
        assert (rank, w, local) == (r, world, r)
        assert ms == 200.0                      # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 1000 / 0.2)


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.aggregate_rate(500, 1, 250.0) == pytest.approx(2000.0)
