"""Multi-rank bookkeeping of bench.py on CPU: two gloo ranks each report their
own device time; both get the slowest rank's time and the whole-job rate
(units of all ranks over that time).  No GPU needed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [40.0, 50.0][rank]
    q.put((rank, bench.combine_ranks(local_ms, 1000, 10)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        t, value = out[r]
        assert t == 50.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.050)


def test_single_rank_is_unchanged(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "1")
    import bench
    t, v = bench.combine_ranks(20.0, 100, 5)
    assert t == 20.0 and v == pytest.approx(100 * 5 / 0.020)
