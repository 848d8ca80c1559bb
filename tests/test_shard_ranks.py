"""Runs sharded by system (forests, request streams): independent systems are
dealt to ranks by bh_partition_systems, each rank runs its shard on its own GPU
with the single-GPU forest code, and only results are gathered on the host.

CPU tests: the assignment covers every system exactly once, is deterministic,
and keeps the largest rank cost within the longest-first bound; two gloo ranks
each take their shard and together cover every system once.  GPU tests: two
ranks (processes) share one GPU; each runs its shard's forest through graph
steps, and rank 0 finds every gathered system bit-identical to the same system
in one forest of all of them; and the benchmark's batched and served legs run
sharded over the two ranks and report the same whole-job figures on both.  No
kernel of one rank waits on another rank.
"""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1109_5190_gb300 import binding as B  # noqa: E402


def _cost(n):
    return n * math.log2(max(n, 2))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_covers_every_system_once_and_balances(world):
    rng = np.random.default_rng(world)
    sizes = np.rint(np.exp(rng.uniform(math.log(256), math.log(65536), 512))).astype(np.int64)
    r = B.bh_partition_systems(sizes, world)
    assert r.shape == (512,) and r.min() >= 0 and r.max() < world
    assert np.array_equal(r, B.bh_partition_systems(sizes, world))  # deterministic
    load = np.zeros(world)
    for s, q in enumerate(r):
        load[q] += _cost(int(sizes[s]))
    # longest-first greedy: the largest load exceeds the mean by at most one system
    assert load.max() <= load.sum() / world + max(_cost(int(x)) for x in sizes) + 1e-6
    # and against brute force on a small case: within 4/3 of the best split
    small = sizes[:9]
    rs = B.bh_partition_systems(small, 2)
    got = max(sum(_cost(int(small[s])) for s in range(9) if rs[s] == q) for q in (0, 1))
    best = min(max(sum(_cost(int(small[s])) for s in range(9) if (m >> s) & 1),
                   sum(_cost(int(small[s])) for s in range(9) if not (m >> s) & 1))
               for m in range(1 << 9))
    assert got <= 4 / 3 * best + 1e-6


def test_partition_edge_cases():
    assert B.bh_partition_systems([], 4).size == 0
    assert list(B.bh_partition_systems([10, 10, 10], 5)) == [0, 1, 2]
    assert list(B.bh_partition_systems([7, 9], 1)) == [0, 0]
    with pytest.raises(B.BHError):
        B.bh_partition_systems([5, 0], 2)
    with pytest.raises(B.BHError):
        B.bh_partition_systems([5], 0)


def _shard_rank(rank, world, port, sizes, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = bench.shard_of(B, sizes, world, rank)
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, mine, got))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_shards_covering_every_system():
    sizes = [int(x) for x in np.random.default_rng(9).integers(256, 65536, 101)]
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, sizes, qu)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, mine, got = qu.get(timeout=120)
        out[rank] = (mine, got)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == out[1][1]  # both ranks saw the same shards
    s0, s1 = out[0][0], out[1][0]
    assert sorted(s0 + s1) == list(range(len(sizes))) and not set(s0) & set(s1)
    assert s0 and s1


def _forest_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    systems = synth.forest_systems(24, 256, 4096, seed=21, theta=0.6, eps=0.01)
    mine = bench.shard_of(B, [s.n for s in systems], world, rank)
    descs = [dict(pos_mass=systems[k].pos_mass, vel=systems[k].vel, eps=0.01, theta=0.6, dt=1e-3)
             for k in mine]
    f = B.bh_forest_create(descs)
    try:
        B.bh_forest_step(f, 5, 1e-3, True)
        states = {}
        for i, k in enumerate(mine):
            x = np.zeros((systems[k].n, 4), np.float32)
            a = np.zeros_like(x)
            B.bh_forest_get_state(f, i, x, None, a)
            states[k] = (x, a)
    finally:
        B.bh_forest_destroy(f)
    got = [None] * world
    dist.gather_object(states, got if rank == 0 else None, dst=0)
    if rank == 0:
        q.put({k: v for part in got for k, v in part.items()})
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_sharded_forest_equals_one_forest():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import synth
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_forest_rank, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = qu.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    systems = synth.forest_systems(24, 256, 4096, seed=21, theta=0.6, eps=0.01)
    assert sorted(gathered) == list(range(len(systems)))
    f = B.bh_forest_create([dict(pos_mass=s.pos_mass, vel=s.vel, eps=0.01, theta=0.6, dt=1e-3)
                            for s in systems])
    try:
        B.bh_forest_step(f, 5, 1e-3, True)
        for k, s in enumerate(systems):
            x = np.zeros((s.n, 4), np.float32)
            a = np.zeros_like(x)
            B.bh_forest_get_state(f, k, x, None, a)
            assert np.array_equal(gathered[k][0], x) and np.array_equal(gathered[k][1], a), k
    finally:
        B.bh_forest_destroy(f)


def _bench_rank(rank, world, port, q):
    import argparse
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import bench
    args = argparse.Namespace(forest_systems=12, forest_steps=4, plain_steps=2)
    batched = bench.bench_batched(args, B, torch, None)
    served = bench.serve_stream(B, 200.0, 0.05, 5, bench.serve_pools(), budget_gb=4.0)
    q.put((rank, batched, served))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_bench_sharded_legs_on_two_ranks():
    # The benchmark's batched and served legs with two ranks (sharing one GPU
    # here, each with its own forest or server): both ranks report the same
    # whole-job figures, over every system and every request.
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import synth
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, batched, served = qu.get(timeout=900)
        out[rank] = (batched, served)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    b0, s0 = out[0]
    b1, s1 = out[1]
    total = sum(s.n for s in synth.forest_systems(12, 256, 65536, seed=4, theta=0.5, eps=0.01,
                                                  materialise=False))
    for b in (b0, b1):
        assert b["ranks"] == 2 and f"(sum {total})" in b["workload"]
    assert b0["value"] == b1["value"] and b0["plain_sequential_graph"] == b1["plain_sequential_graph"]
    assert b0["err_p99"] <= 1e-5 and b0["err_max"] <= 1e-3  # rank 0 checks its share
    nreq = len(synth.request_stream(rate_hz=200.0, duration_s=0.05, seed=5))
    for s in (s0, s1):
        assert s["ranks"] == 2 and s["requests"] == nreq
    assert s0["value"] == s1["value"] and s0["p99_latency_s"] == s1["p99_latency_s"]
