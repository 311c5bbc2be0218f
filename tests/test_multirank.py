"""Multi-rank host logic of bench.py, on CPU ranks (gloo backend, world size 2). The batch
workload's scene shards partition the job's scenes with no scene on two ranks, and balance
the tet counts. The timing reduction takes the maximum over ranks, and the sweep totals
are summed. A single scene runs as one replica per rank, and the reference arm runs on
rank 0 alone."""
import importlib.util
import os
import socket

import pytest

import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, n_per_rank, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        sizes = [scenes.blob_tet_target(i) for i in range(n_per_rank * world)]
        mine = bench.shard_scenes(sizes, world)[rank]
        every = [None] * world
        dist.all_gather_object(every, mine)
        dist.barrier()
        mx = bench.over_ranks(10.0 + 5.0 * rank, "max")
        sm = bench.over_ranks(1.0 + rank, "sum")
        q.put((rank, every, mx, sm, sizes))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port, n = 2, _free_port(), 64
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort()
    shards = out[0][1]
    assert out[1][1] == shards  # every rank computes the same assignment
    flat = sorted(i for sh in shards for i in sh)
    assert flat == list(range(n * world))  # a partition: no scene on two ranks, none left out
    sizes = out[0][4]
    loads = [sum(sizes[i] for i in sh) for sh in shards]
    assert max(loads) - min(loads) <= max(sizes)  # largest-first greedy bound
    assert all(o[2] == 15.0 for o in out)  # max over ranks of 10 + 5 rank
    assert all(o[3] == 3.0 for o in out)  # sum over ranks of 1 + rank


def test_one_rank_keeps_the_whole_batch_in_order():
    bench = _bench()
    sizes = [scenes.blob_tet_target(i) for i in range(256)]
    assert bench.shard_scenes(sizes, 1) == [list(range(256))]
    assert bench.over_ranks(3.5) == 3.5  # no process group: the value itself


def test_reference_arm_runs_on_rank_zero_only():
    bench = _bench()
    assert bench.run_reference(None, rank=1, world=2) is None
