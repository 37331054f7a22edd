"""The N > 1 path of bench.py on CPU: two gloo ranks (127.0.0.1), no GPU.  Each rank gets
its own synthetic pairs (weak scaling, no data-path collective), the step time of the job
is the slowest rank's (max over ranks) and the reported value counts every rank's pairs."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, B, distinct, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        b = _bench()
        seeds = b.rank_pair_seeds(rank, B, distinct)
        everyone = [None] * world
        dist.all_gather_object(everyone, seeds)
        barrier, max_over_ranks = b.rank_reducers(world, dist, "cpu")
        barrier()
        my_ms = 3.0 + 2.0 * rank                 # rank 1 is the slow one
        ms = max_over_ranks(my_ms)
        q.put((rank, everyone, ms, b.whole_job_value(B, world, ms)))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_shard_pairs_and_time_the_slowest():
    world, B, distinct = 2, 64, 16
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, B, distinct, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=100) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, everyone, ms, value in out:
        assert len(everyone) == world
        assert set(everyone[0]).isdisjoint(everyone[1])        # no pair is processed twice
        assert all(len(s) == distinct for s in everyone)
        assert ms == pytest.approx(5.0)                          # the slowest rank's step
        assert value == pytest.approx(B * world / 5e-3)          # every rank's pairs / job time
