"""The N > 1 host logic of bench.py on CPU: two gloo ranks (127.0.0.1) check the rank
environment and the max / sum reductions that turn per-rank step times and pair counts into
the whole-job line (max time over ranks, summed pairs; independent replicas, no data-path
collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        # per-rank step time and pairs of an independent replica
        ms = 100.0 + 25.0 * rank
        pairs = 1000.0 * (rank + 1)
        ms_max = bench.reduce_max_over_ranks(ms, w)
        pairs_all = bench.reduce_sum_over_ranks(pairs, w)
        out.put((r, w, local, ms_max, pairs_all))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, (r, w, local, ms_max, pairs_all) in enumerate(res):
        assert (r, w, local) == (rank, world, rank)
        assert ms_max == 125.0                 # the slowest rank sets the job time
        assert pairs_all == 3000.0             # whole-job units: the sum over ranks


def test_single_rank_reductions_are_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks(3.5, 1) == 3.5
    assert bench.reduce_sum_over_ranks(7.0, 1) == 7.0
