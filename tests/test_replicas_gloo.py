"""Multi-rank path of bench.py on CPU (gloo, world size 2): replicas take their
own seeded problems, the job time is the slowest rank's and the throughput
counts every rank's solves.  No GPU is involved."""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    from paper_1908_07071_gb300.synthetic import make_mesh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 0.5 * rank, world)
        v, k = make_mesh(3, 3, seed=rank, perturb=0.15)
        out.put((rank, t, bench.replica_throughput(t, 5, world), float(v.sum()), float(k.sum())))
    finally:
        dist.destroy_process_group()


def test_two_replicas_gloo():
    world, port = 2, 29500 + os.getpid() % 1000
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time; throughput = all ranks' solves / that time
    assert [r[1] for r in res] == [1.5, 1.5]
    assert [r[2] for r in res] == pytest.approx([2 * 5 / 1.5] * 2)
    # each replica solves its own problem (seed = rank)
    assert res[0][3] != res[1][3] and res[0][4] != res[1][4]


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.replica_throughput(2.0, 4, 1) == 2.0
