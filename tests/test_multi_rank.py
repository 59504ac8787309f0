"""Scenario sharding and the FP64 mean combine on 2 gloo ranks (CPU): the
sharded evaluation equals the single-process evaluation of the whole set."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, per_rank, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2602_05179_gb300 import shard
    from paper_2602_05179_gb300 import workloads as wl
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    s0, s1 = shard.scenario_range(rank, world, per_rank)
    q = wl.split_demands(spec, s0, s1)
    r = oracle.split(tour, spec.Q, q, coords=xy)
    mean = shard.combine_mean(r["cost"].sum(), len(r["cost"]))
    slowest = shard.max_over_ranks(float(rank + 1))
    out[rank] = (mean, slowest)
    dist.destroy_process_group()


def test_two_rank_weak_scaling_mean():
    world, per_rank = 2, 300
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, per_rank, out)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    import oracle
    from paper_2602_05179_gb300 import workloads as wl
    spec = wl.SPLIT_C1
    tour, xy, _ = wl.split_tour(spec)
    full = oracle.split(tour, spec.Q, wl.split_demands(spec, 0, world * per_rank), coords=xy)
    for r in range(world):
        mean, slowest = out[r]
        assert mean == pytest.approx(full["mean"], rel=1e-13)
        assert slowest == float(world)


def test_scenario_range():
    from paper_2602_05179_gb300 import shard
    assert shard.scenario_range(0, 4, 10) == (0, 10)
    assert shard.scenario_range(3, 4, 10) == (30, 40)
    with pytest.raises(ValueError):
        shard.scenario_range(4, 4, 10)
