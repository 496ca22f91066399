"""Replicas over evaluation points with two gloo ranks on the CPU.

Each rank evaluates its shard of a batch (here with the CPU oracle standing
in for the GPU library) and the shards are gathered; the result must equal a
single-process evaluation of the whole batch, point by point."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2204_04678_gb300.replicas import shard, shard_bounds


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from oracle import bta
    from paper_2204_04678_gb300.replicas import gather_results, max_over_ranks, shard
    from synth import build, ccd_design
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mdl = build("r", 2, 4, 1, 80, "gaussian", seed=4)
        pts = ccd_design(mdl.theta_true, 0.1)[:7]
        mine = shard(pts, rank, world)
        vals = np.array([[bta.gaussian(mdl, p, want_grad=True)["f"]] + list(bta.gaussian(mdl, p, want_grad=True)["grad"])
                         for p in mine])
        allv = gather_results(vals, len(pts))
        tmax = max_over_ranks(float(rank + 1))
        if rank == 0:
            q.put((allv, tmax))
    finally:
        dist.destroy_process_group()


def test_shard_bounds_cover_the_batch():
    for n in (0, 1, 7, 9, 25):
        for world in (1, 2, 3, 8):
            b = [shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            sizes = [e - s for s, e in b]
            assert max(sizes) - min(sizes) <= 1
    assert list(shard(list(range(7)), 1, 2)) == [4, 5, 6]


def test_two_gloo_ranks_reproduce_single_process():
    from oracle import bta
    from synth import build, ccd_design
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allv, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mdl = build("r", 2, 4, 1, 80, "gaussian", seed=4)
    pts = ccd_design(mdl.theta_true, 0.1)[:7]
    ref = np.array([[bta.gaussian(mdl, p, want_grad=True)["f"]] + list(bta.gaussian(mdl, p, want_grad=True)["grad"])
                    for p in pts])
    assert np.array_equal(allv, ref)
    assert tmax == 2.0
