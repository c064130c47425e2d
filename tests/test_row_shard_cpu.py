"""The row-sharded multi-GPU design, checked on CPU ranks (gloo, world size 2).

The method shards by voxel rows: each rank holds a contiguous slice of the
rows of D and L, evaluates the forward products, the constraint rows and the
objective terms of its voxels, and the spot-length results are added with
one all-reduce per pass.  The fluence w is replicated.  This test runs that
exchange with two processes and the oracle's own functions on each shard, and
checks that the all-reduced simultaneous step, gradient and objective equal
the unsharded oracle's.  It exercises the design's arithmetic, not a GPU
code path: the library itself drives one GPU per process and runs replicas.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_problem(pl, lo, hi):
    import oracle
    rp = pl.row_ptr[lo:hi + 1] - pl.row_ptr[lo]
    s, e = pl.row_ptr[lo], pl.row_ptr[hi]
    return oracle.build_problem(rp, pl.col[s:e], pl.D[s:e], pl.L[s:e], pl.n_spots, pl.mask[lo:hi],
                                pl.constraints, pl.objective)


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import phantom
    pl = phantom.tiny_plan()
    V = pl.n_vox
    lo, hi = rank * V // world, (rank + 1) * V // world
    P = _shard_problem(pl, lo, hi)
    R = oracle.constraint_rows(P)
    x = np.random.default_rng(5).uniform(0.0, 2.0, pl.n_spots)
    res = {}
    for norm in ("all", "violated"):
        v = R.A @ x
        viol = np.where(R.upper, v > R.b, v < R.b)
        t = np.where(viol, (R.b - v) / R.norm2, 0.0)
        # local sums: the unnormalised projection sum and the priority sums
        u = torch.from_numpy(R.A.T @ (R.p * t))
        W = torch.tensor([R.p.sum() if norm == "all" else R.p[viol].sum()], dtype=torch.float64)
        dist.all_reduce(u)
        dist.all_reduce(W)
        res[norm] = np.maximum(x + 1.0 * u.numpy() / W.item(), 0.0)
    g = torch.from_numpy(oracle.objective_gradient(P, x))
    f = torch.tensor([oracle.objective(P, x)], dtype=torch.float64)
    dist.all_reduce(g)
    dist.all_reduce(f)
    res["grad"] = g.numpy()
    res["f"] = f.item()
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_pass_equals_unsharded_oracle():
    import oracle
    import phantom
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    R = oracle.constraint_rows(P)
    x = np.random.default_rng(5).uniform(0.0, 2.0, pl.n_spots)
    for norm in ("all", "violated"):
        ref = oracle.cimmino_step(R, x, 1.0, norm=norm)
        for r in range(world):
            np.testing.assert_allclose(out[r][norm], ref, rtol=1e-12, atol=1e-14)
    for r in range(world):
        np.testing.assert_allclose(out[r]["grad"], oracle.objective_gradient(P, x), rtol=1e-12, atol=1e-18)
        assert out[r]["f"] == pytest.approx(oracle.objective(P, x), rel=1e-12)
