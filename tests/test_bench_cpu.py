"""Host logic of bench.py's multi-GPU path, run as world_size-2 gloo ranks
on the CPU: every rank runs an independent replica, the timed region is the
maximum over ranks, and the whole-job value counts all ranks' iterations."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms_per_rank, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    m = bench.reduce_max(ms_per_rank[rank])
    v = bench.whole_job_value(100, m, ws)
    out[rank] = (ws, r, m, v)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_iterations():
    world = 2
    port = _free_port()
    ms = [400.0, 500.0]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ms, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ws, rank, m, v = out[r]
        assert ws == 2 and rank == r
        assert m == 500.0                       # slowest rank
        assert v == pytest.approx(2 * 100 / 0.5)  # both replicas' iterations


def test_single_process_value():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.whole_job_value(500, 2500.0, 1) == pytest.approx(200.0)


def test_bench_imports_and_serving_helpers():
    """Everything bench.py imports exists; the serving trace is seeded and its
    summary counts plans per hour and latency percentiles."""
    import numpy as np
    import bench
    import paper_2509_20012_gb300 as pkg
    for name in ("Handle", "Server", "default_params", "footprint_bytes", "DONE"):
        assert hasattr(pkg, name)

    class P:
        def __init__(self, nnz):
            self.nnz = nnz
    lib = [P(3e6), P(3e7), P(5e8)]
    t1 = bench.serving_trace(lib, 50, 2.0, seed=5)
    t2 = bench.serving_trace(lib, 50, 2.0, seed=5)
    assert t1 == t2
    assert all(100 <= r["iters"] <= 500 and r["fmt"] in ("fp32", "bf16") for r in t1)
    assert np.all(np.diff([r["t"] for r in t1]) > 0)
    res = [({"t_submit": float(i), "t_done": float(i) + 1.0 + (i == 9), "status": 3},) for i in range(10)]
    s = bench.serving_summary(res, 10)
    assert s["all_done"] and s["p50_latency_s"] == 1.0 and s["makespan_s"] == 11.0
    assert s["plans_per_hour"] == 10 / 11.0 * 3600
