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
    assert all(100 <= r["iters"] <= 500 and r["fmt"] in ("fp32", "fp16") for r in t1)
    assert {r["fmt"] for r in bench.serving_trace(lib, 50, 2.0, seed=5, fmt16="bf16")} == {"fp32", "bf16"}
    assert np.all(np.diff([r["t"] for r in t1]) > 0)
    res = [({"t_submit": float(i), "t_done": float(i) + 1.0 + (i == 9), "status": 3},) for i in range(10)]
    s = bench.serving_summary(res, 10)
    assert s["all_done"] and s["p50_latency_s"] == 1.0 and s["makespan_s"] == 11.0
    assert s["plans_per_hour"] == 10 / 11.0 * 3600


def test_row_sample_config_and_byte_models():
    """The reference arm's row sample keeps every m-th voxel row bit for bit;
    both arms print the same config for the same plan; the int32 accounting
    counts 12 + 2 vb bytes per nonzero."""
    import numpy as np
    import bench
    import phantom
    pl = phantom.tiny_plan()
    sub = bench.row_sample(pl, 7)
    rows = np.arange(0, pl.n_vox, 7)
    assert sub.n_vox == len(rows) and sub.n_spots == pl.n_spots
    np.testing.assert_array_equal(sub.mask, pl.mask[rows])
    for i in (0, 5, len(rows) - 1):
        r = rows[i]
        s0, s1 = pl.row_ptr[r], pl.row_ptr[r + 1]
        np.testing.assert_array_equal(sub.col[sub.row_ptr[i]:sub.row_ptr[i + 1]], pl.col[s0:s1])
        np.testing.assert_array_equal(sub.D[sub.row_ptr[i]:sub.row_ptr[i + 1]], pl.D[s0:s1])
    assert bench.workload_config(10, 3, 100, "fp32", 1) == bench.workload_config(10, 3, 100, "fp32", 1)
    assert bench.pass_bytes_int32(1000, 10, 3, 4) == 1000 * 12 + 10 * 12 + 12
    assert bench.pass_bytes_int32(1000, 10, 3, 2) == 1000 * 8 + 10 * 20 + 12
    info = bench.cpu_info()
    assert info["nproc"] >= 1 and "cpu_model" in info


def test_output_errors_against_the_oracle():
    """The CPU leg's error measure: zero for the oracle's own outputs, the
    dose error in units of the prescription, LETd only above 1% of it."""
    import numpy as np
    import bench
    import oracle
    import phantom
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    w = pl.w0.astype(np.float64)
    d, l = oracle.forward(P, w)
    let = oracle.letd(d, l)
    e = bench.output_errors(P, w, d, let, 2.0)
    assert e["dose_max_frac_of_presc"] == 0.0 and e["letd_max_keV_um"] == 0.0
    d2 = d.copy()
    d2[np.argmax(d)] += 0.002
    e = bench.output_errors(P, w, d2, let, 2.0)
    assert e["dose_max_frac_of_presc"] == pytest.approx(0.001)


def test_serving_accuracy_bar():
    """The serving check compares each served plan's solution with the FP32
    result of the same request through the oracle's FP64 products: equal
    weights pass, a dose difference above 1e-4 of the prescription fails."""
    import numpy as np
    import bench
    from concurrent.futures import ThreadPoolExecutor
    import phantom
    pl = phantom.tiny_plan()
    w = np.random.default_rng(4).uniform(0.5, 1.5, pl.n_spots).astype(np.float32)
    trace = [dict(t=0.0, plan=0, fmt="fp32", iters=100), dict(t=0.5, plan=0, fmt="fp16", iters=100)]
    import oracle
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    d, l = oracle.forward(P, w.astype(np.float64))
    let = oracle.letd(d, l).astype(np.float32)
    serving = {"lib": [pl], "trace": trace, "served_w": [w, w.copy()], "seq_w": [w, w.copy()],
               "served_dose": [d.astype(np.float32)] * 2, "served_letd": [let] * 2}
    with ThreadPoolExecutor(2) as pool:
        ok = bench.serving_accuracy(serving, None, None, 2, pool)
        assert ok["accuracy_ok"] and len(ok["requests"]) == 2
        assert ok["worst_by_format"]["fp16"]["solution_dose_max_frac_of_presc"] == 0.0
        w2 = (w * 1.01).astype(np.float32)        # a 1% different plan: about 1e-2 of the prescription
        serving["served_w"] = [w, w2]
        bad = bench.serving_accuracy(serving, None, None, 2, pool)
    assert not bad["accuracy_ok"]
    assert bad["worst_by_format"]["fp16"]["solution_dose_max_frac_of_presc"] > 1e-3
