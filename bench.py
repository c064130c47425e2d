"""Benchmark: superiorized iterations/s on the clinical-size synthetic plan.

Workload: 200 x 200 x 150 water phantom at 2 mm (6e6 voxels), three coplanar
fields at 0/90/270 degrees, 30000 spots, D and L in FP32 CSR with one shared
pattern (5.6e8 nonzeros each), PTV ellipsoid 150 cc and three OARs with dose
and LETd limits; w0 = 1, alpha 0.99, relaxation 1.  One step = one
superiorized iteration (Fig. 3 around the simultaneous Fig. 2): two fused
forward products and two transposed products over every voxel row.

Output: one JSON line (rank 0).  `value` is device throughput with the plan
resident in HBM; `e2e` is one full plan re-optimisation (500 iterations)
through the public C ABI from pinned host buffers; `roofline` is the dominant
kernel's algorithmic bytes / its CUDA-event time on the library stream;
`cpu_baseline` is the FP64 oracle on a bounded sample (one iteration of the
same plan) on the host cores.  `--impl reference` times that oracle as the
reference arm.  With --gpus N each rank runs an independent replica (the
path has no exchange step): value = all ranks' iterations / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "superiorized iters/s & SpMV %HBM peak; serving plans/hr, p99 latency vs plain FP32"
UNIT = "iters/s"
WORKLOAD = ("clinical: 200x200x150 voxels at 2 mm, 3 fields 0/90/270 deg, 30000 spots, "
            "FP32 CSR D and L (shared pattern), PTV 150 cc + 3 OARs, w0=1, alpha 0.99, relaxation 1")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, device=None) -> float:
    """Maximum of a float over all ranks (identity without a process group)."""
    try:
        import torch.distributed as dist
    except Exception:
        return float(x)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(steps_per_rank: int, max_ms: float, world: int) -> float:
    """Iterations of all replicas per second of the slowest rank (weak scaling)."""
    return world * steps_per_rank / (max_ms * 1e-3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# DRAM bytes per nonzero of one forward launch (dram__bytes_read.sum +
# dram__bytes_write.sum, ncu, half-resolution clinical phantom, average of the
# two forward launches of an iteration), keyed by (storage, index bytes);
# traffic grows with the nonzeros, so it is scaled to the full plan.  A
# stream without a capture reports null.
FWD_TRAFFIC_PER_NNZ = {("fp32", 4): 12.48, ("fp32", 2): 10.17}
# the same for the transposed product (average of its gradient and projection
# launches), keyed by (storage, row index bytes)
BWD_TRAFFIC_PER_NNZ = {("fp32", 2): 8.26}


def fwd_bytes(nnz, rows, vb, ib, n_launch_obj, n_launch_bc):
    """Algorithmic bytes of the forward launches: the shared index stream
    (ib = 2 or 4 B) and both value streams (vb B each) per nonzero; per row
    with nonzeros: row_ptr (8 B), the (Dx, Lx) pair (8 B), mask (4 B) and the
    residual pair written (OBJ) or read (BC) (8 B).  16-bit storage adds the
    two row scales (8 B)."""
    base = nnz * (ib + 2 * vb) + rows * (8 + 8 + 12 + (8 if vb == 2 else 0))
    return (n_launch_obj + n_launch_bc) * base


def bwd_bytes(nnz, n_hot, n_chunks, vb, rb, n_grad, n_proj):
    """Transposed launches: row index (rb = 2 or 4 B) + L (vb) [+ D (vb) for
    the projection pass, and for a gradient with DOSE terms] per nonzero, the
    coefficient pair read once per row with nonzeros (8 B), chunk pointer
    (8 B) and chunk sum (4 B) per chunk.  Based 16-bit rows also read a 4 B
    base per 128 nonzeros (and 512 B per wide block, an encoding cost left
    out here)."""
    hdr = nnz // 128 * 4 if rb == 2 else 0
    g = nnz * (rb + vb) + hdr + n_hot * 8 + n_chunks * 12
    p = nnz * (rb + 2 * vb) + hdr + n_hot * 8 + n_chunks * 12
    return n_grad * g + n_proj * p


SMALL = dict(shape=(100, 100, 75), h=4.0)  # same phantom at half resolution (profiling case)


def make_plan(seed, small=False):
    import phantom
    return phantom.clinical_plan(seed=seed, **(SMALL if small else {}))


def run_gpu_arm(args):
    import torch
    import phantom
    from paper_2509_20012_gb300 import Handle, default_params

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    t_gen = time.perf_counter()
    plan = make_plan(seed=args.seed + rank, small=args.small)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream(device=local)
    hbm, hbm_src = peaks()
    out = {}

    def timed_run(rows, fmt="fp32"):
        h = Handle(local, stream=stream)
        t0 = time.perf_counter()
        h.load_plan(plan, fmt=fmt, rows=rows)
        t_load = time.perf_counter() - t0
        sz = h.sizes()
        ib, rb, _ = h.storage()
        # plain launches with CUDA events around every kernel on the library stream
        h.set_timing(True)
        h.begin(plan.w0, plan.alpha, plan.relaxation)
        h.iterate(args.warmup)
        torch.cuda.synchronize()
        h.set_timing(True)  # reset the counters: only the timed region below counts
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.iterate(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        ms = reduce_max(e0.elapsed_time(e1), device=f"cuda:{local}")
        kt = h.get_timing()
        launches = h.launch_count()
        w, dose, letd, rep = h.end()
        h.close()
        log = None
        vb = 4 if fmt == "fp32" else 2
        nf = kt["forward"][1]
        nb = kt["backward"][1]
        n_iter = args.steps
        hot = np.ones(plan.n_vox, bool) if rows == "all" else plan.mask != 0
        rows_nz = int(np.count_nonzero(hot & (np.diff(plan.row_ptr) > 0)))
        fb = fwd_bytes(sz["nnz_rows"], rows_nz, vb, ib, n_iter, n_iter)
        # chunk count is internal; it is small next to nnz (bounded by nnz/256 + n_spots)
        n_chunks_est = sz["nnz_rows"] // 2048 + sz["n_spots"]
        bb = bwd_bytes(sz["nnz_rows"], rows_nz, n_chunks_est, vb, rb, n_iter, n_iter)
        f_ms, b_ms = kt["forward"][0], kt["backward"][0]
        fw = {"bound": "hbm", "achieved": fb / (f_ms * 1e-3) / 1e9 if f_ms else None, "peak": hbm,
              "unit": "GB/s", "kernel": "k_forward (fused Dx/Lx)", "index_bytes": ib, "launches": nf,
              "ms_total": f_ms,
              "bytes_per_launch": fb / max(1, 2 * n_iter)}
        bw = {"bound": "hbm", "achieved": bb / (b_ms * 1e-3) / 1e9 if b_ms else None, "peak": hbm,
              "unit": "GB/s", "kernel": "k_backward (CSC chunks)", "row_index_bytes": rb, "launches": nb,
              "ms_total": b_ms,
              "bytes_per_launch": bb / max(1, 2 * n_iter)}
        for r in (fw, bw):
            r["frac"] = r["achieved"] / hbm if r["achieved"] else None
        t = FWD_TRAFFIC_PER_NNZ.get((fmt, ib))
        fw["traffic"] = t * sz["nnz_rows"] if t else None
        t = BWD_TRAFFIC_PER_NNZ.get((fmt, rb))
        bw["traffic"] = t * sz["nnz_rows"] if t else None
        return dict(ms=ms, kt=kt, launches=launches, clocks=clocks, rep=rep, sizes=sz, t_load=t_load,
                    fwd=fw, bwd=bw, w=w, dose=dose, letd=letd)

    main = timed_run("all", args.fmt)
    roi = timed_run("roi", args.fmt) if args.roi else None
    prec = {}
    if args.precision:
        # FP64-class reference outputs: the double-float final pass of an FP32
        # handle (the FP32 inputs multiplied in FP64)
        ref = Handle(local, stream=stream)
        ref.load_plan(plan)

        def fp64_outputs(w):
            ref.begin(w, plan.alpha, plan.relaxation)
            _, d, l, _ = ref.end()
            return d.astype(np.float64), l.astype(np.float64)

        d32, l32 = fp64_outputs(main["w"])
        for fmt in ("bf16", "fp16"):
            r = timed_run("all", fmt)
            d_ref, l_ref = fp64_outputs(r["w"])
            sel = d_ref > 0.01 * plan.prescription
            err_d = np.abs(r["dose"] - d_ref) / plan.prescription
            err_l = np.abs(r["letd"] - l_ref)[sel]
            prec[fmt] = {
                "value": whole_job_value(args.steps, r["ms"], ws), "ms_per_step": r["ms"] / args.steps,
                "forward": r["fwd"], "backward": r["bwd"],
                "dose_err_max_frac_of_2Gy": float(err_d.max()), "dose_err_mean_frac_of_2Gy": float(err_d.mean()),
                "letd_err_max_keV_um": float(err_l.max()), "letd_err_mean_keV_um": float(err_l.mean()),
                "letd_err_where": "voxels with dose > 1% of prescription",
                "vs_fp32_solution_dose_max_frac_of_2Gy": float(np.max(np.abs(d_ref - d32)) / plan.prescription),
                "vs_fp32_solution_letd_max_keV_um": float(np.max(np.abs(l_ref - l32)[sel & (d32 > 0.01 * plan.prescription)])),
            }
        ref.close()

    # end to end: one plan re-optimisation from pinned host buffers through the C ABI
    e2e = None
    if args.e2e_iters > 0:
        pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(plan, k))).pin_memory()
               for k in ("row_ptr", "col", "D", "L")}
        pin_mask = torch.from_numpy(plan.mask.view(np.int32)).pin_memory()
        pin_w0 = torch.from_numpy(plan.w0).pin_memory()
        out_w = torch.empty(plan.n_spots, dtype=torch.float32).pin_memory()
        out_d = torch.empty(plan.n_vox, dtype=torch.float32).pin_memory()
        out_l = torch.empty(plan.n_vox, dtype=torch.float32).pin_memory()
        h = Handle(local, stream=stream)
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.load_influence(pin["row_ptr"], pin["col"], pin["D"], pin["L"], pin_mask, plan.n_spots)
        h.set_constraints(plan.constraints)
        h.set_objective(plan.objective)
        h.superiorize(pin_w0, args.e2e_iters, plan.alpha, plan.relaxation, outputs=(out_w, out_d, out_l))
        t_e2e = reduce_max(time.perf_counter() - t0, device=f"cuda:{local}")
        h.close()
        h2d = sum(v.numel() * v.element_size() for v in pin.values()) + pin_mask.numel() * 4 + plan.n_spots * 4
        d2h = (plan.n_spots + 2 * plan.n_vox) * 4
        e2e = {"value": ws * args.e2e_iters / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.e2e_iters, "d2h_bytes_per_step": d2h / args.e2e_iters,
               "what": f"load_influence from pinned host + set_constraints + set_objective + "
                       f"superiorize({args.e2e_iters} iters) with host w0/w/dose/LETd; {t_e2e:.3f} s"}

    sweep = None
    if rank == 0 and args.sweep:
        sweep = sweep_benchmark(plan, local, stream)

    volume = None
    if rank == 0 and args.volume:
        volume = volume_benchmark(plan, main["w"], local, stream, hbm)

    serving = None
    if ws == 1 and args.serve_requests > 0:
        serving = serving_benchmark(args, local, clinical=None if args.small else plan)
    batching = None
    if ws == 1 and args.batch:
        batching = batching_benchmark(args, local)

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_iters > 0:
        cpu = cpu_baseline(plan, args.cpu_iters)

    if rank == 0:
        dom = main["fwd"] if (main["fwd"]["ms_total"] or 0) >= (main["bwd"]["ms_total"] or 0) else main["bwd"]
        value = whole_job_value(args.steps, main["ms"], ws)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": "all voxel rows streamed every pass",
                       "n_vox": main["sizes"]["n_vox"], "n_spots": main["sizes"]["n_spots"],
                       "nnz_per_matrix": main["sizes"]["nnz"], "storage": args.fmt,
                       "l2": "inputs larger than L2 (each forward pass streams %.1f GB, each "
                             "transposed pass %.1f GB on average)" % (
                           main["fwd"]["bytes_per_launch"] / 1e9, main["bwd"]["bytes_per_launch"] / 1e9),
                       "parallelism": f"replicas{ws}", "generate_s": round(t_gen, 2),
                       "load_s": round(main["t_load"], 3)},
            "roofline": {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")} | {
                "kernel": dom["kernel"], "peak_source": hbm_src,
                "forward": main["fwd"], "backward": main["bwd"]},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": main["launches"],
            "clocks": main["clocks"],
            "kernel_ms": {k: v[0] for k, v in main["kt"].items()},
            "final": {"objective": main["rep"]["objective"], "n_violated": main["rep"]["n_violated"],
                      "max_violation": main["rep"]["max_violation"]},
        }
        if volume is not None:
            line["volume_stats"] = volume
        if sweep is not None:
            line["sweep"] = sweep
        if serving is not None:
            line["serving"] = serving
        if batching is not None:
            line["batching"] = batching
        if prec:
            line["precision"] = {"note": ("D and L stored in 16 bits with power-of-two FP32 row scales, "
                                          "16-bit indices (bit-identical to int32 ones), FP32 accumulation, FP64 norms and final "
                                          "check; "
                                          "errors of the outputs at each run's final w against the FP64 "
                                          "product of the FP32 inputs"), **prec}
        if roi is not None:
            line["roi_rows"] = {"value": whole_job_value(args.steps, roi["ms"], ws),
                                "ms_per_step": roi["ms"] / args.steps,
                                "n_rows": roi["sizes"]["n_rows"], "nnz_rows": roi["sizes"]["nnz_rows"],
                                "forward": roi["fwd"], "backward": roi["bwd"], "clocks": roi["clocks"],
                                "max_abs_w_diff_vs_all_rows": float(np.max(np.abs(roi["w"] - main["w"])))}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


SERVE_RES_MM = [8.0, 6.0, 5.0, 4.0, 3.0, 2.4, 2.0]  # clinical phantom family (2 mm = the clinical plan)


def serving_library(clinical=None):
    """Plans between the tiny plan and the clinical plan: the tiny plan and the
    clinical phantom at 7 resolutions of the same geometry (`clinical`, the
    2 mm plan, is reused when given)."""
    import phantom
    lib = [phantom.tiny_plan()]
    for h in SERVE_RES_MM:
        if h == 2.0 and clinical is not None:
            lib.append(clinical)
            continue
        shape = (int(round(400 / h)), int(round(400 / h)), int(round(300 / h)))
        lib.append(phantom.clinical_plan(shape=shape, h=h))
    return lib


def serving_trace(lib, n_req, rate, seed):
    """Poisson arrivals (mean `rate`/s); sizes log-uniform between the smallest
    and the largest plan (nearest plan of the library); FP32/BF16 50:50;
    100-500 iterations."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    lognnz = np.log([p.nnz for p in lib])
    target = rng.uniform(lognnz.min(), lognnz.max(), n_req)
    idx = [int(np.argmin(np.abs(lognnz - x))) for x in target]
    fmt = ["bf16" if u < 0.5 else "fp32" for u in rng.uniform(size=n_req)]
    iters = rng.integers(100, 501, n_req)
    return [dict(t=float(t[i]), plan=idx[i], fmt=fmt[i], iters=int(iters[i])) for i in range(n_req)]


def run_trace(server, lib, trace, force_fp32=False, at_once=False):
    import threading
    tickets = [None] * len(trace)

    def submitter():
        t0 = time.perf_counter()
        for i, r in enumerate(trace):
            d = t0 + r["t"] - time.perf_counter()
            if d > 0 and not at_once:
                time.sleep(d)
            p = lib[r["plan"]]
            tickets[i] = server.submit(p, fmt="fp32" if force_fp32 else r["fmt"], iters=r["iters"])

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    return [server.wait(t, timeout=3600) for t in tickets]


def serving_summary(results, n_req):
    lat = np.array([r[0]["t_done"] - r[0]["t_submit"] for r in results])
    span = max(r[0]["t_done"] for r in results) - min(r[0]["t_submit"] for r in results)
    ok = all(r[0]["status"] == 3 for r in results)
    return {"plans_per_hour": n_req / span * 3600.0, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "makespan_s": span, "all_done": ok}


def serving_benchmark(args, local, clinical=None):
    from paper_2509_20012_gb300 import Server
    lib = serving_library(clinical)
    trace = serving_trace(lib, args.serve_requests, args.serve_rate, args.seed + 1000)
    with Server(local, mem_cap_bytes=180e9, max_active=8, round_iters=10) as srv:
        served = run_trace(srv, lib, trace)
    with Server(local, mem_cap_bytes=180e9, max_active=1, round_iters=10) as srv:
        seq = run_trace(srv, lib, trace, force_fp32=True)
    # capacity: the same requests all submitted at once (saturated queue)
    with Server(local, mem_cap_bytes=180e9, max_active=8, round_iters=10) as srv:
        cap_served = serving_summary(run_trace(srv, lib, trace, at_once=True), len(trace))
    with Server(local, mem_cap_bytes=180e9, max_active=1, round_iters=10) as srv:
        cap_seq = serving_summary(run_trace(srv, lib, trace, force_fp32=True, at_once=True), len(trace))
    # accuracy of the mixed-precision results against the FP32 results of the same requests
    dmax = lmax = 0.0
    for r, a, b in zip(trace, served, seq):
        if r["fmt"] == "fp32":
            continue
        p = lib[r["plan"]]
        sel = b[2] > 0.01 * p.prescription
        dmax = max(dmax, float(np.max(np.abs(a[2] - b[2]))) / p.prescription)
        if sel.any():
            lmax = max(lmax, float(np.max(np.abs(a[3] - b[3])[sel])))
    sizes = [lib[r["plan"]].nnz for r in trace]
    return {
        "trace": (f"{args.serve_requests} requests, Poisson arrivals mean {args.serve_rate}/s, nnz per matrix "
                  f"log-uniform {min(p.nnz for p in lib):.2e}-{max(p.nnz for p in lib):.2e} "
                  f"(tiny plan + clinical phantom at {SERVE_RES_MM} mm), FP32/BF16 50:50, 100-500 iterations, "
                  f"admission cap 180 GB"),
        "requests_nnz_mean": float(np.mean(sizes)),
        "served": serving_summary(served, len(trace)) | {"mode": "continuous batching, mixed FP32/BF16, "
                                                                 "up to 8 plans resident"},
        "sequential_fp32": serving_summary(seq, len(trace)) | {"mode": "one plan at a time, FP32"},
        "capacity_plans_per_hour": {"served": cap_served["plans_per_hour"],
                                    "sequential_fp32": cap_seq["plans_per_hour"],
                                    "how": "the same requests submitted at once (saturated queue)"},
        "bf16_vs_fp32_dose_max_frac_of_2Gy": dmax, "bf16_vs_fp32_letd_max_keV_um": lmax,
    }


def batching_benchmark(args, local):
    """Batching workloads: (a) 16 independent plans, PTV 20-400 cc, nnz 6e5-7e7,
    BF16, tiles autotuned per plan, run one after another vs as one batch
    graph per iteration; (b) 27 robustness scenarios stacked into one robust
    plan (one w meets the constraints in every scenario), BF16."""
    import phantom
    from paper_2509_20012_gb300 import Batch, Handle
    iters = args.batch_iters
    plans = phantom.batch_plans(16, seed=args.seed)
    # one after another: each plan alone
    seq_ms, seq_w, tiles = 0.0, [], []
    for p in plans:
        with Handle(local) as h:
            h.load_plan(p, fmt="bf16")
            tiles.append(h.autotune(reps=3))
            h.begin(p.w0, p.alpha, p.relaxation)
            h.iterate(iters)
            w, d, l, rep = h.end()
            seq_ms += rep["device_ms"]
            seq_w.append(w)
    # all plans as one graph per iteration
    hs = []
    for p in plans:
        h = Handle(local)
        h.load_plan(p, fmt="bf16")
        h.autotune(reps=3)
        h.begin(p.w0, p.alpha, p.relaxation, use_graphs=0)
        hs.append(h)
    with Batch(hs) as b:
        b.iterate(3)       # warm-up, then the timed iterations continue the same solves
        b.sync()
        t0 = b.sync()
        b.iterate(iters - 3)
        bat_ms = b.sync() - t0
    same = True
    for h, w_ref in zip(hs, seq_w):
        w, *_ = h.end()
        same = same and bool(np.array_equal(w, w_ref))
        h.close()
    total_iters = iters * len(plans)
    out = {"independent": {
        "plans": len(plans), "nnz_per_matrix": [int(p.nnz) for p in plans], "storage": "bf16",
        "iterations_per_plan": iters, "tiles_row_chunk_weight": tiles,
        "sequential_plan_iters_per_s": total_iters / (seq_ms * 1e-3),
        "batched_plan_iters_per_s": (iters - 3) * len(plans) / (bat_ms * 1e-3),
        "batch_graph_results_identical_to_sequential": same}}
    out["independent"]["batched_speedup"] = (out["independent"]["batched_plan_iters_per_s"]
                                             / out["independent"]["sequential_plan_iters_per_s"])
    if args.robust:
        t = time.perf_counter()
        rp, per = phantom.robust_plan(seed=args.seed)
        t_gen = time.perf_counter() - t
        with Handle(local) as h:
            t = time.perf_counter()
            h.load_plan(rp, fmt="bf16")
            t_load = time.perf_counter() - t
            tune = h.autotune(reps=2)
            ib = h.storage()[0]
            h.set_timing(True)
            h.begin(rp.w0, rp.alpha, rp.relaxation)
            h.iterate(3)
            h.get_timing()
            h.set_timing(True)
            h.iterate(iters)
            kt = h.get_timing()
            w, d, l, rep = h.end()
        ms = sum(v[0] for v in kt.values())
        hbm, _ = peaks()
        fb = kt["forward"][0]
        f_bytes = 2 * iters * (rp.nnz * (ib + 4) + int(np.count_nonzero(np.diff(rp.row_ptr) > 0)) * 36)
        out["robust_stacked"] = {
            "scenarios": len(per), "nnz_per_scenario_matrix": int(np.mean(per)), "nnz_stacked": int(rp.nnz),
            "rows_stacked": int(rp.n_vox), "n_spots": int(rp.n_spots), "storage": "bf16", "index_bytes": ib,
            "tiles": tune,
            "iters_per_s": iters / (ms * 1e-3), "forward_GBps": f_bytes / (fb * 1e-3) / 1e9,
            "forward_frac_of_hbm": f_bytes / (fb * 1e-3) / 1e9 / hbm,
            "generate_s": round(t_gen, 1), "load_s": round(t_load, 2),
            "final_max_violation": rep["max_violation"], "final_objective": rep["objective"]}
    return out


def volume_benchmark(plan, w, local, stream, hbm, reps=20):
    """Volume statistics of the final fluence (Sec. 2.4.1): 1000-bin DVH,
    cDLVH and LVH of every structure, and the values at volume a plan review
    reads (PTV D98/D95/D50/D2, OAR cDL30 and D2), timed by class with CUDA
    events on the library stream."""
    from paper_2509_20012_gb300 import Handle
    h = Handle(local, stream=stream)
    h.load_plan(plan)
    bits = sorted({s["bit"] for s in plan.structures})
    oars = [s["bit"] for s in plan.structures if s["role"] == "oar"]
    ptv = [s["bit"] for s in plan.structures if s["role"] == "target"][0]
    top = {"DOSE": 1.3 * plan.prescription, "CDL": 0.5, "LETD": 15.0}
    hist = [{"quantity": q, "struct_bit": b, "edges": np.linspace(0.0, top[q], 1001, dtype=np.float32)}
            for b in bits for q in ("DOSE", "CDL", "LETD")]
    sel = ([{"quantity": "DOSE", "struct_bit": ptv, "fracs": [0.98, 0.95, 0.5, 0.02]}] +
           [{"quantity": "CDL", "struct_bit": b, "fracs": [0.30]} for b in oars] +
           [{"quantity": "DOSE", "struct_bit": b, "fracs": [0.02]} for b in oars])
    out = {}
    any_bits = np.uint32(sum(1 << b for b in bits))
    n_struct = int(np.count_nonzero(plan.mask & any_bits))
    for name, reqs, n_pass in (("histograms", hist, 1), ("values_at_volume", sel, 5)):
        for _ in range(3):
            res = h.volume_stats(reqs, w)
        h.set_timing(True)
        t0 = time.perf_counter()
        for _ in range(reps):
            res = h.volume_stats(reqs, w)
        wall = (time.perf_counter() - t0) / reps
        kt = h.get_timing()
        h.set_timing(False)
        other_ms = kt["other"][0] / reps
        # each pass reads the mask of every streamed row and the FP64 pair of the structure rows
        by = n_pass * (plan.n_vox * 4 + n_struct * 16)
        out[name] = {"requests": len(reqs), "ms_per_call": wall * 1e3, "final_pass_ms": kt["forward"][0] / reps,
                     "stats_kernels_ms": other_ms, "stats_launches": 1 if n_pass == 1 else 9,
                     "stats_bytes": by, "stats_achieved_gbs": by / (other_ms * 1e-3) / 1e9 if other_ms else None,
                     "peak": hbm}
        if name == "values_at_volume":
            out[name]["results"] = {f"{r['quantity']}:{r['struct_bit']}": [float(x) for x in v["at_volume"]]
                                    for r, v in zip(reqs, res)}
    h.close()
    out["note"] = ("%d structure voxels of %d rows; the statistics kernels read 4 B of mask per row and 16 B of "
                   "FP64 (Dw, Lw) per structure voxel per pass, mostly from L2 right after the final pass: "
                   "launch- and L2-bound, not an HBM roofline" % (n_struct, plan.n_vox))
    return out


def sweep_benchmark(plan, local, stream, iters=100, warmup=5):
    """Superiorized iterations with the block-iterative feasibility sweep
    (sweep_blocks voxel blocks visited in turn) against the simultaneous step,
    clinical plan in ROI-row mode (the sweep's blocks are structure voxels)."""
    import torch
    from paper_2509_20012_gb300 import Handle
    out = {}
    for m in (0, 16, 64, 256):
        h = Handle(local, stream=stream)
        h.load_plan(plan, rows="roi")
        h.begin(plan.w0, plan.alpha, plan.relaxation, sweep_blocks=m)
        h.iterate(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.iterate(iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches_per_iter = None
        _, _, _, rep = h.end()
        # per-class device time from a short run with events around every launch
        h.set_timing(True)
        h.begin(plan.w0, plan.alpha, plan.relaxation, sweep_blocks=m)
        n0 = h.launch_count()
        h.iterate(10)
        torch.cuda.synchronize()
        launches_per_iter = (h.launch_count() - n0) / 10
        kt = h.get_timing()
        h.close()
        out["simultaneous" if m == 0 else f"sweep{m}"] = {
            "iters_per_s": iters / (ms * 1e-3), "ms_per_iter": ms / iters, "launches_per_iter": launches_per_iter,
            "kernel_ms_per_iter": {k: v[0] / 10 for k, v in kt.items()},
            "max_violation_after": rep["max_violation"], "n_violated_after": rep["n_violated"]}
    out["note"] = (f"clinical plan, ROI rows, {iters} superiorized iterations after {warmup} warm-up, CUDA graph "
                   "replay; kernel_ms_per_iter from a 10-iteration run with events around every launch "
                   "(sweep: forward = block forward products, backward = block column updates)")
    return out


def cpu_baseline(plan, iters):
    """FP64 oracle, as it stands, on `iters` iterations of the same plan."""
    import oracle
    P = oracle.build_problem(plan.row_ptr, plan.col, plan.D, plan.L, plan.n_spots, plan.mask,
                             plan.constraints, plan.objective)
    R = oracle.constraint_rows(P)
    t0 = time.perf_counter()
    oracle.superiorize(P, plan.w0, iters, plan.alpha, plan.relaxation, rows=R)
    dt = time.perf_counter() - t0
    return {"value": iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{iters} superiorized iteration(s) of the clinical plan (FP64 numpy/scipy, "
                      f"single-threaded sparse products), {dt:.1f} s; setup excluded"}


def run_reference_arm(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    plan = make_plan(seed=args.seed, small=args.small)
    P = oracle.build_problem(plan.row_ptr, plan.col, plan.D, plan.L, plan.n_spots, plan.mask,
                             plan.constraints, plan.objective)
    R = oracle.constraint_rows(P)
    w = plan.w0.astype(np.float64)
    s = 0
    beta0 = 0.1 * float(np.linalg.norm(w))
    k = 0
    for _ in range(args.ref_warmup):
        w, log = oracle.superiorize(P, w, 1, plan.alpha, plan.relaxation, rows=R, beta0=beta0, s0=s, k0=k)
        s, k = log[-1]["s"], k + 1
    t0 = time.perf_counter()
    for _ in range(args.ref_steps):
        w, log = oracle.superiorize(P, w, 1, plan.alpha, plan.relaxation, rows=R, beta0=beta0, s0=s, k0=k)
        s, k = log[-1]["s"], k + 1
    dt = time.perf_counter() - t0
    v = args.ref_steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.ref_steps, "warmup": args.ref_warmup, "ms_per_step": dt * 1e3 / args.ref_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "rows": "all voxel rows"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.ref_steps} timed iteration(s) after {args.ref_warmup} "
                                       f"warm-up, FP64 oracle, single-threaded sparse products"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-roi", dest="roi", action="store_false")
    ap.add_argument("--e2e-iters", type=int, default=500)
    ap.add_argument("--cpu-iters", type=int, default=1)
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the serving trace (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="mean arrivals per second")
    ap.add_argument("--no-precision", dest="precision", action="store_false",
                    help="skip the BF16/FP16 storage runs")
    ap.add_argument("--fmt", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="value storage of the main timed run (profiling of the 16-bit streams)")
    ap.add_argument("--small", action="store_true",
                    help="half-resolution phantom (100x100x75 at 4 mm) for profiler captures")
    ap.add_argument("--batching", action="store_true",
                    help="run only the batching workloads (16 independent plans; 27 stacked robustness scenarios)")
    ap.add_argument("--no-batch", dest="batch", action="store_false",
                    help="skip the batching workloads in the default run")
    ap.add_argument("--no-robust", dest="robust", action="store_false")
    ap.add_argument("--batch-iters", type=int, default=100)
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the block-iterative sweep timing")
    ap.add_argument("--no-volume", dest="volume", action="store_false",
                    help="skip the volume-statistics timing (DVH, values at volume)")
    args = ap.parse_args()
    if args.batching:
        import torch
        ws, rank, local = dist_env()
        torch.cuda.set_device(local)
        res = batching_benchmark(args, local)
        print(json.dumps({"metric": "batching", "n_gpus": 1, "data": "synthetic", **res}))
        return
    if args.warmup < 3:
        args.warmup = 3
    # the reference arm (FP64 oracle on the host cores) is bounded: one
    # iteration of the clinical plan takes ~10-20 s
    args.ref_steps = max(1, min(args.steps, 2))
    args.ref_warmup = 0
    if args.impl == "reference":
        run_reference_arm(args)
    else:
        run_gpu_arm(args)


if __name__ == "__main__":
    main()
