"""Benchmark: superiorized iterations/s on the clinical-size synthetic plan.

Workload: 200 x 200 x 150 water phantom at 2 mm (6e6 voxels), three coplanar
fields at 0/90/270 degrees, 30000 spots, D and L in FP32 CSR with one shared
pattern (5.6e8 nonzeros each), PTV ellipsoid 150 cc and three OARs with dose
and LETd limits; w0 = 1, alpha 0.99, relaxation 1.  One step = one
superiorized iteration (Fig. 3 around the simultaneous Fig. 2): two fused
forward products and two transposed products over every voxel row.

Output: one JSON line (rank 0).  `value` is device throughput with the plan
resident in HBM, timed over K graph replays of the iteration (the library's
path); `e2e` is one full plan re-optimisation (500 iterations) through the
public C ABI from pinned host buffers; `roofline` is the dominant kernel's
algorithmic bytes / its CUDA-event time on the library stream, from a second
timed pass over the same iterations whose graph holds an event pair around
every kernel (`kernel_timing`).
Other entries: ROI-row mode, 16-bit storage (both index widths),
convergence of the violations, the block-iterative sweep, volume statistics,
continuous-batching serving against sequential FP32, and batching.

The CPU leg runs last, on rank 0 alone: it times the FP64 oracle on the host
cores (one core and all cores) on a bounded sample of the same plan, and
evaluates the GPU results against it (16-bit storage errors, short
trajectories, the accuracy of every served plan).  `--impl reference` times
that oracle as the reference arm.  With --gpus N each rank runs an
independent replica (the path has no exchange step): value = all ranks'
iterations / max rank time.
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
FWD_TRAFFIC_PER_NNZ = {("fp32", 4): 12.48, ("fp32", 2): 10.17, ("bf16", 2): 6.18, ("fp16", 2): 6.18}
# the same for the transposed product (average of its gradient and projection
# launches), keyed by (storage, row index bytes)
BWD_TRAFFIC_PER_NNZ = {("fp32", 2): 8.28, ("bf16", 2): 5.23, ("fp16", 2): 5.23}


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


def pass_bytes_int32(nnz, rows, n_spots, vb):
    """Bytes of one pass under 32-bit index accounting: the index and both
    value streams per nonzero (4 + 2 vb), per row with nonzeros a 4-byte
    pointer, the 8-byte (Dx, Lx) pair (+ 8 bytes of row scales for 16-bit
    storage), and the 4-byte spot vector."""
    return nnz * (4 + 2 * vb) + rows * (12 + (8 if vb == 2 else 0)) + n_spots * 4


BYTES_MODEL = ("forward: nnz*(ib + 2*vb) + 28 B per row with nonzeros (+8 for 16-bit row scales); "
               "transposed: nnz*(rb + vb) [gradient, L only] or nnz*(rb + 2*vb) [projection] + 4 B per 128 "
               "nonzeros of block headers (rb = 2) + 8 B coefficient pair per row + 12 B per chunk; "
               "ib, rb = 2 (16-bit column indices, based 16-bit row offsets) or 4, vb = 4 (FP32) or 2; "
               "int32 accounting: nnz*(4 + 2*vb) + 12 B per row (+8 scales) + 4 B per spot for every pass")


def workload_config(n_vox, n_spots, nnz, fmt, ws):
    """The `config` of both arms (identical for the same plan and storage)."""
    return {"workload": WORKLOAD, "rows": "all voxel rows streamed every pass", "n_vox": int(n_vox),
            "n_spots": int(n_spots), "nnz_per_matrix": int(nnz), "storage": fmt,
            "l2": "inputs larger than L2 (each pass streams at least %.1f GB)" % (nnz * 4 / 1e9),
            "parallelism": f"replicas{ws}"}


SMALL = dict(shape=(100, 100, 75), h=4.0)  # same phantom at half resolution (profiling case)
SHORT_ITERS = 3  # iterations of the short runs compared with the oracle's trajectory


def make_plan(seed, small=False):
    import phantom
    return phantom.clinical_plan(seed=seed, **(SMALL if small else {}))


def run_gpu_arm(args):
    import torch
    from paper_2509_20012_gb300 import Handle

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

    def timed_run(rows, fmt="fp32", index32=False, steps=None):
        steps = args.steps if steps is None else steps
        h = Handle(local, stream=stream)
        t0 = time.perf_counter()
        h.load_plan(plan, fmt=fmt, rows=rows, index32=index32)
        t_load = time.perf_counter() - t0
        sz = h.sizes()
        ib, rb, _ = h.storage()
        def region(timed, clock=False):
            # W warm-up iterations from w0, then the K timed ones between CUDA events on the library
            # stream; each iteration is one replay of the handle's CUDA graph (the library's path)
            h.set_timing(timed)
            h.begin(plan.w0, plan.alpha, plan.relaxation)
            h.iterate(args.warmup)
            torch.cuda.synchronize()
            h.set_timing(timed)  # reset the counters: only the timed region below counts
            if ws > 1:
                import torch.distributed as dist
                dist.barrier()
            torch.cuda.synchronize()
            sampler = ClockSampler(local) if clock else None
            if sampler:
                sampler.start()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.iterate(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            clocks = sampler.stop() if sampler else None
            return reduce_max(e0.elapsed_time(e1), device=f"cuda:{local}"), clocks

        # (a) the step time: plain graph replays, as a user's solve runs them
        ms, clocks = region(False, clock=True)
        launches = h.launch_count()
        w, dose, letd, rep = h.end()
        # (b) the kernel durations: the same iterations from w0 again, the graph holding an
        # event-record node before and after every kernel (each pair costs ~3 us of pipeline
        # drain, so (a) runs without them)
        ms_ev, _ = region(True)
        kt = h.get_timing()
        w_ev, *_ = h.end()
        h.close()
        same = bool(np.array_equal(w, w_ev))
        vb = 4 if fmt == "fp32" else 2
        nf = kt["forward"][1]
        nb = kt["backward"][1]
        hot = np.ones(plan.n_vox, bool) if rows == "all" else plan.mask != 0
        rows_nz = int(np.count_nonzero(hot & (np.diff(plan.row_ptr) > 0)))
        fb = fwd_bytes(sz["nnz_rows"], rows_nz, vb, ib, steps, steps)
        # chunk count is internal; it is small next to nnz (bounded by nnz/256 + n_spots)
        n_chunks_est = sz["nnz_rows"] // 2048 + sz["n_spots"]
        bb = bwd_bytes(sz["nnz_rows"], rows_nz, n_chunks_est, vb, rb, steps, steps)
        b32 = 2 * steps * pass_bytes_int32(sz["nnz_rows"], rows_nz, sz["n_spots"], vb)
        f_ms, b_ms = kt["forward"][0], kt["backward"][0]
        fw = {"bound": "hbm", "achieved": fb / (f_ms * 1e-3) / 1e9 if f_ms else None, "peak": hbm,
              "unit": "GB/s", "kernel": "k_forward (fused Dx/Lx)", "index_bytes": ib, "launches": nf,
              "ms_total": f_ms, "bytes_per_launch": fb / max(1, 2 * steps),
              "achieved_int32_accounting": b32 / (f_ms * 1e-3) / 1e9 if f_ms else None}
        bw = {"bound": "hbm", "achieved": bb / (b_ms * 1e-3) / 1e9 if b_ms else None, "peak": hbm,
              "unit": "GB/s", "kernel": "k_backward (CSC chunks)", "row_index_bytes": rb, "launches": nb,
              "ms_total": b_ms, "bytes_per_launch": bb / max(1, 2 * steps),
              "achieved_int32_accounting": b32 / (b_ms * 1e-3) / 1e9 if b_ms else None}
        for r in (fw, bw):
            r["frac"] = r["achieved"] / hbm if r["achieved"] else None
            r["frac_int32_accounting"] = (r["achieved_int32_accounting"] / hbm
                                          if r["achieved_int32_accounting"] else None)
        t = FWD_TRAFFIC_PER_NNZ.get((fmt, ib))
        fw["traffic"] = t * sz["nnz_rows"] if t else None
        t = BWD_TRAFFIC_PER_NNZ.get((fmt, rb))
        bw["traffic"] = t * sz["nnz_rows"] if t else None
        return dict(ms=ms, ms_ev=ms_ev, same=same, kt=kt, launches=launches, clocks=clocks, rep=rep, sizes=sz,
                    t_load=t_load, fwd=fw, bwd=bw, w=w, dose=dose, letd=letd, fmt=fmt, index_bytes=ib)

    main = timed_run("all", args.fmt)
    roi = timed_run("roi", args.fmt) if args.roi else None
    prec = {}
    if args.precision:
        for fmt in ("bf16", "fp16"):
            for index32 in (False, True):
                prec[f"{fmt}_idx{32 if index32 else 16}"] = timed_run("all", fmt, index32)

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

    convergence = None
    if rank == 0 and args.convergence:
        convergence = convergence_benchmark(plan, local, stream)

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

    # short runs of each storage from w0, compared with the oracle's first
    # iterations in the CPU leg
    short = {}
    if rank == 0 and ws == 1 and args.cpu_iters > 0:
        for fmt in ("fp32", "bf16", "fp16"):
            with Handle(local, stream=stream) as h:
                h.load_plan(plan, fmt=fmt)
                w, d, l, rep = h.superiorize(plan.w0, SHORT_ITERS, plan.alpha, plan.relaxation)
                short[fmt] = (w, h.get_log())

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_iters > 0:
        cpu = cpu_leg(args, plan, main, prec, short, serving)

    if rank == 0:
        dom = main["fwd"] if (main["fwd"]["ms_total"] or 0) >= (main["bwd"]["ms_total"] or 0) else main["bwd"]
        value = whole_job_value(args.steps, main["ms"], ws)
        sz = main["sizes"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sz["n_vox"], sz["n_spots"], sz["nnz"], args.fmt, ws),
            "timing_s": {"generate": round(t_gen, 2), "load": round(main["t_load"], 3)},
            "roofline": {k: dom[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")} | {
                "frac_int32_accounting": dom["frac_int32_accounting"], "bytes_model": BYTES_MODEL,
                "kernel": dom["kernel"], "peak_source": hbm_src,
                "forward": main["fwd"], "backward": main["bwd"]},
            "cpu_baseline": cpu["cpu_baseline"] if cpu else None,
            "e2e": e2e,
            "gpu_launches": main["launches"],
            "clocks": main["clocks"],
            "kernel_ms": {k: v[0] for k, v in main["kt"].items()},
            "kernel_timing": {
                "what": ("value and ms_per_step: K plain graph replays; kernel_ms and roofline: the same K "
                         "iterations from w0 again with an event-record node before and after every kernel "
                         "of the graph (CUDA events on the library stream)"),
                "ms_per_step_with_kernel_events": main["ms_ev"] / args.steps,
                "results_identical": main["same"]},
            "final": {"objective": main["rep"]["objective"], "n_violated": main["rep"]["n_violated"],
                      "max_violation": main["rep"]["max_violation"]},
        }
        if convergence is not None:
            line["convergence"] = convergence
        if volume is not None:
            line["volume_stats"] = volume
        if sweep is not None:
            line["sweep"] = sweep
        if serving is not None:
            line["serving"] = serving["summary"]
            if cpu and cpu.get("serving_accuracy"):
                line["serving"]["accuracy"] = cpu["serving_accuracy"]
        if batching is not None:
            line["batching"] = batching
        if prec:
            entries = {}
            for key, r in prec.items():
                e = {"value": whole_job_value(args.steps, r["ms"], ws), "ms_per_step": r["ms"] / args.steps,
                     "ms_per_step_with_kernel_events": r["ms_ev"] / args.steps,
                     "index_bytes": r["index_bytes"], "forward": r["fwd"], "backward": r["bwd"]}
                if cpu and key in cpu.get("precision_vs_oracle", {}):
                    e.update(cpu["precision_vs_oracle"][key])
                entries[key] = e
            line["precision"] = {
                "note": ("D and L stored in 16 bits with power-of-two FP32 row scales; 16-bit (idx16) or int32 "
                         "(idx32) indices, the two giving bit-identical results; FP32 accumulation; FP64 "
                         "projection divides and scalar reductions; row moments and the final dose/LETd pass in "
                         "double-float (pairs of FP32, about 48 bits). Errors: each run's outputs and solution "
                         "against the FP64 oracle's products of the FP32 inputs (CPU leg)"),
                **entries}
            if cpu and cpu.get("short_trajectories"):
                line["precision"]["short_trajectories"] = cpu["short_trajectories"]
        if roi is not None:
            line["roi_rows"] = {"value": whole_job_value(args.steps, roi["ms"], ws),
                                "ms_per_step": roi["ms"] / args.steps,
                                "ms_per_step_with_kernel_events": roi["ms_ev"] / args.steps,
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


def serving_trace(lib, n_req, rate, seed, fmt16="fp16"):
    """Poisson arrivals (mean `rate`/s); sizes log-uniform between the smallest
    and the largest plan (nearest plan of the library); FP32/16-bit storage
    50:50; 100-500 iterations."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    lognnz = np.log([p.nnz for p in lib])
    target = rng.uniform(lognnz.min(), lognnz.max(), n_req)
    idx = [int(np.argmin(np.abs(lognnz - x))) for x in target]
    fmt = [fmt16 if u < 0.5 else "fp32" for u in rng.uniform(size=n_req)]
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
    """Continuous batching of a traced request stream, mixed FP32/16-bit
    storage, against the same requests served one at a time in FP32, traced
    (arrivals kept) and saturated (all submitted at once).  Returns the
    summary and the per-request results (the CPU leg checks the accuracy of
    every served plan against the FP32 result of the same request)."""
    from paper_2509_20012_gb300 import Server
    lib = serving_library(clinical)
    trace = serving_trace(lib, args.serve_requests, args.serve_rate, args.seed + 1000, args.serve_fmt)
    with Server(local, mem_cap_bytes=180e9, max_active=8, round_iters=10) as srv:
        served = run_trace(srv, lib, trace)
    with Server(local, mem_cap_bytes=180e9, max_active=1, round_iters=10) as srv:
        seq = run_trace(srv, lib, trace, force_fp32=True)
    # capacity: the same requests all submitted at once (saturated queue)
    with Server(local, mem_cap_bytes=180e9, max_active=8, round_iters=10) as srv:
        cap_served = serving_summary(run_trace(srv, lib, trace, at_once=True), len(trace))
    with Server(local, mem_cap_bytes=180e9, max_active=1, round_iters=10) as srv:
        cap_seq = serving_summary(run_trace(srv, lib, trace, force_fp32=True, at_once=True), len(trace))
    sizes = [lib[r["plan"]].nnz for r in trace]
    summary = {
        "trace": (f"{args.serve_requests} requests, Poisson arrivals mean {args.serve_rate}/s, nnz per matrix "
                  f"log-uniform {min(p.nnz for p in lib):.2e}-{max(p.nnz for p in lib):.2e} "
                  f"(tiny plan + clinical phantom at {SERVE_RES_MM} mm), FP32/{args.serve_fmt.upper()} 50:50, "
                  f"100-500 iterations, admission cap 180 GB"),
        "requests_nnz_mean": float(np.mean(sizes)),
        "served": serving_summary(served, len(trace)) | {
            "mode": f"continuous batching, mixed FP32/{args.serve_fmt.upper()}, up to 8 plans resident"},
        "sequential_fp32": serving_summary(seq, len(trace)) | {"mode": "one plan at a time, FP32"},
        "capacity": {"served": cap_served, "sequential_fp32": cap_seq,
                     "how": "the same requests submitted at once (saturated queue)"},
        "capacity_plans_per_hour": {"served": cap_served["plans_per_hour"],
                                    "sequential_fp32": cap_seq["plans_per_hour"],
                                    "ratio": cap_served["plans_per_hour"] / cap_seq["plans_per_hour"]},
    }
    return {"summary": summary, "lib": lib, "trace": trace,
            "served_w": [r[1] for r in served], "served_dose": [r[2] for r in served],
            "served_letd": [r[3] for r in served], "seq_w": [r[1] for r in seq]}


def batching_benchmark(args, local):
    """Batching workloads: (a) 16 independent plans, PTV 20-400 cc, nnz 6e5-7e7,
    BF16, tiles autotuned per plan, run one after another (whole-GPU launch
    shapes) vs as one batch graph per iteration and as graphs of 10
    iterations (plans loaded with FREDOPT_SHARED launch shapes); (b) 27
    robustness scenarios stacked into one robust plan (one w meets the
    constraints in every scenario), BF16."""
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
    # the same solves alone with the batch's launch shapes: the batch must match them bit for bit
    shared_w = []
    for p in plans:
        with Handle(local) as h:
            h.load_plan(p, fmt="bf16", shared=True)
            w, *_ = h.superiorize(p.w0, iters, p.alpha, p.relaxation)
            shared_w.append(w)
    shapes_rel = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)) for a, b in zip(shared_w, seq_w))
    # all plans as one graph per iteration, then as graphs of 10 iterations
    batched = {}
    same = True
    for depth in (1, 10):
        hs = []
        for p, tile in zip(plans, tiles):
            h = Handle(local)
            h.load_plan(p, fmt="bf16", shared=True)
            h.autotune(reps=3)
            h.begin(p.w0, p.alpha, p.relaxation, use_graphs=0)
            hs.append(h)
        with Batch(hs, depth=depth) as b:
            b.iterate(depth if depth > 1 else 3)   # warm-up; the timed iterations continue the same solves
            t0 = b.sync()
            b.iterate(iters - (depth if depth > 1 else 3))
            bat_ms = b.sync() - t0
        for h, w_ref in zip(hs, shared_w):
            w, *_ = h.end()
            same = same and bool(np.array_equal(w, w_ref))
            h.close()
        batched[depth] = (iters - (depth if depth > 1 else 3)) * len(plans) / (bat_ms * 1e-3)
    total_iters = iters * len(plans)
    out = {"independent": {
        "plans": len(plans), "nnz_per_matrix": [int(p.nnz) for p in plans], "storage": "bf16",
        "iterations_per_plan": iters, "tiles_row_chunk_weight": tiles,
        "sequential_plan_iters_per_s": total_iters / (seq_ms * 1e-3),
        "batched_plan_iters_per_s": batched[1],
        "batched_10_iteration_graph_plan_iters_per_s": batched[10],
        "batch_graph_results_identical_to_alone": same,
        "launch_shapes": "one after another: whole GPU per plan; batched: FREDOPT_SHARED (about one SM per 2e5 "
                         "nonzeros); the batch matches each plan alone with the same shapes bit for bit",
        "max_rel_l2_w_shared_vs_whole_gpu_shapes": shapes_rel}}
    out["independent"]["batched_speedup"] = (out["independent"]["batched_plan_iters_per_s"]
                                             / out["independent"]["sequential_plan_iters_per_s"])
    out["independent"]["batched_10_speedup"] = (batched[10] / out["independent"]["sequential_plan_iters_per_s"])
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


def convergence_benchmark(plan, local, stream, iters=500, marks=(1, 10, 50, 100, 200, 300, 400, 500)):
    """Violated rows and the largest row violation after k superiorized
    iterations (the per-iteration log), for the Cimmino weights over all
    reachable rows (norm 'all') and over the rows violated at each point
    (norm 'violated'), streaming every row or only the structure rows."""
    from paper_2509_20012_gb300 import Handle
    out = {}
    for rows in ("all", "roi"):
        for norm in ("all", "violated"):
            with Handle(local, stream=stream) as h:
                h.load_plan(plan, rows=rows)
                h.begin(plan.w0, plan.alpha, plan.relaxation, cimmino_norm=norm)
                h.iterate(iters)
                log = h.get_log()
                w, d, l, rep = h.end()
            by_k = {e["k"] + 1: e for e in log}
            out[f"{rows}_rows_norm_{norm}"] = {
                "n_violated": {k: int(by_k[k]["n_violated"]) for k in marks if k in by_k},
                "max_violation": {k: float(by_k[k]["max_violation"]) for k in marks if k in by_k},
                "final_n_violated": int(rep["n_violated"]), "final_max_violation_by_constraint": rep["max_violation"],
                "final_objective": rep["objective"]}
    out["note"] = ("clinical plan, %d iterations from w0 = 1; n_violated and max_violation are the log entries of "
                   "iteration k (rows violated at the point the feasibility step starts from; violations in the "
                   "bound's unit, Gy or keV/um); final_* from the final pass at the returned w" % iters)
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


def cpu_info():
    """Host cores and CPU model of this machine."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def oracle_problem(plan):
    """The FP64 oracle's problem and constraint rows of a plan."""
    import oracle
    P = oracle.build_problem(plan.row_ptr, plan.col, plan.D, plan.L, plan.n_spots, plan.mask,
                             plan.constraints, plan.objective)
    return P, oracle.constraint_rows(P)


def output_errors(P, w, dose, letd, presc, ref=None):
    """Largest and mean |dose - oracle dose| / presc and |LETd - oracle LETd|
    (keV/um, voxels above 1% of the prescription) of outputs at fluence w."""
    import oracle
    d_o, l_o = oracle.forward(P, np.asarray(w, np.float64)) if ref is None else ref
    let_o = oracle.letd(d_o, l_o)
    sel = d_o > 0.01 * presc
    ed = np.abs(np.asarray(dose, np.float64) - d_o) / presc
    el = np.abs(np.asarray(letd, np.float64) - let_o)[sel]
    return {"dose_max_frac_of_presc": float(ed.max()), "dose_mean_frac_of_presc": float(ed.mean()),
            "letd_max_keV_um": float(el.max()) if el.size else 0.0,
            "letd_mean_keV_um": float(el.mean()) if el.size else 0.0}


def cpu_leg(args, plan, main, prec, short, serving):
    """The CPU leg (rank 0, after every GPU measurement): the FP64 oracle on
    the host cores, as it stands, timed on one core and on all cores (its
    sparse products split over row shards, oracle/parallel.py) over a bounded
    sample of the clinical plan (its first iterations), and the checks of the
    GPU results against it."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    from oracle import parallel
    info = cpu_info()
    n = max(1, int(info["nproc"] or 1))
    presc = plan.prescription
    t = time.perf_counter()
    P, R = oracle_problem(plan)
    t_build = time.perf_counter() - t
    pool = ThreadPoolExecutor(n)
    Pt, Rt = parallel.threaded(P, n, pool), parallel.threaded_rows(R, n, pool)
    t = time.perf_counter()
    w_or, log_or = oracle.superiorize(Pt, plan.w0, SHORT_ITERS, plan.alpha, plan.relaxation, rows=Rt)
    dt_all = time.perf_counter() - t
    t = time.perf_counter()
    oracle.superiorize(P, plan.w0, args.cpu_iters, plan.alpha, plan.relaxation, rows=R)
    dt_one = time.perf_counter() - t
    cpu = {"value": SHORT_ITERS / dt_all, "unit": UNIT, "cores": n, "kind": "oracle",
           "sample": (f"the first {SHORT_ITERS} superiorized iterations of the clinical plan from w0 on all {n} "
                      f"host cores ({dt_all:.1f} s; FP64 numpy/scipy, sparse products over {n} row shards on "
                      f"threads); problem setup ({t_build:.1f} s) excluded"),
           "single_core": {"value": args.cpu_iters / dt_one, "unit": UNIT, "cores": 1,
                           "sample": f"the first {args.cpu_iters} iterations on one core, {dt_one:.1f} s"},
           **info}
    out = {"cpu_baseline": cpu}

    # 16-bit storage against the oracle: the outputs of each run at its final
    # w, and the solution (the FP64 dose and LETd of its w) against the FP32 run's
    ref32 = oracle.forward(Pt, main["w"].astype(np.float64))
    let32 = oracle.letd(*ref32)
    sel32 = ref32[0] > 0.01 * presc
    pv = {}
    for key, r in list(prec.items()) + [("fp32", main)]:
        ref = oracle.forward(Pt, r["w"].astype(np.float64))
        let = oracle.letd(*ref)
        e = {"outputs_vs_oracle": output_errors(Pt, r["w"], r["dose"], r["letd"], presc, ref)}
        e["solution_vs_fp32_run"] = {
            "dose_max_frac_of_presc": float(np.max(np.abs(ref[0] - ref32[0])) / presc),
            "letd_max_keV_um": float(np.max(np.abs(let - let32)[sel32])),
            "w_rel_l2": float(np.linalg.norm(r["w"].astype(np.float64) - main["w"]) / np.linalg.norm(main["w"]))}
        pv[key] = e
    out["precision_vs_oracle"] = pv

    # the first iterations of each storage against the oracle's
    traj = {}
    for fmt, (w, log) in short.items():
        ref = oracle.forward(Pt, w.astype(np.float64))
        ref_or = oracle.forward(Pt, w_or)
        traj[fmt] = {"iterations": SHORT_ITERS,
                     "w_rel_l2_vs_oracle": float(np.linalg.norm(w - w_or) / np.linalg.norm(w_or)),
                     "trial_counters_equal": [e["s"] for e in log] == [e["s"] for e in log_or],
                     "dose_max_frac_of_presc": float(np.max(np.abs(ref[0] - ref_or[0])) / presc)}
    out["short_trajectories"] = traj

    if serving is not None:
        out["serving_accuracy"] = serving_accuracy(serving, plan, Pt, n, pool)
    pool.shutdown()
    return out


# accuracy bar of a served plan: its solution's FP64 dose within 1e-4 of the
# prescription and its LETd within 2e-3 keV/um of the FP32 result of the same
# request (the parity tolerances)
SERVE_DOSE_TOL = 1e-4
SERVE_LETD_TOL = 2e-3


def serving_accuracy(serving, clinical, P_clinical, n, pool):
    """Every served plan against the FP32 result of the same request: the FP64
    dose and LETd of both solutions (oracle products of the FP32 inputs), and
    the error of the served outputs themselves."""
    import oracle
    from oracle import parallel
    lib, trace = serving["lib"], serving["trace"]
    worst = {}
    per = []
    for pi, p in enumerate(lib):
        reqs = [i for i, r in enumerate(trace) if r["plan"] == pi]
        if not reqs:
            continue
        P = P_clinical if p is clinical else parallel.threaded(oracle.build_problem(
            p.row_ptr, p.col, p.D, p.L, p.n_spots, p.mask, p.constraints, p.objective), n, pool)
        for i in reqs:
            fmt = trace[i]["fmt"]
            d_s, l_s = oracle.forward(P, serving["served_w"][i].astype(np.float64))
            d_q, l_q = oracle.forward(P, serving["seq_w"][i].astype(np.float64))
            sel = d_q > 0.01 * p.prescription
            dd = float(np.max(np.abs(d_s - d_q)) / p.prescription)
            dl = float(np.max(np.abs(oracle.letd(d_s, l_s) - oracle.letd(d_q, l_q))[sel])) if sel.any() else 0.0
            ev = output_errors(P, serving["served_w"][i], serving["served_dose"][i], serving["served_letd"][i],
                               p.prescription, (d_s, l_s))
            per.append({"request": i, "nnz": int(p.nnz), "fmt": fmt, "iters": trace[i]["iters"],
                        "solution_dose_max_frac_of_presc": dd, "solution_letd_max_keV_um": dl,
                        "outputs_dose_max_frac_of_presc": ev["dose_max_frac_of_presc"],
                        "outputs_letd_max_keV_um": ev["letd_max_keV_um"]})
            w = worst.setdefault(fmt, {"solution_dose_max_frac_of_presc": 0.0, "solution_letd_max_keV_um": 0.0,
                                       "outputs_dose_max_frac_of_presc": 0.0, "outputs_letd_max_keV_um": 0.0})
            for k in w:
                w[k] = max(w[k], per[-1][k])
        del P
    ok = all(r["solution_dose_max_frac_of_presc"] <= SERVE_DOSE_TOL and r["solution_letd_max_keV_um"] <= SERVE_LETD_TOL
             for r in per)
    return {"accuracy_ok": ok,
            "bar": (f"each served plan's solution (FP64 oracle products of the FP32 inputs at its w) within "
                    f"{SERVE_DOSE_TOL:g} of the prescription in dose and {SERVE_LETD_TOL:g} keV/um in LETd "
                    f"(voxels above 1% of the prescription) of the FP32 sequential result of the same request"),
            "worst_by_format": worst, "requests": per}


def row_sample(plan, m):
    """The plan restricted to every m-th voxel row (same spots, structures,
    constraints and objective): a bounded sample of its work."""
    import dataclasses
    rows = np.arange(0, plan.n_vox, m)
    lens = np.diff(plan.row_ptr)[rows]
    rp = np.zeros(len(rows) + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    take = np.concatenate([np.arange(plan.row_ptr[r], plan.row_ptr[r + 1]) for r in rows]) if rp[-1] else \
        np.zeros(0, np.int64)
    return dataclasses.replace(plan, shape=(len(rows), 1, 1), row_ptr=rp, col=plan.col[take], D=plan.D[take],
                               L=plan.L[take], mask=plan.mask[rows])


def run_reference_arm(args):
    """The reference arm: the FP64 oracle, as it stands, on all host cores
    (sparse products over row shards), on the same workload, metric and
    config as the GPU arm.  W warm-up steps, then K timed steps, each one
    superiorized iteration continuing the solve.  When K + W full-size
    iterations would not finish within about four minutes, the steps after
    the first two run on a row sample of the plan (every m-th voxel row) and the
    rate is scaled to the full plan by the nonzeros."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    from oracle import parallel
    info = cpu_info()
    n = max(1, int(info["nproc"] or 1))
    pool = ThreadPoolExecutor(n)
    plan = make_plan(seed=args.seed, small=args.small)
    full = (plan.n_vox, plan.n_spots, plan.nnz)
    budget_s = 240.0

    def prepare(pl):
        P, R = oracle_problem(pl)
        return parallel.threaded(P, n, pool), parallel.threaded_rows(R, n, pool)

    P, R = prepare(plan)
    beta0 = 0.1 * float(np.linalg.norm(plan.w0.astype(np.float64)))
    state = {"w": plan.w0.astype(np.float64), "s": 0, "k": 0}

    def step(P, R, pl):
        w, log = oracle.superiorize(P, state["w"], 1, pl.alpha, pl.relaxation, rows=R, beta0=beta0,
                                    s0=state["s"], k0=state["k"])
        state.update(w=w, s=log[-1]["s"], k=state["k"] + 1)

    t1 = 0.0
    for _ in range(2):                  # the first two warm-up steps, full size
        t = time.perf_counter()
        step(P, R, plan)
        t1 = max(t1, time.perf_counter() - t)
    scale, sample = 1.0, "the full clinical plan"
    est = (args.steps + args.warmup - 2) * t1
    if est > budget_s:
        m = int(np.ceil(est / budget_s))
        sub = row_sample(plan, m)
        scale = sub.nnz / plan.nnz
        P, R = prepare(sub)
        state.update(w=sub.w0.astype(np.float64), s=0, k=0)
        plan = sub
        sample = f"a row sample of the clinical plan: every {m}-th voxel row ({sub.nnz:.3e} of {full[2]:.3e} nonzeros)"
    for _ in range(args.warmup - 2):
        step(P, R, plan)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(P, R, plan)
    dt = time.perf_counter() - t0
    pool.shutdown()
    v = args.steps / dt * scale
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(*full, "fp32", ws),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": n, "kind": "oracle",
                             "sample": (f"{args.steps} timed superiorized iterations after {args.warmup} warm-up "
                                        f"on {sample}, FP64 oracle with sparse products over {n} row shards on "
                                        f"threads; the slower of the first two warm-up iterations took {t1:.2f} s at full size"),
                             **info},
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
    ap.add_argument("--cpu-iters", type=int, default=2,
                    help="iterations of the one-core oracle timing in the CPU leg (0 skips the CPU leg)")
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the serving trace (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=2.0, help="mean arrivals per second")
    ap.add_argument("--serve-fmt", default="fp16", choices=["bf16", "fp16"],
                    help="16-bit storage of half of the served requests")
    ap.add_argument("--no-convergence", dest="convergence", action="store_false",
                    help="skip the convergence runs (violations against the iteration count)")
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
    if args.impl == "reference":
        run_reference_arm(args)
    else:
        run_gpu_arm(args)


if __name__ == "__main__":
    main()
