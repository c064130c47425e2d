"""Oracle parity of the widened forms: the stacked robust plan, batches of
plans in mixed storage formats, requests served by the continuous-batching
server, and 16-bit trajectories.

Each GPU result is compared with the FP64 oracle (`oracle.superiorize`) run
on the matrix the GPU actually multiplies: the FP32 inputs for FP32 storage,
and for BF16/FP16 storage the dequantised matrix (stored 16-bit value x its
power-of-two row scale, exact in binary32) rebuilt from the handle's CSC
copy.  The bar is the one of the single-plan parity tests: identical trial
counters and accept/reject decisions, w within 1e-4 relative L2, dose within
1e-4 x prescription and per-constraint violations within 1e-4 x prescription
(dose) or 2e-3 keV/um (LETd).
"""
import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu

PRESC = 2.0
ITERS = 20


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt


@pytest.fixture(scope="module")
def robust():
    plan, per = phantom.small_robust_plan()
    return plan


def stored_matrix(lib, plan, fmt):
    """(row_ptr, col, D, L) in voxel order of the values the library stores
    for `plan` in format `fmt`, read back through fredopt_get_csc (device rows
    mapped to voxels through fredopt_get_rows); one shared pattern."""
    if fmt == "fp32":
        return plan.row_ptr, plan.col, plan.D, plan.L
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt)
        cp, row, DT, LT = h.get_csc()
        vox, _ = h.get_rows()
    spot = np.repeat(np.arange(plan.n_spots, dtype=np.int64), np.diff(cp))
    rows = vox[row]
    order = np.lexsort((spot, rows))
    rp = np.zeros(plan.n_vox + 1, np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=plan.n_vox))
    col = spot[order].astype(np.int32)
    # same pattern as the input plan (the quantisation keeps every element)
    np.testing.assert_array_equal(rp, plan.row_ptr)
    np.testing.assert_array_equal(col, plan.col)
    return rp, col, DT[order], LT[order]


def oracle_run(lib, plan, fmt, iters, **kw):
    rp, col, D, L = stored_matrix(lib, plan, fmt)
    P = oracle.build_problem(rp, col, D, L, plan.n_spots, plan.mask, plan.constraints, plan.objective)
    R = oracle.constraint_rows(P)
    w, log = oracle.superiorize(P, plan.w0, iters, plan.alpha, plan.relaxation, rows=R, **kw)
    return P, R, w, log


def violation_by_kind(plan, P, w):
    """Largest violation per constraint in its physical unit: Gy for dose,
    keV/um for LETd (LETd = Lw/Dw, Eq. 1)."""
    dose, lw = oracle.forward(P, w)
    let = oracle.letd(dose, lw)
    out = {}
    for ci, c in enumerate(plan.constraints):
        sel = ((plan.mask >> np.uint32(c["struct_bit"])) & 1).astype(bool)
        if c["kind"] == "DOSE_MIN":
            v = c["bound"] - dose[sel]
        elif c["kind"] == "DOSE_MAX":
            v = dose[sel] - c["bound"]
        elif c["kind"] == "LETD_MAX":
            sel = sel & (dose > 0)
            v = let[sel] - c["bound"]
        else:
            continue
        out[ci] = float(max(v.max(), 0.0)) if v.size else 0.0
    return out


def assert_matches_oracle(plan, P, w_ref, log_ref, w, dose, log=None, report=None):
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    assert rel <= 1e-4, rel
    if log is not None:
        assert [e["s"] for e in log] == [e["s"] for e in log_ref]
        assert [e["accepted"] for e in log] == [e["accepted"] for e in log_ref]
    if report is not None:
        assert report["s"] == log_ref[-1]["s"]
        assert report["accepted"] == sum(e["accepted"] for e in log_ref)
    d_ref, _ = oracle.forward(P, w_ref)
    assert np.max(np.abs(dose - d_ref)) <= 1e-4 * PRESC
    vg = violation_by_kind(plan, P, w.astype(np.float64))
    vr = violation_by_kind(plan, P, w_ref)
    for ci in vr:
        tol = 1e-4 * PRESC if plan.constraints[ci]["kind"].startswith("DOSE") else 2e-3
        assert abs(vg[ci] - vr[ci]) <= tol, (ci, vg[ci], vr[ci])


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_robust_stacked_plan_vs_oracle(lib, robust, fmt):
    """27 robustness scenarios (x/y setup shifts x range factors, Sec. 2.5)
    stacked into one plan: one w meets every scenario's constraints."""
    plan = robust
    P, R, w_ref, log_ref = oracle_run(lib, plan, fmt, ITERS)
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt)
        w, dose, letd, rep = h.superiorize(plan.w0, ITERS, plan.alpha, plan.relaxation)
        log = h.get_log()
    assert rep["n_rows"] == R.A.shape[0]
    assert rep["unreachable_rows"] == R.unreachable
    assert_matches_oracle(plan, P, w_ref, log_ref, w, dose, log)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_16bit_trajectory_vs_oracle(lib, fmt):
    """100 superiorized iterations of the tiny plan with 16-bit storage, with
    16-bit and with 32-bit indices, against the FP64 oracle on the stored
    values."""
    plan = phantom.tiny_plan()
    P, R, w_ref, log_ref = oracle_run(lib, plan, fmt, 100)
    for index32 in (False, True):
        with lib.Handle(0) as h:
            h.load_plan(plan, fmt=fmt, index32=index32)
            w, dose, letd, rep = h.superiorize(plan.w0, 100, plan.alpha, plan.relaxation)
            log = h.get_log()
        assert_matches_oracle(plan, P, w_ref, log_ref, w, dose, log)
        # the final pass reports the oracle's objective of the returned w
        assert rep["objective"] == pytest.approx(oracle.objective(P, w.astype(np.float64)), rel=1e-9)


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_shared_launch_shapes_trajectory_vs_oracle(lib, fmt):
    """FREDOPT_SHARED launch shapes (the tiny plan then runs on about five SMs'
    worth of CTAs, with other tiles and chunk partials): 100 iterations keep
    the oracle's trial counters and decisions, w, dose and violations."""
    plan = phantom.tiny_plan()
    P, R, w_ref, log_ref = oracle_run(lib, plan, fmt, 100)
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt, shared=True)
        w, dose, letd, rep = h.superiorize(plan.w0, 100, plan.alpha, plan.relaxation)
        log = h.get_log()
    assert_matches_oracle(plan, P, w_ref, log_ref, w, dose, log)


def _mixed_plans():
    from test_gpu_serving import small_plan
    return [(phantom.tiny_plan(), "fp32"), (phantom.tiny_plan(seed=3), "bf16"),
            (phantom.tiny_plan(seed=5), "fp16"), (small_plan(3000, 257, 0.2, 31, ITERS), "bf16")]


def test_batch_mixed_formats_vs_oracle(lib):
    """One batch graph per iteration over plans stored in FP32, BF16 and FP16."""
    specs = _mixed_plans()
    hs = []
    try:
        for p, f in specs:
            h = lib.Handle(0)
            h.load_plan(p, fmt=f)
            hs.append(h)
        outs = lib.superiorize_batch(hs, [p.w0 for p, _ in specs], ITERS, 0.99, 1.0)
        logs = [h.get_log() for h in hs]
    finally:
        for h in hs:
            h.close()
    for (p, f), (w, d, l, rep), log in zip(specs, outs, logs):
        p.alpha, p.relaxation = 0.99, 1.0
        P, R, w_ref, log_ref = oracle_run(lib, p, f, ITERS)
        assert_matches_oracle(p, P, w_ref, log_ref, w, d, log)


def test_served_requests_vs_oracle(lib):
    """Requests of each storage format served together by the
    continuous-batching server (their rounds interleave on the GPU)."""
    specs = _mixed_plans()
    with lib.Server(0, mem_cap_bytes=32e9, max_active=4, round_iters=7) as srv:
        tickets = [srv.submit(p, fmt=f, iters=ITERS) for p, f in specs]
        out = [srv.wait(t, timeout=300) for t in tickets]
    for (p, f), (info, w, dose, letd) in zip(specs, out):
        assert info["status"] == lib.DONE
        P, R, w_ref, log_ref = oracle_run(lib, p, f, ITERS)
        assert_matches_oracle(p, P, w_ref, log_ref, w, dose, report=info["report"])


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_16bit_sweep_vs_oracle(lib, fmt):
    """The block-iterative sweep (R13) with 16-bit storage: one sweep of 37
    blocks from the same x within 2e-5 relative L2 of the oracle's sweep on
    the stored values, and 15 superiorized iterations with a 16-block sweep
    as the feasibility operator matching the oracle's trial counters and w."""
    plan = phantom.tiny_plan()
    rp, col, D, L = stored_matrix(lib, plan, fmt)
    P = oracle.build_problem(rp, col, D, L, plan.n_spots, plan.mask, plan.constraints, plan.objective)
    R = oracle.constraint_rows(P)
    x = np.random.default_rng(37).uniform(0.2, 2.5, plan.n_spots).astype(np.float32)
    ref = oracle.block_iterative_sweep(R, x.astype(np.float64), 1.0, oracle.sweep_blocks(P, R, 37), prio_scale=0.8)
    w_ref, log_ref = oracle.superiorize(P, plan.w0, 15, plan.alpha, plan.relaxation, rows=R, sweep=16)
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt)
        sw = h.sweep_step(x, 37, relaxation=1.0, prio_scale=0.8)
        w, dose, letd, rep = h.superiorize(plan.w0, 15, plan.alpha, plan.relaxation, sweep_blocks=16)
        log = h.get_log()
    assert np.linalg.norm(sw - ref) / np.linalg.norm(ref) <= 2e-5
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref) <= 1e-4


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_16bit_quantity_maps_vs_oracle(lib, fmt):
    """Dose, cDL and LETd maps of 16-bit storage (the double-float final pass
    over the stored values, rounded once to FP32) within 1e-6 relative of the
    oracle's FP64 maps of the stored matrix."""
    plan = phantom.tiny_plan()
    rp, col, D, L = stored_matrix(lib, plan, fmt)
    P = oracle.build_problem(rp, col, D, L, plan.n_spots, plan.mask, plan.constraints, plan.objective)
    w = np.random.default_rng(12).uniform(0.0, 2.0, plan.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt)
        maps = {q: h.quantity_map(w, q) for q in ("DOSE", "CDL", "LETD")}
    for q, name in (("DOSE", "dose"), ("CDL", "cdl"), ("LETD", "letd")):
        ref = oracle.quantity(P, w, name)
        assert np.all(np.abs(maps[q] - ref) <= 1e-6 * np.abs(ref) + 1e-12), q
