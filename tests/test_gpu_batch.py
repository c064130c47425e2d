"""Batches of plans (CUDA graphs of one or several iterations of all plans)
and tile autotuning: results are bit-identical to running each plan alone
with the default tiles."""
import numpy as np
import pytest

import phantom
from test_gpu_serving import small_plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt


def alone(lib, plan, fmt, iters, shared=False):
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt, shared=shared)
        return h.superiorize(plan.w0, iters, 0.99, 1.0)


def test_autotune_changes_speed_not_results(lib):
    pl = phantom.tiny_plan()
    ref = alone(lib, pl, "fp32", 20)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        rc, cc = h.autotune(reps=2)
        assert rc in (16, 32, 64, 128, 256, 512) and cc in (4, 16, 64, 256, 1024)
        assert h.tuning() == (rc, cc)
        w, dose, letd, rep = h.superiorize(pl.w0, 20, 0.99, 1.0)
    np.testing.assert_array_equal(w, ref[0])
    np.testing.assert_array_equal(dose, ref[1])
    # tuning after begin (mid-solve) does not change the trajectory either
    with lib.Handle(0) as h:
        h.load_plan(pl)
        h.begin(pl.w0, 0.99, 1.0)
        h.iterate(7)
        h.autotune(reps=1)
        h.iterate(13)
        w2, *_ = h.end()
    np.testing.assert_array_equal(w2, ref[0])


@pytest.mark.parametrize("shared", [False, True])
def test_batch_matches_each_plan_alone(lib, shared):
    """With whole-GPU launch shapes and with FREDOPT_SHARED ones (small plans
    on few SMs' worth of CTAs), compared with each plan alone loaded the same
    way."""
    specs = [(phantom.tiny_plan(), "fp32"), (small_plan(3000, 257, 0.2, 31, 0), "bf16"),
             (small_plan(20000, 1500, 0.05, 32, 0), "fp32"), (phantom.tiny_plan(seed=5), "fp16")]
    iters = 17
    refs = [alone(lib, p, f, iters, shared) for p, f in specs]
    hs = []
    for p, f in specs:
        h = lib.Handle(0)
        h.load_plan(p, fmt=f, shared=shared)
        hs.append(h)
    outs = lib.superiorize_batch(hs, [p.w0 for p, _ in specs], iters, 0.99, 1.0, use_graphs=0)
    for (w, d, l, rep), (wr, dr, lr, rr) in zip(outs, refs):
        np.testing.assert_array_equal(w, wr)
        np.testing.assert_array_equal(d, dr)
        assert rep["iters"] == iters
    # the explicit form, continued in two pieces, then finished per plan;
    # graphs of one iteration and of 4 iterations of every plan
    for depth in (1, 4):
        for h, (p, f) in zip(hs, specs):
            h.begin(p.w0, 0.99, 1.0, use_graphs=0)
        with lib.Batch(hs, depth=depth) as b:
            b.iterate(10)
            b.iterate(iters - 10)
            ms = b.sync()
        assert ms > 0
        for h, (wr, dr, lr, rr) in zip(hs, refs):
            w, d, l, rep = h.end()
            np.testing.assert_array_equal(w, wr)
            assert rep["iters"] == iters
    for h in hs:
        h.close()
