"""Serving loop (continuous batching): each result is the same alone and in
the mix; admission respects the memory cap; a failing request does not
disturb the others."""
import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt


def small_plan(n_rows, n_cols, density, seed, iters):
    rp, col, D, L = phantom.random_csr(n_rows, n_cols, density, seed=seed, empty_rows=n_rows // 10)
    rng = np.random.default_rng(seed)
    mask = rng.integers(0, 4, n_rows).astype(np.uint32)
    cons = [dict(struct_bit=0, kind="DOSE_MIN", bound=2.0, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MAX", bound=3.0, priority=2.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=4.0, priority=0.5)]
    obj = [dict(struct_bit=1, quantity="CDL", target=0.0, weight=1.0)]
    return phantom.Plan(name=f"p{seed}", shape=(n_rows, 1, 1), h_mm=1.0, params=None, row_ptr=rp, col=col,
                        D=D, L=L, mask=mask, structures=[], constraints=cons, objective=obj,
                        w0=np.ones(n_cols, np.float32), iters=iters, alpha=0.95, relaxation=1.0)


def alone(lib, plan, fmt, shared=True):
    """The plan alone, loaded as a server with several plans in flight loads
    it (FREDOPT_SHARED launch shapes)."""
    with lib.Handle(0) as h:
        h.load_plan(plan, fmt=fmt, shared=shared)
        return h.superiorize(plan.w0, plan.iters, plan.alpha, plan.relaxation)


def test_results_same_alone_and_in_the_mix(lib):
    plans = [(phantom.tiny_plan(iters=40), "fp32"), (phantom.tiny_plan(seed=3, iters=25), "bf16"),
             (small_plan(3000, 257, 0.2, 1, 60), "fp32"), (small_plan(800, 33, 0.5, 2, 90), "fp16"),
             (small_plan(20000, 1500, 0.05, 4, 30), "bf16")]
    ref = [alone(lib, p, f) for p, f in plans]
    with lib.Server(0, mem_cap_bytes=64e9, max_active=3, round_iters=7) as srv:
        tickets = [srv.submit(p, fmt=f) for p, f in plans]
        out = [srv.wait(t, timeout=300) for t in tickets]
    for (info, w, dose, letd), (wr, dr, lr, rep) in zip(out, ref):
        assert info["status"] == lib.DONE
        np.testing.assert_array_equal(w, wr)
        np.testing.assert_array_equal(dose, dr)
        np.testing.assert_array_equal(letd, lr)
        assert info["report"]["iters"] == rep["iters"]
        assert info["report"]["objective"] == rep["objective"]
        assert info["t_submit"] <= info["t_admit"] <= info["t_start"] <= info["t_done"]


def test_admission_by_footprint(lib):
    plans = [small_plan(20000, 1500, 0.05, 10 + i, 20) for i in range(4)]
    fps = [lib.footprint_bytes(p.n_vox, p.n_spots, p.nnz) for p in plans]
    cap = int(max(fps) * 1.5)          # room for one plan at a time
    with lib.Server(0, mem_cap_bytes=cap, max_active=4, round_iters=5) as srv:
        tickets = [srv.submit(p) for p in plans]
        infos = [srv.wait(t, timeout=300)[0] for t in tickets]
        big = small_plan(200000, 3000, 0.2, 99, 5)
        with pytest.raises(lib.FredoptError) as e:
            srv.submit(big)      # can never fit under the cap
        assert e.value.code == -6
    for a, b in zip(infos, infos[1:]):
        # FIFO, and the next plan is admitted only once the previous one freed its memory
        assert b["t_admit"] >= a["t_done"]
        assert a["status"] == lib.DONE and b["status"] == lib.DONE


def test_failing_request_does_not_disturb_others(lib):
    good = small_plan(3000, 257, 0.2, 21, 15)
    bad = small_plan(3000, 257, 0.2, 22, 15)
    bad.col = bad.col.copy()
    bad.col[3] = 10_000              # column out of range: the load fails
    ref = alone(lib, good, "fp32")
    with lib.Server(0, mem_cap_bytes=16e9, max_active=2, round_iters=4) as srv:
        tb = srv.submit(bad)
        tg = srv.submit(good)
        ib = srv.wait(tb, timeout=120)[0]
        ig, w, dose, letd = srv.wait(tg, timeout=120)
    assert ib["status"] == -3
    assert ig["status"] == lib.DONE
    np.testing.assert_array_equal(w, ref[0])
