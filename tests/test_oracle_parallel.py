"""The all-core timing variant of the oracle (oracle/parallel.py) computes
what the oracle computes: forward products bit-identical, transposed
products and whole superiorized runs equal to rounding, with identical trial
logs.  CPU only."""
import numpy as np

import oracle
import phantom
from oracle import parallel


def test_threaded_products_and_run_match_the_oracle():
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    R = oracle.constraint_rows(P)
    Pt = parallel.threaded(P, 4)
    Rt = parallel.threaded_rows(R, 4)
    rng = np.random.default_rng(0)
    w = rng.uniform(0.0, 2.0, pl.n_spots)
    d, l = oracle.forward(P, w)
    dt, lt = oracle.forward(Pt, w)
    np.testing.assert_array_equal(d, dt)
    np.testing.assert_array_equal(l, lt)
    g = oracle.objective_gradient(P, w)
    gt = oracle.objective_gradient(Pt, w)
    np.testing.assert_allclose(gt, g, rtol=1e-12, atol=1e-14 * np.abs(g).max())
    x = oracle.cimmino_step(R, w, 1.0)
    xt = oracle.cimmino_step(Rt, w, 1.0)
    np.testing.assert_allclose(xt, x, rtol=1e-12, atol=1e-14)
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 6, pl.alpha, pl.relaxation, rows=R)
    w_t, log_t = oracle.superiorize(Pt, pl.w0, 6, pl.alpha, pl.relaxation, rows=Rt)
    assert [e["s"] for e in log_t] == [e["s"] for e in log_ref]
    assert [e["accepted"] for e in log_t] == [e["accepted"] for e in log_ref]
    np.testing.assert_allclose(w_t, w_ref, rtol=1e-10, atol=1e-12)
    # rows built from the threaded problem are the same rows
    R2 = oracle.constraint_rows(Pt)
    assert (R2.A != R.A).nnz == 0 and R2.unreachable == R.unreachable
