"""Parity at the largest workload: the 27-scenario robust plan with every
scenario's rows stacked (3.89e7 rows, 8192 spots, 1.56e9 nonzeros per matrix,
close to the 2^31 nonzero limit of the CSR), FP32 storage, all rows streamed
with the default claimed tiles.

Sampled forward rows against FP64 dot products of the CSR rows (1e-5
relative); sampled columns of the transposed product against FP64 sums over
the CSR (1e-5 of the sum of absolute products); a few superiorized iterations
hold the non-ascent property and stay finite.  The full FP64 oracle run is
out of reach at this size; the clinical plan's three-iteration comparison
covers the trajectory.
"""
import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def robust():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    pl, per = phantom.robust_plan()
    return fredopt, pl


def test_maxsize_forward_backward_and_iterations(robust):
    lib, pl = robust
    assert pl.nnz > 1.5e9 and pl.nnz < 2 ** 31
    rng = np.random.default_rng(3)
    w = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    a = rng.normal(size=pl.n_vox).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        dose, lw = h.forward(w)
        w_out, d_out, l_out, rep = h.superiorize(pl.w0, 4, pl.alpha, pl.relaxation)
        log = h.get_log()
        u = h.backward(a, a)
    # forward: sampled rows, including rows of the first and last scenario
    rl = np.diff(pl.row_ptr)
    nz = np.nonzero(rl > 0)[0]
    sample = np.concatenate([rng.choice(nz, 1500, replace=False), nz[:50], nz[-50:]])
    w64 = w.astype(np.float64)
    for i in sample:
        s, e = pl.row_ptr[i], pl.row_ptr[i + 1]
        c = pl.col[s:e]
        d_ref = float(pl.D[s:e].astype(np.float64) @ w64[c])
        l_ref = float(pl.L[s:e].astype(np.float64) @ w64[c])
        assert abs(dose[i] - d_ref) <= 1e-5 * abs(d_ref) + 1e-30, i
        assert abs(lw[i] - l_ref) <= 1e-5 * abs(l_ref) + 1e-30, i
    # transposed product: sampled columns summed over the whole CSR in FP64
    rows = np.repeat(np.arange(pl.n_vox, dtype=np.int64), rl)
    for j in rng.choice(pl.n_spots, 6, replace=False):
        sel = np.nonzero(pl.col == j)[0]
        ar = a[rows[sel]].astype(np.float64)
        ref = float(pl.D[sel].astype(np.float64) @ ar + pl.L[sel].astype(np.float64) @ ar)
        bound = float(np.abs(pl.D[sel]).astype(np.float64) @ np.abs(ar) + np.abs(pl.L[sel]).astype(np.float64) @ np.abs(ar))
        assert abs(u[j] - ref) <= 1e-5 * bound + 1e-30, j
    # iterations: the perturbation never ascends, everything finite
    assert len(log) == 4
    for e in log:
        assert e["f_end"] <= e["f_start"]
    assert np.all(np.isfinite(w_out)) and np.all(w_out >= 0)
    assert np.isfinite(rep["objective"])
