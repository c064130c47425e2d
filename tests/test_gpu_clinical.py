"""Parity at the benchmark's full size: the clinical plan (6e6 voxels, 30000
spots, 5.6e8 nonzeros per matrix), loaded exactly as bench.py loads it
(FP32, every row streamed, same kernels and launch shapes).

Sampled forward rows are checked one by one against FP64 dot products of
the CSR rows; the transposed product against scipy's FP64 transposed
product; three superiorized iterations against the FP64 oracle (identical
trial counters, w within 1e-4 relative L2); ROI-row mode against all-row
mode.
"""
import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clinical():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    pl = phantom.clinical_plan()
    return fredopt, pl


def test_clinical_forward_sampled_rows(clinical):
    lib, pl = clinical
    rng = np.random.default_rng(0)
    w = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        dose, lw = h.forward(w)
    rl = np.diff(pl.row_ptr)
    struct_rows = np.nonzero(pl.mask)[0]
    sample = np.concatenate([rng.choice(np.nonzero(rl > 0)[0], 1500, replace=False),
                             rng.choice(struct_rows, 500, replace=False),
                             rng.choice(np.nonzero(rl == 0)[0], 100, replace=False)])
    w64 = w.astype(np.float64)
    for i in sample:
        s, e = pl.row_ptr[i], pl.row_ptr[i + 1]
        c = pl.col[s:e]
        d_ref = float(pl.D[s:e].astype(np.float64) @ w64[c])
        l_ref = float(pl.L[s:e].astype(np.float64) @ w64[c])
        assert abs(dose[i] - d_ref) <= 1e-5 * abs(d_ref) + 1e-30, i
        assert abs(lw[i] - l_ref) <= 1e-5 * abs(l_ref) + 1e-30, i


def test_clinical_backward(clinical):
    lib, pl = clinical
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, [], [])
    rng = np.random.default_rng(1)
    aD = rng.normal(size=pl.n_vox).astype(np.float32)
    aL = rng.normal(size=pl.n_vox).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        u = h.backward(aD, aL)
    ref = P.D.T @ aD.astype(np.float64) + P.L.T @ aL.astype(np.float64)
    bound = abs(P.D).T @ np.abs(aD.astype(np.float64)) + abs(P.L).T @ np.abs(aL.astype(np.float64))
    assert np.all(np.abs(u - ref) <= 1e-5 * bound + 1e-30)


def test_clinical_three_iterations_match_oracle(clinical):
    lib, pl = clinical
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints,
                             pl.objective)
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 3, pl.alpha, pl.relaxation)
    out = {}
    for rows in ("all", "roi"):
        with lib.Handle(0) as h:
            h.load_plan(pl, rows=rows)
            w, dose, letd, rep = h.superiorize(pl.w0, 3, pl.alpha, pl.relaxation)
            out[rows] = (w, h.get_log())
    for rows, (w, log) in out.items():
        assert [e["s"] for e in log] == [e["s"] for e in log_ref], rows
        assert np.linalg.norm(w - w_ref) <= 1e-4 * np.linalg.norm(w_ref), rows
        for e in log:
            assert e["f_end"] <= e["f_start"]
    np.testing.assert_allclose(out["roi"][0], out["all"][0], rtol=1e-5, atol=1e-6)
