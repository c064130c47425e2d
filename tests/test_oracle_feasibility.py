"""The LP feasibility check of a plan's constraint set (oracle/feasibility.py),
pinned to brute-force vertex enumeration on 2-4 spots x 10 voxels, then
applied to the clinical phantom at 8 mm.  CPU only."""
import numpy as np
import pytest

import oracle
import phantom
from oracle import feasibility
from test_oracle_pins import _as_inequalities, _vertex_feasible, small_problem


@pytest.mark.parametrize("seed", range(8))
def test_lp_feasibility_agrees_with_vertex_enumeration(seed):
    rng = np.random.default_rng(300 + seed)
    n = 2 + seed % 3
    n_vox = 10
    D = rng.uniform(0.1, 1.0, (n_vox, n))
    L = rng.uniform(1.0, 8.0, (n_vox, n)) * D
    mask = np.where(np.arange(n_vox) < 5, 1, 2).astype(np.uint32)
    z = rng.uniform(0.5, 1.5, n)
    dz = D @ z
    lo = float(dz[:5].min()) * 0.9
    hi = float(dz[:5].max()) * (1.1 if seed % 2 == 0 else 0.7)   # odd seeds: an empty PTV window
    cons = [dict(struct_bit=0, kind="DOSE_MIN", bound=lo, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MAX", bound=hi, priority=1.0),
            dict(struct_bit=1, kind="DOSE_MAX", bound=float(dz[5:].max()) * 1.2, priority=1.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=float(((L @ z) / dz)[5:].max()) * 1.05, priority=1.0)]
    P = small_problem(D, L, mask, cons)
    R = oracle.constraint_rows(P)
    G, h = _as_inequalities(P)
    vert = _vertex_feasible(G, h, n)
    ok, w, v = feasibility.is_feasible(R)
    assert ok == (vert is not None)
    f, _ = feasibility.min_total_violation(R)
    if ok:
        assert np.all(w >= -1e-12) and v <= 1e-7 and f <= 1e-7
    else:
        assert f > 1e-6


def test_clinical_phantom_constraints_are_feasible_at_8mm():
    """The clinical geometry (PTV 150 cc within [0.95, 1.07] x 2 Gy; brainstem-,
    chiasm- and eye-like OARs with their dose and LETd limits) at 8 mm: some
    spot weights meet every row, so a run that still violates rows has not
    converged yet; it does not face an empty set.  Emptying the PTV window
    makes the same check fail."""
    pl = phantom.clinical_plan(shape=(50, 50, 38), h=8.0)
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    R = oracle.constraint_rows(P)
    assert {c["kind"] for c in pl.constraints} >= {"DOSE_MIN", "DOSE_MAX", "LETD_MAX"}
    ok, w, v = feasibility.is_feasible(R)
    assert ok, v
    bad = [dict(c) for c in pl.constraints]
    bad[0]["bound"] = 1.2 * bad[1]["bound"]          # PTV minimum above its maximum
    P2 = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, bad, pl.objective)
    ok2, _, v2 = feasibility.is_feasible(oracle.constraint_rows(P2))
    assert not ok2 and v2 > 1e-3
