"""Pins of the FP64 oracle against what the paper and mathematics fix
(worked examples, closed forms, invariants, brute force), CPU only.

Each test is chosen so that a plausible mistake in the oracle (a dropped
term, a wrong sign, a transposed operand, a wrong weight or index) fails it.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize as opt
import scipy.sparse as sp

import oracle
import phantom

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_problem(D, L, mask, constraints, objective=(), c=oracle.C_CDL):
    D = sp.csr_matrix(np.asarray(D, np.float64))
    L = sp.csr_matrix(np.asarray(L, np.float64))
    # shared pattern: union of both patterns
    pat = (abs(D) + abs(L)).tocsr()
    pat.sort_indices()
    rp, col = pat.indptr.astype(np.int64), pat.indices.astype(np.int32)
    Dv = np.asarray(D[np.repeat(np.arange(D.shape[0]), np.diff(rp)), col]).ravel()
    Lv = np.asarray(L[np.repeat(np.arange(L.shape[0]), np.diff(rp)), col]).ravel()
    return oracle.build_problem(rp, col, Dv, Lv, D.shape[1], np.asarray(mask, np.uint32),
                                list(constraints), list(objective), c=c)


# ------------------------------------------------------------ worked examples

def load_worked():
    with open(os.path.join(GOLD, "cimmino_worked.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("case", load_worked()["cases"], ids=lambda c: c["name"])
def test_worked_projection_examples(case):
    """Hand-derived single Cimmino steps (Fig. 2, readings R1, R3)."""
    P = small_problem(case["D"], case["L"], case["mask"], case["constraints"])
    R = oracle.constraint_rows(P)
    xn = oracle.cimmino_step(R, case["x"], case["lam"])
    np.testing.assert_allclose(xn, case["expected"], rtol=0, atol=1e-12)


def test_worked_letd_limit_reached():
    """After the LETd projection the physical LETd (Eq. 1 ratio) equals the limit."""
    case = [c for c in load_worked()["cases"] if c["constraints"][0]["kind"] == "LETD_MAX"][0]
    P = small_problem(case["D"], case["L"], case["mask"], case["constraints"])
    xn = oracle.cimmino_step(oracle.constraint_rows(P), case["x"], 1.0)
    dose, lw = oracle.forward(P, xn)
    assert oracle.letd(dose, lw)[0] == pytest.approx(case["constraints"][0]["bound"], abs=1e-12)


def test_worked_trial_loop():
    """Fig. 3 trial sequence on a one-voxel objective, derived by hand."""
    t = load_worked()["trials"]
    P = small_problem(t["D"], t["L"], t["mask"], [], t["objective"])
    w, log = oracle.superiorize(P, t["w0"], 2, t["alpha"], 1.0, beta0=t["beta0"])
    np.testing.assert_allclose(w, t["expected_w"], atol=1e-15)
    for got, exp in zip(log, t["expected_log"]):
        for key, val in exp.items():
            assert got[key] == pytest.approx(val, abs=1e-15), key


@pytest.mark.parametrize("case", load_worked()["cases"], ids=lambda c: c["name"])
def test_worked_violations(case):
    """Row violations at the worked points, derived by hand: the amount an
    upper bound is exceeded (a.x - b) or a lower bound missed (b - a.x), 0
    when satisfied; LETd rows in Gy keV/um (R10)."""
    P = small_problem(case["D"], case["L"], case["mask"], case["constraints"])
    R = oracle.constraint_rows(P)
    np.testing.assert_allclose(oracle.violations(R, case["x"]), case["expected_violations"], rtol=0, atol=1e-12)


def test_worked_final_report():
    """final_report on a hand-derived case: dose, Lw and LETd (Eq. 1, 0 where
    the dose is 0), rows in constraint-table then voxel order with one row
    per (structure, constraint) of an overlapping voxel (R11), unreachable
    rows dropped (R10), the largest violation per constraint, the number of
    violated rows and the Eq. 2 objective with its weight."""
    t = load_worked()["report"]
    P = small_problem(t["D"], t["L"], t["mask"], t["constraints"], t["objective"])
    R = oracle.constraint_rows(P)
    e = t["expected"]
    np.testing.assert_array_equal(R.voxel, e["row_voxels"])
    np.testing.assert_allclose(oracle.violations(R, t["w"]), e["row_violations"], rtol=0, atol=1e-12)
    rep = oracle.final_report(P, t["w"], rows=R)
    for k in ("dose", "lw", "letd"):
        np.testing.assert_allclose(rep[k], e[k], rtol=0, atol=1e-12)
    assert rep["max_violation"] == {int(k): pytest.approx(v, abs=1e-12) for k, v in e["max_violation"].items()}
    assert rep["n_violated"] == e["n_violated"]
    assert rep["unreachable"] == e["unreachable"]
    assert rep["objective"] == pytest.approx(e["objective"], abs=1e-12)
    # the same report without precomputed rows
    rep2 = oracle.final_report(P, t["w"])
    assert rep2["n_violated"] == e["n_violated"] and rep2["unreachable"] == e["unreachable"]


def test_violations_sign_and_letd_units():
    """Violations are nonnegative and zero exactly on the feasible side; in
    physical units they are dose - bound (upper), bound - dose (lower),
    bound - cDL (lower cDL) and, for a LETd row divided by the dose,
    LETd - Lambda (R10, Eq. 1)."""
    rng = np.random.default_rng(8)
    D = rng.uniform(0.1, 1.0, (6, 4))
    L = D * rng.uniform(1.0, 9.0, (6, 4))
    cons = [dict(struct_bit=0, kind="DOSE_MAX", bound=2.0, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MIN", bound=1.0, priority=1.0),
            dict(struct_bit=0, kind="LETD_MAX", bound=4.0, priority=1.0),
            dict(struct_bit=0, kind="CDL_MIN", bound=0.1, priority=1.0)]
    P = small_problem(D, L, np.ones(6, np.uint32), cons)
    R = oracle.constraint_rows(P)
    for _ in range(20):
        x = rng.uniform(0.0, 2.0, 4)
        v = oracle.violations(R, x)
        ax = R.A @ x
        assert np.all(v >= 0)
        np.testing.assert_array_equal(v == 0, np.where(R.upper, ax <= R.b, ax >= R.b))
        dose, lw = oracle.forward(P, x)
        let = oracle.letd(dose, lw)
        sel = R.cidx == 2
        np.testing.assert_allclose(v[sel] / dose[R.voxel[sel]], np.maximum(let[R.voxel[sel]] - 4.0, 0.0),
                                   rtol=1e-12, atol=1e-12)
        sel = R.cidx == 0
        np.testing.assert_allclose(v[sel], np.maximum(dose[R.voxel[sel]] - 2.0, 0.0), rtol=0, atol=1e-12)
        sel = R.cidx == 1
        np.testing.assert_allclose(v[sel], np.maximum(1.0 - dose[R.voxel[sel]], 0.0), rtol=0, atol=1e-12)
        sel = R.cidx == 3
        np.testing.assert_allclose(v[sel], np.maximum(0.1 - oracle.C_CDL * lw[R.voxel[sel]], 0.0), rtol=0,
                                   atol=1e-12)


# ------------------------------------------------------------ one half-space

def _rand_row_problem(seed, kind, n=7):
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.1, 1.0, (1, n)) * (rng.uniform(size=(1, n)) < 0.7)
    D[0, 0] = 0.5
    let = rng.uniform(1.0, 10.0, (1, n))
    L = let * D
    x = rng.uniform(0.5, 2.0, n)
    # bound placed so that x violates the row
    P0 = small_problem(D, L, [1], [])
    dose, lw = oracle.forward(P0, x)
    if kind == "DOSE_MAX":
        bound = 0.5 * dose[0]
    elif kind == "DOSE_MIN":
        bound = 2.0 * dose[0]
    elif kind == "CDL_MAX":
        bound = 0.5 * oracle.C_CDL * lw[0]
    elif kind == "CDL_MIN":
        bound = 2.0 * oracle.C_CDL * lw[0]
    elif kind == "LETD_MAX":
        bound = 0.8 * lw[0] / dose[0]
    else:  # LETD_MIN
        bound = 1.2 * lw[0] / dose[0]
    P = small_problem(D, L, [1], [dict(struct_bit=0, kind=kind, bound=bound, priority=1.0)])
    return P, x, bound


def _physical_value(P, x, kind):
    dose, lw = oracle.forward(P, x)
    if kind.startswith("DOSE"):
        return dose[0]
    if kind.startswith("CDL"):
        return oracle.C_CDL * dose[0] * oracle.letd(dose, lw)[0]
    return oracle.letd(dose, lw)[0]


KINDS = ["DOSE_MAX", "DOSE_MIN", "CDL_MAX", "CDL_MIN", "LETD_MAX", "LETD_MIN"]


@pytest.mark.parametrize("kind", KINDS)
def test_projection_is_nearest_point_on_boundary(kind):
    """lam = 1, one violated half-space, no clip: the step equals the nearest
    point of the half-space, found here by a generic constrained solver
    (SLSQP), and the physical quantity (dose, c*dose*LETd, LETd) sits on its
    bound."""
    P, x, bound = _rand_row_problem(3, kind)
    R = oracle.constraint_rows(P)
    xn = oracle.cimmino_step(R, x, 1.0, clip=False)
    assert _physical_value(P, xn, kind) == pytest.approx(bound, rel=1e-10)
    a = R.A.toarray()[0]
    b = R.b[0]
    sign = 1.0 if R.upper[0] else -1.0
    res = opt.minimize(lambda y: 0.5 * np.sum((y - x) ** 2), x, jac=lambda y: y - x, method="SLSQP",
                       constraints=[dict(type="ineq", fun=lambda y: sign * (b - a @ y), jac=lambda y: -sign * a)],
                       options=dict(ftol=1e-14, maxiter=200))
    np.testing.assert_allclose(xn, res.x, atol=1e-7)


@pytest.mark.parametrize("kind", KINDS)
def test_projection_moves_toward_bound(kind):
    """A violated MIN row raises its quantity, a MAX row lowers it (the sign
    fix of reading R3), with any 0 < lam <= 2 (no clip)."""
    P, x, bound = _rand_row_problem(5, kind)
    R = oracle.constraint_rows(P)
    before = _physical_value(P, x, kind)
    for lam in (0.3, 1.0, 1.7):
        after = _physical_value(P, oracle.cimmino_step(R, x, lam, clip=False), kind)
        if kind.endswith("MAX"):
            assert after < before
        else:
            assert after > before


def test_relaxation_two_reflects():
    P, x, bound = _rand_row_problem(7, "DOSE_MAX")
    R = oracle.constraint_rows(P)
    a, b = R.A.toarray()[0], R.b[0]
    xn = oracle.cimmino_step(R, x, 2.0, clip=False)
    assert a @ xn - b == pytest.approx(-(a @ x - b), rel=1e-12)


def test_satisfied_row_leaves_point_unchanged():
    P, x, bound = _rand_row_problem(9, "DOSE_MAX")
    con = dict(P.constraints[0], bound=1e6)
    P2 = small_problem(P.D.toarray(), P.L.toarray(), [1], [con])
    xn = oracle.cimmino_step(oracle.constraint_rows(P2), x, 1.0)
    np.testing.assert_array_equal(xn, x)


# ------------------------------------------------------------ Cimmino step

def _rand_problem(seed, n_vox=12, n_spots=5):
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.05, 1.0, (n_vox, n_spots)) * (rng.uniform(size=(n_vox, n_spots)) < 0.8)
    L = rng.uniform(1.0, 10.0, (n_vox, n_spots)) * D
    mask = rng.integers(1, 8, n_vox).astype(np.uint32)      # overlapping structures
    cons = [
        dict(struct_bit=0, kind="DOSE_MIN", bound=1.0, priority=2.0),
        dict(struct_bit=0, kind="DOSE_MAX", bound=1.5, priority=1.0),
        dict(struct_bit=1, kind="CDL_MAX", bound=0.2, priority=0.5),
        dict(struct_bit=2, kind="LETD_MAX", bound=4.0, priority=1.5),
    ]
    return small_problem(D, L, mask, cons), rng


def test_cimmino_is_weighted_average_of_projections():
    """lam = 1, norm 'all': the step equals sum_r omega_r P_r(x) with
    sum omega = 1, where each P_r(x) is the nearest point of half-space r
    computed by a generic solver (satisfied rows: P_r(x) = x)."""
    P, rng = _rand_problem(11)
    R = oracle.constraint_rows(P)
    x = rng.uniform(0.0, 3.0, P.n_spots)
    A = R.A.toarray()
    avg = np.zeros_like(x)
    W = R.p.sum()
    for r in range(A.shape[0]):
        a, b = A[r], R.b[r]
        sign = 1.0 if R.upper[r] else -1.0
        res = opt.minimize(lambda y: 0.5 * np.sum((y - x) ** 2), x, jac=lambda y: y - x, method="SLSQP",
                           constraints=[dict(type="ineq", fun=lambda y, a=a, b=b, s=sign: s * (b - a @ y),
                                             jac=lambda y, a=a, s=sign: -s * a)],
                           options=dict(ftol=1e-15, maxiter=300))
        avg += R.p[r] / W * res.x
    np.testing.assert_allclose(oracle.cimmino_step(R, x, 1.0, clip=False), avg, atol=1e-7)


def test_overlapping_structures_give_one_row_each():
    """A voxel in k constrained structures contributes one row per constraint."""
    P, _ = _rand_problem(12)
    R = oracle.constraint_rows(P)
    expect = 0
    for con in P.constraints:
        for i in range(P.n_vox):
            if (int(P.mask[i]) >> con["struct_bit"]) & 1:
                row_d = P.D.toarray()[i]
                row_l = P.L.toarray()[i]
                if con["kind"].startswith("DOSE"):
                    a = row_d
                elif con["kind"].startswith("CDL"):
                    a = oracle.C_CDL * row_l
                else:
                    a = row_l - con["bound"] * row_d
                expect += int(np.dot(a, a) > 0)
    assert R.A.shape[0] == expect


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.9])
def test_fejer_monotone_towards_feasible_point(lam):
    """For a point z inside every half-space (z >= 0), one step (projections
    and clip are nonexpansive) never moves away from z."""
    rng = np.random.default_rng(21)
    n_vox, n = 15, 6
    D = rng.uniform(0.05, 1.0, (n_vox, n))
    L = rng.uniform(1.0, 10.0, (n_vox, n)) * D
    z = rng.uniform(0.2, 1.0, n)
    dz, lz = D @ z, L @ z
    mask = np.ones(n_vox, np.uint32) * 3
    mask[::2] = 1
    cons = [dict(struct_bit=0, kind="DOSE_MAX", bound=float(dz.max()) * 1.01, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MIN", bound=float(dz.min()) * 0.99, priority=2.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=float((lz / dz).max()) * 1.01, priority=1.0)]
    P = small_problem(D, L, mask, cons)
    R = oracle.constraint_rows(P)
    for trial in range(20):
        x = rng.uniform(0.0, 4.0, n)
        for norm in ("all", "violated"):
            xn = oracle.cimmino_step(R, x, lam, norm=norm)
            assert np.linalg.norm(xn - z) <= np.linalg.norm(x - z) + 1e-12


def test_eta_scales_the_step():
    """Priorities are multiplied by eta^k (Fig. 3, w_k = eta^k w)."""
    P, x, bound = _rand_row_problem(13, "DOSE_MIN")
    R = oracle.constraint_rows(P)
    full = oracle.cimmino_step(R, x, 1.0, clip=False) - x
    part = oracle.cimmino_step(R, x, 1.0, prio_scale=0.25, clip=False) - x
    np.testing.assert_allclose(part, 0.25 * full, rtol=1e-13)
    P2 = small_problem(P.D.toarray(), P.L.toarray(), [1], P.constraints, [])
    w3, _ = oracle.superiorize(P2, x, 3, 0.9, 0.5, eta=0.5, reductions=0)
    # by hand: one half-space a.x >= b that stays violated; iteration k moves
    # the point lam*eta^k of the way to the hyperplane, so the gap shrinks by
    # (1 - 0.5*1)(1 - 0.5*0.5)(1 - 0.5*0.25)
    a = R.A.toarray()[0]
    gap0 = R.b[0] - a @ x
    assert R.b[0] - a @ w3 == pytest.approx(gap0 * 0.5 * 0.75 * 0.875, rel=1e-12)


# ------------------------------------------------------------ brute-force feasibility

def _vertex_feasible(G, h, n, tol=1e-9):
    """Brute force: is {x : G x <= h} (which includes x >= 0) non-empty and
    bounded?  Enumerate every n-subset of constraints as equalities, solve,
    and check the vertex.  Returns a feasible vertex or None."""
    m = G.shape[0]
    for idx in itertools.combinations(range(m), n):
        Gs = G[list(idx)]
        if abs(np.linalg.det(Gs)) < 1e-12:
            continue
        v = np.linalg.solve(Gs, h[list(idx)])
        if np.all(G @ v <= h + tol):
            return v
    return None


def _as_inequalities(P):
    rows = []
    rhs = []
    Dd, Ld = P.D.toarray(), P.L.toarray()
    for con in P.constraints:
        for i in range(P.n_vox):
            if not (int(P.mask[i]) >> con["struct_bit"]) & 1:
                continue
            k = con["kind"]
            a = Dd[i] if k.startswith("DOSE") else (P.c * Ld[i] if k.startswith("CDL") else Ld[i] - con["bound"] * Dd[i])
            b = 0.0 if k.startswith("LETD") else con["bound"]
            if k.endswith("MAX"):
                rows.append(a); rhs.append(b)
            else:
                rows.append(-a); rhs.append(-b)
    n = P.n_spots
    G = np.vstack(rows + [-np.eye(n)])
    h = np.concatenate([rhs, np.zeros(n)])
    return G, h


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_feasibility_vs_cimmino(seed):
    """2-4 spots x 10 voxels.  Vertex enumeration decides whether the plan's
    feasible set is non-empty (cross-checked with an LP).  If it has an
    interior, plain Cimmino drives every physical violation (dose, LETd,
    cDL evaluated from their definitions) to ~0; if it is empty the largest
    violation stays at or above the LP's minimum achievable value."""
    rng = np.random.default_rng(100 + seed)
    n = 2 + seed % 3
    n_vox = 10
    D = rng.uniform(0.1, 1.0, (n_vox, n))
    LET = rng.uniform(1.0, 8.0, (n_vox, n))
    L = LET * D
    mask = np.where(np.arange(n_vox) < 5, 1, 2).astype(np.uint32)
    z = rng.uniform(0.5, 1.5, n)
    dz = D @ z
    feasible_case = seed % 2 == 0
    lo = float(dz[:5].min()) * 0.9
    # infeasible case: the PTV dose window is empty for the hottest voxel's row
    hi = float(dz[:5].max()) * 1.1 if feasible_case else lo * 0.8
    oar_max = float(dz[5:].max()) * 1.2
    let_lim = float(((L @ z) / dz)[5:].max()) * 1.05
    cons = [dict(struct_bit=0, kind="DOSE_MIN", bound=lo, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MAX", bound=hi, priority=1.0),
            dict(struct_bit=1, kind="DOSE_MAX", bound=oar_max, priority=1.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=let_lim, priority=1.0)]
    P = small_problem(D, L, mask, cons)
    G, h = _as_inequalities(P)
    vert = _vertex_feasible(G, h, n)
    lp = opt.linprog(np.zeros(n), A_ub=G, b_ub=h, bounds=[(None, None)] * n, method="highs")
    assert (vert is not None) == (lp.status == 0)
    w, _ = oracle.superiorize(P, np.ones(n), 3000, 0.99, 1.5, reductions=0)
    dose, lw = oracle.forward(P, w)
    let = oracle.letd(dose, lw)
    phys_viol = max(lo - dose[:5].min(), dose[:5].max() - hi, dose[5:].max() - oar_max,
                    let[5:].max() - let_lim, 0.0)
    if feasible_case:
        assert vert is not None
        assert phys_viol <= 1e-7
    else:
        assert vert is None
        # minimum achievable max-violation t*: min t s.t. G x - t <= h (x>=0 rows exact)
        m_c = G.shape[0] - n
        Gt = np.hstack([G, np.concatenate([-np.ones(m_c), np.zeros(n)])[:, None]])
        lp2 = opt.linprog(np.r_[np.zeros(n), 1.0], A_ub=Gt, b_ub=h, bounds=[(None, None)] * (n + 1),
                          method="highs")
        assert lp2.status == 0 and lp2.fun > 1e-6
        assert np.max(G[:m_c] @ w - h[:m_c]) >= lp2.fun - 1e-9


# ------------------------------------------------------------ products and LETd

def test_forward_matches_bruteforce_loops():
    row_ptr, col, D, L = phantom.random_csr(64, 16, 0.3, seed=1, empty_rows=3)
    P = oracle.build_problem(row_ptr, col, D, L, 16, np.zeros(64, np.uint32), [], [])
    w = np.random.default_rng(2).uniform(0, 2, 16)
    dose, lw = oracle.forward(P, w)
    for i in range(64):
        sd = sl = 0.0
        for p in range(row_ptr[i], row_ptr[i + 1]):
            sd += float(D[p]) * w[col[p]]
            sl += float(L[p]) * w[col[p]]
        assert dose[i] == pytest.approx(sd, rel=1e-14, abs=1e-300)
        assert lw[i] == pytest.approx(sl, rel=1e-14, abs=1e-300)


def test_dose_is_linear_in_w():
    pl = phantom.tiny_plan(noise=0.01)
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, [], [])
    rng = np.random.default_rng(3)
    w1, w2 = rng.uniform(0, 1, pl.n_spots), rng.uniform(0, 1, pl.n_spots)
    d1, l1 = oracle.forward(P, w1)
    d2, l2 = oracle.forward(P, w2)
    d3, l3 = oracle.forward(P, 0.7 * w1 - 1.3 * w2)
    scale = np.abs(d1).max() + np.abs(d2).max()
    np.testing.assert_allclose(d3, 0.7 * d1 - 1.3 * d2, atol=1e-13 * scale)
    np.testing.assert_allclose(l3, 0.7 * l1 - 1.3 * l2, atol=1e-13 * (np.abs(l1).max() + np.abs(l2).max()))


def test_letd_is_dose_weighted_mean_within_spot_let_range():
    """Eq. (1): LETd_i lies between the smallest and largest LET of the spots
    that deliver dose to voxel i; with a single spot it equals that LET."""
    row_ptr, col, D, L = phantom.random_csr(200, 30, 0.2, seed=4, empty_rows=5)
    P = oracle.build_problem(row_ptr, col, D, L, 30, np.zeros(200, np.uint32), [], [])
    w = np.random.default_rng(5).uniform(0, 1, 30)
    w[::4] = 0.0
    dose, lw = oracle.forward(P, w)
    ld = oracle.letd(dose, lw)
    for i in range(200):
        s, e = row_ptr[i], row_ptr[i + 1]
        m = w[col[s:e]] > 0
        if not m.any():
            assert ld[i] == 0.0
            continue
        let = (L[s:e].astype(np.float64) / D[s:e].astype(np.float64))[m]
        assert let.min() * (1 - 1e-12) <= ld[i] <= let.max() * (1 + 1e-12)
    j = 7
    e = np.zeros(30)
    e[j] = 2.5
    dose, lw = oracle.forward(P, e)
    ld = oracle.letd(dose, lw)
    for i in range(200):
        s, t = row_ptr[i], row_ptr[i + 1]
        hit = np.nonzero(col[s:t] == j)[0]
        if hit.size:
            assert ld[i] == pytest.approx(float(L[s + hit[0]]) / float(D[s + hit[0]]), rel=1e-14)


def test_csc_transpose_bit_exact_and_involutive():
    row_ptr, col, D, L = phantom.random_csr(50, 20, 0.3, seed=6, empty_rows=2)
    cp, rows, DT, LT = oracle.transpose_csr(row_ptr, col, 20, D, L)
    dense = np.zeros((50, 20), np.float32)
    for i in range(50):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            dense[i, col[p]] = D[p]
    for j in range(20):
        s, e = cp[j], cp[j + 1]
        assert np.all(np.diff(rows[s:e]) > 0)
        for p in range(s, e):
            assert DT[p] == dense[rows[p], j]            # bit-exact move
        assert e - s == np.count_nonzero(dense[:, j])
    rp2, c2, D2, L2 = oracle.transpose_csr(cp, rows, 50, DT, LT)
    np.testing.assert_array_equal(rp2, row_ptr)
    np.testing.assert_array_equal(c2, col)
    np.testing.assert_array_equal(D2, D)
    np.testing.assert_array_equal(L2, L)


# ------------------------------------------------------------ objective

def test_objective_from_physical_quantities():
    """Eq. (2): OAR term built from dose and LETd (cDL = c*dose*LETd) and PTV
    term from dose, evaluated here via LETd rather than the LET-weighted dose."""
    P, rng = _rand_problem(31)
    P.objective = [dict(struct_bit=0, quantity="DOSE", target=2.0, weight=3.0),
                   dict(struct_bit=1, quantity="CDL", target=0.1, weight=0.5)]
    x = rng.uniform(0, 2, P.n_spots)
    dose, lw = oracle.forward(P, x)
    ld = oracle.letd(dose, lw)
    f = 0.0
    for i in range(P.n_vox):
        if int(P.mask[i]) & 1:
            f += 3.0 * (2.0 - dose[i]) ** 2
        if int(P.mask[i]) & 2:
            f += 0.5 * (0.1 - oracle.C_CDL * dose[i] * ld[i]) ** 2
    assert oracle.objective(P, x) == pytest.approx(f, rel=1e-12)


def test_gradient_matches_finite_differences():
    P, rng = _rand_problem(32)
    P.objective = [dict(struct_bit=0, quantity="DOSE", target=2.0, weight=3.0),
                   dict(struct_bit=1, quantity="CDL", target=0.1, weight=0.5),
                   dict(struct_bit=2, quantity="CDL", target=0.0, weight=1.0)]
    x = rng.uniform(0, 2, P.n_spots)
    g = oracle.objective_gradient(P, x)
    h = 1e-5
    for j in range(P.n_spots):
        e = np.zeros(P.n_spots)
        e[j] = h
        fd = (oracle.objective(P, x + e) - oracle.objective(P, x - e)) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-7, abs=1e-9)


# ------------------------------------------------------------ superiorization

@pytest.fixture(scope="module")
def tiny():
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    return pl, P, oracle.constraint_rows(P)


def test_superiorization_non_ascent_and_beta_schedule(tiny):
    """f(x^{k,N}) <= f(w^k) every iteration; each accepted step is
    beta0*alpha^(s-1) with s the global trial counter (Fig. 3, R5)."""
    pl, P, R = tiny
    beta0 = 0.1 * float(np.linalg.norm(pl.w0.astype(np.float64)))
    w, log = oracle.superiorize(P, pl.w0, 12, pl.alpha, pl.relaxation, rows=R)
    s_prev = 0
    for e in log:
        assert e["f_end"] <= e["f_start"]
        assert e["s"] >= s_prev
        if e["accepted"]:
            assert e["beta"] == beta0 * pl.alpha ** (e["s"] - 1)
        s_prev = e["s"]
    assert log[0]["accepted"] == 1


def test_zero_perturbation_reduces_to_plain_cimmino(tiny):
    """reductions = 0 and beta0 = 0 both give the plain feasibility iteration,
    bit for bit."""
    pl, P, R = tiny
    x = pl.w0.astype(np.float64)
    for k in range(4):
        x = oracle.cimmino_step(R, x, pl.relaxation)
    w0_, _ = oracle.superiorize(P, pl.w0, 4, pl.alpha, pl.relaxation, reductions=0, rows=R)
    wb, logb = oracle.superiorize(P, pl.w0, 4, pl.alpha, pl.relaxation, beta0=0.0, rows=R)
    np.testing.assert_array_equal(w0_, x)
    np.testing.assert_array_equal(wb, x)
    # beta = 0 leaves f unchanged, which "does not ascend": the first trial
    # of every iteration is accepted (R7), so s counts one trial per iteration
    assert [e["s"] for e in logb] == [1, 2, 3, 4]
    assert all(e["accepted"] == 1 for e in logb)


def test_superiorization_reduces_objective_vs_plain(tiny):
    pl, P, R = tiny
    ws, _ = oracle.superiorize(P, pl.w0, 15, pl.alpha, pl.relaxation, rows=R)
    wp, _ = oracle.superiorize(P, pl.w0, 15, pl.alpha, pl.relaxation, reductions=0, rows=R)
    assert oracle.objective(P, ws) < oracle.objective(P, wp)


def test_resume_reproduces_uninterrupted_run(tiny):
    pl, P, R = tiny
    beta0 = 0.1 * float(np.linalg.norm(pl.w0.astype(np.float64)))
    w_all, log_all = oracle.superiorize(P, pl.w0, 6, pl.alpha, pl.relaxation, rows=R, eta=0.9)
    w_a, log_a = oracle.superiorize(P, pl.w0, 3, pl.alpha, pl.relaxation, rows=R, eta=0.9)
    w_b, log_b = oracle.superiorize(P, w_a, 3, pl.alpha, pl.relaxation, rows=R, eta=0.9, beta0=beta0,
                                    s0=log_a[-1]["s"], k0=3)
    np.testing.assert_array_equal(w_b, w_all)


def test_sequential_sweep_single_row_equals_projection():
    P, x, bound = _rand_row_problem(41, "DOSE_MAX")
    R = oracle.constraint_rows(P)
    np.testing.assert_allclose(oracle.sequential_ams_sweep(R, x, 1.0),
                               oracle.cimmino_step(R, x, 1.0), rtol=1e-14)


def test_sequential_sweep_orthogonal_rows_each_on_bound():
    """Two rows with disjoint spots: the row-action sweep puts each dose on
    its bound (the second update cannot disturb the first)."""
    D = [[1.0, 2.0, 0.0, 0.0], [0.0, 0.0, 3.0, 1.0]]
    cons = [dict(struct_bit=0, kind="DOSE_MAX", bound=1.0, priority=1.0),
            dict(struct_bit=1, kind="DOSE_MIN", bound=9.0, priority=1.0)]
    P = small_problem(D, D, [1, 2], cons)
    xn = oracle.sequential_ams_sweep(oracle.constraint_rows(P), [1.0, 1.0, 1.0, 1.0], 1.0)
    dose, _ = oracle.forward(P, xn)
    np.testing.assert_allclose(dose, [1.0, 9.0], rtol=1e-14)


# ------------------------------------------------------------ block-iterative sweep (R13)

@pytest.mark.parametrize("norm", ["all", "violated"])
def test_block_sweep_single_block_is_cimmino(norm):
    P, rng = _rand_problem(51)
    R = oracle.constraint_rows(P)
    x = rng.uniform(0.0, 3.0, P.n_spots)
    one = [np.arange(R.A.shape[0])]
    np.testing.assert_allclose(oracle.block_iterative_sweep(R, x, 1.3, one, prio_scale=0.7, norm=norm),
                               oracle.cimmino_step(R, x, 1.3, prio_scale=0.7, norm=norm), rtol=1e-13, atol=1e-15)


def test_block_sweep_singletons_are_the_row_action_sweep():
    """One row per block with unit priorities is Fig. 2's sweep row by row."""
    P, rng = _rand_problem(52)
    for c in P.constraints:
        c["priority"] = 1.0
    R = oracle.constraint_rows(P)
    x = rng.uniform(0.0, 3.0, P.n_spots)
    singles = [np.array([r]) for r in range(R.A.shape[0])]
    np.testing.assert_allclose(oracle.block_iterative_sweep(R, x, 1.0, singles),
                               oracle.sequential_ams_sweep(R, x, 1.0), rtol=1e-13, atol=1e-15)


def test_block_sweep_later_block_sees_earlier_update():
    """Two blocks sharing a spot: the second block projects from the point the
    first block produced, so its row lands exactly on its bound (lam = 1)."""
    D = [[1.0, 1.0, 0.0], [0.0, 1.0, 1.0]]
    cons = [dict(struct_bit=0, kind="DOSE_MAX", bound=1.0, priority=1.0),
            dict(struct_bit=1, kind="DOSE_MIN", bound=5.0, priority=1.0)]
    P = small_problem(D, D, [1, 2], cons)
    R = oracle.constraint_rows(P)
    x = np.array([1.0, 1.0, 1.0])
    xn = oracle.block_iterative_sweep(R, x, 1.0, [np.array([0]), np.array([1])])
    dose, _ = oracle.forward(P, xn)
    assert abs(dose[1] - 5.0) < 1e-14            # the last projection is exact
    x1 = x + (1.0 - 2.0) / 2.0 * np.array([1.0, 1.0, 0.0])  # first block by hand
    x2 = x1 + (5.0 - (x1[1] + x1[2])) / 2.0 * np.array([0.0, 1.0, 1.0])
    np.testing.assert_allclose(xn, np.maximum(x2, 0.0), rtol=1e-15)


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.9])
def test_block_sweep_fejer_monotone(lam):
    rng = np.random.default_rng(53)
    n_vox, n = 16, 6
    D = rng.uniform(0.05, 1.0, (n_vox, n))
    L = rng.uniform(1.0, 10.0, (n_vox, n)) * D
    z = rng.uniform(0.2, 1.0, n)
    dz, lz = D @ z, L @ z
    mask = np.ones(n_vox, np.uint32) * 3
    mask[::3] = 1
    cons = [dict(struct_bit=0, kind="DOSE_MAX", bound=float(dz.max()) * 1.01, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MIN", bound=float(dz.min()) * 0.99, priority=2.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=float((lz / dz).max()) * 1.01, priority=1.0)]
    P = small_problem(D, L, mask, cons)
    R = oracle.constraint_rows(P)
    for trial in range(10):
        x = rng.uniform(0.0, 4.0, n)
        for nb in (2, 5, 16):
            for norm in ("all", "violated"):
                xn = oracle.block_iterative_sweep(R, x, lam, oracle.sweep_blocks(P, R, nb), norm=norm)
                assert np.linalg.norm(xn - z) <= np.linalg.norm(x - z) + 1e-12


def test_sweep_blocks_group_consecutive_structure_voxels(tiny):
    pl, P, R = tiny
    nz = np.diff(pl.row_ptr) > 0
    C = [v for v in range(pl.n_vox) if pl.mask[v] != 0 and nz[v]]
    for nb in (1, 3, 7, 64, len(C) + 5):
        blocks = oracle.sweep_blocks(P, R, nb)
        S = -(-len(C) // nb)
        assert len(blocks) == -(-len(C) // S) and len(blocks) <= nb
        seen = np.concatenate(blocks)
        assert sorted(seen.tolist()) == list(range(R.A.shape[0]))   # a partition of the rows
        pos = {v: i for i, v in enumerate(C)}
        for b, B in enumerate(blocks):
            for r in B:
                assert pos[int(R.voxel[r])] // S == b                 # voxel group of S


def test_superiorize_with_one_sweep_block_is_plain_superiorize(tiny):
    pl, P, R = tiny
    w_a, log_a = oracle.superiorize(P, pl.w0, 4, pl.alpha, pl.relaxation, rows=R)
    w_b, log_b = oracle.superiorize(P, pl.w0, 4, pl.alpha, pl.relaxation, rows=R, sweep=1)
    np.testing.assert_allclose(w_b, w_a, rtol=1e-12, atol=1e-14)
    assert [e["s"] for e in log_a] == [e["s"] for e in log_b]


# ------------------------------------------------------------ inputs

def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            out = phantom.philox4x32_10(w[0:4], w[4:6])
            assert out.tolist() == w[6:10]


def test_tiny_masks_by_integer_geometry():
    m = phantom.tiny_masks()
    n_ball = 0
    for k in range(32):
        for j in range(32):
            for i in range(32):
                inside = (i - 16) ** 2 + (j - 16) ** 2 + (k - 16) ** 2 <= 64
                n_ball += inside
                assert bool(m[(k * 32 + j) * 32 + i] & 1) == inside
    assert n_ball == int((m & 1).astype(bool).sum())
    n_cyl = sum(1 for k in range(32) for i in range(32) if (i - 16) ** 2 + (k - 29) ** 2 <= 16) * 32
    assert int(((m >> 1) & 1).sum()) == n_cyl


def test_generator_physics():
    """Noise-free tiny plan: w = 1 gives 2 Gy at the isocentre; the dose
    peaks near the nominal range; LET rises toward the end of range; L/D is
    the per-element LET and is the same for the noise-free and noisy D."""
    p = phantom.tiny_params(noise=0.0)
    rp, col, D, L = phantom.generate(p)
    P = oracle.build_problem(rp, col, D, L, 2250, np.zeros(32 ** 3, np.uint32), [], [])
    dose, _ = oracle.forward(P, np.ones(2250))
    # exact up to the entries dropped by the 1e-4 truncation
    assert dose[(16 * 32 + 16) * 32 + 16] == pytest.approx(2.0, rel=2e-3)
    dd, let = phantom.layer_table(p, 0, 9)
    R_mm = p.range_last_mm[0]
    z_peak = np.argmax(dd) * 0.1
    assert R_mm - 3.0 < z_peak <= R_mm
    i_mid = int(0.5 * R_mm / 0.1)
    i_peak = int(z_peak / 0.1)
    assert let[i_mid] < let[i_peak] <= 15.0
    rp2, col2, D2, L2 = phantom.generate(phantom.tiny_params(noise=0.01))
    np.testing.assert_array_equal(rp2, rp)
    np.testing.assert_array_equal(col2, col)
    assert np.max(np.abs(D2 / D - 1)) <= 0.0100001
