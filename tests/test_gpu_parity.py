"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: bit-exact for masks, row order, sparsity pattern and the CSC
copy; <= 1e-5 relative for one FP32 product (relative to the sum of absolute
products of the row or column, which equals |result| for nonnegative
operands); <= 1e-4 relative L2 for w after 100 iterations; final constraint
violations and dose within 1e-4 x prescription (2 Gy) of the oracle's.
"""
import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu

PRESC = 2.0


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt


@pytest.fixture(scope="module")
def tiny():
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints,
                             pl.objective)
    return pl, P, oracle.constraint_rows(P)


def handle(lib, plan, fmt="fp32", rows="all"):
    h = lib.Handle(0)
    h.load_plan(plan, fmt=fmt, rows=rows)
    return h


def abs_sum_bound(Mabs, xabs):
    return Mabs @ xabs


def hot_rows(plan, rows):
    """Streamed rows in device order: rows with nonzeros, then rows without,
    each ascending by voxel."""
    hot = np.ones(plan.n_vox, bool) if rows == "all" else plan.mask != 0
    nz = np.diff(plan.row_ptr) > 0
    return np.concatenate([np.nonzero(hot & nz)[0], np.nonzero(hot & ~nz)[0]])


# ---------------------------------------------------------------- setup (K5)

@pytest.mark.parametrize("rows", ["all", "roi"])
def test_rows_masks_bit_exact(lib, tiny, rows):
    pl, P, R = tiny
    with handle(lib, pl, rows=rows) as h:
        vox, mask = h.get_rows()
    np.testing.assert_array_equal(vox, hot_rows(pl, rows))
    np.testing.assert_array_equal(mask, pl.mask[vox])


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_csc_bit_exact(lib, tiny, rows):
    pl, P, R = tiny
    hr = hot_rows(pl, rows)
    sub_D = P.D[hr]
    sub_L = P.L[hr]
    rp = sub_D.indptr.astype(np.int64)
    col = sub_D.indices.astype(np.int32)
    Dv = sub_D.data.astype(np.float32)
    Lv = sub_L.data.astype(np.float32)
    cp, row, DT, LT = oracle.transpose_csr(rp, col, pl.n_spots, Dv, Lv)
    with handle(lib, pl, rows=rows) as h:
        gcp, grow, gD, gL = h.get_csc()
    np.testing.assert_array_equal(gcp, cp)
    np.testing.assert_array_equal(grow, row)
    np.testing.assert_array_equal(gD.view(np.uint32), DT.view(np.uint32))
    np.testing.assert_array_equal(gL.view(np.uint32), LT.view(np.uint32))


def _csc_of_device_rows(rp, col, D, L, n_cols):
    """The CSC copy the library must build: rows with nonzeros first, then
    the rest (ALL-row mode), transposed stably.  Moving the empty rows back
    keeps the nonzero stream in its order."""
    lens = np.diff(rp)
    lens = np.concatenate([lens[lens > 0], lens[lens == 0]])
    rp2 = np.zeros(len(lens) + 1, np.int64)
    rp2[1:] = np.cumsum(lens)
    return oracle.transpose_csr(rp2, col, n_cols, D, L)


@pytest.mark.parametrize("case", ["wide", "long_rows", "many_short_rows"])
@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
def test_csc_bit_exact_shapes(lib, case, fmt):
    """Shapes that take the transpose's other paths: column tables too large
    for shared memory (the row-by-row fill with bulk-copy windows), 16-row
    steps with more entries than the registers hold (the loop form of the
    row-step fill), and blocks with more rows than one staged row-pointer
    chunk."""
    rng = np.random.default_rng(17)
    if case == "wide":
        rp, col, D, L = phantom.random_csr(300, 60000, 0.02, seed=1, empty_rows=20)
    elif case == "long_rows":
        n_cols, lens = 30000, [25000, 3, 29999, 0, 17000, 1]
        cols = [np.sort(rng.choice(n_cols, k, replace=False)).astype(np.int32) for k in lens]
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        col = np.concatenate(cols)
        D = rng.uniform(0.1, 1.0, len(col)).astype(np.float32)
        L = (D * rng.uniform(1.0, 9.0, len(col))).astype(np.float32)
    else:
        n = 400000
        c1 = rng.integers(0, 32, n)
        c2 = rng.integers(32, 64, n)
        col = np.stack([c1, c2], 1).ravel().astype(np.int32)
        rp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
        D = rng.uniform(0.1, 1.0, 2 * n).astype(np.float32)
        L = (D * rng.uniform(1.0, 9.0, 2 * n)).astype(np.float32)
    n_cols = int(col.max()) + 1 if len(col) else 1
    n_cols = max(n_cols, 60000 if case == "wide" else n_cols)
    mask = np.ones(len(rp) - 1, np.uint32)
    with lib.Handle(0) as h:
        h.load_influence(rp, col, D, L, mask, n_cols, fmt=fmt)
        gcp, grow, gD, gL = h.get_csc()
        if fmt != "fp32":
            vox, _ = h.get_rows()
    if fmt == "fp32":
        cp, row, DT, LT = _csc_of_device_rows(rp, col, D, L, n_cols)
        np.testing.assert_array_equal(gcp, cp)
        np.testing.assert_array_equal(grow, row)
        np.testing.assert_array_equal(gD.view(np.uint32), DT.view(np.uint32))
        np.testing.assert_array_equal(gL.view(np.uint32), LT.view(np.uint32))
    else:
        # pattern and row order bit-exact; values are the dequantised stored values
        cp, row, DT, LT = _csc_of_device_rows(rp, col, D, L, n_cols)
        np.testing.assert_array_equal(gcp, cp)
        np.testing.assert_array_equal(grow, row)
        assert np.all(np.abs(gD - DT) <= 2.0 ** -8 * np.abs(DT) * 1.0001)


def test_moments_fp64(lib, tiny):
    pl, P, R = tiny
    with handle(lib, pl, rows="roi") as h:
        dd, ll, dl = h.get_moments()
    hr = hot_rows(pl, "roi")
    D, L = P.D[hr], P.L[hr]
    np.testing.assert_allclose(dd, np.asarray(D.multiply(D).sum(1)).ravel(), rtol=1e-12)
    np.testing.assert_allclose(ll, np.asarray(L.multiply(L).sum(1)).ravel(), rtol=1e-12)
    np.testing.assert_allclose(dl, np.asarray(D.multiply(L).sum(1)).ravel(), rtol=1e-12)


# ---------------------------------------------------------------- single passes

@pytest.mark.parametrize("rows", ["all", "roi"])
def test_forward_fp32(lib, tiny, rows):
    pl, P, R = tiny
    rng = np.random.default_rng(1)
    w = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    with handle(lib, pl, rows=rows) as h:
        dose, lw = h.forward(w)
    d_ref, l_ref = oracle.forward(P, w)
    np.testing.assert_array_less(np.abs(dose - d_ref), 1e-5 * np.abs(d_ref) + 1e-30)
    np.testing.assert_array_less(np.abs(lw - l_ref), 1e-5 * np.abs(l_ref) + 1e-30)
    # signed input: bound by the sum of absolute products
    w2 = rng.normal(size=pl.n_spots).astype(np.float32)
    with handle(lib, pl, rows=rows) as h:
        dose, lw = h.forward(w2)
    d_ref, l_ref = oracle.forward(P, w2)
    bd = abs(P.D) @ np.abs(w2.astype(np.float64))
    bl = abs(P.L) @ np.abs(w2.astype(np.float64))
    assert np.all(np.abs(dose - d_ref) <= 1e-5 * bd + 1e-30)
    assert np.all(np.abs(lw - l_ref) <= 1e-5 * bl + 1e-30)


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_backward_fp32(lib, tiny, rows):
    pl, P, R = tiny
    rng = np.random.default_rng(2)
    aD = rng.normal(size=pl.n_vox).astype(np.float32)
    aL = rng.normal(size=pl.n_vox).astype(np.float32)
    hr = hot_rows(pl, rows)
    mD = np.zeros(pl.n_vox)
    mL = np.zeros(pl.n_vox)
    mD[hr] = aD[hr]
    mL[hr] = aL[hr]
    ref = P.D.T @ mD + P.L.T @ mL
    bound = abs(P.D).T @ np.abs(mD) + abs(P.L).T @ np.abs(mL)
    with handle(lib, pl, rows=rows) as h:
        u = h.backward(aD, aL)
    assert np.all(np.abs(u - ref) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("norm", ["all", "violated"])
def test_feasibility_step(lib, tiny, norm):
    pl, P, R = tiny
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    for lam, ps in ((1.0, 1.0), (1.7, 0.6)):
        ref = oracle.cimmino_step(R, x, lam, prio_scale=ps, norm=norm)
        with handle(lib, pl) as h:
            got = h.feasibility_step(x, lam, ps, norm)
        step = np.linalg.norm(ref - x)
        assert np.linalg.norm(got - ref) <= 1e-5 * max(step, 1e-12) + 1e-6 * np.linalg.norm(ref)


def test_objective_and_gradient(lib, tiny):
    pl, P, R = tiny
    rng = np.random.default_rng(4)
    x = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    P2 = oracle.Problem(P.D, P.L, P.mask, P.constraints,
                        [dict(struct_bit=0, quantity="DOSE", target=2.0, weight=0.5)] + list(pl.objective))
    for prob, terms in ((P, pl.objective), (P2, P2.objective)):
        with lib.Handle(0) as h:
            h.load_plan(pl)
            h.set_objective(terms)
            f, g = h.objective(x)
        f_ref = oracle.objective(prob, x)
        g_ref = oracle.objective_gradient(prob, x)
        assert f == pytest.approx(f_ref, rel=1e-5)
        assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)


# ---------------------------------------------------------------- whole loop

def run_gpu(lib, pl, iters, rows="all", fmt="fp32", **params):
    with handle(lib, pl, fmt=fmt, rows=rows) as h:
        w, dose, letd, rep = h.superiorize(pl.w0, iters, pl.alpha, pl.relaxation, **params)
        log = h.get_log()
    return w, dose, letd, rep, log


def violation_by_kind(pl, P, w):
    dose, lw = oracle.forward(P, w)
    let = oracle.letd(dose, lw)
    out = {}
    for ci, c in enumerate(pl.constraints):
        sel = ((pl.mask >> np.uint32(c["struct_bit"])) & 1).astype(bool)
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


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_superiorize_100_iterations(lib, tiny, rows):
    pl, P, R = tiny
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 100, pl.alpha, pl.relaxation, rows=R)
    w, dose, letd, rep, log = run_gpu(lib, pl, 100, rows=rows)
    rel = np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)
    assert rel <= 1e-4, rel
    # identical accept/reject decisions and trial counters
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert [e["accepted"] for e in log] == [e["accepted"] for e in log_ref]
    for e, r in zip(log, log_ref):
        assert e["f_end"] <= e["f_start"]
        assert e["f_start"] == pytest.approx(r["f_start"], rel=1e-4, abs=1e-12)
    d_ref, l_ref = oracle.forward(P, w_ref)
    assert np.max(np.abs(dose - d_ref)) <= 1e-4 * PRESC
    vg = violation_by_kind(pl, P, w.astype(np.float64))
    vr = violation_by_kind(pl, P, w_ref)
    for ci in vr:
        # dose: 1e-4 of prescription; LETd (keV/um, up to 15): the 1e-4 relative
        # tolerance of w carried to a 15 keV/um LETd, rounded up
        tol = 1e-4 * PRESC if pl.constraints[ci]["kind"].startswith("DOSE") else 2e-3
        assert abs(vg[ci] - vr[ci]) <= tol, (ci, vg[ci], vr[ci])
    assert rep["iters"] == 100
    assert rep["objective"] == pytest.approx(oracle.objective(P, w.astype(np.float64)), rel=1e-9)
    assert rep["unreachable_rows"] == R.unreachable
    assert rep["n_rows"] == R.A.shape[0]


def test_plain_cimmino_matches(lib, tiny):
    pl, P, R = tiny
    w_ref, _ = oracle.superiorize(P, pl.w0, 30, pl.alpha, pl.relaxation, rows=R, reductions=0)
    w, *_ = run_gpu(lib, pl, 30, reductions=0)
    assert np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref) <= 1e-4


@pytest.mark.parametrize("opts", [dict(reductions=2), dict(eta=0.95), dict(cimmino_norm="violated"),
                                  dict(grad_normalize=0, beta0=50.0), dict(beta0=1.0, max_trials=3)],
                         ids=["N2", "eta", "violated", "raw_grad", "cap"])
def test_variants_match(lib, tiny, opts):
    pl, P, R = tiny
    o = dict(opts)
    norm = o.pop("cimmino_norm", "all")
    kw = dict(eta=o.get("eta", 1.0), reductions=o.get("reductions", 1), norm=norm,
              grad_normalize=bool(o.get("grad_normalize", 1)), max_trials=o.get("max_trials", 50))
    if "beta0" in o:
        kw["beta0"] = o["beta0"]
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 15, pl.alpha, pl.relaxation, rows=R, **kw)
    w, d, l, rep, log = run_gpu(lib, pl, 15, cimmino_norm=norm, **o)
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref) <= 1e-4


def test_deterministic_and_graph_equals_plain(lib, tiny):
    pl, P, R = tiny
    w1, *_ = run_gpu(lib, pl, 20)
    w2, *_ = run_gpu(lib, pl, 20)
    w3, *_ = run_gpu(lib, pl, 20, use_graphs=0)
    np.testing.assert_array_equal(w1, w2)
    np.testing.assert_array_equal(w1, w3)


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_claimed_tiles_equal_static_tiles(lib, tiny, rows):
    """Warps claiming row tiles dynamically (the default) and one static tile
    per warp give bit-identical iterates: a row's sums do not depend on the
    warp that streams them.  The FP64 objective adds per-tile partials, so
    the two tilings may group its sum differently (last-bit differences)."""
    pl, P, R = tiny
    w1, d1, l1, rep1, log1 = run_gpu(lib, pl, 12, rows=rows, tile_balance=2)
    w0, d0, l0, rep0, log0 = run_gpu(lib, pl, 12, rows=rows, tile_balance=0)
    np.testing.assert_array_equal(w1, w0)
    np.testing.assert_array_equal(d1, d0)
    for a, b in zip(log1, log0):
        for k in a:
            if k in ("f_start", "f_end"):
                assert a[k] == pytest.approx(b[k], rel=1e-14, abs=0)
            else:
                assert a[k] == b[k], k
    # each tiling on its own is deterministic, objective included
    w2, *_, log2 = run_gpu(lib, pl, 12, rows=rows, tile_balance=2)
    np.testing.assert_array_equal(w2, w1)
    assert log2 == log1


@pytest.mark.parametrize("fmt", ["fp32", "bf16"])
@pytest.mark.parametrize("rows", ["all", "roi"])
def test_index16_equals_index32(lib, tiny, fmt, rows):
    """16-bit indices (forward columns when the spots fit; transposed-product
    rows as offsets from per-block bases) and 32-bit ones stream the same
    elements in the same order: forward and transposed products, sweeps,
    iterates, logs and final outputs are bit-identical."""
    pl, P, R = tiny
    x = np.random.default_rng(11).uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    out = []
    for index32 in (False, True):
        with lib.Handle(0) as h:
            h.load_plan(pl, fmt=fmt, rows=rows, index32=index32)
            assert h.storage() == (4, 4, 4 if fmt == "fp32" else 2) if index32 else \
                h.storage() == (2, 2, 4 if fmt == "fp32" else 2)
            dose, lw = h.forward(x)
            u = h.backward(dose, lw)
            sw = h.sweep_step(x, 16)
            w, d, l, rep = h.superiorize(pl.w0, 15, pl.alpha, pl.relaxation)
            out.append((dose, lw, u, sw, w, d, l, h.get_log()))
    a, b = out
    for u, v in zip(a[:7], b[:7]):
        np.testing.assert_array_equal(u, v)
    assert a[7] == b[7]


@pytest.mark.parametrize("n_cols,index_bytes", [(1, 2), (58000, 2), (60000, 4), (70000, 4)])
def test_index_width_by_spot_count(lib, n_cols, index_bytes):
    """16-bit indices need x in the forward kernel's shared memory (up to about
    58000 spots); past that the forward keeps 32-bit indices and reads x
    through L1.  Both match FP64 products of the CSR rows."""
    rp, col, D, L = phantom.random_csr(300, n_cols, min(0.5, 40.0 / n_cols), seed=n_cols, empty_rows=7)
    mask = np.ones(300, np.uint32)
    x = np.random.default_rng(2).uniform(0.0, 2.0, n_cols).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_influence(rp, col, D, L, mask, n_cols)
        assert h.storage()[0] == index_bytes
        dose, lw = h.forward(x)
    x64 = x.astype(np.float64)
    for i in range(300):
        s, e = rp[i], rp[i + 1]
        d_ref = D[s:e].astype(np.float64) @ x64[col[s:e]]
        l_ref = L[s:e].astype(np.float64) @ x64[col[s:e]]
        assert abs(dose[i] - d_ref) <= 1e-5 * abs(d_ref) + 1e-30
        assert abs(lw[i] - l_ref) <= 1e-5 * abs(l_ref) + 1e-30


@pytest.mark.parametrize("n_rows,n_cols,density", [(300000, 20, 0.0004), (200000, 40, 0.01), (70000, 3, 0.9)])
def test_based_row_indices_wide_blocks(lib, n_rows, n_cols, density):
    """Transposed product with based 16-bit row indices on columns whose
    blocks of 128 nonzeros span 65536 rows or more (sparse columns over
    300000 rows; blocks across column boundaries): bit-identical to the
    32-bit stream and within 1e-5 of the FP64 column sums."""
    rp, col, D, L = phantom.random_csr(n_rows, n_cols, density, seed=n_rows + n_cols, empty_rows=11)
    mask = np.ones(n_rows, np.uint32)
    rng = np.random.default_rng(3)
    aD = rng.normal(size=n_rows).astype(np.float32)
    aL = rng.normal(size=n_rows).astype(np.float32)
    out = []
    for index32 in (False, True):
        with lib.Handle(0) as h:
            h.load_influence(rp, col, D, L, mask, n_cols, index32=index32)
            assert h.storage()[1] == (4 if index32 else 2)
            out.append(h.backward(aD, aL))
    np.testing.assert_array_equal(out[0], out[1])
    rows = np.repeat(np.arange(n_rows), np.diff(rp))
    tD = D.astype(np.float64) * aD[rows]
    tL = L.astype(np.float64) * aL[rows]
    ref = np.bincount(col, weights=tD + tL, minlength=n_cols)
    bound = np.bincount(col, weights=np.abs(tD) + np.abs(tL), minlength=n_cols)
    assert np.all(np.abs(out[0] - ref) <= 1e-5 * bound + 1e-30)


def test_checkpoint_resume_bit_exact(lib, tiny):
    pl, P, R = tiny
    with handle(lib, pl) as h:
        h.begin(pl.w0, pl.alpha, pl.relaxation)
        h.iterate(20)
        w_full, *_ = h.end()
    with handle(lib, pl) as h:
        h.begin(pl.w0, pl.alpha, pl.relaxation)
        h.iterate(10)
        w_mid, k, s = h.get_state()
    assert k == 10
    beta0 = 0.1 * float(np.linalg.norm(pl.w0.astype(np.float64)))
    with handle(lib, pl) as h:
        h.begin(w_mid, pl.alpha, pl.relaxation, beta0=beta0)
        h.set_state(w_mid, k, s)
        h.iterate(10)
        w_res, *_ = h.end()
    np.testing.assert_array_equal(w_res, w_full)


def test_trial_steps_past_the_step_table(lib, tiny):
    """The trial loop takes beta0 alpha^s from a table for s < 65536 and from
    the FP64 expression beyond: a solve resumed at s = 65526 crosses the end
    of the table and keeps the oracle's trial counters, decisions and w
    (Fig. 3; alpha = 0.9999 keeps the steps large enough to matter)."""
    pl, P, R = tiny
    alpha, s0, iters = 0.9999, 65536 - 10, 25
    beta0 = 0.1 * float(np.linalg.norm(pl.w0.astype(np.float64)))
    with handle(lib, pl) as h:
        h.begin(pl.w0, alpha, pl.relaxation, beta0=beta0)
        h.set_state(pl.w0, 0, s0)
        h.iterate(iters)
        w, *_ = h.end()
        log = h.get_log()
    w_ref, log_ref = oracle.superiorize(P, pl.w0, iters, alpha, pl.relaxation, beta0=beta0, rows=R, s0=s0)
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert [e["accepted"] for e in log] == [e["accepted"] for e in log_ref]
    assert log[0]["s"] < 65536 < log[-1]["s"]
    assert np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref) <= 1e-4


def test_device_pointers(lib, tiny):
    torch = pytest.importorskip("torch")
    pl, P, R = tiny
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    with lib.Handle(0) as h:
        h.load_influence(t(pl.row_ptr), t(pl.col), t(pl.D), t(pl.L), t(pl.mask.view(np.int32)), pl.n_spots)
        h.set_constraints(pl.constraints)
        h.set_objective(pl.objective)
        w, dose, letd, rep = h.superiorize(t(pl.w0), 10, pl.alpha, pl.relaxation)
        assert w.is_cuda
    w_host, *_ = run_gpu(lib, pl, 10)
    np.testing.assert_array_equal(w.cpu().numpy(), w_host)


# ---------------------------------------------------------------- precision

@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_quantized_storage(lib, tiny, fmt):
    """16-bit storage with power-of-two row scales: the product equals the
    FP64 product of the dequantised matrix within FP32 accumulation error,
    the CSC copy is the exact transpose of the stored values, and the dose
    error against the FP32 oracle is reported (bounded by the format)."""
    pl, P, R = tiny
    with handle(lib, pl, fmt=fmt) as h:
        cp, row, DT, LT = h.get_csc()
        vox, _ = h.get_rows()
        dose, lw = h.forward(pl.w0)
    # the dequantised matrix, rebuilt from the exact CSC values (CSC rows are
    # device rows; vox maps them to voxels)
    import scipy.sparse as sp
    Dq = sp.csc_matrix((DT.astype(np.float64), vox[row], cp), shape=(pl.n_vox, pl.n_spots))
    d_ref = Dq @ pl.w0.astype(np.float64)
    np.testing.assert_array_less(np.abs(dose - d_ref), 1e-5 * np.abs(d_ref) + 1e-30)
    # element-wise rounding of the stored values against the FP32 inputs, in device order
    sub = P.D[vox]
    cp32, row32, DT32 = oracle.transpose_csr(sub.indptr, sub.indices, pl.n_spots, sub.data.astype(np.float32))
    np.testing.assert_array_equal(row32, row)
    rel_elem = np.abs(DT.astype(np.float64) - DT32) / np.abs(DT32)
    assert rel_elem.max() <= (2.0 ** -8 if fmt == "bf16" else 2.0 ** -11) * 1.0001
    d32, _ = oracle.forward(P, pl.w0)
    err = np.max(np.abs(dose - d32)) / PRESC
    assert err <= (4e-3 if fmt == "bf16" else 5e-4)


# ---------------------------------------------------------------- edge cases

def small_plan(row_ptr, col, D, L, n_spots, mask, cons, obj, iters=5):
    return phantom.Plan(name="small", shape=(len(row_ptr) - 1, 1, 1), h_mm=1.0, params=None,
                        row_ptr=row_ptr, col=col, D=D, L=L, mask=mask, structures=[], constraints=cons,
                        objective=obj, w0=np.ones(n_spots, np.float32), iters=iters, alpha=0.9,
                        relaxation=1.0)


@pytest.mark.parametrize("n_rows,n_cols,density,empty", [(37, 5, 0.5, 4), (300, 129, 0.2, 30),
                                                         (1000, 1, 0.7, 100), (64, 3000, 0.3, 0)])
def test_ragged_random_plans(lib, n_rows, n_cols, density, empty):
    rp, col, D, L = phantom.random_csr(n_rows, n_cols, density, seed=n_rows + n_cols, empty_rows=empty)
    rng = np.random.default_rng(5)
    mask = rng.integers(0, 4, n_rows).astype(np.uint32)
    cons = [dict(struct_bit=0, kind="DOSE_MIN", bound=2.0, priority=1.0),
            dict(struct_bit=0, kind="DOSE_MAX", bound=3.0, priority=2.0),
            dict(struct_bit=1, kind="CDL_MAX", bound=0.5, priority=1.0),
            dict(struct_bit=1, kind="LETD_MAX", bound=4.0, priority=0.5)]
    obj = [dict(struct_bit=1, quantity="CDL", target=0.0, weight=1.0),
           dict(struct_bit=0, quantity="DOSE", target=2.5, weight=0.3)]
    pl = small_plan(rp, col, D, L, n_cols, mask, cons, obj)
    P = oracle.build_problem(rp, col, D, L, n_cols, mask, cons, obj)
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 8, 0.9, 1.0)
    for rows in ("all", "roi"):
        w, dose, letd, rep, log = run_gpu(lib, pl, 8, rows=rows)
        assert [e["s"] for e in log] == [e["s"] for e in log_ref]
        assert np.linalg.norm(w - w_ref) <= 1e-4 * max(np.linalg.norm(w_ref), 1e-12)
        d_ref, l_ref = oracle.forward(P, w_ref)
        np.testing.assert_allclose(dose, d_ref, rtol=1e-4, atol=1e-6)
        lt = oracle.letd(d_ref, l_ref)
        np.testing.assert_allclose(letd, lt, rtol=1e-4, atol=1e-6)


def test_empty_matrix_and_no_constraints(lib):
    rp = np.zeros(11, np.int64)
    pl = small_plan(rp, np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32), 6,
                    np.ones(10, np.uint32), [], [])
    w, dose, letd, rep, log = run_gpu(lib, pl, 3)
    np.testing.assert_array_equal(w, np.ones(6, np.float32))
    np.testing.assert_array_equal(dose, 0)
    np.testing.assert_array_equal(letd, 0)


def test_input_errors_leave_handle_usable(lib, tiny):
    pl, P, R = tiny
    bad_col = pl.col.copy()
    bad_col[5] = pl.n_spots + 3
    with lib.Handle(0) as h:
        with pytest.raises(lib.FredoptError) as e:
            h.load_influence(pl.row_ptr, bad_col, pl.D, pl.L, pl.mask, pl.n_spots)
        assert e.value.code == -3
        unsorted = pl.col.copy()
        r = int(np.nonzero(np.diff(pl.row_ptr) >= 2)[0][0])
        p0 = pl.row_ptr[r]
        unsorted[p0], unsorted[p0 + 1] = unsorted[p0 + 1], unsorted[p0]
        with pytest.raises(lib.FredoptError) as e:
            h.load_influence(pl.row_ptr, unsorted, pl.D, pl.L, pl.mask, pl.n_spots)
        assert e.value.code == -3
        nanD = pl.D.copy()
        nanD[7] = np.nan
        with pytest.raises(lib.FredoptError) as e:
            h.load_influence(pl.row_ptr, pl.col, nanD, pl.L, pl.mask, pl.n_spots)
        assert e.value.code == -4
        bad_rp = pl.row_ptr.copy()
        bad_rp[10] = bad_rp[11] + 1
        with pytest.raises(lib.FredoptError) as e:
            h.load_influence(bad_rp, pl.col, pl.D, pl.L, pl.mask, pl.n_spots)
        assert e.value.code == -3
        with pytest.raises(lib.FredoptError) as e:
            h.iterate(1)
        assert e.value.code == -5
        h.load_plan(pl)
        for bad in (dict(alpha=1.0), dict(alpha=0.0), dict(relaxation=2.5), dict(relaxation=0.0)):
            a = bad.get("alpha", 0.99)
            lam = bad.get("relaxation", 1.0)
            with pytest.raises(lib.FredoptError) as e:
                h.begin(pl.w0, a, lam)
            assert e.value.code == -1
        neg = pl.w0.copy()
        neg[0] = -1
        with pytest.raises(lib.FredoptError):
            h.begin(neg, 0.99, 1.0)
        with pytest.raises(lib.FredoptError):
            h.set_constraints([dict(struct_bit=40, kind="DOSE_MAX", bound=1.0, priority=1.0)])
        # still usable
        w, dose, letd, rep = h.superiorize(pl.w0, 5, 0.99, 1.0)
    w_ok, *_ = run_gpu(lib, pl, 5)
    np.testing.assert_array_equal(w, w_ok)


@pytest.mark.parametrize("use_graphs", [1, 0])
def test_launch_count_and_timing(lib, tiny, use_graphs):
    """Timed iterations, as graph replays with an event pair around each
    kernel or as plain launches: every kernel is counted and timed, and w is
    bit-identical to an untimed graph run."""
    pl, P, R = tiny
    with handle(lib, pl) as h:
        h.set_timing(True)
        h.begin(pl.w0, pl.alpha, pl.relaxation, use_graphs=use_graphs)
        h.iterate(1)
        h.iterate(3)
        w, *_ = h.end()
        t = h.get_timing()
        n = h.launch_count()
    # per iteration: 2 forward, 2 transposed, 2 column finishes, 1 scalar finish, 1 constraint kernel
    assert t["forward"][1] == 2 * 4 + 1
    assert t["backward"][1] == 2 * 4
    assert t["constraints"][1] == 4
    assert t["finish"][1] == 4
    assert n >= 8 * 4
    assert all(ms >= 0 for ms, c in t.values())
    assert t["forward"][0] > 0 and t["backward"][0] > 0
    w_ref, *_ = run_gpu(lib, pl, 4)
    np.testing.assert_array_equal(w, w_ref)


def test_final_pass_is_fp64_product_of_fp32_inputs(lib, tiny):
    """With FP32 storage the final pass (double-float accumulation: exact
    products, <= 3 * 2^-48 relative error per addition) equals the FP64
    oracle product up to the FP32 rounding of its outputs; bench.py uses it
    as the FP64-class reference of the 16-bit storage errors."""
    pl, P, R = tiny
    rng = np.random.default_rng(9)
    w = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    with handle(lib, pl) as h:
        h.begin(w, pl.alpha, pl.relaxation)
        w_out, dose, letd, rep = h.end()
    np.testing.assert_array_equal(w_out, w)
    d_ref, l_ref = oracle.forward(P, w)
    lt_ref = oracle.letd(d_ref, l_ref)
    np.testing.assert_allclose(dose, d_ref.astype(np.float32), rtol=2 ** -23, atol=0)
    sel = d_ref > 0
    np.testing.assert_allclose(letd[sel], lt_ref[sel].astype(np.float32), rtol=2 ** -22, atol=0)
    assert np.all(letd[~sel] == 0)


def test_loaded_code_is_sm_103a(lib):
    """The code object the CUDA runtime loads for the hot kernels is sm_103a
    SASS (cudaFuncGetAttributes binaryVersion 103), not a JIT of PTX for
    another architecture."""
    fwd, bwd, ptx = lib.kernel_arch(0)
    assert fwd == 103 and bwd == 103, (fwd, bwd, ptx)
