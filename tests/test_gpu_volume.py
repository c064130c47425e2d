"""Parity of the volume statistics (Sec. 2.4.1: DVH, LVH, cDLVH, the value
received by a fraction of a structure's volume, the PTV coverage rule and the
cDL30 limits) with the oracle, through the C ABI.

Tolerances: the voxel maps are FP64 sums of the stored FP32 values rounded
once to FP32, so they sit within 1e-6 relative (plus 1e-12 absolute) of the
oracle's FP64 values.  Counts and values at volume are integer decisions
taken on those FP32 maps: they are compared bit for bit with the oracle run
on the same FP32 maps.
"""
import math

import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu

QTY = {"DOSE": "dose", "CDL": "cdl", "LETD": "letd"}
FRACS = [1e-6, 0.02, 0.05, 0.14, 0.3, 0.5, 0.95, 0.98, 1.0]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt


@pytest.fixture(scope="module")
def tiny():
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    w = np.random.default_rng(11).uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    return pl, P, w


def edges_for(values, mask, bit, n):
    """Bins whose inner edges include values that occur in the map (half-open test)."""
    v = np.sort(values[oracle.structure_voxels(mask, bit)])
    hi = float(v[-1]) if len(v) else 1.0
    e = np.linspace(0.0, hi * 1.01 + 1e-6, n + 1).astype(np.float32)
    if len(v) > 10:
        e[1:-1:7] = v[np.linspace(0, len(v) - 1, len(e[1:-1:7])).astype(int)]
        e = np.maximum.accumulate(e)
    e[-1] = np.inf
    return e


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_maps_match_oracle_and_final_outputs(lib, tiny, rows):
    pl, P, w = tiny
    with lib.Handle(0) as h:
        h.load_plan(pl, rows=rows)
        maps = {q: h.quantity_map(w, q) for q in QTY}
        _, dose, letd, _ = h.superiorize(w, 0, pl.alpha, pl.relaxation)
    for q, m in maps.items():
        ref = oracle.quantity(P, w, QTY[q])
        assert m.dtype == np.float32 and m.shape == (pl.n_vox,)
        assert np.all(np.abs(m - ref) <= 1e-6 * np.abs(ref) + 1e-12), q
    # the maps are the final pass's own outputs, bit for bit
    np.testing.assert_array_equal(maps["DOSE"], dose)
    np.testing.assert_array_equal(maps["LETD"], letd)


@pytest.mark.parametrize("rows", ["all", "roi"])
def test_histograms_and_values_at_volume_bit_exact(lib, tiny, rows):
    pl, P, w = tiny
    with lib.Handle(0) as h:
        h.load_plan(pl, rows=rows)
        maps = {q: h.quantity_map(w, q) for q in QTY}
        reqs = []
        for bit in (0, 1):
            for q in QTY:
                reqs.append({"quantity": q, "struct_bit": bit, "edges": edges_for(maps[q], pl.mask, bit, 50),
                             "fracs": FRACS})
        res = h.volume_stats(reqs, w)
    for r, out in zip(reqs, res):
        m = maps[r["quantity"]]
        n = len(oracle.structure_voxels(pl.mask, r["struct_bit"]))
        assert out["n_voxels"] == n
        np.testing.assert_array_equal(out["counts"], oracle.volume_histogram(m, pl.mask, r["struct_bit"], r["edges"]))
        want = [oracle.value_at_volume(m, pl.mask, r["struct_bit"], f) for f in FRACS]
        np.testing.assert_array_equal(out["at_volume"], np.array(want, np.float32))


def test_ties_negative_edges_and_empty_structure(lib):
    # every voxel of structure 0 gets the same dose (ties), structure 5 is empty
    V, n = 300, 4
    rp = np.arange(V + 1, dtype=np.int64)
    col = (np.arange(V) % n).astype(np.int32)
    D = np.ones(V, np.float32)
    L = np.full(V, 3.0, np.float32)
    mask = np.where(np.arange(V) < 200, 1, 2).astype(np.uint32)
    w = np.ones(n, np.float32)
    with lib.Handle(0) as h:
        h.load_influence(rp, col, D, L, mask, n)
        res = h.volume_stats([
            {"quantity": "DOSE", "struct_bit": 0, "edges": [-np.inf, -1.0, 1.0, 1.0, 2.0], "fracs": [0.5, 1.0]},
            {"quantity": "LETD", "struct_bit": 1, "edges": [0.0, 3.0, np.inf], "fracs": [1e-3]},
            {"quantity": "CDL", "struct_bit": 5, "edges": [0.0, 1.0], "fracs": [0.3]},
        ], w)
    assert res[0]["n_voxels"] == 200
    assert res[0]["counts"].tolist() == [0, 0, 0, 200]  # [1, 1) is empty, 1.0 falls in [1, 2)
    assert res[0]["at_volume"].tolist() == [1.0, 1.0]
    assert res[1]["n_voxels"] == 100 and res[1]["counts"].tolist() == [0, 100]
    assert res[1]["at_volume"][0] == np.float32(3.0)
    assert res[2]["n_voxels"] == 0 and res[2]["counts"].tolist() == [0]
    assert math.isnan(res[2]["at_volume"][0])


def test_current_iterate_device_pointer_and_bf16(lib, tiny):
    import torch
    pl, P, w = tiny
    reqs = [{"quantity": "CDL", "struct_bit": 1, "edges": np.linspace(0, 0.2, 41, dtype=np.float32),
             "fracs": [0.3, 0.98]}]
    with lib.Handle(0) as h:
        h.load_plan(pl)
        h.begin(pl.w0, pl.alpha, pl.relaxation)
        h.iterate(5)
        cur = h.volume_stats(reqs)  # the current iterate
        w5, _, _, _ = h.end()
        host = h.volume_stats(reqs, w5)
        dev = h.volume_stats(reqs, torch.from_numpy(w5).cuda())
        dmap = h.quantity_map(torch.from_numpy(w5).cuda(), "CDL")
        hmap = h.quantity_map(w5, "CDL")
    for a in (host, dev):
        np.testing.assert_array_equal(cur[0]["counts"], a[0]["counts"])
        np.testing.assert_array_equal(cur[0]["at_volume"], a[0]["at_volume"])
    np.testing.assert_array_equal(dmap.cpu().numpy(), hmap)
    # 16-bit storage: the statistics are still exact functions of the map
    with lib.Handle(0) as h:
        h.load_plan(pl, fmt="bf16")
        m = h.quantity_map(w, "DOSE")
        r = h.volume_stats([{"quantity": "DOSE", "struct_bit": 0, "edges": edges_for(m, pl.mask, 0, 30),
                             "fracs": FRACS}], w)[0]
    np.testing.assert_array_equal(r["counts"], oracle.volume_histogram(m, pl.mask, 0, edges_for(m, pl.mask, 0, 30)))
    np.testing.assert_array_equal(r["at_volume"],
                                  np.array([oracle.value_at_volume(m, pl.mask, 0, f) for f in FRACS], np.float32))


def test_cdl30_limits_and_coverage(lib, tiny):
    pl, P, w = tiny
    with lib.Handle(0) as h:
        h.load_plan(pl)
        cons = h.derive_cdl_limits(w, [1])
        cmap = h.quantity_map(w, "CDL")
        dmap = h.quantity_map(w, "DOSE")
        d98, n_cov, n_ptv, ok = h.coverage(0, 2.0, w)
    ref = oracle.derive_cdl_limits(P, w, [1])
    assert cons[0]["kind"] == "CDL_MAX" and cons[0]["struct_bit"] == 1
    assert cons[0]["bound"] == float(oracle.value_at_volume(cmap, pl.mask, 1, 0.3))
    assert abs(cons[0]["bound"] - ref[0]["bound"]) <= 1e-6 * abs(ref[0]["bound"]) + 1e-12
    assert d98 == float(oracle.value_at_volume(dmap, pl.mask, 0, 0.98))
    t = np.float32(0.95 * 2.0)
    assert n_cov == int(np.count_nonzero(dmap[oracle.structure_voxels(pl.mask, 0)] >= t))
    assert n_ptv == len(oracle.structure_voxels(pl.mask, 0))
    assert ok == (n_cov >= oracle.at_volume_rank(0.98, n_ptv))  # the two statements of the rule agree


def test_request_errors_leave_handle_usable(lib, tiny):
    pl, P, w = tiny
    bad = [
        [{"quantity": "DOSE", "struct_bit": 32}],
        [{"quantity": "DOSE", "struct_bit": 0, "edges": [1.0, 0.5]}],
        [{"quantity": "DOSE", "struct_bit": 0, "edges": [0.0, np.nan, 1.0]}],
        [{"quantity": "DOSE", "struct_bit": 0, "fracs": [0.0]}],
        [{"quantity": "DOSE", "struct_bit": 0, "fracs": [1.5]}],
        [{"quantity": "DOSE", "struct_bit": 0, "edges": np.arange(lib.VOLUME_MAX_BINS + 2, dtype=np.float32)}],
        [{"quantity": "DOSE", "struct_bit": 0, "fracs": [0.5] * (lib.VOLUME_MAX_FRACS + 1)}],
        [{"quantity": "DOSE", "struct_bit": 0}] * (lib.VOLUME_MAX_REQUESTS + 1),
    ]
    with lib.Handle(0) as h:
        h.load_plan(pl)
        for reqs in bad:
            with pytest.raises(lib.FredoptError) as e:
                h.volume_stats(reqs, w)
            assert e.value.code == -1
        with pytest.raises(lib.FredoptError):
            h.volume_stats([{"quantity": "DOSE", "struct_bit": 0}])  # no begun solve, w = None
        out = np.empty(pl.n_vox, np.float32)
        assert h.lib.fredopt_quantity_map(h.h, w.ctypes.data, 7, out.ctypes.data, 0) == -1  # unknown quantity
        assert h.lib.fredopt_quantity_map(h.h, w.ctypes.data, 0, None, 0) == -1             # no output
        ok = h.volume_stats([{"quantity": "DOSE", "struct_bit": 0, "fracs": [0.5]}], w)
    assert ok[0]["n_voxels"] == len(oracle.structure_voxels(pl.mask, 0))


def test_clinical_volume_stats(lib):
    pl = phantom.clinical_plan()
    rng = np.random.default_rng(12)
    w = rng.uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        maps = {q: h.quantity_map(w, q) for q in QTY}
        reqs = [{"quantity": q, "struct_bit": b, "edges": edges_for(maps[q], pl.mask, b, 200), "fracs": FRACS}
                for b in range(4) for q in QTY]
        res = h.volume_stats(reqs[:6], w) + h.volume_stats(reqs[6:], w)  # at most 64 fractions per call
    for r, out in zip(reqs, res):
        m = maps[r["quantity"]]
        assert out["n_voxels"] == len(oracle.structure_voxels(pl.mask, r["struct_bit"]))
        np.testing.assert_array_equal(out["counts"], oracle.volume_histogram(m, pl.mask, r["struct_bit"], r["edges"]))
        want = [oracle.value_at_volume(m, pl.mask, r["struct_bit"], f) for f in FRACS]
        np.testing.assert_array_equal(out["at_volume"], np.array(want, np.float32))
    # sampled voxels of the maps against FP64 dot products of the CSR rows
    sample = rng.choice(np.nonzero(pl.mask)[0], 400, replace=False)
    w64 = w.astype(np.float64)
    for i in sample:
        s, e = pl.row_ptr[i], pl.row_ptr[i + 1]
        c = pl.col[s:e]
        d = float(pl.D[s:e].astype(np.float64) @ w64[c])
        lw = float(pl.L[s:e].astype(np.float64) @ w64[c])
        assert abs(maps["DOSE"][i] - d) <= 1e-6 * abs(d) + 1e-12
        assert abs(maps["CDL"][i] - oracle.C_CDL * lw) <= 1e-6 * abs(oracle.C_CDL * lw) + 1e-12
        let = lw / d if d > 0 else 0.0
        assert abs(maps["LETD"][i] - let) <= 1e-6 * abs(let) + 1e-12
