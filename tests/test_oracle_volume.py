"""Pins of the volume-statistics oracle (Sec. 2.4.1): histogram counts by
brute force, the value-at-volume by its defining property and by the closed
form on a permutation of 1..n, the equivalence of the two statements of the
PTV coverage rule, LETd and cDL identities, and the defining property of the
derived cDL30 limits."""
import math

import numpy as np
import pytest

import oracle
import phantom


def _brute_hist(values, mask, bit, edges):
    counts = [0] * (len(edges) - 1)
    for v, m in zip(values, mask):
        if not (int(m) >> bit) & 1:
            continue
        for b in range(len(edges) - 1):
            if edges[b] <= v < edges[b + 1]:
                counts[b] += 1
    return counts


def test_histogram_brute_force_and_half_open_edges():
    rng = np.random.default_rng(3)
    v = rng.integers(0, 10, 200).astype(np.float32) / 2  # many values sit exactly on an edge
    mask = rng.integers(0, 4, 200).astype(np.uint32)
    edges = np.array([0.0, 0.5, 1.0, 2.5, 4.0, np.inf], np.float32)
    for bit in (0, 1):
        got = oracle.volume_histogram(v, mask, bit, edges)
        assert got.tolist() == _brute_hist(v, mask, bit, edges)
        assert got.sum() == len(oracle.structure_voxels(mask, bit))
    # a value equal to an edge belongs to the bin that starts there
    assert oracle.volume_histogram(np.array([1.0]), np.array([1], np.uint32), 0, [0.0, 1.0, 2.0]).tolist() == [0, 1]


def test_cumulative_volume_matches_histogram_tail():
    rng = np.random.default_rng(4)
    v = rng.gamma(2.0, 1.0, 500)
    mask = np.ones(500, np.uint32)
    edges = np.concatenate([np.linspace(0, 8, 33), [np.inf]])
    counts = oracle.volume_histogram(v, mask, 0, edges)
    cum = oracle.cumulative_volume(v, mask, 0, edges[:-1])
    tail = np.cumsum(counts[::-1])[::-1] / 500.0
    np.testing.assert_array_equal(cum, tail)
    assert np.all(np.diff(cum) <= 0)


@pytest.mark.parametrize("n", [1, 7, 10, 50, 333])
def test_value_at_volume_closed_form_on_permutation(n):
    rng = np.random.default_rng(n)
    v = rng.permutation(np.arange(1, n + 1)).astype(np.float64)
    mask = np.ones(n, np.uint32)
    for j in range(1, n + 1):
        frac = float(f"{j / n:.12g}")  # the decimal a user would type for j of n voxels
        assert oracle.value_at_volume(v, mask, 0, frac) == n - j + 1
    assert oracle.value_at_volume(v, mask, 0, 1.0) == 1.0          # whole volume: the minimum
    assert oracle.value_at_volume(v, mask, 0, 1e-9) == float(n)    # vanishing volume: the maximum


def test_value_at_volume_is_largest_threshold_reaching_the_fraction():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(1, 40))
        v = rng.integers(0, 6, n).astype(np.float64)  # ties
        mask = np.ones(n, np.uint32)
        frac = float(rng.choice([0.02, 0.05, 0.3, 0.5, 0.95, 0.98, 1.0, rng.uniform(0.01, 1)]))
        need = oracle.at_volume_rank(frac, n)
        # brute force over thresholds: the largest d with #(v >= d) >= need
        best = max(d for d in v if np.count_nonzero(v >= d) >= need)
        assert oracle.value_at_volume(v, mask, 0, frac) == best
    assert math.isnan(oracle.value_at_volume([1.0, 2.0], np.zeros(2, np.uint32), 0, 0.5))
    with pytest.raises(ValueError):
        oracle.at_volume_rank(0.0, 10)


def test_at_volume_rank_reads_decimal_fractions():
    # ceil(x * n) with x * n taken in FP64 would give 8 here (0.14 * 50 = 7.000000000000001)
    assert oracle.at_volume_rank(0.14, 50) == 7
    assert oracle.at_volume_rank(0.3, 10) == 3
    assert oracle.at_volume_rank(0.98, 2145) == 2103          # 2102.1 -> 2103
    assert oracle.at_volume_rank(0.5, 3) == 2
    assert oracle.at_volume_rank(1.0, 5) == 5 and oracle.at_volume_rank(1e-12, 5) == 1


def test_coverage_rule_two_statements_agree():
    rng = np.random.default_rng(6)
    rx = 2.0
    for n in (37, 50, 200, 1000):
        for trial in range(40):
            dose = rng.normal(rx, 0.06 * rng.uniform(0.2, 2.0), n)
            mask = np.ones(n, np.uint32)
            d98, v95, ok = oracle.coverage(dose, mask, 0, rx)
            assert ok == (v95 >= 0.98), (n, trial, d98, v95)


def test_single_spot_letd_and_cdl_identity():
    # one spot: LETd_i is the spot's LET_ij exactly (Eq. 1); cDL = c * dose * LETd
    rng = np.random.default_rng(7)
    V = 64
    d = rng.uniform(0.1, 1.0, V)
    let = rng.uniform(1.0, 8.0, V)
    rp = np.arange(V + 1)
    P = oracle.build_problem(rp, np.zeros(V, np.int32), d, d * let, 1, np.ones(V, np.uint32), [], [])
    w = np.array([1.7])
    np.testing.assert_allclose(oracle.quantity(P, w, "letd"), let, rtol=1e-14)
    dose = oracle.quantity(P, w, "dose")
    np.testing.assert_allclose(oracle.quantity(P, w, "cdl"), oracle.C_CDL * dose * let, rtol=1e-14)
    np.testing.assert_allclose(dose, 1.7 * d, rtol=1e-15)


def test_derived_cdl30_limits_hold_their_definition():
    pl = phantom.tiny_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    oar_bits = sorted({c["struct_bit"] for c in pl.constraints if c["kind"] in ("DOSE_MAX", "LETD_MAX")})
    cons = oracle.derive_cdl_limits(P, pl.w0, oar_bits)
    cdl = oracle.quantity(P, pl.w0, "cdl")
    for c in cons:
        v = cdl[oracle.structure_voxels(P.mask, c["struct_bit"])]
        assert c["kind"] == "CDL_MAX" and c["bound"] >= 0
        assert np.count_nonzero(v >= c["bound"]) >= 0.3 * len(v)
        assert np.count_nonzero(v > c["bound"]) < 0.3 * len(v)
