"""Parity of the block-iterative sweep (the block form of Fig. 2's row-action
sweep, reading R13) with the oracle, through the C ABI.

Tolerances: one sweep from the same x within 2e-5 relative L2 of the FP64
oracle (every block re-evaluates its rows with an FP32 product of <= 1e-5
relative error); superiorized runs as for the simultaneous step: identical
trial counters and w within 1e-4 relative L2.
"""
import numpy as np
import pytest

import oracle
import phantom

pytestmark = pytest.mark.gpu


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
    return pl, P, oracle.constraint_rows(P)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("rows", ["all", "roi"])
@pytest.mark.parametrize("n_blocks", [1, 4, 37, 1024])
@pytest.mark.parametrize("norm", ["all", "violated"])
def test_one_sweep_matches_oracle(lib, tiny, rows, n_blocks, norm):
    pl, P, R = tiny
    x = np.random.default_rng(n_blocks).uniform(0.2, 2.5, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl, rows=rows)
        w = h.sweep_step(x, n_blocks, relaxation=1.0, prio_scale=0.8, norm=norm)
    ref = oracle.block_iterative_sweep(R, x.astype(np.float64), 1.0, oracle.sweep_blocks(P, R, n_blocks),
                                       prio_scale=0.8, norm=norm)
    assert rel(w, ref) <= 2e-5, rel(w, ref)
    assert np.all(w >= 0)


def test_single_block_is_the_simultaneous_step(lib, tiny):
    pl, P, R = tiny
    x = np.random.default_rng(3).uniform(0.2, 2.5, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        a = h.sweep_step(x, 1, relaxation=1.5)
        b = h.feasibility_step(x, relaxation=1.5)
    # same forward values and coefficients; only the transposed sum's order differs
    np.testing.assert_allclose(a, b, rtol=2e-6, atol=1e-7)


def test_sweep_blocks_differ_from_simultaneous_and_reduce_violation(lib, tiny):
    """A sweep of many blocks moves further toward feasibility than one
    simultaneous step (later blocks see earlier updates)."""
    pl, P, R = tiny
    x = pl.w0.astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        one = h.sweep_step(x, 1)
        many = h.sweep_step(x, 256)
    v0 = np.linalg.norm(oracle.violations(R, x.astype(np.float64)))
    v1 = np.linalg.norm(oracle.violations(R, one.astype(np.float64)))
    vm = np.linalg.norm(oracle.violations(R, many.astype(np.float64)))
    assert vm < v1 < v0


@pytest.mark.parametrize("n_blocks", [8, 64])
def test_superiorize_with_sweep_matches_oracle(lib, tiny, n_blocks):
    pl, P, R = tiny
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 25, pl.alpha, pl.relaxation, rows=R, sweep=n_blocks)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        w, dose, letd, rep = h.superiorize(pl.w0, 25, pl.alpha, pl.relaxation, sweep_blocks=n_blocks)
        log = h.get_log()
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert [e["accepted"] for e in log] == [e["accepted"] for e in log_ref]
    assert rel(w, w_ref) <= 1e-4, rel(w, w_ref)
    for e in log:
        assert e["f_end"] <= e["f_start"]
    assert rep["iters"] == 25


def test_sweep_graph_plain_deterministic_and_launch_count(lib, tiny):
    pl, P, R = tiny
    out = []
    for use_graphs in (1, 1, 0):
        with lib.Handle(0) as h:
            h.load_plan(pl)
            h.set_timing(False)
            h.begin(pl.w0, pl.alpha, pl.relaxation, sweep_blocks=16, use_graphs=use_graphs)
            n0 = h.launch_count()
            h.iterate(6)
            n1 = h.launch_count()
            w, *_ = h.end()
            out.append((w, n1 - n0))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][0], out[2][0])
    nb = len(oracle.sweep_blocks(P, R, 16))
    # perturbation (forward, transposed, column finish, forward of g, scalar finish) + start + 3 per block + finish
    assert out[0][1] == 6 * (5 + 1 + 3 * nb + 1)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_sweep_with_16bit_storage(lib, tiny, fmt):
    pl, P, R = tiny
    x = np.random.default_rng(4).uniform(0.2, 2.5, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl, fmt=fmt)
        w = h.sweep_step(x, 16)
    ref = oracle.block_iterative_sweep(R, x.astype(np.float64), 1.0, oracle.sweep_blocks(P, R, 16))
    assert rel(w, ref) <= (2e-2 if fmt == "bf16" else 4e-3)


def test_sweep_errors(lib, tiny):
    pl, P, R = tiny
    with lib.Handle(0) as h:
        h.load_plan(pl)
        for bad in (0, lib.MAX_SWEEP_BLOCKS + 1):
            with pytest.raises(lib.FredoptError):
                h.sweep_step(pl.w0, bad)
            with pytest.raises(lib.FredoptError):
                h.begin(pl.w0, pl.alpha, pl.relaxation, sweep_blocks=bad if bad else -1)
        h.begin(pl.w0, pl.alpha, pl.relaxation, sweep_blocks=8)
        with pytest.raises(lib.FredoptError):
            h.sweep_step(pl.w0, 9)      # the begun solve's graph uses 8 blocks
        h.sweep_step(pl.w0, 8)          # the same count is fine
        h.iterate(2)
        w, *_ = h.end()
    assert np.all(np.isfinite(w))


def test_clinical_sweep_roi(lib):
    pl = phantom.clinical_plan()
    P = oracle.build_problem(pl.row_ptr, pl.col, pl.D, pl.L, pl.n_spots, pl.mask, pl.constraints, pl.objective)
    R = oracle.constraint_rows(P)
    w_ref, log_ref = oracle.superiorize(P, pl.w0, 2, pl.alpha, pl.relaxation, rows=R, sweep=32)
    with lib.Handle(0) as h:
        h.load_plan(pl, rows="roi")
        w, *_ = h.superiorize(pl.w0, 2, pl.alpha, pl.relaxation, sweep_blocks=32)
        log = h.get_log()
    assert [e["s"] for e in log] == [e["s"] for e in log_ref]
    assert rel(w, w_ref) <= 1e-4, rel(w, w_ref)
