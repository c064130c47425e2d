"""Failure detection on the GPU without a fault.

The library's one kind of device-side wait, the mbarrier phase that a bulk
copy completes, polls a bounded number of times; when it gives up the kernel
sets the handle's error word and returns.  `fredopt_check_wait` runs that wait
on a phase that nothing completes, so these tests make it run out for real and
check that the status comes back as FREDOPT_ERR_TIMEOUT, that the context and
the handle stay usable, and that results after the failure equal those of a
fresh handle.  No kernel here traps, asserts or touches a bad address.
"""
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


def test_completed_wait_is_ok(lib):
    with lib.Handle(0) as h:
        for spins in (0, 1):
            rc, ms = h.check_wait(True, spins)
            assert rc == 0 and ms >= 0.0


def test_wait_that_gives_up_reports_timeout_and_handle_stays_usable(lib):
    pl = phantom.tiny_plan()
    w = np.random.default_rng(8).uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    with lib.Handle(0) as h:
        h.load_plan(pl)
        d0, l0 = h.forward(w)
        rc, _ = h.check_wait(False, 1 << 12)
        assert rc == lib.ERR_TIMEOUT
        # the error word was reported once and cleared: the next calls succeed
        assert h.check_wait(True)[0] == 0
        d1, l1 = h.forward(w)
        np.testing.assert_array_equal(d0, d1)
        np.testing.assert_array_equal(l0, l1)
        # a failure in the middle of a begun solve: the solve goes on and
        # ends where an undisturbed one ends
        h.begin(pl.w0, pl.alpha, pl.relaxation)
        h.iterate(5)
        assert h.check_wait(False, 1 << 10)[0] == lib.ERR_TIMEOUT
        h.iterate(5)
        wa, da, la = h.end()[:3]
    with lib.Handle(0) as g:
        g.load_plan(pl)
        g.begin(pl.w0, pl.alpha, pl.relaxation)
        g.iterate(10)
        wb, db, lb = g.end()[:3]
    np.testing.assert_array_equal(wa, wb)
    np.testing.assert_array_equal(da, db)
    np.testing.assert_array_equal(la, lb)


def test_kernels_bound_gives_up_in_bounded_time(lib):
    """The bound the kernels use ends a stuck wait within a few seconds.
    Its time is predicted from a short wait first and the full one runs only
    when the prediction is under 10 s."""
    with lib.Handle(0) as h:
        rc, ms_short = h.check_wait(False, 1 << 12)
        assert rc == lib.ERR_TIMEOUT
        predicted = ms_short * lib.WAIT_POLLS / (1 << 12)
        if predicted > 10000.0:
            pytest.skip(f"predicted give-up time {predicted:.0f} ms")
        rc, ms = h.check_wait(False, 0)
        assert rc == lib.ERR_TIMEOUT
        assert ms < 5000.0
        print(f"bounded wait gave up after {ms:.1f} ms ({ms_short:.3f} ms for 2^12 polls)")
        assert h.check_wait(True)[0] == 0
