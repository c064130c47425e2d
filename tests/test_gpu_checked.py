"""Checked build (FO_CHECKED=1) of the streaming kernels.

compute-sanitizer is not available on the GPU pool, so the library has a
debug build in place of its memory check.  In it, the forward and transposed
products check three things:
- every tile's element range against the allocated length;
- every gathered index (spot or streamed row) against its table;
- every overflow slot of the based row offsets.

A failure sets bit 1 of the device error word, skips the access, and comes
back as FREDOPT_ERR_PATTERN.  This test runs the parity workloads through the
checked library and through the default one, each in a child process (the
binding loads one library per process).  It requires that no violation is
reported and that every output is bit-identical: the checks change no
arithmetic.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.path.join(ROOT, "_build", "checked", "libfredopt_checked.so")
WORKER = os.path.join(ROOT, "tests", "checked_worker.py")


def run_worker(tmp_path, name, lib=None):
    out = str(tmp_path / f"{name}.npz")
    cmd = [sys.executable, WORKER, out] + ([lib] if lib else [])
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_checked_build_reports_nothing_and_matches(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import _build
    os.makedirs(os.path.dirname(CHECKED), exist_ok=True)
    _build.build(force=True, lib=CHECKED, defines=["FO_CHECKED=1"])
    ref = run_worker(tmp_path, "default")
    chk = run_worker(tmp_path, "checked", CHECKED)
    assert sorted(ref.files) == sorted(chk.files)
    for k in ref.files:
        np.testing.assert_array_equal(chk[k], ref[k], err_msg=k)
