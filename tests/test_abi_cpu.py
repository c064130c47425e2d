"""CPU checks of the C ABI: the library builds, loads and exports every
function that include/fredopt.h declares; argument errors that need no GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return fredopt.load_library()


def declared_functions():
    with open(os.path.join(ROOT, "include", "fredopt.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fredopt_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fredopt_load_influence", "fredopt_set_constraints", "fredopt_superiorize",
                     "fredopt_create", "fredopt_destroy", "fredopt_get_state", "fredopt_set_state",
                     "fredopt_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2509_20012_gb300 import fredopt
    assert set(declared_functions()) <= set(fredopt._SIGS)


def test_strerror_and_defaults(lib):
    from paper_2509_20012_gb300 import fredopt
    assert lib.fredopt_strerror(0) == b"ok"
    assert lib.fredopt_strerror(-3) == b"pattern"
    assert lib.fredopt_strerror(-99) == b"unknown error"
    p = fredopt.default_params()
    assert p.beta0 < 0 and p.eta == 1.0 and p.reductions == 1 and p.max_trials == 50
    assert p.c_cdl == pytest.approx(0.04) and p.use_graphs == 1


def test_null_and_bad_arguments_without_gpu(lib):
    assert lib.fredopt_create(None, 0, None) == -1
    assert lib.fredopt_destroy(None) == -1
    assert lib.fredopt_launch_count(None) == -1
    h = ctypes.c_void_p()
    # no device with this index (and on a CPU-only machine none at all)
    assert lib.fredopt_create(ctypes.byref(h), 1 << 20, None) == -1
    assert lib.fredopt_iterate(None, 1) == -1
    assert lib.fredopt_check_wait(None, 0, 0, None) == -1
    # no CUDA device here: the architecture query fails cleanly
    assert lib.fredopt_kernel_arch(0, None, None, None) == -7


def test_binding_error_constant_matches_header():
    from paper_2509_20012_gb300 import fredopt
    text = open(os.path.join(ROOT, "include", "fredopt.h")).read()
    assert int(re.search(r"#define FREDOPT_ERR_TIMEOUT \((-?\d+)\)", text).group(1)) == fredopt.ERR_TIMEOUT
    assert 1 << int(re.search(r"#define FREDOPT_WAIT_POLLS \(1 << (\d+)\)", text).group(1)) == fredopt.WAIT_POLLS
    assert int(re.search(r"#define FREDOPT_INDEX32 (0x[0-9a-fA-F]+)", text).group(1), 16) == fredopt.INDEX32
    assert int(re.search(r"#define FREDOPT_ROWS_ROI (0x[0-9a-fA-F]+)", text).group(1), 16) == fredopt.ROWS["roi"]
    assert int(re.search(r"#define FREDOPT_SHARED (0x[0-9a-fA-F]+)", text).group(1), 16) == fredopt.SHARED


def test_footprint_covers_the_load_peak(lib):
    """The memory estimate the server admits by (a host function: no GPU)
    covers the load's peak: CSR + CSC + one CSC-build record per nonzero
    (16 bytes with FP32 values, 8 with 16-bit), at least 40 and 24 bytes per
    nonzero; it grows with the plan and rejects bad sizes."""
    fp = lib.fredopt_footprint_bytes
    nnz = 10_000_000
    assert fp(1000, 100, nnz, 0) >= 40 * nnz
    assert fp(1000, 100, nnz, 1) >= 24 * nnz
    assert fp(1000, 100, nnz, 2) == fp(1000, 100, nnz, 1)
    assert fp(1000, 100, 2 * nnz, 0) > fp(1000, 100, nnz, 0)
    assert fp(2_000_000, 100, nnz, 0) > fp(1000, 100, nnz, 0)
    # the launch-shape and index flags do not change the estimate
    assert fp(1000, 100, nnz, 0x400) == fp(1000, 100, nnz, 0)
    assert fp(-1, 100, nnz, 0) == -1 and fp(1000, 0, nnz, 0) == -1 and fp(1000, 100, -1, 0) == -1


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the public structs have the C sizes and offsets."""
    import ctypes
    import subprocess
    from paper_2509_20012_gb300 import fredopt as f
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "fredopt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(fredopt_params), sizeof(fredopt_report),
         sizeof(fredopt_request), sizeof(fredopt_ticket_info), sizeof(fredopt_log_entry),
         sizeof(fredopt_constraint), sizeof(fredopt_objective_term), offsetof(fredopt_request, params),
         offsetof(fredopt_request, w_out), offsetof(fredopt_request, alpha), offsetof(fredopt_ticket_info, report),
         sizeof(fredopt_volume_request), offsetof(fredopt_volume_request, edges),
         offsetof(fredopt_volume_request, n_voxels));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    c = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    py = [ctypes.sizeof(f.Params), ctypes.sizeof(f.Report), ctypes.sizeof(f.Request), ctypes.sizeof(f.TicketInfo),
          ctypes.sizeof(f.LogEntry), ctypes.sizeof(f.Constraint), ctypes.sizeof(f.ObjectiveTerm),
          f.Request.params.offset, f.Request.w_out.offset, f.Request.alpha.offset, f.TicketInfo.report.offset,
          ctypes.sizeof(f.VolumeRequest), f.VolumeRequest.edges.offset, f.VolumeRequest.n_voxels.offset]
    assert c == py
