"""The allocation-free transposed product (fredopt_backward_noalloc).

It serves callers that cannot allocate device memory where they need the
product (their own pool owns the GPU, or cudaMalloc/cudaFree must stay out
of a latency-critical loop).  The test feeds it the CSC copy that a handle
built, through the C ABI with device pointers, twice in a row, and compares
each result with the handle's own transposed product (fredopt_backward)
within the FP32 product tolerance of the other parity tests: 1e-5 of the
sum of absolute products of each column.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu


def test_backward_noalloc_matches_backward_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    lib = fredopt.load_library()
    pl = phantom.tiny_plan()
    rng = np.random.default_rng(11)
    dev = torch.device("cuda:0")
    with fredopt.Handle(0) as h:
        h.load_plan(pl)
        cp, row, DT, LT = h.get_csc()
        vox, _ = h.get_rows()
        n_rows = int(vox.shape[0])
        t_cp = torch.from_numpy(cp).to(dev)
        t_row = torch.from_numpy(row).to(dev)
        t_D = torch.from_numpy(DT).to(dev)
        t_L = torch.from_numpy(LT).to(dev)
        for call in range(2):
            aD = rng.normal(size=pl.n_vox).astype(np.float32)
            aL = rng.normal(size=pl.n_vox).astype(np.float32)
            u_ref = h.backward(aD, aL)
            # coefficients in the CSC's row order (device rows -> voxels)
            t_aD = torch.from_numpy(aD[vox]).to(dev)
            t_aL = torch.from_numpy(aL[vox]).to(dev)
            u = torch.full((pl.n_spots,), float("nan"), dtype=torch.float32, device=dev)
            stream = torch.cuda.current_stream(dev).cuda_stream
            rc = lib.fredopt_backward_noalloc(n_rows, pl.n_spots, int(row.shape[0]), t_cp.data_ptr(),
                                              t_row.data_ptr(), t_D.data_ptr(), t_L.data_ptr(),
                                              t_aD.data_ptr(), t_aL.data_ptr(), u.data_ptr(),
                                              ctypes.c_void_p(stream))
            assert rc == 0
            torch.cuda.synchronize(dev)
            got = u.cpu().numpy()
            bound = np.zeros(pl.n_spots)
            absD, absL = np.abs(DT.astype(np.float64)), np.abs(LT.astype(np.float64))
            wD, wL = np.abs(aD[vox][row].astype(np.float64)), np.abs(aL[vox][row].astype(np.float64))
            np.add.at(bound, np.repeat(np.arange(pl.n_spots), np.diff(cp)), absD * wD + absL * wL)
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - u_ref) <= 1e-5 * bound + 1e-30)


def test_backward_noalloc_rejects_sizes_beyond_its_scratch():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    lib = fredopt.load_library()
    # more columns than the fixed scratch holds: refused before any device work
    assert lib.fredopt_backward_noalloc(10, 70000, 0, None, None, None, None, None, None, None, None) == -2
    assert lib.fredopt_backward_noalloc(10, 100, 1 << 33, None, None, None, None, None, None, None, None) == -2
