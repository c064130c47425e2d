"""The allocation-free transposed product (fredopt_backward_noalloc).

It serves callers that cannot allocate device memory where they need the
product (their own pool owns the GPU, or cudaMalloc/cudaFree must stay out
of a latency-critical loop).  Its scratch is one fixed device array shared
by every call.  The tests call it through the C ABI with device pointers and
compare it with the FP64 product sum_i D_ij a_D[i] + L_ij a_L[i] computed on
the host, within the FP32 product tolerance of the other parity tests: 1e-5
of the sum of absolute products of each column.  They cover:
- the CSC copy a handle built for the tiny plan, with the handle's own
  transposed product (fredopt_backward) beside it, two calls in a row;
- columns of up to about 40000 nonzeros (up to 10 chunks of 4096, so a
  column's chunks are summed across warps and added in order) next to empty
  columns, with and without a_D;
- the largest column count accepted (65536 columns), and the sizes just past
  each limit, which are refused before any device work;
- the same inputs twice give the same bits.
This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import phantom

pytestmark = pytest.mark.gpu

MAX_COLS = 65536
CHUNK = 4096
MAX_CHUNKS = 1 << 20


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2509_20012_gb300 import fredopt
    return torch, fredopt, fredopt.load_library()


def fp64_product(cp, row, D, L, aD, aL, n_cols):
    """(exact-ish FP64 column sums, sums of absolute products) of the CSC pair."""
    col = np.repeat(np.arange(n_cols), np.diff(cp))
    tD = D.astype(np.float64) * (aD[row].astype(np.float64) if aD is not None else 0.0)
    tL = L.astype(np.float64) * aL[row].astype(np.float64)
    ref = np.bincount(col, weights=tD + tL, minlength=n_cols)
    bound = np.bincount(col, weights=np.abs(tD) + np.abs(tL), minlength=n_cols)
    return ref, bound


def call_noalloc(env, n_rows, cp, row, D, L, aD, aL):
    torch, fredopt, lib = env
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n_cols = len(cp) - 1
    keep = [t(cp), t(row), t(D), t(L), t(aD) if aD is not None else None, t(aL)]
    u = torch.full((n_cols,), float("nan"), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    ptr = lambda x: x.data_ptr() if x is not None else None
    rc = lib.fredopt_backward_noalloc(n_rows, n_cols, int(len(row)), ptr(keep[0]), ptr(keep[1]), ptr(keep[2]),
                                      ptr(keep[3]), ptr(keep[4]), ptr(keep[5]), u.data_ptr(),
                                      ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize(dev)
    return u.cpu().numpy()


def test_backward_noalloc_matches_fp64_and_backward_twice(env):
    torch, fredopt, lib = env
    pl = phantom.tiny_plan()
    rng = np.random.default_rng(11)
    with fredopt.Handle(0) as h:
        h.load_plan(pl)
        cp, row, DT, LT = h.get_csc()
        vox, _ = h.get_rows()
        n_rows = int(vox.shape[0])
        for call in range(2):
            aD = rng.normal(size=pl.n_vox).astype(np.float32)
            aL = rng.normal(size=pl.n_vox).astype(np.float32)
            u_lib = h.backward(aD, aL)
            # coefficients in the CSC's row order (device rows -> voxels)
            got = call_noalloc(env, n_rows, cp, row, DT, LT, aD[vox], aL[vox])
            ref, bound = fp64_product(cp, row, DT, LT, aD[vox], aL[vox], pl.n_spots)
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)
            assert np.all(np.abs(got - u_lib) <= 2e-5 * bound + 1e-30)


def long_column_csc(n_rows, lens, seed):
    """CSC pair with the given nonzeros per column (ascending distinct rows)."""
    rng = np.random.default_rng(seed)
    rows = [np.sort(rng.choice(n_rows, size=k, replace=False)).astype(np.int32) for k in lens]
    cp = np.zeros(len(lens) + 1, np.int64)
    cp[1:] = np.cumsum(lens)
    row = np.concatenate(rows) if cp[-1] else np.zeros(0, np.int32)
    D = rng.uniform(0.01, 1.0, size=row.shape[0]).astype(np.float32)
    L = (D * rng.uniform(0.5, 12.0, size=row.shape[0])).astype(np.float32)
    return cp, row, D, L


@pytest.mark.parametrize("with_aD", [True, False])
def test_multi_chunk_columns_and_empty_columns(env, with_aD):
    """Columns longer than one chunk of 4096 nonzeros (the chunk offset of a
    later chunk, the column search landing on it, and the in-order sum of a
    column's chunk sums), among empty columns and one-element columns."""
    n_rows = 60000
    lens = [40000, 0, 4096, 4097, 1, 0, 12289, 8191, 0, 33333, 2, 16384]
    cp, row, D, L = long_column_csc(n_rows, lens, seed=7)
    rng = np.random.default_rng(3)
    aD = rng.normal(size=n_rows).astype(np.float32) if with_aD else None
    aL = rng.normal(size=n_rows).astype(np.float32)
    got = call_noalloc(env, n_rows, cp, row, D, L, aD, aL)
    ref, bound = fp64_product(cp, row, D, L, aD, aL, len(lens))
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)
    assert np.all(got[np.array(lens) == 0] == 0.0)
    # deterministic: the same inputs give the same bits
    again = call_noalloc(env, n_rows, cp, row, D, L, aD, aL)
    np.testing.assert_array_equal(got, again)


def test_largest_column_count(env):
    """65536 columns, the most the scratch's offset table holds."""
    n_rows = 12000
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 40, MAX_COLS)
    lens[[0, 777, MAX_COLS - 1]] = [9000, 4097, 5000]   # a few multi-chunk columns
    cp, row, D, L = long_column_csc(n_rows, lens, seed=9)
    aD = rng.normal(size=n_rows).astype(np.float32)
    aL = rng.normal(size=n_rows).astype(np.float32)
    got = call_noalloc(env, n_rows, cp, row, D, L, aD, aL)
    ref, bound = fp64_product(cp, row, D, L, aD, aL, MAX_COLS)
    assert np.all(np.abs(got - ref) <= 1e-5 * bound + 1e-30)


def test_backward_noalloc_rejects_sizes_beyond_its_scratch(env):
    """Sizes past either limit are refused before any device work (no
    pointer is read)."""
    torch, fredopt, lib = env
    args = (None,) * 8
    assert lib.fredopt_backward_noalloc(10, MAX_COLS + 1, 0, *args) == -2
    # chunk bound nnz / 4096 + n_cols <= 2^20: one past it, with one column
    nnz = (MAX_CHUNKS - 1 + 1) * CHUNK
    assert lib.fredopt_backward_noalloc(10, 1, nnz, *args) == -2
    assert lib.fredopt_backward_noalloc(10, 100, 1 << 33, *args) == -2
    assert lib.fredopt_backward_noalloc(10, 0, 0, *args) == -2
