"""All-core timing variant of the FP64 oracle.

TEST INFRASTRUCTURE ONLY: bench.py's CPU-baseline and reference legs and
tests/ use it; nothing in the CUDA library imports it.

The oracle's sparse products are its only heavy steps.  `threaded(P, n)`
returns a copy of the problem whose matrices D and L compute their products
with vectors over n row shards of about equal nonzeros on a thread pool
(scipy's sparse kernels release the interpreter lock), and `threaded_rows`
does the same for the constraint rows.  Every other step of the oracle runs
unchanged.  A row shard computes each output of D @ w exactly as the whole
matrix does, so forward products are bit-identical; the transposed product
D.T @ r adds the shards' partial sums in shard order, so its rounding order
differs from the single-threaded product (agreement to about 1e-15
relative).  The variant is not tuned beyond this split.
"""
from __future__ import annotations

import dataclasses
from concurrent.futures import ThreadPoolExecutor

import numpy as np


class RowSharded:
    """A CSR matrix whose products with vectors run over row shards."""

    def __init__(self, M, pool: ThreadPoolExecutor, n_shards: int):
        self.M = M
        indptr = np.asarray(M.indptr)
        targets = np.linspace(0, indptr[-1], n_shards + 1)
        b = np.searchsorted(indptr, targets, side="left")
        b[0], b[-1] = 0, M.shape[0]
        self.bounds = np.maximum.accumulate(b)
        self.shards = [M[self.bounds[i]:self.bounds[i + 1]] for i in range(n_shards)]
        self.pool = pool

    def __getattr__(self, name):
        return getattr(self.M, name)

    def __getitem__(self, idx):
        return self.M[idx]

    def __mul__(self, x):
        return self.M * x

    def __rmul__(self, x):
        return x * self.M

    def __abs__(self):
        return abs(self.M)

    def __matmul__(self, v):
        v = np.asarray(v)
        if v.ndim != 1:
            return self.M @ v
        return np.concatenate(list(self.pool.map(lambda s: s @ v, self.shards)))

    @property
    def T(self):
        return _TransposedShards(self)


class _TransposedShards:
    def __init__(self, rs: RowSharded):
        self.rs = rs

    def __matmul__(self, r):
        r = np.asarray(r)
        b = self.rs.bounds
        parts = list(self.rs.pool.map(lambda i: self.rs.shards[i].T @ r[b[i]:b[i + 1]],
                                      range(len(self.rs.shards))))
        out = np.array(parts[0], dtype=np.float64, copy=True)
        for p in parts[1:]:
            out += p
        return out


def threaded(P, n_threads: int, pool: ThreadPoolExecutor | None = None):
    """The problem P with D and L products split over n_threads row shards."""
    pool = pool or ThreadPoolExecutor(n_threads)
    return dataclasses.replace(P, D=RowSharded(P.D, pool, n_threads), L=RowSharded(P.L, pool, n_threads))


def threaded_rows(R, n_threads: int, pool: ThreadPoolExecutor | None = None):
    """The constraint rows R with their products split over row shards."""
    pool = pool or ThreadPoolExecutor(n_threads)
    return dataclasses.replace(R, A=RowSharded(R.A, pool, n_threads))
