"""Child process of tests/test_gpu_checked.py: runs the streaming workloads of
the parity tests through one library (argv[2], default: the package's own)
and saves every output to argv[1] (.npz).  Any library error raises, so a
violation reported by a checked build fails the child."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import phantom  # noqa: E402
from paper_2509_20012_gb300 import fredopt  # noqa: E402


def main(out_path, lib_path=None):
    if lib_path:
        fredopt.load_library(lib_path)
    out = {}
    pl = phantom.tiny_plan()
    x = np.random.default_rng(11).uniform(0.0, 2.0, pl.n_spots).astype(np.float32)
    for fmt in ("fp32", "bf16"):
        for rows in ("all", "roi"):
            for index32 in (False, True):
                key = f"{fmt}_{rows}_{int(index32)}"
                with fredopt.Handle(0) as h:
                    h.load_plan(pl, fmt=fmt, rows=rows, index32=index32)
                    dose, lw = h.forward(x)
                    out[key + "_dose"], out[key + "_lw"] = dose, lw
                    out[key + "_u"] = h.backward(dose, lw)
                    out[key + "_sweep"] = h.sweep_step(x, 16)
                    w, d, l, _ = h.superiorize(pl.w0, 10, pl.alpha, pl.relaxation)
                    out[key + "_w"], out[key + "_d"], out[key + "_l"] = w, d, l
    # wide blocks of based row offsets; a forward with x read through L1
    for n_rows, n_cols, dens in ((300000, 20, 0.0004), (70000, 3, 0.9), (300, 60000, 40.0 / 60000)):
        rp, col, D, L = phantom.random_csr(n_rows, n_cols, dens, seed=n_rows + n_cols, empty_rows=11)
        rng = np.random.default_rng(3)
        xs = rng.uniform(0.0, 2.0, n_cols).astype(np.float32)
        a = rng.normal(size=n_rows).astype(np.float32)
        with fredopt.Handle(0) as h:
            h.load_influence(rp, col, D, L, np.ones(n_rows, np.uint32), n_cols)
            key = f"rand_{n_rows}_{n_cols}"
            out[key + "_dose"], out[key + "_lw"] = h.forward(xs)
            out[key + "_u"] = h.backward(a, a)
    np.savez(out_path, **out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2] if len(sys.argv) > 2 else None)
