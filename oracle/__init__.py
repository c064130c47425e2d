"""FP64 CPU oracle of the superiorized simultaneous feasibility-seeking loop.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only tests/, __graft_entry__.smoke() and bench.py (its CPU-baseline and
reference legs) may use it.  It shares no code with the CUDA library.
"""
from .fredopt_oracle import (  # noqa: F401
    C_CDL, Problem, build_problem, constraint_rows, forward, letd, objective,
    objective_gradient, cimmino_step, sequential_ams_sweep, superiorize, transpose_csr,
    final_report, sweep_blocks, block_iterative_sweep, violations,
)
from .volume import (  # noqa: F401
    QUANTITIES, at_volume_rank, coverage, cumulative_volume, derive_cdl_limits, quantity,
    structure_voxels, value_at_volume, volume_histogram,
)
