"""GB300 (sm_103a) superiorized simultaneous dose + LETd plan optimisation
(arXiv 2509.20012).  The compute lives in libfredopt.so (CUDA kernels behind
the C ABI of include/fredopt.h); `fredopt` is its argument-marshalling
binding."""
from .fredopt import (  # noqa: F401
    Batch, DEVICE_PTR, DONE, FORMATS, KINDS, NORMS, QUANTITIES, ROWS, FredoptError, Handle, Params, Server,
    default_params, footprint_bytes, load_library, superiorize_batch,
)
