"""Thin ctypes binding of libfredopt (include/fredopt.h): argument
marshalling only.  Every step of the method runs in the library's CUDA
kernels; nothing here computes.

Arrays may be numpy arrays (host) or torch tensors; CUDA tensors are passed
as device pointers (FREDOPT_DEVICE_PTR), everything else as host memory.
If libfredopt.so is missing the import fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfredopt.so")

# ---- constants (values of include/fredopt.h) ----
OK = 0
DEVICE_PTR = 0x1
FORMATS = {"fp32": 0, "bf16": 1, "fp16": 2}
ROWS = {"all": 0x000, "roi": 0x100}
INDEX32 = 0x200  # keep 32-bit indices in the forward and transposed streams
SHARED = 0x400   # launch shapes for running beside other plans (batches, servers)
KINDS = {"DOSE_MIN": 0, "DOSE_MAX": 1, "CDL_MIN": 2, "CDL_MAX": 3, "LETD_MIN": 4, "LETD_MAX": 5}
QUANTITIES = {"DOSE": 0, "CDL": 1, "LETD": 2}  # LETD: volume statistics only
VOLUME_MAX_REQUESTS, VOLUME_MAX_BINS, VOLUME_MAX_FRACS = 64, 16384, 64
MAX_SWEEP_BLOCKS = 1024
NORMS = {"all": 0, "violated": 1}
KCLASS_N = 6
KCLASS_NAMES = ["forward", "backward", "constraints", "colfinish", "finish", "other"]
ERR_TIMEOUT = -8  # FREDOPT_ERR_TIMEOUT: a bounded device-side wait gave up
WAIT_POLLS = 1 << 18  # FREDOPT_WAIT_POLLS


class FredoptError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fredopt error {code}: {msg}")
        self.code = code


class Constraint(ctypes.Structure):
    _fields_ = [("struct_bit", ctypes.c_uint32), ("kind", ctypes.c_int32),
                ("bound", ctypes.c_double), ("priority", ctypes.c_double)]


class ObjectiveTerm(ctypes.Structure):
    _fields_ = [("struct_bit", ctypes.c_uint32), ("quantity", ctypes.c_int32),
                ("target", ctypes.c_double), ("weight", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("beta0", ctypes.c_double), ("eta", ctypes.c_double),
                ("reductions", ctypes.c_int32), ("max_trials", ctypes.c_int32),
                ("cimmino_norm", ctypes.c_int32), ("grad_normalize", ctypes.c_int32),
                ("c_cdl", ctypes.c_double), ("log_capacity", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("sweep_blocks", ctypes.c_int32), ("tile_balance", ctypes.c_int32)]


class LogEntry(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("s", ctypes.c_int64), ("accepted", ctypes.c_int32),
                ("n_violated", ctypes.c_int32), ("beta", ctypes.c_double),
                ("f_start", ctypes.c_double), ("f_end", ctypes.c_double),
                ("gnorm", ctypes.c_double), ("max_violation", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("s", ctypes.c_int64), ("accepted", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("unreachable_rows", ctypes.c_int64),
                ("n_violated", ctypes.c_int64), ("objective", ctypes.c_double),
                ("max_violation", ctypes.c_double * 6), ("beta0", ctypes.c_double),
                ("device_ms", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["max_violation"] = list(self.max_violation)
        return d


class Request(ctypes.Structure):
    _fields_ = [("n_vox", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_spots", ctypes.c_int32),
                ("format", ctypes.c_int32), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("D_val", ctypes.c_void_p), ("L_val", ctypes.c_void_p), ("voxel_mask", ctypes.c_void_p),
                ("n_constraints", ctypes.c_int32), ("n_objective", ctypes.c_int32),
                ("constraints", ctypes.POINTER(Constraint)), ("objective", ctypes.POINTER(ObjectiveTerm)),
                ("w0", ctypes.c_void_p), ("iters", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("relaxation", ctypes.c_double), ("params", Params),
                ("w_out", ctypes.c_void_p), ("dose_out", ctypes.c_void_p), ("letd_out", ctypes.c_void_p)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("pad", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint_bytes", ctypes.c_int64), ("report", Report)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("pad", "report")}
        d["report"] = self.report.as_dict()
        return d


class VolumeRequest(ctypes.Structure):
    _fields_ = [("quantity", ctypes.c_int32), ("struct_bit", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("n_fracs", ctypes.c_int32), ("edges", ctypes.c_void_p), ("fracs", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("at_volume", ctypes.c_void_p), ("n_voxels", ctypes.c_int64)]


QUEUED, LOADING, RUNNING, DONE = 0, 1, 2, 3

_lib = None

_SIGS = {
    "fredopt_default_params": (None, [ctypes.POINTER(Params)]),
    "fredopt_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fredopt_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fredopt_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]),
    "fredopt_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fredopt_load_influence": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]),
    "fredopt_set_constraints": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Constraint)]),
    "fredopt_set_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ObjectiveTerm)]),
    "fredopt_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(Params), ctypes.c_uint32]),
    "fredopt_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fredopt_end": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.POINTER(Report), ctypes.c_uint32]),
    "fredopt_superiorize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(Params), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Report),
                                           ctypes.c_uint32]),
    "fredopt_get_log": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(LogEntry), ctypes.c_int]),
    "fredopt_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_uint32]),
    "fredopt_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_uint32]),
    "fredopt_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_uint32]),
    "fredopt_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_uint32]),
    "fredopt_feasibility_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32]),
    "fredopt_sweep_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_uint32]),
    "fredopt_objective": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p, ctypes.c_uint32]),
    "fredopt_volume_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int,
                                            ctypes.POINTER(VolumeRequest)]),
    "fredopt_quantity_map": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_uint32]),
    "fredopt_get_sizes": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int64)] * 5),
    "fredopt_get_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fredopt_get_csc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "fredopt_get_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fredopt_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fredopt_get_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fredopt_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "fredopt_kernel_arch": (ctypes.c_int, [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3),
    "fredopt_get_storage": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 3),
    "fredopt_check_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
    "fredopt_footprint_bytes": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_int]),
    "fredopt_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64,
                                             ctypes.c_int, ctypes.c_int]),
    "fredopt_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int64)]),
    "fredopt_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(TicketInfo)]),
    "fredopt_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double,
                                           ctypes.POINTER(TicketInfo)]),
    "fredopt_server_drain": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "fredopt_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "fredopt_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fredopt_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "fredopt_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "fredopt_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_int]),
    "fredopt_batch_create_depth": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                                  ctypes.c_int, ctypes.c_int]),
    "fredopt_batch_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fredopt_batch_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "fredopt_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fredopt_superiorize_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.POINTER(Params),
                                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(Report),
                                                 ctypes.c_uint32]),
    "fredopt_backward_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH):
    """Load libfredopt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libfredopt.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def default_params(**overrides) -> Params:
    p = Params()
    load_library().fredopt_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "cimmino_norm" and isinstance(v, str):
            v = NORMS[v]
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _on_device(x) -> bool:
    return _is_torch(x) and x.is_cuda


def _ptr(x, dtype):
    """(pointer, keepalive) of a contiguous array of the given numpy dtype."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.int64: torch.int64, np.int32: torch.int32,
               np.uint32: torch.int32, np.float64: torch.float64}[dtype]
        if x.dtype != tdt and not (dtype is np.uint32 and x.dtype in (torch.int32, torch.uint32)):
            raise TypeError(f"expected {tdt}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if not x.is_cuda:
            return x.data_ptr(), x
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


class Handle:
    """One plan on one GPU (a fredopt_t)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        h = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        rc = self.lib.fredopt_create(ctypes.byref(h), device, s)
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        self.h = h
        self.device = device
        self.n_vox = self.n_spots = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.fredopt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc < 0:
            msg = self.lib.fredopt_last_error(self.h)
            raise FredoptError(rc, f"{self.lib.fredopt_strerror(rc).decode()}: {msg.decode() if msg else ''}")
        return rc

    # ---------------------------------------------------------- plan
    def load_influence(self, row_ptr, col, D, L, mask, n_spots, fmt="fp32", rows="all", index32=False,
                       shared=False):
        dev = _on_device(row_ptr)
        n_vox = int(row_ptr.shape[0]) - 1
        nnz = int(col.shape[0])
        p_rp, k1 = _ptr(row_ptr, np.int64)
        p_c, k2 = _ptr(col, np.int32)
        p_d, k3 = _ptr(D, np.float32)
        p_l, k4 = _ptr(L, np.float32)
        p_m, k5 = _ptr(mask, np.uint32)
        code = FORMATS[fmt] | ROWS[rows] | (INDEX32 if index32 else 0) | (SHARED if shared else 0)
        self._check(self.lib.fredopt_load_influence(self.h, n_vox, int(n_spots), nnz, p_rp, p_c, p_d, p_l,
                                                    p_m, code, DEVICE_PTR if dev else 0))
        self.n_vox, self.n_spots = n_vox, int(n_spots)

    def set_constraints(self, constraints):
        arr = (Constraint * max(1, len(constraints)))()
        for i, c in enumerate(constraints):
            arr[i] = Constraint(int(c["struct_bit"]), KINDS[c["kind"]], float(c["bound"]), float(c["priority"]))
        self._check(self.lib.fredopt_set_constraints(self.h, len(constraints), arr))

    def set_objective(self, terms):
        arr = (ObjectiveTerm * max(1, len(terms)))()
        for i, t in enumerate(terms):
            arr[i] = ObjectiveTerm(int(t["struct_bit"]), QUANTITIES[t["quantity"]], float(t["target"]),
                                   float(t["weight"]))
        self._check(self.lib.fredopt_set_objective(self.h, len(terms), arr))

    def load_plan(self, plan, fmt="fp32", rows="all", index32=False, shared=False):
        """Load a phantom.Plan-like object (row_ptr, col, D, L, mask, constraints, objective)."""
        self.load_influence(plan.row_ptr, plan.col, plan.D, plan.L, plan.mask, plan.n_spots, fmt=fmt, rows=rows,
                            index32=index32, shared=shared)
        self.set_constraints(plan.constraints)
        self.set_objective(plan.objective)

    def storage(self):
        """(column index bytes of the forward stream, row index bytes of the
        transposed product's stream, value bytes) of the loaded plan."""
        ib, rb, vb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.fredopt_get_storage(self.h, ctypes.byref(ib), ctypes.byref(rb), ctypes.byref(vb)))
        return ib.value, rb.value, vb.value

    def sizes(self):
        v = [ctypes.c_int64() for _ in range(5)]
        self._check(self.lib.fredopt_get_sizes(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["n_vox", "n_spots", "nnz", "n_rows", "nnz_rows"], [x.value for x in v]))

    # ---------------------------------------------------------- outputs
    def _out(self, like_dev, n, dtype=np.float32):
        if like_dev:
            import torch
            return torch.empty(n, dtype=torch.float32, device=f"cuda:{self.device}")
        return np.empty(n, dtype)

    # ---------------------------------------------------------- solve
    def begin(self, w0, alpha, relaxation, params: Params | None = None, **kw):
        if params is None:
            params = default_params(**kw)
        dev = _on_device(w0)
        p, keep = _ptr(w0, np.float32)
        self._check(self.lib.fredopt_begin(self.h, p, float(alpha), float(relaxation), ctypes.byref(params),
                                           DEVICE_PTR if dev else 0))
        self._dev = dev

    def iterate(self, iters: int):
        self._check(self.lib.fredopt_iterate(self.h, int(iters)))

    def end(self, outputs=None):
        """Returns (w, dose, letd, report dict); outputs=(w, dose, letd) to fill."""
        dev = getattr(self, "_dev", False)
        if outputs is None:
            outputs = (self._out(dev, self.n_spots), self._out(dev, self.n_vox), self._out(dev, self.n_vox))
        w, d, l = outputs
        dev = _on_device(w)
        rep = Report()
        self._check(self.lib.fredopt_end(self.h, _ptr(w, np.float32)[0], _ptr(d, np.float32)[0] if d is not None else None,
                                         _ptr(l, np.float32)[0] if l is not None else None, ctypes.byref(rep),
                                         DEVICE_PTR if dev else 0))
        return w, d, l, rep.as_dict()

    def superiorize(self, w0, iters, alpha, relaxation, params: Params | None = None, outputs=None, **kw):
        """One call: begin + iterate + end (fredopt_superiorize)."""
        if params is None:
            params = default_params(**kw)
        dev = _on_device(w0)
        if outputs is None:
            outputs = (self._out(dev, self.n_spots), self._out(dev, self.n_vox), self._out(dev, self.n_vox))
        w, d, l = outputs
        rep = Report()
        p0, keep = _ptr(w0, np.float32)
        self._check(self.lib.fredopt_superiorize(self.h, p0, int(iters), float(alpha), float(relaxation),
                                                 ctypes.byref(params), _ptr(w, np.float32)[0],
                                                 _ptr(d, np.float32)[0], _ptr(l, np.float32)[0],
                                                 ctypes.byref(rep), DEVICE_PTR if dev else 0))
        self._dev = dev
        return w, d, l, rep.as_dict()

    def get_log(self, max_entries=1 << 20):
        arr = (LogEntry * max_entries)()
        n = self._check(self.lib.fredopt_get_log(self.h, arr, max_entries))
        return [{k: getattr(arr[i], k) for k, _ in LogEntry._fields_} for i in range(n)]

    def get_state(self):
        w = np.empty(self.n_spots, np.float32)
        k, s = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.fredopt_get_state(self.h, w.ctypes.data, ctypes.byref(k), ctypes.byref(s), 0))
        return w, k.value, s.value

    def set_state(self, w, k, s):
        dev = _on_device(w)
        p, keep = _ptr(w, np.float32)
        self._check(self.lib.fredopt_set_state(self.h, p, int(k), int(s), DEVICE_PTR if dev else 0))

    # ---------------------------------------------------------- single passes
    def forward(self, w):
        dev = _on_device(w)
        d, l = self._out(dev, self.n_vox), self._out(dev, self.n_vox)
        self._check(self.lib.fredopt_forward(self.h, _ptr(w, np.float32)[0], _ptr(d, np.float32)[0],
                                             _ptr(l, np.float32)[0], DEVICE_PTR if dev else 0))
        return d, l

    def backward(self, a_D, a_L):
        dev = _on_device(a_D if a_D is not None else a_L)
        u = self._out(dev, self.n_spots)
        self._check(self.lib.fredopt_backward(self.h, _ptr(a_D, np.float32)[0], _ptr(a_L, np.float32)[0],
                                              _ptr(u, np.float32)[0], DEVICE_PTR if dev else 0))
        return u

    def feasibility_step(self, x, relaxation=1.0, prio_scale=1.0, norm="all"):
        dev = _on_device(x)
        w = self._out(dev, self.n_spots)
        self._check(self.lib.fredopt_feasibility_step(self.h, _ptr(x, np.float32)[0], float(relaxation),
                                                      float(prio_scale), NORMS[norm], _ptr(w, np.float32)[0],
                                                      DEVICE_PTR if dev else 0))
        return w

    def sweep_step(self, x, n_blocks, relaxation=1.0, prio_scale=1.0, norm="all"):
        """One block-iterative sweep of Fig. 2 over n_blocks voxel blocks from x."""
        dev = _on_device(x)
        w = self._out(dev, self.n_spots)
        self._check(self.lib.fredopt_sweep_step(self.h, _ptr(x, np.float32)[0], float(relaxation),
                                                float(prio_scale), NORMS[norm], int(n_blocks),
                                                _ptr(w, np.float32)[0], DEVICE_PTR if dev else 0))
        return w

    def objective(self, x):
        dev = _on_device(x)
        g = self._out(dev, self.n_spots)
        f = ctypes.c_double()
        self._check(self.lib.fredopt_objective(self.h, _ptr(x, np.float32)[0], ctypes.byref(f),
                                               _ptr(g, np.float32)[0], DEVICE_PTR if dev else 0))
        return f.value, g

    # ---------------------------------------------------------- volume statistics
    def volume_stats(self, requests, w=None):
        """fredopt_volume_stats.  requests: dicts with quantity ("DOSE", "CDL",
        "LETD"), struct_bit, and optional edges (n_bins + 1 floats) and fracs.
        w: fluence (host or CUDA), None = the current iterate of a begun solve.
        Returns one dict per request: counts (int64[n_bins]), at_volume
        (float32[n_fracs]), n_voxels."""
        arr = (VolumeRequest * max(1, len(requests)))()
        keep, outs = [], []
        for i, r in enumerate(requests):
            edges = None if r.get("edges") is None else np.ascontiguousarray(r["edges"], np.float32)
            fracs = None if r.get("fracs") is None else np.ascontiguousarray(r["fracs"], np.float64)
            nb = 0 if edges is None else max(0, len(edges) - 1)
            nf = 0 if fracs is None else len(fracs)
            counts = np.zeros(max(1, nb), np.int64)
            at = np.zeros(max(1, nf), np.float32)
            keep += [edges, fracs]
            outs.append((counts, at, nb, nf))
            arr[i] = VolumeRequest(QUANTITIES[r["quantity"]], int(r["struct_bit"]), nb, nf,
                                   edges.ctypes.data if nb else None, fracs.ctypes.data if nf else None,
                                   counts.ctypes.data, at.ctypes.data, 0)
        dev = w is not None and _on_device(w)
        p, kw = _ptr(w, np.float32)
        self._check(self.lib.fredopt_volume_stats(self.h, p, DEVICE_PTR if dev else 0, len(requests), arr))
        return [{"counts": c[:nb], "at_volume": a[:nf], "n_voxels": int(arr[i].n_voxels)}
                for i, (c, a, nb, nf) in enumerate(outs)]

    def quantity_map(self, w, quantity):
        """fredopt_quantity_map: the per-voxel DOSE, CDL or LETD map (voxel order)
        of fluence w (None = the current iterate of a begun solve)."""
        dev = w is not None and _on_device(w)
        out = self._out(dev, self.n_vox)
        self._check(self.lib.fredopt_quantity_map(self.h, _ptr(w, np.float32)[0], QUANTITIES[quantity],
                                                  _ptr(out, np.float32)[0], DEVICE_PTR if dev else 0))
        return out

    def derive_cdl_limits(self, w, oar_bits, frac=0.30, priority=1.0):
        """CDL_MAX constraints at the cDL value received by `frac` of each OAR's
        volume for fluence w (cDL30 for frac = 0.3)."""
        res = self.volume_stats([{"quantity": "CDL", "struct_bit": b, "fracs": [frac]} for b in oar_bits], w)
        return [{"struct_bit": int(b), "kind": "CDL_MAX", "bound": float(r["at_volume"][0]),
                 "priority": float(priority)} for b, r in zip(oar_bits, res)]

    def coverage(self, ptv_bit, prescription, w=None, volume=0.98, level=0.95):
        """PTV coverage rule: (value received by `volume` of the PTV, voxels at
        or above level * prescription, PTV voxels, rule satisfied)."""
        t = np.float32(level * prescription)
        r = self.volume_stats([{"quantity": "DOSE", "struct_bit": ptv_bit, "fracs": [volume],
                                "edges": [t, np.inf]}], w)[0]
        d = float(r["at_volume"][0])
        return d, int(r["counts"][0]), r["n_voxels"], bool(d >= t)

    # ---------------------------------------------------------- inspection
    def get_rows(self):
        sz = self.sizes()
        vox = np.empty(sz["n_rows"], np.int64)
        mask = np.empty(sz["n_rows"], np.uint32)
        self._check(self.lib.fredopt_get_rows(self.h, vox.ctypes.data, mask.ctypes.data))
        return vox, mask

    def get_csc(self):
        sz = self.sizes()
        cp = np.empty(sz["n_spots"] + 1, np.int64)
        row = np.empty(max(1, sz["nnz_rows"]), np.int32)
        D = np.empty(max(1, sz["nnz_rows"]), np.float32)
        L = np.empty(max(1, sz["nnz_rows"]), np.float32)
        self._check(self.lib.fredopt_get_csc(self.h, cp.ctypes.data, row.ctypes.data, D.ctypes.data, L.ctypes.data))
        m = sz["nnz_rows"]
        return cp, row[:m], D[:m], L[:m]

    def get_moments(self):
        n = self.sizes()["n_rows"]
        a, b, c = (np.empty(max(1, n), np.float64) for _ in range(3))
        self._check(self.lib.fredopt_get_moments(self.h, a.ctypes.data, b.ctypes.data, c.ctypes.data))
        return a[:n], b[:n], c[:n]

    def set_timing(self, enable: bool):
        self._check(self.lib.fredopt_set_timing(self.h, 1 if enable else 0))

    def get_timing(self):
        ms = (ctypes.c_double * KCLASS_N)()
        cnt = (ctypes.c_int64 * KCLASS_N)()
        self._check(self.lib.fredopt_get_timing(self.h, ms, cnt))
        return {KCLASS_NAMES[i]: (ms[i], cnt[i]) for i in range(KCLASS_N)}

    def launch_count(self) -> int:
        return int(self.lib.fredopt_launch_count(self.h))

    def check_wait(self, arrive: bool, spins: int = 0):
        """Run the bounded device-side wait alone (fredopt_check_wait).
        Returns (status, device ms): status 0 when the wait completed,
        ERR_TIMEOUT when it gave up (the handle stays usable); any other
        error raises FredoptError."""
        ms = ctypes.c_float()
        rc = self.lib.fredopt_check_wait(self.h, int(bool(arrive)), int(spins), ctypes.byref(ms))
        if rc != ERR_TIMEOUT:
            self._check(rc)
        return rc, ms.value

    def autotune(self, reps: int = 3):
        """Time candidate tile weights and keep the fastest (results unchanged)."""
        r, c = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.fredopt_autotune(self.h, int(reps), ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def tuning(self):
        r, c = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.fredopt_get_tuning(self.h, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value


def kernel_arch(device: int = 0):
    """(forward binary, transposed-product binary, PTX) architecture versions
    of the library's kernels on `device` (fredopt_kernel_arch; 103 = sm_103)."""
    lib = load_library()
    v = [ctypes.c_int() for _ in range(3)]
    rc = lib.fredopt_kernel_arch(int(device), *[ctypes.byref(x) for x in v])
    if rc != OK:
        raise FredoptError(rc, lib.fredopt_strerror(rc).decode())
    return tuple(x.value for x in v)


def footprint_bytes(n_vox, n_spots, nnz, fmt="fp32") -> int:
    return int(load_library().fredopt_footprint_bytes(int(n_vox), int(n_spots), int(nnz), FORMATS[fmt]))


class Server:
    """Continuous-batching server on one GPU (fredopt_server_*).  Host arrays
    of a request are kept referenced here until the request is done."""

    def __init__(self, device: int = 0, mem_cap_bytes: float = 180e9, max_active: int = 8, round_iters: int = 10):
        self.lib = load_library()
        s = ctypes.c_void_p()
        rc = self.lib.fredopt_server_create(ctypes.byref(s), device, int(mem_cap_bytes), max_active, round_iters)
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        self.s = s
        self._keep = {}

    def submit(self, plan, fmt="fp32", rows="all", iters=None, alpha=None, relaxation=None, w0=None,
               params: Params | None = None, **kw) -> int:
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(x, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        r = Request()
        r.n_vox = plan.n_vox
        r.nnz = plan.nnz
        r.n_spots = plan.n_spots
        r.format = FORMATS[fmt] | ROWS[rows]
        r.row_ptr = arr(plan.row_ptr, np.int64)
        r.col = arr(plan.col, np.int32)
        r.D_val = arr(plan.D, np.float32)
        r.L_val = arr(plan.L, np.float32)
        r.voxel_mask = arr(plan.mask, np.uint32)
        con = (Constraint * max(1, len(plan.constraints)))()
        for i, c in enumerate(plan.constraints):
            con[i] = Constraint(int(c["struct_bit"]), KINDS[c["kind"]], float(c["bound"]), float(c["priority"]))
        obj = (ObjectiveTerm * max(1, len(plan.objective)))()
        for i, t in enumerate(plan.objective):
            obj[i] = ObjectiveTerm(int(t["struct_bit"]), QUANTITIES[t["quantity"]], float(t["target"]),
                                   float(t["weight"]))
        keep += [con, obj]
        r.n_constraints, r.n_objective = len(plan.constraints), len(plan.objective)
        r.constraints, r.objective = con, obj
        r.w0 = arr(plan.w0 if w0 is None else w0, np.float32)
        r.iters = int(plan.iters if iters is None else iters)
        r.alpha = float(plan.alpha if alpha is None else alpha)
        r.relaxation = float(plan.relaxation if relaxation is None else relaxation)
        r.params = params if params is not None else default_params(**kw)
        out = (np.empty(plan.n_spots, np.float32), np.empty(plan.n_vox, np.float32), np.empty(plan.n_vox, np.float32))
        keep += list(out)
        r.w_out, r.dose_out, r.letd_out = (o.ctypes.data for o in out)
        t = ctypes.c_int64()
        rc = self.lib.fredopt_server_submit(self.s, ctypes.byref(r), ctypes.byref(t))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        self._keep[t.value] = (keep, out)
        return t.value

    def poll(self, ticket) -> dict:
        info = TicketInfo()
        rc = self.lib.fredopt_server_poll(self.s, ticket, ctypes.byref(info))
        if rc != OK:
            raise FredoptError(rc, "bad ticket")
        return info.as_dict()

    def wait(self, ticket, timeout=600.0):
        """Returns (info, w, dose, letd) once the request is done (or failed)."""
        info = TicketInfo()
        rc = self.lib.fredopt_server_wait(self.s, ticket, float(timeout), ctypes.byref(info))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        keep, out = self._keep.pop(ticket)
        return (info.as_dict(),) + tuple(out)

    def drain(self, timeout=3600.0):
        rc = self.lib.fredopt_server_drain(self.s, float(timeout))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())

    def stats(self):
        m, a, q = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
        self.lib.fredopt_server_stats(self.s, ctypes.byref(m), ctypes.byref(a), ctypes.byref(q))
        return dict(mem_used=m.value, active=a.value, queued=q.value)

    def close(self):
        if getattr(self, "s", None):
            self.lib.fredopt_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Iterations of several begun plans as CUDA graphs of one iteration, or
    of `depth` iterations, of every plan (fredopt_batch_*)."""

    def __init__(self, handles, depth: int = 1):
        self.lib = load_library()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.h for h in self.handles])
        b = ctypes.c_void_p()
        rc = self.lib.fredopt_batch_create_depth(ctypes.byref(b), arr, len(self.handles), int(depth))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        self.b = b

    def iterate(self, iters: int):
        rc = self.lib.fredopt_batch_iterate(self.b, int(iters))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())

    def sync(self) -> float:
        ms = ctypes.c_double()
        rc = self.lib.fredopt_batch_sync(self.b, ctypes.byref(ms))
        if rc != OK:
            raise FredoptError(rc, self.lib.fredopt_strerror(rc).decode())
        return ms.value

    def close(self):
        if getattr(self, "b", None):
            self.lib.fredopt_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def superiorize_batch(handles, w0s, iters, alpha, relaxation, params: Params | None = None, **kw):
    """fredopt_superiorize_batch with host arrays; returns [(w, dose, letd, report)]."""
    lib = load_library()
    n = len(handles)
    if params is None:
        params = default_params(**kw)
    hs = (ctypes.c_void_p * n)(*[h.h for h in handles])
    w0a = [np.ascontiguousarray(w, np.float32) for w in w0s]
    outs = [(np.empty(h.n_spots, np.float32), np.empty(h.n_vox, np.float32), np.empty(h.n_vox, np.float32))
            for h in handles]
    ptr = lambda xs: (ctypes.c_void_p * n)(*[x.ctypes.data for x in xs])
    reps = (Report * n)()
    rc = lib.fredopt_superiorize_batch(hs, n, ptr(w0a), int(iters), float(alpha), float(relaxation),
                                       ctypes.byref(params), ptr([o[0] for o in outs]), ptr([o[1] for o in outs]),
                                       ptr([o[2] for o in outs]), reps, 0)
    if rc != OK:
        raise FredoptError(rc, lib.fredopt_strerror(rc).decode())
    return [o + (reps[i].as_dict(),) for i, o in enumerate(outs)]
