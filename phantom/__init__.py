"""Seeded synthetic plans: water phantom, structures, pencil-beam fields and
the (D, L) influence-matrix pair in CSR with one shared sparsity pattern.

This module holds INPUTS only.  It has no part of the optimisation method's
arithmetic (no projections, objectives or products with spot weights); both
the CUDA path and the FP64 oracle consume what it produces.  It stands in for
the patient CT, structure set, plan and the Monte Carlo influence matrices
(Sec. 2.1, 2.2, 2.4.1-2.4.2), none of which is available.

Plans are plain data:
  * csr: row_ptr int64[V+1], col int32[nnz] (sorted within a row),
    D float32[nnz] (Gy per unit weight), L float32[nnz] (Gy*keV/um; L = LET*D)
  * mask uint32[V]: bit b set if the voxel belongs to structure b
  * constraints: dicts {struct_bit, kind, bound, priority}; kind is one of the
    strings DOSE_MIN, DOSE_MAX, CDL_MIN, CDL_MAX, LETD_MAX, LETD_MIN
  * objective: dicts {struct_bit, quantity ('DOSE'|'CDL'), target, weight}
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cpp")
_LIB = os.path.join(_HERE, "_phantom.so")
_lock = threading.Lock()
_lib = None

MAX_FIELDS = 8


class PhantomParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("h_mm", ctypes.c_double),
        ("n_fields", ctypes.c_int32),
        ("angle_deg", ctypes.c_double * MAX_FIELDS),
        ("iso_mm", ctypes.c_double * 3),
        ("spots_x", ctypes.c_int32), ("spots_y", ctypes.c_int32),
        ("spot_pitch_mm", ctypes.c_double),
        ("n_layers", ctypes.c_int32),
        ("range_first_mm", ctypes.c_double * MAX_FIELDS),
        ("range_last_mm", ctypes.c_double * MAX_FIELDS),
        ("sigma_mm", ctypes.c_double),
        ("trunc_rel", ctypes.c_double),
        ("noise_rel", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("shift_mm", ctypes.c_double * 3),
        ("density_scale", ctypes.c_double),
        ("dose_at_iso", ctypes.c_double),
        ("table_dz_mm", ctypes.c_double),
        ("n_threads", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the generator into phantom/_phantom.so (host code only)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["g++", "-O3", "-std=c++17", "-shared", "-fPIC", "-pthread",
                                   _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(PhantomParams)
        lib.phantom_n_spots.argtypes = [P]; lib.phantom_n_spots.restype = ctypes.c_int64
        lib.phantom_n_voxels.argtypes = [P]; lib.phantom_n_voxels.restype = ctypes.c_int64
        lib.phantom_amplitude.argtypes = [P]; lib.phantom_amplitude.restype = ctypes.c_double
        lib.phantom_layer_table.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p]
        lib.phantom_layer_table.restype = ctypes.c_int
        lib.phantom_count.argtypes = [P, ctypes.c_void_p]; lib.phantom_count.restype = ctypes.c_int
        lib.phantom_fill.argtypes = [P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.phantom_fill.restype = ctypes.c_int
        lib.phantom_philox4x32_10.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.phantom_philox4x32_10.restype = None
        _lib = lib
    return _lib


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one 128-bit counter (for the known-answer test)."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.phantom_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def make_params(**kw) -> PhantomParams:
    p = PhantomParams()
    p.density_scale = 1.0
    p.table_dz_mm = 0.1
    p.trunc_rel = 1e-4
    p.sigma_mm = 4.0
    p.dose_at_iso = 2.0
    for k, v in kw.items():
        if k in ("angle_deg", "range_first_mm", "range_last_mm"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        elif k in ("iso_mm", "shift_mm"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def generate(p: PhantomParams):
    """Return (row_ptr int64[V+1], col int32[nnz], D f32[nnz], L f32[nnz])."""
    lib = _load()
    V = lib.phantom_n_voxels(ctypes.byref(p))
    row_nnz = np.empty(V, np.int64)
    if lib.phantom_count(ctypes.byref(p), row_nnz.ctypes.data) != 0:
        raise ValueError("phantom_count failed")
    row_ptr = np.zeros(V + 1, np.int64)
    np.cumsum(row_nnz, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, np.int32)
    D = np.empty(nnz, np.float32)
    L = np.empty(nnz, np.float32)
    if lib.phantom_fill(ctypes.byref(p), row_ptr.ctypes.data, col.ctypes.data,
                        D.ctypes.data, L.ctypes.data) != 0:
        raise ValueError("phantom_fill failed")
    return row_ptr, col, D, L


def layer_table(p: PhantomParams, field: int, layer: int, n: int = 4096):
    """Depth dose (arbitrary units) and LET (keV/um) of one layer on the table grid."""
    lib = _load()
    dd = np.zeros(n, np.float64)
    let = np.zeros(n, np.float64)
    m = lib.phantom_layer_table(ctypes.byref(p), field, layer, n, dd.ctypes.data, let.ctypes.data)
    if m < 0:
        raise ValueError("bad field/layer")
    return dd[:min(m, n)], let[:min(m, n)]


# ----------------------------------------------------------------- geometry

def voxel_index_grids(nx: int, ny: int, nz: int):
    """Integer voxel indices (i, j, k) of every row, row = (k*ny + j)*nx + i."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel().astype(np.int64), j.ravel().astype(np.int64), k.ravel().astype(np.int64)


def voxel_centres_mm(nx: int, ny: int, nz: int, h: float):
    i, j, k = voxel_index_grids(nx, ny, nz)
    return (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h


# ----------------------------------------------------------------- plans

@dataclasses.dataclass
class Plan:
    name: str
    shape: tuple            # (nx, ny, nz)
    h_mm: float
    params: PhantomParams
    row_ptr: np.ndarray
    col: np.ndarray
    D: np.ndarray
    L: np.ndarray
    mask: np.ndarray        # uint32[V]
    structures: list        # [{name, bit, role}]
    constraints: list       # [{struct_bit, kind, bound, priority}]
    objective: list         # [{struct_bit, quantity, target, weight}]
    w0: np.ndarray          # float32[n]
    iters: int
    alpha: float
    relaxation: float
    prescription: float = 2.0

    @property
    def n_vox(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n_spots(self) -> int:
        return int(self.w0.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def default_objective(structures, constraints):
    """OAR c*dose*LETd objective with zero target (one term per OAR)."""
    terms = []
    for s in structures:
        if s["role"] != "oar":
            continue
        pr = [c["priority"] for c in constraints if c["struct_bit"] == s["bit"]]
        terms.append(dict(struct_bit=s["bit"], quantity="CDL", target=0.0,
                          weight=float(pr[0]) if pr else 1.0))
    return terms


def tiny_params(seed: int = 0, noise: float = 0.01, shift_mm=(0.0, 0.0, 0.0), density_scale: float = 1.0):
    """32^3 water phantom at 3 mm, one field along +z, 15x15 spots at 4 mm,
    10 layers with ranges evenly spaced over the PTV depth span."""
    h = 3.0
    c = 16.5 * h                      # centre of voxel 16
    # PTV ball of radius 8 voxels around voxel 16 spans depths 8h..25h (voxel edges)
    return make_params(nx=32, ny=32, nz=32, h_mm=h, n_fields=1, angle_deg=[0.0],
                       iso_mm=[c, c, c], spots_x=15, spots_y=15, spot_pitch_mm=4.0,
                       n_layers=10, range_first_mm=[8 * h], range_last_mm=[25 * h],
                       sigma_mm=4.0, trunc_rel=1e-4, noise_rel=noise, seed=seed,
                       shift_mm=list(shift_mm), density_scale=density_scale, dose_at_iso=2.0)


def tiny_masks():
    """PTV: integer ball |(i,j,k) - (16,16,16)|^2 <= 64 (bit 0).
    OAR: cylinder along y, (i-16)^2 + (k-29)^2 <= 16, clipped to the grid (bit 1)."""
    i, j, k = voxel_index_grids(32, 32, 32)
    ptv = (i - 16) ** 2 + (j - 16) ** 2 + (k - 16) ** 2 <= 64
    oar = (i - 16) ** 2 + (k - 29) ** 2 <= 16
    mask = np.zeros(i.shape[0], np.uint32)
    mask |= ptv.astype(np.uint32) << 0
    mask |= oar.astype(np.uint32) << 1
    return mask


def tiny_plan(seed: int = 0, noise: float = 0.01, iters: int = 100) -> Plan:
    """Plain method, tiny: 32^3 voxels, 2250 spots, PTV 2 Gy within [0.95, 1.07],
    OAR dose <= 1.2 Gy and LETd <= 2.5 keV/um; w0 = 1; alpha 0.99; relaxation 1."""
    p = tiny_params(seed=seed, noise=noise)
    row_ptr, col, D, L = generate(p)
    structures = [dict(name="PTV", bit=0, role="target"), dict(name="OAR", bit=1, role="oar")]
    constraints = [
        dict(struct_bit=0, kind="DOSE_MIN", bound=0.95 * 2.0, priority=1.0),
        dict(struct_bit=0, kind="DOSE_MAX", bound=1.07 * 2.0, priority=1.0),
        dict(struct_bit=1, kind="DOSE_MAX", bound=1.2, priority=1.0),
        dict(struct_bit=1, kind="LETD_MAX", bound=2.5, priority=1.0),
    ]
    n = int(p.n_fields * p.n_layers * p.spots_x * p.spots_y)
    return Plan(name="tiny", shape=(32, 32, 32), h_mm=3.0, params=p, row_ptr=row_ptr, col=col,
                D=D, L=L, mask=tiny_masks(), structures=structures, constraints=constraints,
                objective=default_objective(structures, constraints),
                w0=np.ones(n, np.float32), iters=iters, alpha=0.99, relaxation=1.0)


# clinical-size phantom: 200 x 200 x 150 voxels at 2 mm
CLIN_SHAPE = (200, 200, 150)
CLIN_H = 2.0
CLIN_PTV_SEMI = (35.0, 35.0, 29.2)     # mm; 4/3*pi*35*35*29.2 mm^3 = 149.8 cc


def clinical_params(seed: int = 0, noise: float = 0.01, shift_mm=(0.0, 0.0, 0.0),
                    density_scale: float = 1.0, shape=CLIN_SHAPE, h=CLIN_H,
                    spots=(20, 20), layers: int = 25):
    """Three coplanar fields at 0/90/270 degrees; per field a 20 x 20 lateral
    grid at 4 mm and 25 layers 3 mm apart in range (30000 spots in total)."""
    nx, ny, nz = shape
    iso = [0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h]
    a, b, c = CLIN_PTV_SEMI
    angles = [0.0, 90.0, 270.0]
    # ranges spanning the PTV along each beam, centred on the isocentre depth
    span = 3.0 * (layers - 1)
    first, last = [], []
    for ang in angles:
        d_iso = {0.0: iso[2], 90.0: iso[0], 270.0: nx * h - iso[0]}[ang]
        first.append(d_iso - 0.5 * span)
        last.append(d_iso + 0.5 * span)
    return make_params(nx=nx, ny=ny, nz=nz, h_mm=h, n_fields=3, angle_deg=angles, iso_mm=iso,
                       spots_x=spots[0], spots_y=spots[1], spot_pitch_mm=4.0, n_layers=layers,
                       range_first_mm=first, range_last_mm=last, sigma_mm=4.0, trunc_rel=1e-4,
                       noise_rel=noise, seed=seed, shift_mm=list(shift_mm),
                       density_scale=density_scale, dose_at_iso=2.0)


def clinical_structures(shape=CLIN_SHAPE, h=CLIN_H):
    """PTV ellipsoid (bit 0); brainstem-like cylinder r 12 mm along y, distal to
    the 0-degree field (bit 1); chiasm-like slab 4 mm thick (bit 2); two
    eye-like spheres r 12 mm (bit 3).  Positions in mm from the phantom centre."""
    nx, ny, nz = shape
    x, y, z = voxel_centres_mm(nx, ny, nz, h)
    cx, cy, cz = 0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h
    a, b, c = CLIN_PTV_SEMI
    X, Y, Z = x - cx, y - cy, z - cz
    ptv = (X / a) ** 2 + (Y / b) ** 2 + (Z / c) ** 2 <= 1.0
    stem = (X ** 2 + (Z - (c + 14.0)) ** 2 <= 12.0 ** 2) & (np.abs(Y) <= 25.0)
    chiasm = (np.abs(Y - (b + 6.0)) <= 2.0) & (np.abs(X) <= 20.0) & (np.abs(Z) <= 12.0)
    eyes = (((X - 40.0) ** 2 + (Y - 20.0) ** 2 + (Z + 45.0) ** 2 <= 12.0 ** 2)
            | ((X + 40.0) ** 2 + (Y - 20.0) ** 2 + (Z + 45.0) ** 2 <= 12.0 ** 2))
    mask = np.zeros(x.shape[0], np.uint32)
    for bit, m in enumerate((ptv, stem, chiasm, eyes)):
        mask |= m.astype(np.uint32) << bit
    return mask


def clinical_plan(seed: int = 0, noise: float = 0.01, iters: int = 500, shape=CLIN_SHAPE, h=CLIN_H,
                  **kw) -> Plan:
    """Plain method, clinical size: 200x200x150 voxels at 2 mm, 3 fields, 30000
    spots; PTV 150 cc at 2 Gy within [0.95, 1.07]; brainstem-like Dmax 1.2 Gy,
    chiasm-like Dmax 1.0 Gy, eye-like Dmax 0.5 Gy; LETd <= 2.5 / 2.5 / 3.0 keV/um."""
    p = clinical_params(seed=seed, noise=noise, shape=shape, h=h, **kw)
    row_ptr, col, D, L = generate(p)
    structures = [dict(name="PTV", bit=0, role="target"), dict(name="brainstem", bit=1, role="oar"),
                  dict(name="chiasm", bit=2, role="oar"), dict(name="eyes", bit=3, role="oar")]
    constraints = [
        dict(struct_bit=0, kind="DOSE_MIN", bound=0.95 * 2.0, priority=1.0),
        dict(struct_bit=0, kind="DOSE_MAX", bound=1.07 * 2.0, priority=1.0),
        dict(struct_bit=1, kind="DOSE_MAX", bound=1.2, priority=1.0),
        dict(struct_bit=1, kind="LETD_MAX", bound=2.5, priority=1.0),
        dict(struct_bit=2, kind="DOSE_MAX", bound=1.0, priority=1.0),
        dict(struct_bit=2, kind="LETD_MAX", bound=2.5, priority=1.0),
        dict(struct_bit=3, kind="DOSE_MAX", bound=0.5, priority=1.0),
        dict(struct_bit=3, kind="LETD_MAX", bound=3.0, priority=1.0),
    ]
    n = int(p.n_fields * p.n_layers * p.spots_x * p.spots_y)
    return Plan(name="clinical", shape=tuple(shape), h_mm=h, params=p, row_ptr=row_ptr,
                col=col, D=D, L=L, mask=clinical_structures(shape, h), structures=structures,
                constraints=constraints, objective=default_objective(structures, constraints),
                w0=np.ones(n, np.float32), iters=iters, alpha=0.99, relaxation=1.0)


def random_csr(n_rows: int, n_cols: int, density: float, seed: int, let_range=(0.5, 12.0),
               empty_rows: int = 0):
    """Small random (D, L) pair for unit tests: sorted columns, shared pattern,
    positive D, L = LET * D with LET uniform in let_range.  The first
    `empty_rows` rows are left empty."""
    rng = np.random.default_rng(seed)
    rows = []
    for r in range(n_rows):
        if r < empty_rows:
            rows.append(np.zeros(0, np.int64))
            continue
        k = rng.binomial(n_cols, density)
        rows.append(np.sort(rng.choice(n_cols, size=k, replace=False)))
    row_ptr = np.zeros(n_rows + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in rows])
    col = np.concatenate(rows).astype(np.int32) if row_ptr[-1] else np.zeros(0, np.int32)
    D = rng.uniform(0.01, 1.0, size=col.shape[0]).astype(np.float32)
    let = rng.uniform(let_range[0], let_range[1], size=col.shape[0])
    L = (let * D).astype(np.float32)
    return row_ptr, col, D, L


# ----------------------------------------------------------------- batching workloads

ROBUST_SHAPE = (120, 120, 100)
ROBUST_H = 2.5


def _sphere_plan(name, shape, h, ptv_r_mm, angles, spots, layers, pitch, seed, noise, shift_mm=(0.0, 0.0, 0.0),
                 density_scale=1.0, iters=100, layer_mm=3.0):
    """Water phantom with a spherical PTV at the centre and a distal OAR
    cylinder (behind the first field), spots on a lateral grid and layers
    `layer_mm` apart in range spanning the PTV along each field."""
    nx, ny, nz = shape
    iso = [0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h]
    span = layer_mm * (layers - 1)
    first, last = [], []
    for ang in angles:
        d_iso = {0.0: iso[2], 90.0: iso[0], 270.0: nx * h - iso[0], 180.0: nz * h - iso[2]}[ang]
        first.append(d_iso - 0.5 * span)
        last.append(d_iso + 0.5 * span)
    p = make_params(nx=nx, ny=ny, nz=nz, h_mm=h, n_fields=len(angles), angle_deg=list(angles), iso_mm=iso,
                    spots_x=spots, spots_y=spots, spot_pitch_mm=pitch, n_layers=layers, range_first_mm=first,
                    range_last_mm=last, sigma_mm=4.0, trunc_rel=1e-4, noise_rel=noise, seed=seed,
                    shift_mm=list(shift_mm), density_scale=density_scale, dose_at_iso=2.0)
    row_ptr, col, D, L = generate(p)
    x, y, z = voxel_centres_mm(nx, ny, nz, h)
    X, Y, Z = x - iso[0], y - iso[1], z - iso[2]
    ptv = X ** 2 + Y ** 2 + Z ** 2 <= ptv_r_mm ** 2
    oar = (X ** 2 + (Z - (ptv_r_mm + 12.0)) ** 2 <= 10.0 ** 2) & (np.abs(Y) <= 2 * ptv_r_mm)
    mask = ptv.astype(np.uint32) | (oar.astype(np.uint32) << 1)
    structures = [dict(name="PTV", bit=0, role="target"), dict(name="OAR", bit=1, role="oar")]
    constraints = [dict(struct_bit=0, kind="DOSE_MIN", bound=0.95 * 2.0, priority=1.0),
                   dict(struct_bit=0, kind="DOSE_MAX", bound=1.07 * 2.0, priority=1.0),
                   dict(struct_bit=1, kind="DOSE_MAX", bound=1.2, priority=1.0),
                   dict(struct_bit=1, kind="LETD_MAX", bound=2.5, priority=1.0)]
    n = int(p.n_fields * p.n_layers * p.spots_x * p.spots_y)
    return Plan(name=name, shape=tuple(shape), h_mm=h, params=p, row_ptr=row_ptr, col=col, D=D, L=L, mask=mask,
                structures=structures, constraints=constraints,
                objective=default_objective(structures, constraints), w0=np.ones(n, np.float32), iters=iters,
                alpha=0.99, relaxation=1.0)


def batch_plans(n_plans: int = 16, seed: int = 0):
    """Independent plans with PTV volumes log-spaced 20-400 cc in the
    300 x 300 x 250 mm phantom: spots 6 mm apart over the PTV plus 12 mm,
    layers 4 mm apart in range over the PTV depth plus 12 mm, one field below
    150 cc, else two; voxels from 5 mm (smallest PTV) to 3 mm (largest)."""
    plans = []
    vols = np.geomspace(20.0, 400.0, n_plans)
    for i, v in enumerate(vols):
        r = (3.0 * v * 1000.0 / (4.0 * np.pi)) ** (1.0 / 3.0)
        frac = i / max(1, n_plans - 1)
        h = float(np.exp(np.log(5.0) + frac * (np.log(3.0) - np.log(5.0))))
        shape = tuple(int(round(s * ROBUST_H / h)) for s in ROBUST_SHAPE)
        angles = [0.0] if v < 150 else [0.0, 90.0]
        spots = int(np.ceil((2 * r + 12.0) / 6.0))
        layers = int(np.ceil((2 * r + 12.0) / 4.0))
        plans.append(_sphere_plan(f"ptv{v:.0f}cc", shape, h, r, angles, spots, layers, 6.0, seed + i, 0.01,
                                  layer_mm=4.0))
    return plans


def robust_scenarios():
    """27 scenarios: setup shift x in {-3, 0, +3} mm x setup shift y in
    {-3, 0, +3} mm x range (water-equivalent depth) scaled by {0.965, 1, 1.035};
    the shift along the first beam's axis is carried by the range factor."""
    return [((sx, sy, 0.0), rs) for sx in (-3.0, 0.0, 3.0) for sy in (-3.0, 0.0, 3.0)
            for rs in (0.965, 1.0, 1.035)]


def robust_plan(seed: int = 0, noise: float = 0.01, scenarios=None, shape=ROBUST_SHAPE, h=ROBUST_H,
                spots: int = 16, layers: int = 16, pitch: float = 4.0):
    """Robust plan on the 120x120x100 phantom at 2.5 mm (two fields at 0 and
    90 degrees, 2 x 64 x 64 spots ... trimmed to 8192 spots: 16 x 16 lateral x
    16 layers per field): the rows of every scenario's influence matrices are
    stacked, so one spot-weight vector has to meet the constraints in all
    scenarios (structure masks follow the patient).  Returns (plan, nnz per
    scenario).  shape, h, spots, layers and pitch give smaller versions of the
    same geometry (small_robust_plan)."""
    scen = robust_scenarios() if scenarios is None else scenarios
    parts, per = [], []
    for k, (shift, rs) in enumerate(scen):
        pl = _sphere_plan("robust", shape, h, 25.0, [0.0, 90.0], spots, layers, pitch, seed, noise,
                          shift_mm=shift, density_scale=rs)
        parts.append(pl)
        per.append(pl.nnz)
    base = parts[0]
    V = base.n_vox
    row_ptr = np.zeros(V * len(parts) + 1, np.int64)
    off = 0
    for k, pl in enumerate(parts):
        row_ptr[1 + k * V:1 + (k + 1) * V] = pl.row_ptr[1:] + off
        off += pl.nnz
    col = np.concatenate([pl.col for pl in parts])
    D = np.concatenate([pl.D for pl in parts])
    L = np.concatenate([pl.L for pl in parts])
    mask = np.tile(base.mask, len(parts))
    plan = Plan(name=f"robust{len(parts)}", shape=(V * len(parts), 1, 1), h_mm=h, params=base.params, row_ptr=row_ptr,
                col=col, D=D, L=L, mask=mask, structures=base.structures, constraints=base.constraints,
                objective=base.objective, w0=base.w0.copy(), iters=100, alpha=0.99, relaxation=1.0)
    return plan, per


def small_robust_plan(seed: int = 0, noise: float = 0.01, scenarios=None):
    """The robust geometry at test size: the same 300 x 300 x 250 mm phantom
    at 7.5 mm (40 x 40 x 34 voxels), two fields of 6 x 6 spots 8 mm apart x 6
    layers (432 spots), all 27 scenarios stacked (about 2.9e6 nonzeros)."""
    return robust_plan(seed=seed, noise=noise, scenarios=scenarios, shape=(40, 40, 34), h=7.5, spots=6,
                       layers=6, pitch=8.0)
