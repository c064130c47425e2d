"""Plain FP64 CPU oracle of the plan-evaluation statistics the paper uses to
select constraints and judge plans (Sec. 2.4.1): volume histograms of dose,
LETd and c x dose x LETd (DVH, LVH, cDLVH), the value received by a given
fraction of a structure's volume (e.g. cDL30, D98), the PTV coverage rule,
and the derivation of OAR cDL upper limits from an initial plan.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs are the only users.  Nothing here is shared with,
or imported by, the CUDA library.

Definitions (where the paper states the idea but not the formula):
  V1  The voxel quantities are dose = Dw, LETd = Lw/Dw (0 where Dw = 0,
      Eq. 1) and cDL = c * dose * LETd = c * Lw (Sec. 2.4, c = 0.04 um/keV).
  V2  A structure S is the set of voxels whose mask has bit S set.
  V3  Histogram bin b of edges e counts the voxels of S with
      e[b] <= v < e[b+1] (half-open; a last edge of +inf makes the last bin
      cumulative).  The cumulative volume histogram at d is the fraction of
      S with v >= d.
  V4  "The value received by a fraction x of the volume" is the largest d
      with at least that fraction of S at v >= d, i.e. the k-th largest value
      of S with k = ceil(x * n), n = |S|, k kept in [1, n].  The product
      t = x * n is taken in FP64; a t within 1e-9 * max(1, t) of an integer
      counts as that integer, so that a decimal fraction such as 0.14 of 50
      voxels means 7 voxels, not 8 (0.14 * 50 rounds to 7.000000000000001).
      For n = 0 the value is NaN.
  V5  PTV coverage (Sec. 2.4.1): at least 98% of the PTV receives at least
      95% of the prescribed dose, i.e. D98 >= 0.95 * prescription.
  V6  The OAR cDL limit is cDL30: the cDL value received by 30% of the OAR's
      volume in the initial plan, used as a CDL_MAX bound (Sec. 2.4.1).
"""
from __future__ import annotations

import math

import numpy as np

from .fredopt_oracle import Problem, forward, letd

QUANTITIES = ("dose", "letd", "cdl")


def quantity(P: Problem, w, which: str):
    """Per-voxel dose, LETd or cDL of fluence w in FP64 (V1)."""
    dose, lw = forward(P, w)
    if which == "dose":
        return dose
    if which == "letd":
        return letd(dose, lw)
    if which == "cdl":
        return P.c * lw
    raise ValueError(which)


def structure_voxels(mask, bit: int):
    """Voxel indices of structure `bit` (V2)."""
    mask = np.asarray(mask, np.uint32)
    return np.nonzero((mask >> np.uint32(bit)) & np.uint32(1))[0]


def volume_histogram(values, mask, bit: int, edges):
    """Counts per half-open bin [edges[b], edges[b+1]) over structure `bit` (V3)."""
    v = np.asarray(values)[structure_voxels(mask, bit)]
    edges = np.asarray(edges)
    counts = np.zeros(len(edges) - 1, np.int64)
    for b in range(len(edges) - 1):
        counts[b] = int(np.count_nonzero((v >= edges[b]) & (v < edges[b + 1])))
    return counts


def cumulative_volume(values, mask, bit: int, thresholds):
    """Fraction of structure `bit` with value >= d, for each d (V3)."""
    v = np.asarray(values)[structure_voxels(mask, bit)]
    if len(v) == 0:
        return np.full(len(thresholds), np.nan)
    return np.array([np.count_nonzero(v >= d) / len(v) for d in thresholds])


def at_volume_rank(frac: float, n: int) -> int:
    """k of V4: the rank (1 = largest) of the value received by `frac` of n voxels."""
    if not (0.0 < frac <= 1.0):
        raise ValueError("fraction must lie in (0, 1]")
    t = float(np.float64(frac) * np.float64(n))
    r = math.floor(t + 0.5)
    k = r if abs(t - r) <= 1e-9 * max(1.0, t) else math.ceil(t)
    return min(max(k, 1), n)


def value_at_volume(values, mask, bit: int, frac: float):
    """The value received by fraction `frac` of structure `bit`: its k-th
    largest value (V4).  The values keep their dtype (an FP32 map gives an
    FP32 result)."""
    v = np.asarray(values)[structure_voxels(mask, bit)]
    n = len(v)
    if n == 0:
        return np.nan
    k = at_volume_rank(frac, n)
    return np.sort(v, kind="stable")[::-1][k - 1]


def coverage(dose, mask, ptv_bit: int, prescription: float, volume: float = 0.98, level: float = 0.95):
    """PTV coverage rule (V5): returns (D_volume, fraction of the PTV at or
    above level * prescription, rule satisfied)."""
    d = value_at_volume(dose, mask, ptv_bit, volume)
    v = cumulative_volume(dose, mask, ptv_bit, [level * prescription])[0]
    return float(d), float(v), bool(d >= level * prescription)


def derive_cdl_limits(P: Problem, w, oar_bits, frac: float = 0.30, priority: float = 1.0):
    """CDL_MAX constraints at cDL_{frac} of each OAR for the initial fluence w (V6)."""
    cdl = quantity(P, w, "cdl")
    return [{"struct_bit": int(b), "kind": "CDL_MAX", "bound": float(value_at_volume(cdl, P.mask, b, frac)),
             "priority": float(priority)} for b in oar_bits]
