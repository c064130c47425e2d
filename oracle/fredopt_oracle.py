"""Plain FP64 CPU oracle of simultaneous dose and LETd plan optimisation by
superiorized feasibility seeking (Sec. 2.4.3, Fig. 2, Fig. 3, Eq. 2).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs are the only users.  Nothing here is shared with,
or imported by, the CUDA library.

Everything is FP64; the influence values (FP32 inputs) are read as FP64.
Library primitives used as single steps: scipy sparse matrix-vector products
and a stable numpy sort.  There is no blocking, fusion or reordering.

Readings of the paper taken here (where it is silent, garbled or
inconsistent):
  R1  The projections are simultaneous (Cimmino): every row is evaluated at
      the same point and the relaxed projections are averaged with weights
      omega_r = p_S / W, W = sum of p_S over all reachable rows (textbook
      Cimmino); option norm='violated' takes W over the currently violated
      rows.  The literal row-action sweep of Fig. 2 is `sequential_ams_sweep`.
  R2  Fig. 2's U_{c,i} in the dose-upper update is U_{D,i}; the dose-lower
      update's L_{cDLET} is L_{D,i}; the cDL upper update's bound is
      U_{cDLET,i}.
  R3  Lower-bound updates move TOWARD the bound: every violated half-space
      a.x <= b or a.x >= b is projected as x + lam*omega*(b - a.x)/|a|^2 * a
      (Fig. 2 prints a sign that would push the dose further below the bound).
  R4  The feasibility step of Fig. 3 is applied to the perturbed point
      fluence^{k,N} (the text says the perturbations are inserted into the
      feasibility-seeking iteration; as printed, Fig. 3 would discard them).
  R5  Trial steps are beta = beta0 * alpha^s with one global trial counter s
      that advances on every trial (Fig. 3 starts at s = -1 and increments
      before use, so the first step is beta0 * alpha^0); beta0 defaults to
      0.1 * ||w0||_2.
  R6  The perturbation direction is the unit negative gradient -g/||g||
      (bounded perturbations, Sec. 2.3); grad_normalize=False gives Fig. 3's
      raw -grad.
  R7  A trial is accepted when the objective does not ascend (f_new <= f);
      the trial loop is capped at max_trials; when the cap is hit the point
      is unchanged and s has still advanced.  A zero gradient skips the step.
  R8  reductionsN defaults to 1; eta defaults to 1 and multiplies the
      priorities (w_k = eta^k w).
  R9  Objective (Eq. 2, generalised): f(x) = sum over terms, over voxels i of
      the term's structure, of weight * (q_i(x) - target)^2 with q = Dx
      (DOSE) or c*Lx (CDL).  The default plan objective is the OAR cDL term
      with target 0; Eq. 2 literal is PTV DOSE (target = prescription) plus
      OAR CDL (target = the cDL limit).
  R10 The LETd limit LETd <= Lam is the half-space (L_i - Lam*D_i).x <= 0;
      LETD_MIN the reverse.  Rows whose |a_r|^2 is zero are unreachable and
      are skipped (not counted in W).
  R11 A voxel in several structures contributes one row per (structure,
      constraint); rows are ordered by constraint table order, then voxel.
  R12 LETd output = Lw/Dw where Dw > 0, else 0 (Eq. 1 with the denominator
      taken as the dose, Sec. 2.2).
  R13 Block-iterative form of Fig. 2 (`block_iterative_sweep`): the rows are
      split into blocks that are visited in turn; inside a block the rows are
      projected simultaneously at the block's starting point with weights
      p_r / W_B (W_B over the block's reachable rows, or its violated rows),
      so a single block is R1's Cimmino step and one row per block is Fig. 2's
      row-action sweep with unit priorities.  Fluence >= 0 is imposed once,
      after the sweep, as in Fig. 2's last loop.  The blocks used for plans
      (`sweep_blocks`) are groups of S = ceil(|C| / n_blocks) consecutive
      voxels of C, the voxels that lie in a structure and have influence
      entries, in ascending voxel order; all rows of a voxel share its block.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

C_CDL = 0.04  # um/keV: the constant c in cDL = c * dose * LETd (Sec. 2.4)

_MAX_KINDS = ("DOSE_MAX", "CDL_MAX", "LETD_MAX")
_MIN_KINDS = ("DOSE_MIN", "CDL_MIN", "LETD_MIN")


@dataclasses.dataclass
class Problem:
    D: sp.csr_matrix          # V x n, FP64
    L: sp.csr_matrix          # V x n, FP64 (LET-weighted dose)
    mask: np.ndarray          # uint32[V]
    constraints: list
    objective: list
    c: float = C_CDL

    @property
    def n_vox(self) -> int:
        return self.D.shape[0]

    @property
    def n_spots(self) -> int:
        return self.D.shape[1]


def build_problem(row_ptr, col, D, L, n_spots, mask, constraints, objective, c=C_CDL) -> Problem:
    V = len(row_ptr) - 1
    Dm = sp.csr_matrix((np.asarray(D, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(V, n_spots))
    Lm = sp.csr_matrix((np.asarray(L, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(V, n_spots))
    return Problem(D=Dm, L=Lm, mask=np.asarray(mask, np.uint32), constraints=list(constraints),
                   objective=list(objective), c=float(c))


# ---------------------------------------------------------------- products

def forward(P: Problem, w):
    """Dose Dw and LET-weighted dose Lw of every voxel (Sec. 2.2; Fig. 2's
    inner products <D_i, fluence>)."""
    w = np.asarray(w, np.float64)
    return P.D @ w, P.L @ w


def letd(dose, lw):
    """Dose-averaged LET = (LET-weighted dose)/(dose), Eq. (1); 0 where dose is 0."""
    dose = np.asarray(dose, np.float64)
    out = np.zeros_like(dose)
    nz = dose > 0
    out[nz] = np.asarray(lw, np.float64)[nz] / dose[nz]
    return out


def transpose_csr(row_ptr, col, n_cols, *vals):
    """CSC copy of a CSR matrix: column pointers, row indices ascending within
    each column, and the values moved bit-exactly (stable sort by column of the
    row-major nonzero stream)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    n_rows = len(row_ptr) - 1
    rows = np.repeat(np.arange(n_rows, dtype=np.int64), np.diff(row_ptr))
    order = np.argsort(col, kind="stable")
    col_ptr = np.zeros(n_cols + 1, np.int64)
    col_ptr[1:] = np.cumsum(np.bincount(col, minlength=n_cols))
    return (col_ptr, rows[order].astype(np.int32)) + tuple(np.asarray(v)[order] for v in vals)


# ---------------------------------------------------------------- constraints

@dataclasses.dataclass
class Rows:
    A: sp.csr_matrix     # m x n, one half-space normal per row
    b: np.ndarray        # bounds
    upper: np.ndarray    # True: a.x <= b ; False: a.x >= b
    p: np.ndarray        # structure priority of the row
    voxel: np.ndarray    # voxel index
    cidx: np.ndarray     # index into the constraint table
    norm2: np.ndarray    # |a_r|^2
    unreachable: int     # rows dropped because |a_r|^2 == 0


def constraint_rows(P: Problem) -> Rows:
    """All half-spaces of the plan (Fig. 2 with the spec LETd rows).

    DOSE_*: a = D_i,        b = bound      (Gy)
    CDL_* : a = c * L_i,    b = bound      (Gy)
    LETD_*: a = L_i - Lam*D_i, b = 0, Lam = bound (keV/um)
    """
    blocks, bs, ups, ps, vox, cid, n2s = [], [], [], [], [], [], []
    dropped = 0
    for ci, con in enumerate(P.constraints):
        kind = con["kind"]
        idx = np.nonzero((P.mask >> np.uint32(con["struct_bit"])) & np.uint32(1))[0]
        Di = P.D[idx]
        Li = P.L[idx]
        if kind.startswith("DOSE"):
            A, b = Di, float(con["bound"])
        elif kind.startswith("CDL"):
            A, b = P.c * Li, float(con["bound"])
        elif kind.startswith("LETD"):
            A, b = Li - float(con["bound"]) * Di, 0.0
        else:
            raise ValueError(f"unknown constraint kind {kind}")
        A = sp.csr_matrix(A)
        n2 = np.asarray(A.multiply(A).sum(axis=1)).ravel()
        keep = n2 > 0
        dropped += int((~keep).sum())
        blocks.append(A[keep])
        k = int(keep.sum())
        bs.append(np.full(k, b))
        ups.append(np.full(k, kind in _MAX_KINDS))
        ps.append(np.full(k, float(con["priority"])))
        vox.append(idx[keep])
        cid.append(np.full(k, ci))
        n2s.append(n2[keep])
    if blocks:
        A = sp.vstack(blocks).tocsr()
    else:
        A = sp.csr_matrix((0, P.n_spots))
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return Rows(A=A, b=cat(bs, np.float64), upper=cat(ups, bool), p=cat(ps, np.float64),
                voxel=cat(vox, np.int64), cidx=cat(cid, np.int64), norm2=cat(n2s, np.float64),
                unreachable=dropped)


def violations(R: Rows, x):
    """Amount by which each row is violated at x (0 if satisfied)."""
    v = R.A @ np.asarray(x, np.float64)
    return np.where(R.upper, np.maximum(v - R.b, 0.0), np.maximum(R.b - v, 0.0))


def cimmino_step(R: Rows, x, lam: float, prio_scale: float = 1.0, norm: str = "all", clip: bool = True):
    """One simultaneous relaxed projection step from x, then fluence >= 0.

    Each violated row r is projected as t_r = (b_r - a_r.x)/|a_r|^2 (R3);
    x+ = x + lam * sum_r omega_r t_r a_r with omega_r = prio_scale*p_r/W (R1);
    then every negative component is set to 0 (Fig. 2, last loop).
    """
    x = np.asarray(x, np.float64)
    v = R.A @ x
    viol = np.where(R.upper, v > R.b, v < R.b)
    t = np.where(viol, (R.b - v) / np.where(R.norm2 > 0, R.norm2, 1.0), 0.0)
    if norm == "all":
        W = R.p.sum()
    elif norm == "violated":
        W = R.p[viol].sum()
    else:
        raise ValueError(norm)
    if W <= 0:
        step = np.zeros_like(x)
    else:
        omega = prio_scale * R.p / W
        step = R.A.T @ (omega * t)
    xn = x + lam * step
    if clip:
        xn = np.maximum(xn, 0.0)
    return xn


def sequential_ams_sweep(R: Rows, x, lam: float, prio_scale: float = 1.0, clip: bool = True):
    """Fig. 2 literally as a row-action sweep (with R2, R3): rows in table
    order, each projected at the current point with relaxation lam * p_r,
    then fluence >= 0.  Python loop: small cases only."""
    x = np.array(x, np.float64)
    A = R.A
    for r in range(A.shape[0]):
        s, e = A.indptr[r], A.indptr[r + 1]
        cols, vals = A.indices[s:e], A.data[s:e]
        v = float(vals @ x[cols])
        if (R.upper[r] and v > R.b[r]) or ((not R.upper[r]) and v < R.b[r]):
            x[cols] += lam * prio_scale * R.p[r] * (R.b[r] - v) / R.norm2[r] * vals
    if clip:
        x = np.maximum(x, 0.0)
    return x


def sweep_blocks(P: Problem, R: Rows, n_blocks: int):
    """Blocks of R13: row indices of R per block, in visiting order."""
    nz = np.diff(P.D.indptr) > 0
    C = np.nonzero((P.mask != 0) & nz)[0]
    if len(C) == 0:
        return []
    S = -(-len(C) // max(1, int(n_blocks)))
    group = np.full(P.n_vox, -1, np.int64)
    group[C] = np.arange(len(C)) // S
    g = group[R.voxel]
    return [np.nonzero(g == b)[0] for b in range(int(group[C[-1]]) + 1)]


def block_iterative_sweep(R: Rows, x, lam: float, blocks, prio_scale: float = 1.0, norm: str = "all",
                          clip: bool = True):
    """One block-iterative sweep (R13): for each block B in order, from the
    current point x, x <- x + lam * prio_scale * sum_{r in B} (p_r / W_B) t_r a_r
    with t_r = (b_r - a_r.x)/|a_r|^2 for the violated rows of B (R3); then
    fluence >= 0."""
    x = np.array(x, np.float64)
    for B in blocks:
        A = R.A[B]
        v = A @ x
        viol = np.where(R.upper[B], v > R.b[B], v < R.b[B])
        t = np.where(viol, (R.b[B] - v) / R.norm2[B], 0.0)
        if norm == "all":
            W = R.p[B].sum()
        elif norm == "violated":
            W = R.p[B][viol].sum()
        else:
            raise ValueError(norm)
        if W > 0:
            x = x + lam * (A.T @ (prio_scale * R.p[B] / W * t))
    if clip:
        x = np.maximum(x, 0.0)
    return x


# ---------------------------------------------------------------- objective

def _term_rows(P: Problem, term):
    return np.nonzero((P.mask >> np.uint32(term["struct_bit"])) & np.uint32(1))[0]


def objective(P: Problem, x) -> float:
    """Eq. (2) generalised (R9): sum_terms sum_{i in S} weight*(q_i(x) - target)^2."""
    dose, lw = forward(P, x)
    f = 0.0
    for term in P.objective:
        idx = _term_rows(P, term)
        q = dose[idx] if term["quantity"] == "DOSE" else P.c * lw[idx]
        f += float(term["weight"]) * float(np.sum((q - float(term["target"])) ** 2))
    return f


def objective_gradient(P: Problem, x):
    """grad f = sum_terms 2*weight * J^T (q - target), J = D_S or c*L_S."""
    dose, lw = forward(P, x)
    rD = np.zeros(P.n_vox)
    rL = np.zeros(P.n_vox)
    for term in P.objective:
        idx = _term_rows(P, term)
        wgt, tgt = float(term["weight"]), float(term["target"])
        if term["quantity"] == "DOSE":
            rD[idx] += 2.0 * wgt * (dose[idx] - tgt)
        else:
            rL[idx] += 2.0 * wgt * P.c * (P.c * lw[idx] - tgt)
    return P.D.T @ rD + P.L.T @ rL


# ---------------------------------------------------------------- Fig. 3

def superiorize(P: Problem, w0, iters: int, alpha: float, lam: float, beta0: float | None = None,
                eta: float = 1.0, reductions: int = 1, max_trials: int = 50, norm: str = "all",
                grad_normalize: bool = True, sequential: bool = False, rows: Rows | None = None,
                s0: int = 0, k0: int = 0, sweep: int = 0):
    """Superiorized feasibility seeking (Fig. 3 with R4-R8).

    For k = 0..iters-1: perturbation phase from w^k (reductions steps, each a
    trial loop with beta = beta0*alpha^s, s advancing on every trial, accepted
    when f does not ascend, f evaluated afresh at every trial), then one
    feasibility step (Cimmino; the block-iterative sweep of R13 over `sweep`
    blocks if sweep > 0; the Fig. 2 row-action sweep if sequential=True) from
    the perturbed point with priorities scaled by eta^k.

    Returns (w, log); log[k] = dict(k, s, accepted, beta, f_start, f_end, gnorm).
    """
    w = np.asarray(w0, np.float64).copy()
    if beta0 is None:
        beta0 = 0.1 * float(np.linalg.norm(w))
    R = constraint_rows(P) if rows is None else rows
    blocks = sweep_blocks(P, R, sweep) if sweep > 0 else None
    s = int(s0)
    log = []
    for k in range(k0, k0 + iters):
        x = w.copy()
        f_start = objective(P, x) if reductions > 0 else 0.0
        f_x = f_start
        acc, beta_acc, gn = 0, 0.0, 0.0
        for _t in range(reductions):
            g = objective_gradient(P, x)
            gn = float(np.linalg.norm(g))
            if gn == 0.0:
                continue
            v = -g / gn if grad_normalize else -g
            for _trial in range(max_trials):
                beta = beta0 * alpha ** s
                s += 1
                x_new = x + beta * v
                f_new = objective(P, x_new)
                if f_new <= f_x:
                    x, f_x = x_new, f_new
                    acc += 1
                    beta_acc = beta
                    break
        scale = eta ** k
        if sequential:
            w = sequential_ams_sweep(R, x, lam, prio_scale=scale)
        elif blocks is not None:
            w = block_iterative_sweep(R, x, lam, blocks, prio_scale=scale, norm=norm)
        else:
            w = cimmino_step(R, x, lam, prio_scale=scale, norm=norm)
        log.append(dict(k=k, s=s, accepted=acc, beta=beta_acc, f_start=f_start, f_end=f_x, gnorm=gn))
    return w, log


def final_report(P: Problem, w, rows: Rows | None = None):
    """Dose, LETd, objective and the largest violation per constraint kind."""
    R = constraint_rows(P) if rows is None else rows
    dose, lw = forward(P, w)
    viol = violations(R, w)
    maxv = {}
    for ci, con in enumerate(P.constraints):
        sel = R.cidx == ci
        maxv[ci] = float(viol[sel].max()) if sel.any() else 0.0
    return dict(dose=dose, lw=lw, letd=letd(dose, lw), objective=objective(P, w),
                max_violation=maxv, n_violated=int((viol > 0).sum()), unreachable=R.unreachable)
