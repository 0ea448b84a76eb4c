"""Plain FP64 restatement of column-generation DAO (arXiv:1003.5402).

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

Notation follows the paper: voxels j in V, beamlets i in N, apertures k in K,
dose z, aperture intensities y, beamlet intensities x, dual multipliers pi.
``case`` is a ``phantom.Case``-like object with CSR ``indptr/indices/data``
(voxel-major D, FP32 values promoted to FP64 here), per-beam ``rows/cols``,
``voxel_struct`` and per-structure ``is_target, under_w, under_t, over_w,
over_t``.  Beamlet i of beam b, MLC row r, column c is
``i = offset_b + r * cols_b + c`` (beam-major, then row, then column).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np
import scipy.sparse as sp


# ---------------------------------------------------------------------------
# Objective: Eqs. 3-5 in the per-structure form of Eqs. 9-10 (Sec. 4)
# ---------------------------------------------------------------------------

@dataclass
class VoxelTerms:
    """Per-voxel weights and thresholds of the one-sided quadratic penalties.

    alpha[j] = alpha_s / |v_s| for a voxel of target s (Eq. 9), else 0;
    t_under[j] = T_s^-; beta[j] = beta_s / |v_s| (Eq. 10), t_over[j] = T_s^+.
    """
    alpha: np.ndarray
    t_under: np.ndarray
    beta: np.ndarray
    t_over: np.ndarray


def voxel_terms(case, normalize_by_volume: bool = True) -> VoxelTerms:
    """Expand the per-structure criteria of Eqs. 9-10 to voxels.

    Reading: each voxel belongs to exactly one structure (the caller resolved
    overlaps by priority) and |v_s| counts the voxels labelled s.  With
    ``normalize_by_volume=False`` the weights are Eqs. 3-4's per-voxel
    alpha_j = alpha_s, beta_j = beta_s.
    """
    s = np.asarray(case.voxel_struct, dtype=np.int64)
    S = len(case.under_w)
    count = np.bincount(s, minlength=S).astype(np.float64)
    denom = np.where(count > 0, count, 1.0) if normalize_by_volume else np.ones(S)
    is_t = np.asarray(case.is_target, dtype=bool)
    a_s = np.where(is_t, np.asarray(case.under_w, dtype=np.float64), 0.0) / denom
    b_s = np.asarray(case.over_w, dtype=np.float64) / denom
    return VoxelTerms(alpha=a_s[s], t_under=np.asarray(case.under_t, np.float64)[s],
                      beta=b_s[s], t_over=np.asarray(case.over_t, np.float64)[s])


def reoptimisation_terms(T, target_mask=None) -> VoxelTerms:
    """The re-optimisation mode of Sec. 4: Eqs. 3-4 with alpha_j = beta_j = 1 and
    T_j = the planned dose deformed onto the day's anatomy, used as both the
    under- and the over-dose threshold.  Reading: Eq. 3 applies to target
    voxels only (``target_mask``; None means every voxel), Eq. 4 to all."""
    T = np.asarray(T, dtype=np.float64)
    a = np.ones_like(T) if target_mask is None else np.asarray(target_mask, dtype=bool).astype(np.float64)
    return VoxelTerms(alpha=a, t_under=T.copy(), beta=np.ones_like(T), t_over=T.copy())


def objective(z: np.ndarray, vt: VoxelTerms) -> float:
    """F(z) of Eq. 5: sum over voxels of alpha_j max(0, T^-_j - z_j)^2 (Eq. 3/9)
    plus beta_j max(0, z_j - T^+_j)^2 (Eq. 4/10)."""
    under = np.maximum(0.0, vt.t_under - z)
    over = np.maximum(0.0, z - vt.t_over)
    return float(np.sum(vt.alpha * under * under) + np.sum(vt.beta * over * over))


def gradient(z: np.ndarray, vt: VoxelTerms) -> np.ndarray:
    """dF/dz_j = -2 alpha_j max(0, T^-_j - z_j) + 2 beta_j max(0, z_j - T^+_j).

    This is also the dual multiplier pi_j of the constraint z_j = sum_k D_kj y_k
    (Eq. 6, Sec. 2.3): stationarity of the Lagrangian in z gives pi = grad F(z).
    """
    return -2.0 * vt.alpha * np.maximum(0.0, vt.t_under - z) + 2.0 * vt.beta * np.maximum(0.0, z - vt.t_over)


def curvature(z: np.ndarray, vt: VoxelTerms) -> np.ndarray:
    """Generalised second derivative of F_j: 2 alpha_j [z_j < T^-_j] + 2 beta_j [z_j > T^+_j]."""
    return 2.0 * vt.alpha * (z < vt.t_under) + 2.0 * vt.beta * (z > vt.t_over)


# ---------------------------------------------------------------------------
# Dose (Eqs. 1, 2, 7) and the pricing weights w (Eq. 8)
# ---------------------------------------------------------------------------

def csr64(case) -> sp.csr_matrix:
    """D_ij as an FP64 scipy CSR matrix (V x N); FP32 inputs are promoted exactly."""
    V = len(case.indptr) - 1
    N = int(np.sum(np.asarray(case.rows, np.int64) * np.asarray(case.cols, np.int64)))
    return sp.csr_matrix((np.asarray(case.data, np.float64), np.asarray(case.indices, np.int64),
                          np.asarray(case.indptr, np.int64)), shape=(V, N))


def dose(D: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """z_j = sum_i D_ij x_i: Eq. 1 with Eq. 2 substituted, x from Eq. 7."""
    return D @ np.asarray(x, dtype=np.float64)


def beamlet_prices(D: sp.csr_matrix, pi: np.ndarray) -> np.ndarray:
    """w_i = sum_j D_ij pi_j, the bracketed sum of Eq. 8 (Sec. 2.3)."""
    return D.T @ np.asarray(pi, dtype=np.float64)


# ---------------------------------------------------------------------------
# Pricing sub-problem (Eq. 8 and the one-pass row search of Sec. 2.3)
# ---------------------------------------------------------------------------

def kadane_row(w_row) -> Tuple[float, int, int]:
    """The paper's left-to-right search for the consecutive beamlets of one MLC row
    with the smallest sum of w (Sec. 2.3, after Bates & Constable / Bentley).

    State: v (running sum), vbar (largest running sum so far, which starts at the
    empty prefix 0), vstar (best value), l / lstar (left leaf), r / rstar (right
    leaf); beamlets are numbered 1..n.  Both comparisons are strict, so ties keep
    the earliest left leaf of the largest prefix and the earliest right end.

    Returns (vstar, L, R) with the open beamlets as the half-open 0-based range
    [L, R) = [lstar, rstar - 1); a row whose best value is 0 is closed, (0, 0).
    """
    n = len(w_row)
    v = vbar = vstar = 0.0
    l = lstar = 0
    rstar = 1
    for r in range(1, n + 1):
        v = v + float(w_row[r - 1])
        if v > vbar:
            vbar = v
            l = r
        if v - vbar < vstar:
            vstar = v - vbar
            lstar = l
            rstar = r + 1
    if vstar < 0.0:
        return vstar, lstar, rstar - 1
    return 0.0, 0, 0


@dataclass
class Pricing:
    beam: int                      # chosen beam b*
    leaves: np.ndarray             # int32 [rows_b*, 2], half-open [L, R) per MLC row
    reduced_cost: float            # S_b* = sum over rows of v*
    beam_values: np.ndarray        # S_b for every beam
    row_values: List[np.ndarray]   # v* per row, per beam
    row_leaves: List[np.ndarray]   # [L, R) per row, per beam


def price(case, w: np.ndarray, mlc: str = "consecutive") -> Pricing:
    """Solve Eq. 8: every MLC row of every beam runs ``kadane_row``; the per-beam
    sums of v* are compared and the beam with the smallest sum gives the new
    aperture (Sec. 2.3).  Reading: equal beam sums go to the lowest beam index,
    and the per-beam sum adds the rows' v* in row order.

    ``mlc`` other than "consecutive" prices each beam under an MLC hardware
    constraint of Sec. 4 (``oracle.mlc``: "interdigitation", "connected",
    "jaws"); the beam's value then takes the place of the row sum and
    ``row_values`` holds it at the beam's first row (0 in the others)."""
    rows = np.asarray(case.rows, np.int64)
    cols = np.asarray(case.cols, np.int64)
    off = np.concatenate([[0], np.cumsum(rows * cols)])
    sums, rv, rl = [], [], []
    if mlc != "consecutive":
        from .mlc import MODES
        fn = MODES[mlc]
        for b in range(len(rows)):
            v, lv = fn(w[off[b]:off[b + 1]], int(rows[b]), int(cols[b]))
            vals = np.zeros(rows[b])
            vals[0] = v
            sums.append(v)
            rv.append(vals)
            rl.append(lv)
        sums = np.array(sums)
        best = 0
        for b in range(1, len(sums)):
            if sums[b] < sums[best]:
                best = b
        return Pricing(beam=best, leaves=rl[best].copy(), reduced_cost=float(sums[best]),
                       beam_values=sums, row_values=rv, row_leaves=rl)
    for b in range(len(rows)):
        vals = np.zeros(rows[b])
        lv = np.zeros((rows[b], 2), dtype=np.int32)
        total = 0.0
        for r in range(rows[b]):
            base = off[b] + r * cols[b]
            vs, L, R = kadane_row(w[base:base + cols[b]])
            vals[r] = vs
            lv[r] = (L, R)
            total = total + vs
        sums.append(total)
        rv.append(vals)
        rl.append(lv)
    sums = np.array(sums)
    best = 0
    for b in range(1, len(sums)):
        if sums[b] < sums[best]:
            best = b
    return Pricing(beam=best, leaves=rl[best].copy(), reduced_cost=float(sums[best]),
                   beam_values=sums, row_values=rv, row_leaves=rl)


def aperture_mask(case, beam: int, leaves) -> np.ndarray:
    """Indicator of the beamlets of aperture A_k: row r of ``beam`` is open on [L, R)."""
    rows = np.asarray(case.rows, np.int64)
    cols = np.asarray(case.cols, np.int64)
    off = int(np.sum(rows[:beam] * cols[:beam]))
    m = np.zeros(int(np.sum(rows * cols)))
    for r in range(rows[beam]):
        L, R = int(leaves[r][0]), int(leaves[r][1])
        m[off + r * cols[beam] + L: off + r * cols[beam] + R] = 1.0
    return m


def aperture_value(case, w: np.ndarray, beam: int, leaves) -> float:
    """sum_{i in A_k} w_i, the objective of Eq. 8 for one aperture."""
    return float(np.dot(aperture_mask(case, beam, leaves), w))


def aperture_column(D: sp.csr_matrix, case, beam: int, leaves) -> np.ndarray:
    """D_kj = sum_{i in A_k} D_ij (Eq. 2) for all voxels j."""
    return D @ aperture_mask(case, beam, leaves)


def fluence(case, apertures, y) -> np.ndarray:
    """x_i = sum_{k in K_i} y_k (Eq. 7)."""
    x = np.zeros(int(np.sum(np.asarray(case.rows, np.int64) * np.asarray(case.cols, np.int64))))
    for (b, lv), yk in zip(apertures, y):
        x += yk * aperture_mask(case, b, lv)
    return x


def pricing_tolerance(D: sp.csr_matrix, pi: np.ndarray, rel: float = 1e-12) -> float:
    """tau for the optimality test S_b* >= -tau.  Reading (the paper gives none): a
    reduced cost is a sum of terms D_ij pi_j, so it is compared with
    rel * max D * ||pi||_1, the size of its largest possible term sum.  Column
    generation evaluates this once, at pi = grad F(0), so tau is a fixed scale of
    the problem and does not shrink with the rounding noise of pi near F = 0."""
    dmax = float(np.max(D.data)) if D.nnz else 0.0
    return rel * dmax * float(np.sum(np.abs(pi)))


# ---------------------------------------------------------------------------
# Master problem: min F(S y) s.t. y >= 0  (Eqs. 5-6 over the current pool)
# ---------------------------------------------------------------------------

def kkt_residual(y: np.ndarray, g: np.ndarray) -> float:
    """||y - P(y - g)||_inf, zero exactly at a KKT point of min f(y), y >= 0."""
    return float(np.max(np.abs(y - np.maximum(y - g, 0.0)))) if len(y) else 0.0


@dataclass
class MasterResult:
    y: np.ndarray
    z: np.ndarray
    F: float
    pi: np.ndarray
    g: np.ndarray
    kkt: float
    iters: int
    status: str


def solve_master(S, vt: VoxelTerms, y0: Optional[np.ndarray] = None, tol_rel: float = 1e-12,
                 max_iter: int = 500, sigma: float = 1e-4) -> MasterResult:
    """Optimal intensities of the current aperture pool (Sec. 2.2-2.3).

    The paper solves this convex problem with a gradient projection method and
    states no step or stopping rule.  Any convergent method reaches the same
    optimal F and the same pi = grad F(z*) (grad F is constant on the solution
    set of a convex problem with Lipschitz gradient), so the oracle uses the
    projected Newton method of Bertsekas (1982): an epsilon-active set
    {y_k <= eps, g_k > 0} takes the plain gradient step, the free variables a
    Newton step on H = S_F^T diag(h) S_F (h = ``curvature``), and an Armijo rule
    F(P(y + a d)) <= F(y) + sigma g^T (P(y + a d) - y) along the projection arc
    with a = 1, 1/2, 1/4, ...  It stops at ||y - P(y - g)||_inf <= tol_rel times
    the largest |g| at the start.  ``S`` is V x K (dense or sparse).
    """
    K = S.shape[1]
    y = np.zeros(K) if y0 is None else np.maximum(np.asarray(y0, dtype=np.float64), 0.0)
    dense = not sp.issparse(S)

    def evaluate(yv):
        z = S @ yv
        return z, objective(z, vt), gradient(z, vt)

    z, F, pi = evaluate(y)
    g = S.T @ pi
    scale = max(float(np.max(np.abs(g))) if K else 0.0, 1e-300)
    tol = tol_rel * scale
    status = "max_iter"
    it = 0
    for it in range(1, max_iter + 1):
        res = kkt_residual(y, g)
        if res <= tol:
            status = "kkt"
            it -= 1
            break
        eps = min(1e-3, res)
        active = (y <= eps) & (g > 0)
        free = ~active
        d = np.zeros(K)
        d[active] = -g[active]
        if np.any(free):
            h = curvature(z, vt)
            SF = S[:, free] if dense else S[:, np.nonzero(free)[0]]
            if dense:
                H = SF.T @ (h[:, None] * SF)
            else:
                H = (SF.T @ sp.diags(h) @ SF).toarray()
            # plain Cholesky; a singular H (an aperture whose voxels all sit in a
            # flat part of F) gets the smallest diagonal shift that factors
            lam, step = 0.0, 1e-14 * max(float(np.max(np.diag(H))), 1e-300)
            while True:
                try:
                    Lc = np.linalg.cholesky(H + lam * np.eye(H.shape[0]))
                    break
                except np.linalg.LinAlgError:
                    lam = step if lam == 0.0 else lam * 10.0
            d[free] = -np.linalg.solve(Lc.T, np.linalg.solve(Lc, g[free]))
        a = 1.0
        accepted = False
        for _ in range(80):
            y_new = np.maximum(y + a * d, 0.0)
            z_new, F_new, pi_new = evaluate(y_new)
            if F_new <= F + sigma * float(np.dot(g, y_new - y)):
                accepted = True
                break
            a *= 0.5
        if not accepted or np.array_equal(y_new, y):
            status = "stalled"
            break
        y, z, F, pi = y_new, z_new, F_new, pi_new
        g = S.T @ pi
    return MasterResult(y=y, z=z, F=F, pi=pi, g=g, kkt=kkt_residual(y, g), iters=it, status=status)


# ---------------------------------------------------------------------------
# Column generation (Sec. 2.2-2.3, Fig. 1)
# ---------------------------------------------------------------------------

@dataclass
class CGResult:
    apertures: List[Tuple[int, np.ndarray]] = field(default_factory=list)
    y: np.ndarray = field(default_factory=lambda: np.zeros(0))
    z: Optional[np.ndarray] = None
    objective: List[float] = field(default_factory=list)      # F after the master with k apertures
    reduced_cost: List[float] = field(default_factory=list)   # S_b* that admitted aperture k
    kkt: List[float] = field(default_factory=list)
    master_iters: List[int] = field(default_factory=list)
    status: str = "k_max"
    final_reduced_cost: Optional[float] = None
    pi: Optional[np.ndarray] = None


def column_generation(case, k_max: int, normalize_by_volume: bool = True, tol_rel: float = 1e-12,
                      tau_rel: float = 1e-12, teacher=None, callback=None, vt: Optional[VoxelTerms] = None,
                      mlc: str = "consecutive") -> CGResult:
    """Column generation for DAO (Sec. 2.2-2.3): start from an empty pool (y = [],
    z = 0); each iteration prices with pi = grad F(z) (Eq. 8), stops when the
    best reduced cost is not negative (the current plan is optimal over all
    deliverable apertures), otherwise appends the new aperture's column
    D_kj (Eq. 2) and re-solves the master problem warm-started from the previous
    intensities with the new one at 0.

    ``teacher``: optional list of (beam, leaves) added in order instead of the
    priced aperture (pricing still runs and is recorded); used to compare
    another solver's masters on an identical aperture sequence.
    ``callback(k, pricing, result)`` is called after each iteration.
    ``vt``: per-voxel terms used in place of the case's structures (for example
    ``reoptimisation_terms``, the re-optimisation mode of Sec. 4).  ``mlc``:
    the MLC constraint of the pricing (``price``).
    Reading: an aperture identical to one already in the pool ends the loop with
    status "duplicate" (its reduced cost is >= 0 at an exact master optimum).
    """
    D = csr64(case)
    vt = voxel_terms(case, normalize_by_volume) if vt is None else vt
    V = D.shape[0]
    res = CGResult()
    S = np.zeros((V, 0))
    y = np.zeros(0)
    z = np.zeros(V)
    tau = pricing_tolerance(D, gradient(z, vt), tau_rel)
    for k in range(k_max):
        pi = gradient(z, vt)
        w = beamlet_prices(D, pi)
        pr = price(case, w, mlc)
        if teacher is not None:
            b, lv = teacher[k]
            lv = np.asarray(lv, dtype=np.int32)
            rc = aperture_value(case, w, b, lv)
        else:
            b, lv, rc = pr.beam, pr.leaves, pr.reduced_cost
            if rc >= -tau:
                res.status = "optimal"
                res.final_reduced_cost = rc
                break
            if any(b == b2 and np.array_equal(lv, l2) for b2, l2 in res.apertures):
                res.status = "duplicate"
                res.final_reduced_cost = rc
                break
        col = aperture_column(D, case, b, lv)
        S = np.column_stack([S, col])
        y = np.append(y, 0.0)
        m = solve_master(S, vt, y, tol_rel=tol_rel)
        y, z = m.y, m.z
        res.apertures.append((int(b), np.array(lv, dtype=np.int32)))
        res.objective.append(m.F)
        res.reduced_cost.append(float(rc))
        res.kkt.append(m.kkt)
        res.master_iters.append(m.iters)
        if callback is not None:
            callback(k, pr, m)
    res.y, res.z = y, z
    res.pi = gradient(z, vt)
    return res


def fmo(case, normalize_by_volume: bool = True, tol_rel: float = 1e-12, max_iter: int = 500,
        vt: Optional[VoxelTerms] = None) -> MasterResult:
    """Beamlet-level fluence map optimisation min_{x >= 0} F(D x), the model the
    paper calls mathematically the same as DAO with beamlets as the decision
    variables (Sec. 2.2).  Solved by ``solve_master`` with S = D.  Its optimum
    is a lower bound on every DAO objective, and equals the DAO optimum when
    column generation runs to optimality (any non-negative fluence map is a
    non-negative sum of consecutive-leaf apertures)."""
    D = csr64(case).tocsc()
    vt = voxel_terms(case, normalize_by_volume) if vt is None else vt
    return solve_master(D, vt, np.zeros(D.shape[1]), tol_rel=tol_rel, max_iter=max_iter)
