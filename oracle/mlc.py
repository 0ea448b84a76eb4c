"""MLC hardware constraints in the pricing sub-problem (Sec. 4, last paragraph:
the method also handles interdigitation, connectedness and jaws-only delivery
besides the standard consecutiveness of each row's open beamlets).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every function prices ONE beam: ``w`` holds the beam's beamlet prices w_i
(Eq. 8) row by row (R rows of C beamlets).  The objective of Eq. 8 for an
aperture is the sum of its open beamlets' prices; the functions return
(value, leaves) with leaves an int32 [R, 2] array of half-open [L, R) ranges,
closed rows as (0, 0), and value 0 with every row closed when no aperture of
negative value exists (a zero-value aperture is never opened, as in the
row search of Sec. 2.3).

Arithmetic (fixed here so that another implementation can reproduce it bit
for bit): per row the prefix sums P[0] = 0, P[c + 1] = P[c] + w_c in FP64 in
column order, and an interval's sum is P[R] - P[L].

Readings of constraints the paper names but does not define:
  - interdigitation: the leaves of adjacent rows may not cross, L_r <= R_{r+1}
    and L_{r+1} <= R_r (in boundary positions 0..C); a closed row keeps its
    two leaves together at some position p (L = R = p), which takes part in
    the constraint;
  - connectedness: each row is consecutive and the open rows form one
    contiguous block of rows (no closed row between two open rows);
  - jaws-only: the aperture is a rectangle, one column range [L, R) open in a
    contiguous block of rows.
Tie rules: see each function.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from .dao import kadane_row


def row_prefix(w_row) -> np.ndarray:
    """P[0] = 0, P[c + 1] = P[c] + w_c, FP64, in column order."""
    P = [0.0]
    for v in w_row:
        P.append(P[-1] + float(v))
    return np.array(P)


def interval_states(C: int):
    """Leaf states (L, R), 0 <= L <= R <= C, in L-major order (their index is
    the tie-break order of the interdigitation dynamic programme)."""
    return [(L, R) for L in range(C + 1) for R in range(L, C + 1)]


def _closed(R: int) -> np.ndarray:
    return np.zeros((R, 2), np.int32)


def price_interdigitation(w, R: int, C: int) -> Tuple[float, np.ndarray]:
    """Minimum-value aperture under interdigitation, by dynamic programming over
    the rows: f_0(s) = I_0(s), f_r(s') = I_r(s') + min{f_{r-1}(s) : s
    compatible with s'} where (L, R) and (L', R') are compatible iff L <= R'
    and L' <= R, and I_r(L, R) = P_r[R] - P_r[L] (that exact FP64 order).
    Ties: the smallest state index at every choice (the final state, then each
    predecessor while tracing back), i.e. among optimal state sequences the one
    that is smallest read from the last row to the first."""
    w = np.asarray(w, np.float64).reshape(R, C)
    S = interval_states(C)
    Ls = np.array([s[0] for s in S])
    Rs = np.array([s[1] for s in S])
    P = [row_prefix(w[r]) for r in range(R)]
    compat = (Ls[None, :] <= Rs[:, None]) & (Ls[:, None] <= Rs[None, :])   # [s', s]
    f = P[0][Rs] - P[0][Ls]
    back = []
    for r in range(1, R):
        cand = np.where(compat, f[None, :], np.inf)
        arg = np.argmin(cand, axis=1)              # first minimum: the smallest index
        best = cand[np.arange(len(S)), arg]
        f = (P[r][Rs] - P[r][Ls]) + best
        back.append(arg)
    s = int(np.argmin(f))
    value = float(f[s])
    if not value < 0.0:
        return 0.0, _closed(R)
    leaves = np.zeros((R, 2), np.int32)
    for r in range(R - 1, -1, -1):
        L, Rr = S[s]
        leaves[r] = (L, Rr) if L < Rr else (0, 0)
        if r > 0:
            s = int(back[r - 1][s])
    return value, leaves


def price_connected(w, R: int, C: int) -> Tuple[float, np.ndarray]:
    """Minimum-value aperture whose open rows form one contiguous block.  Each
    row r of the block is open at its best non-empty interval, value m_r =
    min over L < R of P_r[R] - P_r[L] (ties: smallest (L, R) in L-major order);
    the block is the paper's one-pass row search (``kadane_row``) run over
    m_0 .. m_{R-1} instead of over beamlets, with its tie rules."""
    w = np.asarray(w, np.float64).reshape(R, C)
    m = np.zeros(R)
    best_lr = np.zeros((R, 2), np.int32)
    for r in range(R):
        P = row_prefix(w[r])
        bv, bl = np.inf, (0, 0)
        for L in range(C):
            for Rr in range(L + 1, C + 1):
                v = P[Rr] - P[L]
                if v < bv:
                    bv, bl = v, (L, Rr)
        m[r] = bv
        best_lr[r] = bl
    value, a, b = kadane_row(m)
    if not value < 0.0:
        return 0.0, _closed(R)
    leaves = _closed(R)
    leaves[a:b] = best_lr[a:b]
    return float(value), leaves


def price_jaws(w, R: int, C: int) -> Tuple[float, np.ndarray]:
    """Minimum-value rectangle: for every column range [L, R), L < R (L-major
    order), the paper's one-pass row search (``kadane_row``) over the rows'
    sums s_r = P_r[R] - P_r[L] gives the best block of rows; the smallest value
    over the column ranges wins, ties to the earliest column range."""
    w = np.asarray(w, np.float64).reshape(R, C)
    P = [row_prefix(w[r]) for r in range(R)]
    bv, best = 0.0, None
    for L in range(C):
        for Rr in range(L + 1, C + 1):
            s = [P[r][Rr] - P[r][L] for r in range(R)]
            v, a, b = kadane_row(s)
            if v < bv:
                bv, best = v, (L, Rr, a, b)
    if best is None:
        return 0.0, _closed(R)
    L, Rr, a, b = best
    leaves = _closed(R)
    leaves[a:b] = (L, Rr)
    return float(bv), leaves


MODES = {"interdigitation": price_interdigitation, "connected": price_connected, "jaws": price_jaws}
