"""Shared helpers of the tests: synthetic cases and FP32 error bounds.

The bounds follow the standard floating-point summation analysis: a sum of n
terms accumulated in FP32 (unit roundoff u = 2^-24) is within
(n + extra) * u * sum|terms| of the exact sum.
"""
import numpy as np
import pytest

import phantom as P

U32 = 2.0 ** -24


class ArrayCase:
    """A case object built from plain arrays (the fields phantom.Case exposes)."""

    def __init__(self, indptr, indices, data, rows, cols, voxel_struct, is_target, under_w, under_t, over_w, over_t):
        self.indptr = np.asarray(indptr, np.int64)
        self.indices = np.asarray(indices, np.int32)
        self.data = np.asarray(data, np.float32)
        self.rows = np.asarray(rows, np.int32)
        self.cols = np.asarray(cols, np.int32)
        self.voxel_struct = np.asarray(voxel_struct, np.int32)
        self.is_target = np.asarray(is_target, np.uint8)
        self.under_w = np.asarray(under_w, np.float64)
        self.under_t = np.asarray(under_t, np.float64)
        self.over_w = np.asarray(over_w, np.float64)
        self.over_t = np.asarray(over_t, np.float64)

    @property
    def n_voxels(self):
        return len(self.indptr) - 1

    @property
    def n_beamlets(self):
        return int(np.sum(self.rows.astype(np.int64) * self.cols))

    @property
    def n_beams(self):
        return len(self.rows)


def random_case(seed, V, rows, cols, mean_row=20.0, S=3):
    """Ragged random D (empty and heavy rows) with a random structure labelling."""
    rows = np.asarray(rows, np.int32)
    cols = np.asarray(cols, np.int32)
    N = int(np.sum(rows.astype(np.int64) * cols))
    ip, ix, d = P.random_csr(seed, V, N, mean_row)
    lab = np.floor(P.uniform(seed + 9, np.arange(V)) * S).astype(np.int32)
    tgt = np.zeros(S, np.uint8)
    tgt[0] = 1
    return ArrayCase(ip, ix, d, rows, cols, lab, tgt, under_w=[10.0] + [0.0] * (S - 1),
                     under_t=[1.0] + [0.0] * (S - 1), over_w=[1.0] * S, over_t=[1.0] + [0.5] * (S - 1))


def sum_abs_rows(case, v):
    """sum_i |D_ji v_i| per voxel row j (FP64)."""
    import scipy.sparse as sp
    V = len(case.indptr) - 1
    N = int(np.sum(case.rows.astype(np.int64) * case.cols))
    A = sp.csr_matrix((np.abs(case.data.astype(np.float64)), case.indices, case.indptr), shape=(V, N))
    return A @ np.abs(np.asarray(v, np.float64)), np.diff(case.indptr)


def sum_abs_cols(case, v):
    """sum_j |D_ji v_j| per beamlet i and the column counts (FP64)."""
    import scipy.sparse as sp
    V = len(case.indptr) - 1
    N = int(np.sum(case.rows.astype(np.int64) * case.cols))
    A = sp.csr_matrix((np.abs(case.data.astype(np.float64)), case.indices, case.indptr), shape=(V, N))
    return A.T @ np.abs(np.asarray(v, np.float64)), np.bincount(case.indices, minlength=N)


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# ---------------------------------------------------------------------------
# 16-bit storage of D written out from its definition: per-beamlet scale
# s_i = max_j |D_ij| (1 for an empty beamlet), stored value RN16(D_ij / s_i)
# with the quotient first rounded to FP32 (IEEE division), round-to-nearest-even.
# ---------------------------------------------------------------------------

def bf16_round(x32):
    """FP32 -> nearest bfloat16 (ties to even), returned as FP32 (finite inputs)."""
    u = np.ascontiguousarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def beamlet_scale(case):
    N = int(np.sum(np.asarray(case.rows, np.int64) * np.asarray(case.cols, np.int64)))
    s = np.zeros(N, np.float32)
    np.maximum.at(s, np.asarray(case.indices, np.int64), np.abs(np.asarray(case.data, np.float32)))
    s[~(s > 0)] = 1.0
    return s


def quantized_case(case, prec):
    """A copy of ``case`` whose D holds the dequantised values s_i * RN16(D_ij / s_i)
    in FP64 (exact: at most 11 + 24 significant bits)."""
    import copy
    s = beamlet_scale(case)
    col = np.asarray(case.indices, np.int64)
    r = (np.asarray(case.data, np.float32) / s[col]).astype(np.float32)
    if prec == "fp16":
        q = r.astype(np.float16).astype(np.float64)
    elif prec == "bf16":
        q = bf16_round(r).astype(np.float64)
    else:
        raise ValueError(prec)
    out = copy.copy(case)
    out.data = q * s[col].astype(np.float64)
    return out
