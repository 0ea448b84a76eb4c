"""The dose-deposition coefficients D_ij of Eq. 2 from a pencil-beam model,
written out from its definition (the stand-in for the paper's finite-size
pencil-beam engine, Sec. 1), as the reference for the GPU's own generation of D.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model (FP64): beam b of B coplanar beams at gantry angle theta_b = 2 pi b / B
about the z axis; direction e = (sin theta, -cos theta), lateral axis
u = (cos theta, sin theta), the beamlet grid (R rows along z, C columns along
u, pitch w) centred on the isocentre.  For voxel j at p = xyz_j - iso:
  depth t_j   = max(0, -s) with s the smallest parameter of the ray
                xyz_j + s e inside the body's z-invariant cross-section
                (box: slab intersection; elliptic cylinder: quadratic root),
  D_ij        = exp(-mu t_j) * L(dv) * L(du) (the product in that order),
  du, dv      = (p . u) - (c + 1/2 - C/2) w,  p_z - (r + 1/2 - R/2) w,
  L(d)        = exp(-d^2 / (2 sigma^2))                       ("gauss"), or
              = [erf((d + w/2) k) - erf((d - w/2) k)] / 2 / erf(w k / 2),
                k = 1 / (sqrt(2) sigma)                       ("strip"),
for beamlet i = b R C + r C + c.  A coefficient is kept when it exceeds 1e-12
and is at least cutoff * max_j D_ij (the beamlet's largest), then multiplied by
1 + jitter (2 U_ij - 1), U_ij = the (j N + i)-th draw of the SplitMix64 stream
``jitter_stream`` (phantom.uniform), and rounded to FP32.  The voxels that can
reach a beamlet are all voxels here (no search window): the reading of "every
voxel and every beamlet" the generator's window must reproduce.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def splitmix_uniform(stream: int, counter) -> np.ndarray:
    """U(0, 1) draws of SplitMix64 (Steele, Lea & Flood 2014) used as a
    counter-based generator: mix(stream + (counter + 1) * golden gamma), top 53
    bits.  Written from the published constants."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def entry_parameter(body_kind: str, center, size, px, py, ex: float, ey: float) -> np.ndarray:
    """Smallest s with (px, py) + s (ex, ey) inside the body cross-section."""
    qx, qy = px - center[0], py - center[1]
    if body_kind == "box":
        s = np.full(np.shape(qx), -np.inf)
        for q, e, h in ((qx, ex, size[0]), (qy, ey, size[1])):
            if abs(e) < 1e-12:
                continue
            s = np.maximum(s, np.minimum((-h - q) / e, (h - q) / e))
        return s
    if body_kind == "ecyl":
        a, b = size[0], size[1]
        A = (ex / a) ** 2 + (ey / b) ** 2
        Bq = 2.0 * (qx * ex / (a * a) + qy * ey / (b * b))
        Cq = (qx / a) ** 2 + (qy / b) ** 2 - 1.0
        return (-Bq - np.sqrt(np.maximum(Bq * Bq - 4.0 * A * Cq, 0.0))) / (2.0 * A)
    raise ValueError(body_kind)


def lateral(profile: str, d, sigma: float, width: float):
    if profile == "gauss":
        return np.exp(-(d * d) / (2.0 * sigma * sigma))
    from scipy.special import erf
    k = 1.0 / (math.sqrt(2.0) * sigma)
    return 0.5 * (erf((d + 0.5 * width) * k) - erf((d - 0.5 * width) * k)) / math.erf(0.5 * width * k)


def beam_coefficients(xyz, iso, b, B, R, C, w, sigma, mu, profile, body_kind, body_center, body_size):
    """Dense [V, R*C] FP64 block of beam b (before cutoff and jitter)."""
    th = 2.0 * math.pi * b / B
    ex, ey = math.sin(th), -math.cos(th)
    ux, uy = math.cos(th), math.sin(th)
    x = np.asarray(xyz, np.float64)
    p = x - np.asarray(iso, np.float64)[None, :]
    u = p[:, 0] * ux + p[:, 1] * uy
    v = p[:, 2]
    depth = np.maximum(-entry_parameter(body_kind, body_center, body_size, x[:, 0], x[:, 1], ex, ey), 0.0)
    att = np.exp(-mu * depth)
    r = np.arange(R)
    c = np.arange(C)
    gv = lateral(profile, v[:, None] - (r[None, :] + 0.5 - 0.5 * R) * w, sigma, w)     # [V, R]
    gu = lateral(profile, u[:, None] - (c[None, :] + 0.5 - 0.5 * C) * w, sigma, w)     # [V, C]
    return ((att[:, None] * gv)[:, :, None] * gu[:, None, :]).reshape(len(x), R * C)


def pencil_matrix(xyz, iso, B, R, C, w, sigma, mu, cutoff, profile, body_kind, body_center, body_size,
                  jitter, jitter_stream, chunk: int = 20000) -> sp.csr_matrix:
    """D as an FP64 CSR matrix whose values are the FP32-rounded coefficients.
    Voxels are evaluated ``chunk`` at a time (twice: the beamlets' maxima, then
    the kept entries) to bound the memory of the dense blocks."""
    V, N = len(xyz), B * R * C
    xyz = np.asarray(xyz)
    rows, cols, vals = [], [], []
    for b in range(B):
        args = (iso, b, B, R, C, w, sigma, mu, profile, body_kind, body_center, body_size)
        bmax = np.zeros(R * C)
        for j0 in range(0, V, chunk):
            blk = beam_coefficients(xyz[j0:j0 + chunk], *args)
            bmax = np.maximum(bmax, np.max(np.where(blk > 1e-12, blk, 0.0), axis=0))
        js, ivs, vs = [], [], []
        for j0 in range(0, V, chunk):
            blk = beam_coefficients(xyz[j0:j0 + chunk], *args)
            keep = (blk > 1e-12) & (blk >= cutoff * bmax[None, :])
            jj, ii = np.nonzero(keep)
            js.append(jj + j0)
            ivs.append(ii)
            vs.append(blk[jj, ii])
        j, i, val = np.concatenate(js), np.concatenate(ivs), np.concatenate(vs)
        gi = i + b * R * C
        if jitter > 0:
            val = val * (1.0 + jitter * (2.0 * splitmix_uniform(jitter_stream, j.astype(np.uint64) * np.uint64(N)
                                                                 + gi.astype(np.uint64)) - 1.0))
        rows.append(j)
        cols.append(gi)
        vals.append(val.astype(np.float32).astype(np.float64))
    j = np.concatenate(rows)
    i = np.concatenate(cols)
    v = np.concatenate(vals)
    return sp.csr_matrix((v, (j, i)), shape=(V, N))
