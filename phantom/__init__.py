"""Seeded synthetic IMRT phantoms for column-generation direct aperture optimization.

This module only makes inputs: a voxel model (structures, priority-resolved labels,
2x2x2 down-sampling of unspecified tissue as in Sec. 3 of Men, Jia & Jiang), a
coplanar parallel-beam MLC geometry and a pencil-beam dose-deposition matrix
``D`` (voxel-major CSR, FP32 values, Eq. 2's ``D_ij``).  It holds none of the DAO
method's arithmetic (objective, gradients, pricing, master problem): the FP64
oracle and the CUDA path both take its output as given.

Random numbers come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
counter-based generator: the n-th draw of stream ``s`` is ``mix(s + n * GAMMA)``,
so every value depends only on (seed, counter) and not on evaluation order.

Dose model (a stand-in for the paper's finite-size pencil-beam engine, which is
not part of the method): for beam ``b`` at gantry angle ``2*pi*b/B`` about the z
axis, a voxel at lateral offset (du, dv) from beamlet ``i``'s central axis and at
depth ``t`` below the body surface along the beam receives
``D_ij = exp(-mu * t) * exp(-(du^2 + dv^2) / (2 sigma^2))`` (the ``gauss``
profile) or the product of two 5 mm strips blurred by the same Gaussian
(``strip`` profile, closer to a finite-size pencil beam).  Entries below
``cutoff * max_j D_ij`` (per-beamlet maximum) are dropped, then each kept entry
is multiplied by a seeded factor in ``[1 - jitter, 1 + jitter]`` so that
symmetric geometries do not produce exact pricing ties.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "GAMMA", "splitmix64", "uniform", "Shape", "StructureSpec", "CaseSpec", "Case",
    "make_case", "spec_tiny", "spec_prostate", "spec_hn", "spec_micro", "perturb",
    "random_csr", "CONFIGS",
]

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output mix of the 64-bit words ``x`` (wrapping arithmetic)."""
    z = np.asarray(x, dtype=np.uint64).copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def uniform(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0, 1): draw ``counter`` (0-based) of stream ``seed``."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GAMMA
    return (splitmix64(state) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# Analytic shapes (millimetres, patient frame: x lateral, y anterior, z superior)
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Shape:
    kind: str                     # sphere | ellipsoid | box | zcyl | ecyl | ering
    center: Tuple[float, float, float]
    size: Tuple[float, ...]       # radii / half-widths; see contains()

    def contains(self, x, y, z) -> np.ndarray:
        cx, cy, cz = self.center
        dx, dy, dz = x - cx, y - cy, z - cz
        s = self.size
        if self.kind == "sphere":
            return dx * dx + dy * dy + dz * dz <= s[0] * s[0]
        if self.kind == "ellipsoid":
            return (dx / s[0]) ** 2 + (dy / s[1]) ** 2 + (dz / s[2]) ** 2 <= 1.0
        if self.kind == "box":
            return (np.abs(dx) <= s[0]) & (np.abs(dy) <= s[1]) & (np.abs(dz) <= s[2])
        if self.kind == "zcyl":       # circular cylinder along z: (radius, half-length)
            return (dx * dx + dy * dy <= s[0] * s[0]) & (np.abs(dz) <= s[1])
        if self.kind == "ecyl":       # elliptic cylinder along z: (a, b, half-length)
            return ((dx / s[0]) ** 2 + (dy / s[1]) ** 2 <= 1.0) & (np.abs(dz) <= s[2])
        if self.kind == "ering":      # anterior half of an elliptic ring: (ao, bo, ai, bi, half-length)
            outer = (dx / s[0]) ** 2 + (dy / s[1]) ** 2 <= 1.0
            inner = (dx / s[2]) ** 2 + (dy / s[3]) ** 2 <= 1.0
            return outer & ~inner & (dy >= 0) & (np.abs(dz) <= s[4])
        raise ValueError(self.kind)

    def scaled(self, f: float) -> "Shape":
        if self.kind in ("sphere", "ellipsoid", "box", "ering"):
            return replace(self, size=tuple(v * f for v in self.size))
        if self.kind == "zcyl":
            return replace(self, size=(self.size[0] * f, self.size[1] * f))
        if self.kind == "ecyl":
            return replace(self, size=tuple(v * f for v in self.size))
        raise ValueError(self.kind)

    def shifted(self, d) -> "Shape":
        return replace(self, center=tuple(float(c + e) for c, e in zip(self.center, d)))


@dataclass(frozen=True)
class StructureSpec:
    name: str
    role: str                     # "target" | "oar" | "body"
    shape: Optional[Shape]        # None for the body (the remainder of the body shape)
    under_w: float = 0.0          # alpha_s (Eq. 9); targets only
    under_t: float = 0.0          # T_s^- (prescription)
    over_w: float = 0.0           # beta_s (Eq. 10)
    over_t: float = 0.0           # T_s^+


@dataclass(frozen=True)
class CaseSpec:
    name: str
    grid: Tuple[int, int, int]    # fine voxels (nx, ny, nz)
    voxel_mm: float
    body: Shape                   # body outline (box or ecyl, z-invariant cross-section)
    structures: Tuple[StructureSpec, ...]   # priority order: listed first wins; body last
    n_beams: int
    rows: int                     # MLC rows per beam (along z)
    cols: int                     # beamlets per row (along the in-plane lateral axis)
    beamlet_mm: float = 5.0
    sigma_mm: float = 3.0
    mu_per_mm: float = 0.005
    cutoff: float = 1e-3
    downsample: bool = False      # 2x2x2 super-voxels for unspecified tissue
    jitter: float = 0.01
    profile: str = "gauss"        # "gauss" | "strip"
    seed: int = 0
    iso_shift_mm: Tuple[float, float, float] = (0.0, 0.0, 0.0)


@dataclass
class Case:
    spec: CaseSpec
    # D: voxel-major CSR, columns sorted; beamlet index = beam-major, then row, then column
    indptr: np.ndarray            # int64 [V+1]
    indices: np.ndarray           # int32 [nnz]
    data: np.ndarray              # float32 [nnz]
    rows: np.ndarray              # int32 [B]
    cols: np.ndarray              # int32 [B]
    voxel_struct: np.ndarray      # int32 [V], index into structure arrays
    is_target: np.ndarray         # uint8 [S]
    under_w: np.ndarray           # float64 [S] alpha_s
    under_t: np.ndarray           # float64 [S] T_s^- (prescription)
    over_w: np.ndarray            # float64 [S] beta_s
    over_t: np.ndarray            # float64 [S] T_s^+
    names: List[str]
    voxel_xyz: np.ndarray         # float32 [V,3], mm, voxel (or super-voxel) centres
    iso: np.ndarray               # float64 [3]

    @property
    def n_voxels(self) -> int:
        return int(self.indptr.shape[0] - 1)

    @property
    def n_beamlets(self) -> int:
        return int(np.sum(self.rows.astype(np.int64) * self.cols))

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    @property
    def n_beams(self) -> int:
        return int(self.rows.shape[0])

    def beam_offsets(self) -> np.ndarray:
        off = np.zeros(self.n_beams + 1, dtype=np.int64)
        off[1:] = np.cumsum(self.rows.astype(np.int64) * self.cols)
        return off

    def summary(self) -> dict:
        s = {"name": self.spec.name, "voxels": self.n_voxels, "beamlets": self.n_beamlets,
             "beams": self.n_beams, "nnz": self.nnz}
        for k, nm in enumerate(self.names):
            s["n_" + nm] = int(np.sum(self.voxel_struct == k))
        return s


# ---------------------------------------------------------------------------
# Ray entry into the (z-invariant) body cross-section
# ---------------------------------------------------------------------------

def _entry_param(body: Shape, px, py, ex, ey):
    """Smallest s with (px, py) + s*(ex, ey) inside the body cross-section.

    The point itself is inside the body, so the answer is <= 0; depth = -s.
    """
    cx, cy = body.center[0], body.center[1]
    qx, qy = px - cx, py - cy
    if body.kind == "box":
        hx, hy = body.size[0], body.size[1]
        s_lo = np.full(qx.shape, -np.inf)
        for q, e, h in ((qx, ex, hx), (qy, ey, hy)):
            if abs(e) < 1e-12:
                continue
            t1 = (-h - q) / e
            t2 = (h - q) / e
            s_lo = np.maximum(s_lo, np.minimum(t1, t2))
        return s_lo
    if body.kind == "ecyl":
        a, b = body.size[0], body.size[1]
        A = (ex / a) ** 2 + (ey / b) ** 2
        Bq = 2.0 * (qx * ex / (a * a) + qy * ey / (b * b))
        C = (qx / a) ** 2 + (qy / b) ** 2 - 1.0
        disc = np.maximum(Bq * Bq - 4.0 * A * C, 0.0)
        return (-Bq - np.sqrt(disc)) / (2.0 * A)
    raise ValueError(body.kind)


def _lateral(profile: str, d, sigma: float, width: float):
    if profile == "gauss":
        return np.exp(-(d * d) / (2.0 * sigma * sigma))
    if profile == "strip":
        from scipy.special import erf
        k = 1.0 / (math.sqrt(2.0) * sigma)
        peak = math.erf(0.5 * width * k)
        return 0.5 * (erf((d + 0.5 * width) * k) - erf((d - 0.5 * width) * k)) / peak
    raise ValueError(profile)


# ---------------------------------------------------------------------------
# Case construction
# ---------------------------------------------------------------------------

def _voxel_model(spec: CaseSpec):
    nx, ny, nz = spec.grid
    h = spec.voxel_mm
    xs = (np.arange(nx) + 0.5 - 0.5 * nx) * h
    ys = (np.arange(ny) + 0.5 - 0.5 * ny) * h
    zs = (np.arange(nz) + 0.5 - 0.5 * nz) * h
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")      # [nx, ny, nz]
    in_body = spec.body.contains(X, Y, Z)
    label = np.full(X.shape, -1, dtype=np.int32)
    body_index = None
    for k, st in enumerate(spec.structures):
        if st.role == "body":
            body_index = k
            continue
        m = st.shape.contains(X, Y, Z) & in_body & (label < 0)
        label[m] = k
    if body_index is None:
        raise ValueError("a case needs a body structure")
    fine_struct = label >= 0
    label[in_body & ~fine_struct] = body_index

    if not spec.downsample:
        ix, iy, iz = np.nonzero(label >= 0)
        key = (iz.astype(np.int64) * ny + iy) * nx + ix
        xyz = np.stack([xs[ix], ys[iy], zs[iz]], axis=1)
        lab = label[ix, iy, iz]
    else:
        if nx % 2 or ny % 2 or nz % 2:
            raise ValueError("down-sampling needs even grid dimensions")
        blk_struct = fine_struct.reshape(nx // 2, 2, ny // 2, 2, nz // 2, 2).any(axis=(1, 3, 5))
        keep_fine = np.repeat(np.repeat(np.repeat(blk_struct, 2, 0), 2, 1), 2, 2) & (label >= 0)
        ix, iy, iz = np.nonzero(keep_fine)
        key_f = (iz.astype(np.int64) * ny + iy) * nx + ix
        xyz_f = np.stack([xs[ix], ys[iy], zs[iz]], axis=1)
        lab_f = label[ix, iy, iz]
        # super-voxels: blocks with no structure voxel whose centre lies in the body
        bx = (np.arange(nx // 2) * 2 + 1 - 0.5 * nx) * h
        by = (np.arange(ny // 2) * 2 + 1 - 0.5 * ny) * h
        bz = (np.arange(nz // 2) * 2 + 1 - 0.5 * nz) * h
        BX, BY, BZ = np.meshgrid(bx, by, bz, indexing="ij")
        keep_b = (~blk_struct) & spec.body.contains(BX, BY, BZ)
        jx, jy, jz = np.nonzero(keep_b)
        key_b = ((2 * jz).astype(np.int64) * ny + 2 * jy) * nx + 2 * jx
        xyz_b = np.stack([bx[jx], by[jy], bz[jz]], axis=1)
        lab_b = np.full(jx.shape, body_index, dtype=np.int32)
        key = np.concatenate([key_f, key_b])
        xyz = np.concatenate([xyz_f, xyz_b])
        lab = np.concatenate([lab_f, lab_b])
    order = np.argsort(key, kind="stable")
    return xyz[order], lab[order].astype(np.int32)


def _iso_center(spec: CaseSpec) -> np.ndarray:
    for st in spec.structures:
        if st.role == "target":
            return np.array(st.shape.center, dtype=np.float64)
    return np.zeros(3)


def _dose_matrix(spec: CaseSpec, xyz: np.ndarray, iso: np.ndarray):
    """COO triplets (voxel j, beamlet i, value) of the pencil-beam model."""
    V = xyz.shape[0]
    R, C, B = spec.rows, spec.cols, spec.n_beams
    w = spec.beamlet_mm
    reach = spec.sigma_mm * math.sqrt(2.0 * math.log(1e7))     # lateral factor >= 1e-7
    win = int(math.ceil(reach / w)) + 1
    p = xyz.astype(np.float64) - iso[None, :]
    rows_j, cols_i, vals = [], [], []
    for b in range(B):
        th = 2.0 * math.pi * b / B
        ex, ey = math.sin(th), -math.cos(th)          # beam direction (source -> patient)
        ux, uy = math.cos(th), math.sin(th)           # in-plane lateral axis (leaf travel)
        t = p[:, 0] * ex + p[:, 1] * ey
        u = p[:, 0] * ux + p[:, 1] * uy
        v = p[:, 2]
        s_in = _entry_param(spec.body, xyz[:, 0].astype(np.float64), xyz[:, 1].astype(np.float64), ex, ey)
        depth = np.maximum(-s_in, 0.0)
        att = np.exp(-spec.mu_per_mm * depth)
        cf = u / w + 0.5 * C - 0.5                    # fractional column of the voxel
        rf = v / w + 0.5 * R - 0.5
        c0 = np.floor(cf).astype(np.int64)
        r0 = np.floor(rf).astype(np.int64)
        jj, ii, vv = [], [], []
        for dr in range(-win, win + 2):
            r = r0 + dr
            okr = (r >= 0) & (r < R)
            dv = v - (r + 0.5 - 0.5 * R) * w
            gv = _lateral(spec.profile, dv, spec.sigma_mm, w)
            for dc in range(-win, win + 2):
                c = c0 + dc
                ok = okr & (c >= 0) & (c < C)
                du = u - (c + 0.5 - 0.5 * C) * w
                val = att * gv * _lateral(spec.profile, du, spec.sigma_mm, w)
                ok &= val > 1e-12
                idx = np.nonzero(ok)[0]
                jj.append(idx)
                ii.append(r[idx] * C + c[idx])
                vv.append(val[idx])
        jj = np.concatenate(jj)
        ii = np.concatenate(ii)
        vv = np.concatenate(vv)
        bmax = np.zeros(R * C)
        np.maximum.at(bmax, ii, vv)
        keep = vv >= spec.cutoff * bmax[ii]
        rows_j.append(jj[keep])
        cols_i.append(ii[keep] + b * R * C)
        vals.append(vv[keep])
    return np.concatenate(rows_j), np.concatenate(cols_i), np.concatenate(vals)


def make_case(spec: CaseSpec) -> Case:
    """Build the voxel model and the dose-deposition matrix of ``spec``."""
    xyz, lab = _voxel_model(spec)
    iso = _iso_center(spec) + np.asarray(spec.iso_shift_mm, dtype=np.float64)
    j, i, val = _dose_matrix(spec, xyz, iso)
    N = spec.n_beams * spec.rows * spec.cols
    V = xyz.shape[0]
    if spec.jitter > 0:
        u = uniform(spec.seed * 0x100000001 + 0x5EED, j.astype(np.uint64) * np.uint64(N) + i.astype(np.uint64))
        val = val * (1.0 + spec.jitter * (2.0 * u - 1.0))
    key = j.astype(np.int64) * N + i
    order = np.argsort(key, kind="stable")
    j, i, val = j[order], i[order], val[order]
    indptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(np.bincount(j, minlength=V), out=indptr[1:])
    S = len(spec.structures)
    return Case(
        spec=spec,
        indptr=indptr,
        indices=i.astype(np.int32),
        data=val.astype(np.float32),
        rows=np.full(spec.n_beams, spec.rows, dtype=np.int32),
        cols=np.full(spec.n_beams, spec.cols, dtype=np.int32),
        voxel_struct=lab,
        is_target=np.array([st.role == "target" for st in spec.structures], dtype=np.uint8),
        under_w=np.array([st.under_w for st in spec.structures], dtype=np.float64),
        under_t=np.array([st.under_t for st in spec.structures], dtype=np.float64),
        over_w=np.array([st.over_w for st in spec.structures], dtype=np.float64),
        over_t=np.array([st.over_t for st in spec.structures], dtype=np.float64),
        names=[st.name for st in spec.structures],
        voxel_xyz=xyz.astype(np.float32),
        iso=iso,
    )


# ---------------------------------------------------------------------------
# The workloads
# ---------------------------------------------------------------------------

def _sub_voxel_shift(seed: int, voxel_mm: float):
    u = uniform(seed, np.arange(3))
    return tuple(float((x - 0.5) * voxel_mm) for x in u)


def spec_tiny(seed: int = 1003) -> CaseSpec:
    """5 beams x 10x10 beamlets, 40x40x12 water box of 2.5 mm voxels, sphere target, two box OARs."""
    h = 2.5
    shift = _sub_voxel_shift(seed, h)
    tgt = Shape("sphere", shift, (15.0,))
    oar1 = Shape("box", (20.0 + 7.5, 0.0, 0.0), (7.5, 10.0, 15.0))       # +x slab, 5 mm off the sphere
    oar2 = Shape("box", (0.0, -(20.0 + 7.5), 0.0), (10.0, 7.5, 15.0))    # -y slab
    return CaseSpec(
        name="tiny", grid=(40, 40, 12), voxel_mm=h,
        body=Shape("box", (0.0, 0.0, 0.0), (50.0, 50.0, 15.0)),
        structures=(
            StructureSpec("ptv", "target", tgt, under_w=10.0, under_t=1.0, over_w=1.0, over_t=1.0),
            StructureSpec("oar_x", "oar", oar1, over_w=1.0, over_t=0.5),
            StructureSpec("oar_y", "oar", oar2, over_w=1.0, over_t=0.5),
            StructureSpec("body", "body", None, over_w=0.1, over_t=0.8),
        ),
        n_beams=5, rows=10, cols=10, seed=seed, downsample=False,
    )


def spec_prostate(seed: int = 5402) -> CaseSpec:
    """9 beams x 20x20 beamlets, 200x120x60 grid of 2.5 mm voxels, prostate-shaped anatomy."""
    h = 2.5
    shift = _sub_voxel_shift(seed, h)
    ptv = Shape("ellipsoid", shift, (35.0, 30.0, 28.0))
    return CaseSpec(
        name="prostate", grid=(200, 120, 60), voxel_mm=h,
        body=Shape("ecyl", (0.0, 0.0, 0.0), (240.0, 145.0, 75.0)),
        structures=(
            StructureSpec("ptv", "target", ptv, under_w=10.0, under_t=1.0, over_w=1.0, over_t=1.0),
            StructureSpec("rectum", "oar", Shape("zcyl", (0.0, -45.0, 0.0), (15.0, 40.0)), over_w=1.0, over_t=0.6),
            StructureSpec("bladder", "oar", Shape("ellipsoid", (0.0, 45.0, 25.0), (40.0, 30.0, 30.0)), over_w=1.0, over_t=0.6),
            StructureSpec("femur_l", "oar", Shape("sphere", (95.0, 0.0, -10.0), (25.0,)), over_w=1.0, over_t=0.5),
            StructureSpec("femur_r", "oar", Shape("sphere", (-95.0, 0.0, -10.0), (25.0,)), over_w=1.0, over_t=0.5),
            StructureSpec("body", "body", None, over_w=0.1, over_t=0.8),
        ),
        n_beams=9, rows=20, cols=20, seed=seed, downsample=True,
    )


def spec_hn(seed: int = 7333) -> CaseSpec:
    """5 beams x 30x30 beamlets, head-and-neck-shaped anatomy with two nested PTVs."""
    h = 2.5
    shift = _sub_voxel_shift(seed, h)
    c = (0.0 + shift[0], 40.0 + shift[1], 0.0 + shift[2])
    return CaseSpec(
        name="hn", grid=(192, 160, 80), voxel_mm=h,
        body=Shape("ecyl", (0.0, 0.0, 0.0), (235.0, 195.0, 100.0)),
        structures=(
            StructureSpec("ptv1", "target", Shape("ellipsoid", c, (28.0, 24.0, 30.0)), under_w=10.0, under_t=1.0, over_w=1.0, over_t=1.0),
            StructureSpec("ptv2", "target", Shape("ellipsoid", c, (55.0, 45.0, 60.0)), under_w=10.0, under_t=0.85, over_w=1.0, over_t=0.85),
            StructureSpec("cord", "oar", Shape("zcyl", (0.0, -35.0, -10.0), (7.0, 70.0)), over_w=1.0, over_t=0.6),
            StructureSpec("brainstem", "oar", Shape("zcyl", (0.0, -25.0, 80.0), (13.0, 18.0)), over_w=1.0, over_t=0.7),
            StructureSpec("parotid_l", "oar", Shape("ellipsoid", (60.0, 15.0, 40.0), (15.0, 20.0, 22.0)), over_w=1.0, over_t=0.5),
            StructureSpec("parotid_r", "oar", Shape("ellipsoid", (-60.0, 15.0, 40.0), (15.0, 20.0, 22.0)), over_w=1.0, over_t=0.5),
            StructureSpec("mandible", "oar", Shape("ering", (0.0, 20.0, -35.0), (60.0, 65.0, 50.0, 55.0, 12.0)), over_w=1.0, over_t=0.9),
            StructureSpec("body", "body", None, over_w=0.1, over_t=0.8),
        ),
        n_beams=5, rows=30, cols=30, seed=seed, downsample=True,
    )


def spec_micro(seed: int = 11, n_beams: int = 3, rows: int = 4, cols: int = 6,
               grid=(24, 24, 10), downsample: bool = False) -> CaseSpec:
    """A small case for parity tests: a few thousand voxels, several tiles, ragged rows."""
    h = 2.5
    shift = _sub_voxel_shift(seed, h)
    nx, ny, nz = grid
    half = (nx * h / 2, ny * h / 2, nz * h / 2)
    r = 0.25 * min(half[0], half[1])
    return CaseSpec(
        name="micro", grid=tuple(grid), voxel_mm=h,
        body=Shape("box", (0.0, 0.0, 0.0), half),
        structures=(
            StructureSpec("ptv", "target", Shape("sphere", shift, (r,)), under_w=10.0, under_t=1.0, over_w=1.0, over_t=1.0),
            StructureSpec("oar", "oar", Shape("box", (0.0, -(r + 0.35 * r + 2.5), 0.0), (r, 0.3 * r, half[2])), over_w=1.0, over_t=0.5),
            StructureSpec("body", "body", None, over_w=0.1, over_t=0.8),
        ),
        n_beams=n_beams, rows=rows, cols=cols, seed=seed, downsample=downsample,
    )


def perturb(spec: CaseSpec, seed: int, shift_mm: float = 5.0, scale_lo: float = 0.9,
            scale_hi: float = 1.1) -> CaseSpec:
    """A re-plan instance: targets shifted by U(-shift, shift) mm per axis, each OAR scaled
    by U(scale_lo, scale_hi) about its centre; the D jitter stream follows ``seed``."""
    u = uniform(seed, np.arange(3))
    d = tuple(float((2 * x - 1) * shift_mm) for x in u)
    new = []
    for k, st in enumerate(spec.structures):
        if st.role == "target":
            new.append(replace(st, shape=st.shape.shifted(d)))
        elif st.role == "oar":
            f = scale_lo + (scale_hi - scale_lo) * float(uniform(seed + 17, k)[()])
            new.append(replace(st, shape=st.shape.scaled(f)))
        else:
            new.append(st)
    return replace(spec, structures=tuple(new), seed=seed, name=f"{spec.name}@{seed}")


CONFIGS = {"tiny": spec_tiny, "prostate": spec_prostate, "hn": spec_hn, "micro": spec_micro}


def random_csr(seed: int, n_rows: int, n_cols: int, mean_row: float, empty_frac: float = 0.05,
               heavy_frac: float = 0.02, heavy_mult: float = 20.0):
    """A seeded random sparse matrix with ragged rows (some empty, some heavy), sorted
    columns and positive FP32 values; returns (indptr int64, indices int32, data float32)."""
    k = np.arange(n_rows, dtype=np.uint64)
    u_len = uniform(seed, k)
    u_kind = uniform(seed + 1, k)
    lens = np.floor(2.0 * mean_row * u_len).astype(np.int64)
    lens[u_kind < empty_frac] = 0
    heavy = u_kind > 1.0 - heavy_frac
    lens[heavy] = np.minimum(n_cols, (lens[heavy] * heavy_mult).astype(np.int64) + 1)
    lens = np.minimum(lens, n_cols)
    indptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    nnz = int(indptr[-1])
    idx = np.empty(nnz, dtype=np.int32)
    ctr = 0
    for r in range(n_rows):
        L = int(lens[r])
        if L == 0:
            continue
        pick = uniform(seed + 2, np.arange(ctr, ctr + 2 * L, dtype=np.uint64))
        ctr += 2 * L
        cand = np.unique(np.floor(pick * n_cols).astype(np.int64))
        if cand.shape[0] < L:
            extra = np.setdiff1d(np.arange(n_cols), cand)[: L - cand.shape[0]]
            cand = np.union1d(cand, extra)
        idx[indptr[r]:indptr[r + 1]] = np.sort(cand[:L])
    data = (0.05 + uniform(seed + 3, np.arange(nnz, dtype=np.uint64))).astype(np.float32)
    return indptr, idx, data
