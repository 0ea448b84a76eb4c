"""ctypes binding of libdao.so (include/dao.h): argument marshalling only.

Every step of column-generation DAO runs in the library's CUDA kernels; this
module converts numpy arrays and torch CUDA tensors to the C structs and
pointers of the ABI and turns status codes into exceptions.  The library must
be built (``paper_1003_5402_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdao.so")

DAO_OK, DAO_OPTIMAL, DAO_DUPLICATE = 0, 1, 2
DAO_EINVAL, DAO_ENOMEM, DAO_ECUDA, DAO_ETIMEOUT, DAO_EBUSY, DAO_ESTATE = -1, -2, -3, -4, -5, -6
DAO_PREC_FP32, DAO_PREC_FP16, DAO_PREC_BF16 = 0, 1, 2
DAO_MLC_CONSECUTIVE, DAO_MLC_INTERDIGITATION, DAO_MLC_CONNECTED, DAO_MLC_JAWS = 0, 1, 2, 3
MLC = {"consecutive": DAO_MLC_CONSECUTIVE, "interdigitation": DAO_MLC_INTERDIGITATION,
       "connected": DAO_MLC_CONNECTED, "jaws": DAO_MLC_JAWS}
DAO_DT_GROUPED, DAO_DT_CONSECUTIVE, DAO_DT_SPLIT = 1, 2, 3
DAO_DOSE_LANES, DAO_DOSE_UNITS, DAO_DOSE_MERGE = 1, 2, 3
DT_MAPS = {DAO_DT_GROUPED: "grouped", DAO_DT_CONSECUTIVE: "consecutive", DAO_DT_SPLIT: "split"}
DOSE_FORMS = {DAO_DOSE_LANES: "lanes", DAO_DOSE_UNITS: "units", DAO_DOSE_MERGE: "merge"}
KC = {"dose": 0, "dt": 1, "price": 2, "column": 3, "master_pass": 4, "master_reduce": 5, "master_step": 6,
      "master_hess": 7, "other": 8, "master_solve": 9}

# every function declared in include/dao.h, with (restype, argtypes)
_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_F64P = C.POINTER(C.c_double)


class dao_csr(C.Structure):
    _fields_ = [("n_voxels", C.c_int32), ("n_beamlets", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", _I32P), ("val", C.POINTER(C.c_float))]


class dao_geometry(C.Structure):
    _fields_ = [("n_beams", C.c_int32), ("rows", _I32P), ("cols", _I32P)]


class dao_structures(C.Structure):
    _fields_ = [("n_structures", C.c_int32), ("voxel_struct", _I32P), ("is_target", C.POINTER(C.c_uint8))]


class dao_weights(C.Structure):
    _fields_ = [("under_w", _F64P), ("over_w", _F64P), ("over_thresh", _F64P), ("normalize_by_volume", C.c_int32)]


class dao_options(C.Structure):
    _fields_ = [("k_max", C.c_int32), ("max_master_iters", C.c_int32), ("master_tol", C.c_double),
                ("price_tol", C.c_double), ("precision", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p),
                ("use_graphs", C.c_int32), ("master_persistent", C.c_int32), ("mlc_constraint", C.c_int32),
                ("master_blocks", C.c_int32), ("dt_threads", C.c_int32), ("dt_map", C.c_int32),
                ("dose_form", C.c_int32), ("column_lanes", C.c_int32),
                ("split_warps", C.c_int32)]


class dao_tuning(C.Structure):
    _fields_ = [("dose_lanes", C.c_int32), ("column_lanes", C.c_int32), ("dt_threads", C.c_int32),
                ("from_cache", C.c_int32), ("dose_form", C.c_int32), ("dt_map", C.c_int32)]


class dao_server_options(C.Structure):
    _fields_ = [("max_slots", C.c_int32), ("queue_capacity", C.c_int32), ("hbm_reserve_bytes", C.c_int64),
                ("hbm_budget_bytes", C.c_int64), ("device", C.c_int32), ("simulate_ms_per_aperture", C.c_double),
                ("plan_options", dao_options), ("prewarm_bytes", C.c_int64), ("solve_slots", C.c_int32)]


class dao_voxel_terms(C.Structure):
    _fields_ = [("under_w", _F64P), ("under_t", _F64P), ("over_w", _F64P), ("over_t", _F64P)]


class dao_pencil_beam(C.Structure):
    _fields_ = [("n_voxels", C.c_int32), ("voxel_xyz", C.POINTER(C.c_float)), ("iso", C.c_double * 3),
                ("n_beams", C.c_int32), ("rows", C.c_int32), ("cols", C.c_int32), ("beamlet_mm", C.c_double),
                ("sigma_mm", C.c_double), ("mu_per_mm", C.c_double), ("cutoff", C.c_double),
                ("profile", C.c_int32), ("body_kind", C.c_int32), ("body_center", C.c_double * 2),
                ("body_size", C.c_double * 2), ("jitter", C.c_double), ("jitter_stream", C.c_uint64)]


class dao_request(C.Structure):
    _fields_ = [("D", dao_csr), ("geometry", dao_geometry), ("structures", dao_structures), ("weights", dao_weights),
                ("prescriptions", _F64P), ("n_apertures", C.c_int32), ("dose_out", C.POINTER(C.c_float)),
                ("intensities_out", _F64P), ("beams_out", _I32P), ("leaves_out", _I32P)]


class dao_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_apertures", C.c_int32), ("objective", C.c_double),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
                ("create_ms", C.c_double), ("solve_ms", C.c_double), ("finish_ms", C.c_double),
                ("gpu_wait_ms", C.c_double), ("error", C.c_char * 256)]


class dao_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64),
                ("active", C.c_int32), ("queued", C.c_int32), ("max_active", C.c_int32),
                ("bytes_in_use", C.c_int64)]


SIGNATURES = {
    "dao_options_default": (None, [C.POINTER(dao_options)]),
    "dao_create": (C.c_int, [C.POINTER(dao_csr), C.POINTER(dao_geometry), C.POINTER(dao_structures),
                             C.POINTER(dao_weights), _F64P, C.POINTER(dao_options), C.POINTER(_P)]),
    "dao_create_voxelwise": (C.c_int, [C.POINTER(dao_csr), C.POINTER(dao_geometry), C.POINTER(dao_voxel_terms),
                                       C.POINTER(dao_options), C.POINTER(_P)]),
    "dao_create_pencil": (C.c_int, [C.POINTER(dao_pencil_beam), C.POINTER(dao_structures), C.POINTER(dao_weights),
                                    _F64P, C.POINTER(dao_options), C.POINTER(_P)]),
    "dao_pencil_generate": (C.c_int, [C.POINTER(dao_pencil_beam), C.c_int32, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), _I32P, C.POINTER(C.c_float)]),
    "dao_destroy": (None, [_P]),
    "dao_release_cached_memory": (C.c_int, [C.c_int32]),
    "dao_check_bounded_wait": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "dao_import_apertures": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dao_reset": (C.c_int, [_P]),
    "dao_price": (C.c_int, [_P, _I32P, _I32P, _F64P]),
    "dao_add_aperture": (C.c_int, [_P, C.c_int32, _I32P, _F64P]),
    "dao_solve": (C.c_int, [_P, C.c_int32, _I32P, _F64P]),
    "dao_dose": (C.c_int, [_P, C.POINTER(C.c_float), _F64P]),
    "dao_intensities": (C.c_int, [_P, _F64P, _I32P]),
    "dao_apertures": (C.c_int, [_P, _I32P, _I32P, _I32P]),
    "dao_sizes": (C.c_int, [_P, _I32P, _I32P, _I32P, _I32P, _I32P, C.POINTER(C.c_int64), _I32P]),
    "dao_fmo": (C.c_int, [_P, C.c_int32, C.c_double, _F64P, _F64P, _I32P, _I32P]),
    "dao_k_dose": (C.c_int, [_P, _P, _P, _P, _F64P]),
    "dao_k_beamlet_prices": (C.c_int, [_P, _P, _P]),
    "dao_k_price": (C.c_int, [_P, _P, _I32P, _I32P, _F64P, _F64P, _I32P]),
    "dao_k_aperture_column": (C.c_int, [_P, C.c_int32, _I32P, _P]),
    "dao_k_state": (C.c_int, [_P, _P, _P]),
    "dao_k_time": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _F64P]),
    "dao_k_time_cold": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P, C.c_int64, _F64P]),
    "dao_profile_enable": (C.c_int, [_P, C.c_int32]),
    "dao_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), _F64P]),
    "dao_launch_count": (C.c_int64, [_P]),
    "dao_master_stats": (C.c_int, [_P, _I32P, _I32P, _F64P, _I32P]),
    "dao_dose_objective_noalloc": (C.c_int, [C.c_int32, C.c_int32, _P, _P, _P, _P, _P, C.c_int32, _F64P, _P, _P,
                                             _P, _P]),
    "dao_batch_solve": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, _I32P, _F64P, _I32P]),
    "dao_batch_solve_persistent": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, _I32P, _F64P, _I32P]),
    "dao_batch_group_size": (C.c_int32, [C.c_int32, C.c_int32]),
    "dao_autotune": (C.c_int, [_P, C.c_char_p, C.POINTER(dao_tuning)]),
    "dao_kernel_forms": (C.c_int, [_P, C.POINTER(dao_tuning)]),
    "dao_server_options_default": (None, [C.POINTER(dao_server_options)]),
    "dao_server_create": (C.c_int, [C.POINTER(dao_server_options), C.POINTER(_P)]),
    "dao_server_submit": (C.c_int, [_P, C.POINTER(dao_request), C.POINTER(C.c_int64)]),
    "dao_server_poll": (C.c_int, [_P, C.c_int64, C.POINTER(dao_result)]),
    "dao_server_wait": (C.c_int, [_P, C.c_int64, C.c_double, C.POINTER(dao_result)]),
    "dao_server_stats_get": (C.c_int, [_P, C.POINTER(dao_server_stats)]),
    "dao_server_footprint": (C.c_int64, [C.POINTER(dao_request), C.POINTER(dao_options)]),
    "dao_server_destroy": (None, [_P]),
    "dao_last_error": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libdao.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1003_5402_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class DaoError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


def _check(st: int, fn: str, ok=(DAO_OK,)):
    if st in ok:
        return st
    raise DaoError(st, fn, load().dao_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _dev(t, dtype_name: str, n: int = 0, device: int = None):
    """Device pointer of a contiguous torch CUDA tensor of at least n elements
    on CUDA device ``device``: the library takes bare pointers, so a short or
    foreign buffer is refused here rather than read or written out of bounds."""
    if not getattr(t, "is_cuda", False):
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype_name} tensor, got {t.dtype}")
    if t.numel() < n:
        raise ValueError(f"expected at least {n} elements, got {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"expected a tensor on cuda:{device}, got {t.device}")
    return C.c_void_p(t.data_ptr())


def _leaves(leaves, n: int) -> np.ndarray:
    """Flat int32 [L, R) pairs with at least n entries (2 per MLC row read)."""
    lr = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32).reshape(-1))
    if lr.size < n:
        raise ValueError(f"expected {n // 2} (L, R) pairs, got {lr.size // 2}")
    return lr


def options(**kw) -> dao_options:
    o = dao_options()
    load().dao_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            v = C.c_void_p(v)
        elif k == "dt_map" and isinstance(v, str):
            v = {n: c for c, n in DT_MAPS.items()}[v]
        elif k == "dose_form" and isinstance(v, str):
            v = {n: c for c, n in DOSE_FORMS.items()}[v]
        setattr(o, k, v)
    return o


def _case_structs(case, normalize_by_volume: bool = True):
    """dao_create's argument structs for a case, and the arrays they point into
    (which must outlive the call)."""
    indptr = np.ascontiguousarray(case.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(case.indices, dtype=np.int32)
    data = np.ascontiguousarray(case.data, dtype=np.float32)
    rows = np.ascontiguousarray(case.rows, dtype=np.int32)
    cols = np.ascontiguousarray(case.cols, dtype=np.int32)
    vs = np.ascontiguousarray(case.voxel_struct, dtype=np.int32)
    tgt = np.ascontiguousarray(case.is_target, dtype=np.uint8)
    uw = np.ascontiguousarray(case.under_w, dtype=np.float64)
    ow = np.ascontiguousarray(case.over_w, dtype=np.float64)
    ot = np.ascontiguousarray(case.over_t, dtype=np.float64)
    rx = np.ascontiguousarray(case.under_t, dtype=np.float64)
    keep = [indptr, indices, data, rows, cols, vs, tgt, uw, ow, ot, rx]
    D = dao_csr(len(indptr) - 1, int(np.sum(rows.astype(np.int64) * cols)), int(indptr[-1]),
                _ptr(indptr, C.c_int64), _ptr(indices, C.c_int32), _ptr(data, C.c_float))
    g = dao_geometry(len(rows), _ptr(rows, C.c_int32), _ptr(cols, C.c_int32))
    s = dao_structures(len(uw), _ptr(vs, C.c_int32), _ptr(tgt, C.c_uint8))
    w = dao_weights(_ptr(uw, C.c_double), _ptr(ow, C.c_double), _ptr(ot, C.c_double), int(normalize_by_volume))
    return D, g, s, w, rx, keep


def pencil_beam(xyz, iso, n_beams: int, rows: int, cols: int, beamlet_mm: float, sigma_mm: float,
                mu_per_mm: float, cutoff: float, profile: str, body_kind: str, body_center, body_size,
                jitter: float, jitter_stream: int):
    """A dao_pencil_beam and the array it points into (keep both alive)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    pb = dao_pencil_beam()
    pb.n_voxels = xyz.shape[0]
    pb.voxel_xyz = _ptr(xyz, C.c_float)
    pb.iso = (C.c_double * 3)(*[float(v) for v in iso])
    pb.n_beams, pb.rows, pb.cols = int(n_beams), int(rows), int(cols)
    pb.beamlet_mm, pb.sigma_mm, pb.mu_per_mm, pb.cutoff = float(beamlet_mm), float(sigma_mm), float(mu_per_mm), \
        float(cutoff)
    pb.profile = {"gauss": 0, "strip": 1}[profile]
    pb.body_kind = {"box": 0, "ecyl": 1}[body_kind]
    pb.body_center = (C.c_double * 2)(*[float(v) for v in body_center[:2]])
    pb.body_size = (C.c_double * 2)(*[float(v) for v in body_size[:2]])
    pb.jitter = float(jitter)
    pb.jitter_stream = int(jitter_stream) & 0xFFFFFFFFFFFFFFFF
    return pb, xyz


def pencil_generate(pb_args: dict, device: int = 0):
    """dao_pencil_generate: D from the pencil-beam model on the device, returned
    as host CSR arrays (int64 row_ptr, int32 col, float32 val)."""
    pb, keep = pencil_beam(**pb_args)
    lib = load()
    nnz = C.c_int64()
    _check(lib.dao_pencil_generate(C.byref(pb), int(device), C.byref(nnz), None, None, None), "dao_pencil_generate")
    rp = np.zeros(pb.n_voxels + 1, np.int64)
    col = np.zeros(max(nnz.value, 1), np.int32)
    val = np.zeros(max(nnz.value, 1), np.float32)
    _check(lib.dao_pencil_generate(C.byref(pb), int(device), C.byref(nnz), _ptr(rp, C.c_int64), _ptr(col, C.c_int32),
                                   _ptr(val, C.c_float)), "dao_pencil_generate")
    return rp, col[: nnz.value], val[: nnz.value]


def release_cached_memory(device: int = 0) -> None:
    """Give the device pool's cached memory and the page-locked free list back
    to the system (dao_release_cached_memory)."""
    _check(load().dao_release_cached_memory(int(device)), "dao_release_cached_memory")


class Plan:
    """One DAO plan context (dao_create ... dao_destroy).

    ``case`` is any object with the fields of ``phantom.Case`` (voxel-major CSR
    ``indptr/indices/data``, ``rows/cols``, ``voxel_struct``, ``is_target``,
    ``under_w/under_t/over_w/over_t``).  Keyword options map to dao_options;
    ``stream`` is a raw cudaStream_t (e.g. ``torch.cuda.current_stream().cuda_stream``).
    """

    def __init__(self, case, normalize_by_volume: bool = True, voxel_terms=None, pencil=None, **opt):
        lib = load()
        D, g, s, w, rx, self._keep = _case_structs(case, normalize_by_volume)
        o = options(**opt)
        h = C.c_void_p()
        if pencil is not None:
            # D generated on the device from the pencil-beam model (keyword
            # arguments of ``pencil_beam``); the case gives structures and weights
            pb, xyz = pencil_beam(**pencil)
            _check(lib.dao_create_pencil(C.byref(pb), C.byref(s), C.byref(w), _ptr(rx, C.c_double), C.byref(o),
                                         C.byref(h)), "dao_create_pencil")
        elif voxel_terms is None:
            _check(lib.dao_create(C.byref(D), C.byref(g), C.byref(s), C.byref(w), _ptr(rx, C.c_double), C.byref(o),
                                  C.byref(h)), "dao_create")
        else:
            # re-optimisation mode: per-voxel (under_w, under_t, over_w, over_t),
            # each n_voxels long, in place of the case's structures and weights
            V = len(case.indptr) - 1
            arr = [np.ascontiguousarray(a, dtype=np.float64) for a in voxel_terms]
            if len(arr) != 4 or any(a.shape != (V,) for a in arr):
                raise ValueError(f"voxel_terms: four arrays of {V} values")
            t = dao_voxel_terms(*[_ptr(a, C.c_double) for a in arr])
            _check(lib.dao_create_voxelwise(C.byref(D), C.byref(g), C.byref(t), C.byref(o), C.byref(h)),
                   "dao_create_voxelwise")
        self.h = h
        self._keep = []
        self.rows = np.array(case.rows, dtype=np.int32)
        self.cols = np.array(case.cols, dtype=np.int32)
        self.device = int(o.device)
        sz = self.sizes()
        self.n_voxels, self.n_beamlets, self.n_beams, self.n_mlc_rows, self.max_rows, self.nnz_stored, self.k_max = sz

    # -- lifetime
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().dao_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- ABI calls
    def sizes(self) -> Tuple[int, ...]:
        v = [C.c_int32() for _ in range(5)]
        nnz = C.c_int64()
        k = C.c_int32()
        _check(load().dao_sizes(self.h, *[C.byref(x) for x in v], C.byref(nnz), C.byref(k)), "dao_sizes")
        return tuple(x.value for x in v) + (nnz.value, k.value)

    def reset(self):
        _check(load().dao_reset(self.h), "dao_reset")

    def price(self):
        """(status, beam, leaves [rows, 2], reduced cost)."""
        beam = C.c_int32()
        lr = np.zeros(2 * self.max_rows, dtype=np.int32)
        rc = C.c_double()
        st = _check(load().dao_price(self.h, C.byref(beam), _ptr(lr, C.c_int32), C.byref(rc)), "dao_price",
                    (DAO_OK, DAO_OPTIMAL))
        b = beam.value
        return st, b, lr[: 2 * self.rows[b]].reshape(-1, 2).copy(), rc.value

    def _rows_of(self, beam: int) -> int:
        """Leaf entries the library reads for ``beam`` (0 for an invalid beam,
        which it refuses before reading)."""
        return 2 * int(self.rows[beam]) if 0 <= int(beam) < len(self.rows) else 0

    def add_aperture(self, beam: int, leaves) -> float:
        lr = _leaves(leaves, self._rows_of(beam))
        F = C.c_double()
        _check(load().dao_add_aperture(self.h, int(beam), _ptr(lr, C.c_int32), C.byref(F)), "dao_add_aperture")
        return F.value

    def import_apertures(self, apertures, y_start=None) -> float:
        """Append saved apertures [(beam, leaves [rows, 2]), ...] and solve the master
        once (dao_import_apertures); returns the objective."""
        n = len(apertures)
        stride = 2 * self.max_rows
        beams = np.array([int(b) for b, _ in apertures], dtype=np.int32)
        lr = np.zeros((max(n, 1), stride), dtype=np.int32)
        for i, (_, lv) in enumerate(apertures):
            flat = np.asarray(lv, dtype=np.int32).reshape(-1)
            lr[i, : flat.size] = flat
        y = None if y_start is None else np.ascontiguousarray(np.asarray(y_start, dtype=np.float64))
        F = C.c_double(float("nan"))
        _check(load().dao_import_apertures(self.h, n, _ptr(beams, C.c_int32), _ptr(lr, C.c_int32),
                                           None if y is None else _ptr(y, C.c_double), C.byref(F)),
               "dao_import_apertures")
        return F.value

    def solve(self, n_apertures: int):
        """(status, apertures added, objective trace)."""
        n = C.c_int32()
        trace = np.full(max(n_apertures, 1), np.nan)
        st = _check(load().dao_solve(self.h, int(n_apertures), C.byref(n), _ptr(trace, C.c_double)), "dao_solve",
                    (DAO_OK, DAO_OPTIMAL, DAO_DUPLICATE))
        return st, n.value, trace[:n_apertures]

    def dose(self):
        z = np.zeros(self.n_voxels, dtype=np.float32)
        F = C.c_double()
        _check(load().dao_dose(self.h, _ptr(z, C.c_float), C.byref(F)), "dao_dose")
        return z, F.value

    def fmo(self, max_iters: int = 300, tol: float = 1e-7):
        """dao_fmo: beamlet-level FMO on the device.  Returns (status, x, F,
        Newton steps, CG iterations); status DAO_OK or DAO_ESTATE (cap hit)."""
        x = np.zeros(self.n_beamlets)
        F = C.c_double()
        it = C.c_int32()
        cg = C.c_int32()
        st = _check(load().dao_fmo(self.h, int(max_iters), float(tol), _ptr(x, C.c_double), C.byref(F), C.byref(it),
                                   C.byref(cg)), "dao_fmo", (DAO_OK, DAO_ESTATE))
        return st, x, F.value, it.value, cg.value

    def intensities(self) -> np.ndarray:
        y = np.zeros(self.k_max)
        k = C.c_int32()
        _check(load().dao_intensities(self.h, _ptr(y, C.c_double), C.byref(k)), "dao_intensities")
        return y[: k.value].copy()

    def apertures(self):
        beams = np.zeros(self.k_max, dtype=np.int32)
        lr = np.zeros((self.k_max, 2 * self.max_rows), dtype=np.int32)
        k = C.c_int32()
        _check(load().dao_apertures(self.h, _ptr(beams, C.c_int32), _ptr(lr, C.c_int32), C.byref(k)),
               "dao_apertures")
        out = []
        for i in range(k.value):
            b = int(beams[i])
            out.append((b, lr[i, : 2 * self.rows[b]].reshape(-1, 2).copy()))
        return out

    # -- kernel-level calls on torch CUDA tensors
    def k_dose(self, x, z, grad=None, objective: bool = True):
        F = C.c_double()
        V, N, d = self.n_voxels, self.n_beamlets, self.device
        _check(load().dao_k_dose(self.h, _dev(x, "float32", N, d), _dev(z, "float32", V, d),
                                 _dev(grad, "float32", V, d) if grad is not None else None,
                                 C.byref(F) if objective else None), "dao_k_dose")
        return F.value if objective else None

    def k_beamlet_prices(self, pi, w):
        d = self.device
        _check(load().dao_k_beamlet_prices(self.h, _dev(pi, "float32", self.n_voxels, d),
                                           _dev(w, "float32", self.n_beamlets, d)), "dao_k_beamlet_prices")

    def k_price(self, w):
        """(status, beam, leaves, reduced cost, row best values, row [L, R))."""
        beam = C.c_int32()
        lr = np.zeros(2 * self.max_rows, dtype=np.int32)
        rc = C.c_double()
        rv = np.zeros(self.n_mlc_rows)
        rl = np.zeros(2 * self.n_mlc_rows, dtype=np.int32)
        st = _check(load().dao_k_price(self.h, _dev(w, "float32", self.n_beamlets, self.device), C.byref(beam),
                                       _ptr(lr, C.c_int32), C.byref(rc),
                                       _ptr(rv, C.c_double), _ptr(rl, C.c_int32)), "dao_k_price",
                    (DAO_OK, DAO_OPTIMAL))
        b = beam.value
        return st, b, lr[: 2 * self.rows[b]].reshape(-1, 2).copy(), rc.value, rv, rl.reshape(-1, 2)

    def k_aperture_column(self, beam: int, leaves, out):
        lr = _leaves(leaves, self._rows_of(beam))
        _check(load().dao_k_aperture_column(self.h, int(beam), _ptr(lr, C.c_int32),
                                            _dev(out, "float32", self.n_voxels, self.device)),
               "dao_k_aperture_column")

    def k_state(self, z, pi):
        V, d = self.n_voxels, self.device
        _check(load().dao_k_state(self.h, _dev(z, "float32", V, d), _dev(pi, "float32", V, d)), "dao_k_state")

    def k_time(self, kc: str, K: int = 0, reps: int = 20) -> float:
        """Average microseconds per launch of one kernel class (dao_k_time)."""
        us = C.c_double()
        _check(load().dao_k_time(self.h, KC[kc], int(K), int(reps), C.byref(us)), "dao_k_time")
        return us.value

    def k_time_cold(self, kc: str, flush, reps: int = 20) -> float:
        """Median cold-cache microseconds of one launch (dao_k_time_cold); ``flush``
        is a CUDA tensor larger than L2 that each repetition overwrites first."""
        us = C.c_double()
        _check(load().dao_k_time_cold(self.h, KC[kc], 0, int(reps), C.c_void_p(flush.data_ptr()),
                                      int(flush.numel() * flush.element_size()), C.byref(us)), "dao_k_time_cold")
        return us.value

    def profile_enable(self, on: bool = True):
        _check(load().dao_profile_enable(self.h, int(on)), "dao_profile_enable")

    def profile_read(self, kc: str):
        n = C.c_int64()
        ms = C.c_double()
        _check(load().dao_profile_read(self.h, KC[kc], C.byref(n), C.byref(ms)), "dao_profile_read")
        return n.value, ms.value

    def launch_count(self) -> int:
        return int(load().dao_launch_count(self.h))

    def autotune(self, cache_path: Optional[str] = None) -> dict:
        """dao_autotune: choose the SpMV launch shapes for this plan (cached by size class)."""
        t = dao_tuning()
        path = cache_path.encode() if cache_path else None
        _check(load().dao_autotune(self.h, path, C.byref(t)), "dao_autotune")
        return {"dose_lanes": t.dose_lanes, "column_lanes": t.column_lanes, "dt_threads": t.dt_threads,
                "dose_form": DOSE_FORMS.get(t.dose_form, t.dose_form), "dt_map": DT_MAPS.get(t.dt_map, t.dt_map),
                "from_cache": bool(t.from_cache)}

    def kernel_forms(self) -> dict:
        """dao_kernel_forms: the SpMV forms and launch shapes this plan runs with."""
        t = dao_tuning()
        _check(load().dao_kernel_forms(self.h, C.byref(t)), "dao_kernel_forms")
        return {"dose_form": DOSE_FORMS.get(t.dose_form, t.dose_form), "dose_lanes": t.dose_lanes,
                "column_lanes": t.column_lanes, "dt_map": DT_MAPS.get(t.dt_map, t.dt_map), "dt_threads": t.dt_threads}

    def master_stats(self):
        """(evaluations, status, relative KKT residual) per master solve since the last reset."""
        ev = np.zeros(self.k_max, dtype=np.int32)
        stt = np.zeros(self.k_max, dtype=np.int32)
        kkt = np.zeros(self.k_max)
        k = C.c_int32()
        _check(load().dao_master_stats(self.h, _ptr(ev, C.c_int32), _ptr(stt, C.c_int32), _ptr(kkt, C.c_double),
                                       C.byref(k)), "dao_master_stats")
        n = k.value
        return ev[:n].copy(), stt[:n].copy(), kkt[:n].copy()


def dose_objective_noalloc(row_ptr, col, val, x, voxel_struct, terms, z, grad=None, objective=None, stream=None):
    """dao_dose_objective_noalloc on torch CUDA tensors (int32 row_ptr / col /
    voxel_struct, float32 val / x / z / grad, float64 objective of one element)
    and a host float64 terms array [n_structures, 4]; returns the status.

    Every tensor must be on one CUDA device; the call runs with that device
    current (the library launches on the current device).  ``stream`` is a
    torch.cuda.Stream of that device, a raw cudaStream_t handle (int) or None
    (the device's current torch stream).  The lengths are checked, col and val
    against row_ptr[-1]; the contents of D (column indices below x's length)
    and the labels are not: the library flags a label outside
    [0, n_structures) with a NaN objective, and an out-of-range column index
    is read out of bounds."""
    import torch
    t = np.ascontiguousarray(terms, dtype=np.float64).reshape(-1, 4)
    V, N, d = int(z.numel()), int(x.numel()), z.device.index
    if col.numel() != val.numel():
        raise ValueError(f"col and val differ in length ({col.numel()} and {val.numel()})")
    nnz = int(row_ptr[-1].item()) if row_ptr.numel() > V else -1
    if nnz < 0 or col.numel() < nnz:
        raise ValueError(f"col and val hold {col.numel()} entries, row_ptr needs {nnz}")
    with torch.cuda.device(d):
        if stream is None:
            handle = torch.cuda.current_stream(d).cuda_stream
        elif isinstance(stream, torch.cuda.Stream):
            if stream.device.index != d:
                raise ValueError(f"the stream is on {stream.device}, the tensors on cuda:{d}")
            handle = stream.cuda_stream
        else:
            handle = int(stream)
        st = load().dao_dose_objective_noalloc(
            V, N, _dev(row_ptr, "int32", V + 1, d), _dev(col, "int32", nnz, d), _dev(val, "float32", nnz, d),
            _dev(x, "float32", N, d), _dev(voxel_struct, "int32", V, d), int(t.shape[0]), _ptr(t, C.c_double),
            _dev(z, "float32", V, d), _dev(grad, "float32", V, d) if grad is not None else None,
            _dev(objective, "float64", 1, d), C.c_void_p(handle) if handle else None)
    return _check(st, "dao_dose_objective_noalloc")


def batch_solve(plans: Sequence["Plan"], n_apertures: int, persistent: bool = False):
    """dao_batch_solve: column generation for several plans at once (each on its
    own stream); ``persistent``: dao_batch_solve_persistent, every round's master
    solves in one launch.  Returns [(status, pool size, objective trace)] per
    plan, as Plan.solve returns them (the trace NaN past the apertures added)."""
    n = len(plans)
    arr = (C.c_void_p * max(n, 1))(*[p.h.value for p in plans])
    n_done = np.zeros(max(n, 1), dtype=np.int32)
    status = np.zeros(max(n, 1), dtype=np.int32)
    traces = np.full((max(n, 1), max(n_apertures, 1)), np.nan)
    fn = load().dao_batch_solve_persistent if persistent else load().dao_batch_solve
    _check(fn(C.cast(arr, C.POINTER(C.c_void_p)), n, int(n_apertures), _ptr(n_done, C.c_int32),
              _ptr(traces, C.c_double), _ptr(status, C.c_int32)), "dao_batch_solve")
    return [(int(status[i]), int(n_done[i]), traces[i, :n_apertures].copy()) for i in range(n)]


class Server:
    """A re-plan server (dao_server_*): requests are queued, admitted while a slot
    is free and their device footprint fits, planned concurrently on their own
    streams and returned as they finish.  Keyword options beyond the server's own
    map to the dao_options of every plan."""

    def __init__(self, max_slots: int = 8, queue_capacity: int = 1024, hbm_reserve_bytes: int = 2 << 30,
                 hbm_budget_bytes: int = 0, device: int = 0, simulate_ms_per_aperture: float = 0.0,
                 prewarm_bytes: Optional[int] = None, solve_slots: int = 0, **plan_opt):
        lib = load()
        o = dao_server_options()
        lib.dao_server_options_default(C.byref(o))
        o.max_slots, o.queue_capacity = int(max_slots), int(queue_capacity)
        o.hbm_reserve_bytes, o.hbm_budget_bytes = int(hbm_reserve_bytes), int(hbm_budget_bytes)
        o.device, o.simulate_ms_per_aperture = int(device), float(simulate_ms_per_aperture)
        if prewarm_bytes is not None:
            o.prewarm_bytes = int(prewarm_bytes)
        o.solve_slots = int(solve_slots)
        o.plan_options = options(**plan_opt)
        self.k_max = o.plan_options.k_max
        h = C.c_void_p()
        _check(lib.dao_server_create(C.byref(o), C.byref(h)), "dao_server_create")
        self.h = h
        self._live = {}

    def _request(self, case, n_apertures: int, outputs: bool = True):
        D, g, s, w, rx, keep = _case_structs(case)
        out = {}
        req = dao_request(D, g, s, w, _ptr(rx, C.c_double), int(n_apertures))
        if outputs:
            max_rows = int(np.max(np.asarray(case.rows)))
            out = {"dose": np.zeros(len(case.indptr) - 1, np.float32), "y": np.zeros(self.k_max),
                   "beams": np.zeros(self.k_max, np.int32),
                   "leaves": np.zeros((self.k_max, max_rows, 2), np.int32)}
            req.dose_out = _ptr(out["dose"], C.c_float)
            req.intensities_out = _ptr(out["y"], C.c_double)
            req.beams_out = _ptr(out["beams"], C.c_int32)
            req.leaves_out = _ptr(out["leaves"], C.c_int32)
        return req, keep, out

    def footprint(self, case, **plan_opt) -> int:
        req, keep, _ = self._request(case, 0, outputs=False)
        o = options(**plan_opt)
        return int(load().dao_server_footprint(C.byref(req), C.byref(o)))

    def submit(self, case, n_apertures: int, outputs: bool = True) -> int:
        """Queue a request; returns its id.  Raises DaoError(DAO_EBUSY) when the queue is full."""
        req, keep, out = self._request(case, n_apertures, outputs)
        rid = C.c_int64()
        _check(load().dao_server_submit(self.h, C.byref(req), C.byref(rid)), "dao_server_submit")
        self._live[rid.value] = (req, keep, out)
        return rid.value

    def _result(self, rid, r):
        req, keep, out = self._live.pop(rid)
        res = {"status": r.status, "n_apertures": r.n_apertures, "objective": r.objective, "queue_ms": r.queue_ms,
               "run_ms": r.run_ms, "latency_ms": r.latency_ms, "create_ms": r.create_ms, "solve_ms": r.solve_ms,
               "finish_ms": r.finish_ms, "gpu_wait_ms": r.gpu_wait_ms, "error": r.error.decode(errors="replace")}
        if out:
            k = max(r.n_apertures, 0)
            res.update(dose=out["dose"], y=out["y"][:k].copy(), beams=out["beams"][:k].copy(),
                       leaves=out["leaves"][:k].copy())
        return res

    def poll(self, rid: int):
        """The finished request's result (a dict), or None while it is queued or running."""
        r = dao_result()
        st = load().dao_server_poll(self.h, int(rid), C.byref(r))
        if st == DAO_EBUSY:
            return None
        _check(st, "dao_server_poll")
        return self._result(rid, r)

    def wait(self, rid: int, timeout_ms: float = -1.0):
        r = dao_result()
        _check(load().dao_server_wait(self.h, int(rid), float(timeout_ms), C.byref(r)), "dao_server_wait")
        return self._result(rid, r)

    def stats(self) -> dict:
        t = dao_server_stats()
        _check(load().dao_server_stats_get(self.h, C.byref(t)), "dao_server_stats_get")
        return {f: getattr(t, f) for f, _ in dao_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().dao_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
