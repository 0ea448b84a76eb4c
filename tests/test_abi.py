"""The C ABI without a GPU: libdao.so loads, exports every function that
include/*.h declares, and rejects malformed inputs on the host (no CUDA call is
reached before validation)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1003_5402_gb300 import build
    build.build()
    from paper_1003_5402_gb300 import binding
    return binding.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(dao_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["dao_create", "dao_price", "dao_add_aperture", "dao_solve", "dao_dose", "dao_destroy",
                     "dao_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1003_5402_gb300 import binding
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, name


def test_options_default_on_host(lib):
    from paper_1003_5402_gb300 import binding
    o = binding.options()
    assert o.k_max == 64 and o.max_master_iters == 50 and o.precision == 0
    assert o.master_tol == 1e-6
    assert o.dt_map == 0 and o.dose_form == 0
    assert binding.options(dt_map="grouped", dose_form="units").dt_map == binding.DAO_DT_GROUPED
    assert binding.options(dose_form="lanes").dose_form == binding.DAO_DOSE_LANES


def _tiny_inputs():
    V, N = 6, 8
    indptr = np.array([0, 2, 3, 3, 5, 6, 8], dtype=np.int64)
    indices = np.array([0, 3, 1, 2, 7, 5, 0, 4], dtype=np.int32)
    data = np.ones(8, dtype=np.float32)
    rows = np.array([2], dtype=np.int32)
    cols = np.array([4], dtype=np.int32)
    vs = np.array([0, 0, 1, 1, 1, 1], dtype=np.int32)
    tgt = np.array([1, 0], dtype=np.uint8)
    return dict(indptr=indptr, indices=indices, data=data, rows=rows, cols=cols, vs=vs, tgt=tgt,
                uw=np.array([10.0, 0.0]), ow=np.array([1.0, 1.0]), ot=np.array([1.0, 0.5]),
                rx=np.array([1.0, 0.0]), V=V, N=N)


def _create(lib, d, **opt):
    from paper_1003_5402_gb300 import binding as b
    P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
    D = b.dao_csr(d["V"], d["N"], int(d["indptr"][-1]), P(d["indptr"], C.c_int64), P(d["indices"], C.c_int32),
                  P(d["data"], C.c_float))
    g = b.dao_geometry(len(d["rows"]), P(d["rows"], C.c_int32), P(d["cols"], C.c_int32))
    s = b.dao_structures(len(d["uw"]), P(d["vs"], C.c_int32), P(d["tgt"], C.c_uint8))
    w = b.dao_weights(P(d["uw"], C.c_double), P(d["ow"], C.c_double), P(d["ot"], C.c_double), 1)
    o = b.options(**opt)
    h = C.c_void_p()
    st = lib.dao_create(C.byref(D), C.byref(g), C.byref(s), C.byref(w), P(d["rx"], C.c_double), C.byref(o),
                        C.byref(h))
    if st == 0:
        lib.dao_destroy(h)
    return st, lib.dao_last_error().decode()


# the per-entry CSR and per-voxel label checks run on the device
# (tests/test_gpu_build.py); these are the host's
@pytest.mark.parametrize("mutate,needle", [
    (lambda d: d["cols"].__setitem__(0, 5), "rows*cols"),
    (lambda d: d["indptr"].__setitem__(0, 1), "row_ptr[0]"),
    (lambda d: d["uw"].__setitem__(0, -1.0), "weights"),
    (lambda d: d["ot"].__setitem__(1, np.inf), "weights"),
])
def test_create_rejects_malformed_inputs(lib, mutate, needle):
    d = _tiny_inputs()
    mutate(d)
    st, msg = _create(lib, d)
    assert st == -1 and needle in msg, (st, msg)


def test_create_rejects_wide_rows_and_pool_sizes(lib):
    d = _tiny_inputs()
    d["rows"] = np.array([1], dtype=np.int32)
    d["cols"] = np.array([8], dtype=np.int32)
    d["N"] = 8
    st, _ = _create(lib, d, k_max=0)
    assert st == -1
    st, _ = _create(lib, d, k_max=65)
    assert st == -1
    d["cols"] = np.array([40], dtype=np.int32)
    d["N"] = 40
    st, msg = _create(lib, d)
    assert st == -1 and "[1, 32]" in msg


@pytest.mark.parametrize("opt,needle", [({"dt_map": 4}, "dt_map"), ({"dt_map": -1}, "dt_map"),
                                        ({"dose_form": 4}, "dose_form"), ({"dt_threads": 96}, "dt_threads"),
                                        ({"column_lanes": 3}, "column_lanes"), ({"column_lanes": 32}, "column_lanes"),
                                        ({"split_warps": -1}, "split_warps")])
def test_create_rejects_unknown_kernel_forms(lib, opt, needle):
    st, msg = _create(lib, _tiny_inputs(), **opt)
    assert st == -1 and needle in msg, (st, msg)


def test_null_arguments(lib):
    assert lib.dao_create(None, None, None, None, None, None, None) == -1
    assert lib.dao_price(None, None, None, None) == -1
    assert lib.dao_solve(None, 5, None, None) == -1
    assert lib.dao_launch_count(None) == 0


def test_batch_and_autotune_validate_on_host(lib):
    """Null and malformed batch arguments are refused before any CUDA call."""
    from paper_1003_5402_gb300 import binding
    assert lib.dao_batch_solve(None, 1, 5, None, None, None) == binding.DAO_EINVAL
    assert lib.dao_batch_solve(None, -1, 5, None, None, None) == binding.DAO_EINVAL
    arr = (C.c_void_p * 2)(None, None)
    assert lib.dao_batch_solve(C.cast(arr, C.POINTER(C.c_void_p)), 2, 5, None, None, None) == binding.DAO_EINVAL
    assert b"null context" in lib.dao_last_error()
    assert lib.dao_batch_solve(None, 0, 5, None, None, None) == binding.DAO_OK
    assert lib.dao_autotune(None, None, None) == binding.DAO_EINVAL
    assert lib.dao_kernel_forms(None, None) == binding.DAO_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libdao.so the binding raises at the first call: there is no CPU
    fallback to route the product path through."""
    from paper_1003_5402_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libdao.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.load()
    with pytest.raises(RuntimeError, match="missing"):
        binding.release_cached_memory(0)


class _FakeCudaTensor:
    """Just the attributes the binding reads from a torch CUDA tensor."""

    def __init__(self, n, dtype="float32", index=0, contiguous=True):
        self.is_cuda = True
        self.dtype = "torch." + dtype
        self._n = n
        self.device = type("Dev", (), {"index": index, "__str__": lambda s: f"cuda:{index}"})()
        self._c = contiguous

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 4096


def test_device_buffers_are_checked_before_the_library_sees_them():
    """The library takes bare device pointers, so the binding refuses a buffer
    that is too short, on another device, of another type or strided."""
    from paper_1003_5402_gb300 import binding
    assert binding._dev(_FakeCudaTensor(10), "float32", 10, 0).value == 4096
    assert binding._dev(_FakeCudaTensor(12), "float32", 10, 0).value == 4096
    with pytest.raises(ValueError, match="at least 10"):
        binding._dev(_FakeCudaTensor(9), "float32", 10, 0)
    with pytest.raises(ValueError, match="cuda:1"):
        binding._dev(_FakeCudaTensor(10, index=0), "float32", 10, 1)
    with pytest.raises(TypeError):
        binding._dev(_FakeCudaTensor(10, dtype="float64"), "float32", 10, 0)
    with pytest.raises(TypeError):
        binding._dev(_FakeCudaTensor(10, contiguous=False), "float32", 10, 0)
    with pytest.raises(TypeError, match="CUDA"):
        binding._dev(np.zeros(10, np.float32), "float32", 10, 0)


def test_leaf_arrays_cover_the_rows_the_library_reads():
    from paper_1003_5402_gb300 import binding
    assert binding._leaves([(0, 2), (1, 3)], 4).tolist() == [0, 2, 1, 3]
    with pytest.raises(ValueError, match="expected 3"):
        binding._leaves([(0, 2), (1, 3)], 6)


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes across the boundary has the size and
    field offsets that a C compiler gives the declaration in include/dao.h
    (a field added on one side only would shift every field after it)."""
    import shutil
    import subprocess
    from paper_1003_5402_gb300 import binding as b
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = ["dao_csr", "dao_geometry", "dao_structures", "dao_weights", "dao_options", "dao_tuning",
               "dao_server_options", "dao_voxel_terms", "dao_pencil_beam", "dao_request", "dao_result",
               "dao_server_stats"]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dao.h"', "int main(void) {"]
    for name in structs:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(b, name)._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c_layout = {}
    for ln in out:
        if ln:
            parts = ln.split()
            c_layout[(parts[0], parts[1])] = int(parts[2])
    for name in structs:
        cls = getattr(b, name)
        assert C.sizeof(cls) == c_layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c_layout[(name, field)], (name, field)
