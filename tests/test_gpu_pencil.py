"""D generated on the device from the pencil-beam model (dao_pencil_generate,
dao_create_pencil; the coefficients D_ij of Eq. 2) against the oracle's
definition of the same model (oracle.pencil, every voxel against every
beamlet in FP64): the same sparsity pattern, except entries whose value lies
within 1e-12 relative of the keep threshold (where the last bits of exp, erf,
sin and cos may decide), and the same FP32 values within one FP32 rounding.
Plans on the generated D meet the oracle's bars at every round."""
import copy
import functools
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
import oracle.pencil as PB
import phantom as P
from _helpers import need_cuda
from test_gpu_cg import _free_running_checked, _plan

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _pb_args(spec, case):
    return dict(xyz=case.voxel_xyz, iso=case.iso, n_beams=spec.n_beams, rows=spec.rows, cols=spec.cols,
                beamlet_mm=spec.beamlet_mm, sigma_mm=spec.sigma_mm, mu_per_mm=spec.mu_per_mm, cutoff=spec.cutoff,
                profile=spec.profile, body_kind=spec.body.kind, body_center=spec.body.center[:2],
                body_size=spec.body.size[:2], jitter=spec.jitter,
                jitter_stream=(spec.seed * 0x100000001 + 0x5EED) & 0xFFFFFFFFFFFFFFFF)


@functools.lru_cache(maxsize=None)
def _workload(name, profile="gauss"):
    spec = replace(P.CONFIGS[name](), profile=profile)
    case = P.make_case(spec)
    a = _pb_args(spec, case)
    ref = PB.pencil_matrix(xyz=a["xyz"], iso=a["iso"], B=spec.n_beams, R=spec.rows, C=spec.cols, w=spec.beamlet_mm,
                           sigma=spec.sigma_mm, mu=spec.mu_per_mm, cutoff=spec.cutoff, profile=profile,
                           body_kind=spec.body.kind, body_center=spec.body.center[:2],
                           body_size=spec.body.size[:2], jitter=spec.jitter, jitter_stream=a["jitter_stream"])
    return spec, case, a, ref


def _compare(rp, col, val, ref, spec):
    """Pattern and values of a generated CSR against the oracle's matrix; returns
    (entries only on one side, largest value difference in FP32 ulps)."""
    V = len(rp) - 1
    g = {}
    for j in range(V):
        for p in range(rp[j], rp[j + 1]):
            g[(j, int(col[p]))] = float(val[p])
    r = ref.tocoo()
    o = {(int(j), int(i)): float(v) for j, i, v in zip(r.row, r.col, r.data)}
    only = set(g) ^ set(o)
    ulps = 0
    for k in set(g) & set(o):
        a, b = np.float32(g[k]), np.float32(o[k])
        ulps = max(ulps, abs(int(a.view(np.int32)) - int(b.view(np.int32))))
    return only, ulps


@pytest.mark.parametrize("name,profile", [("micro", "gauss"), ("tiny", "gauss"), ("tiny", "strip"),
                                          ("prostate", "gauss")])
def test_generated_matrix_matches_the_oracle(torch, name, profile):
    from paper_1003_5402_gb300 import binding
    spec, case, a, ref = _workload(name, profile)
    rp, col, val = binding.pencil_generate(a)
    assert len(rp) == case.n_voxels + 1 and rp[0] == 0 and np.all(np.diff(rp) >= 0)
    for j in range(0, case.n_voxels, max(1, case.n_voxels // 997)):   # columns increasing in each row
        assert np.all(np.diff(col[rp[j]:rp[j + 1]]) > 0)
    if name == "prostate":   # full size: counts, then sampled rows and every beamlet's column sums
        assert abs(len(col) - ref.nnz) <= 1e-6 * ref.nnz + 4
        D = ref.tocsr()
        rng = np.random.default_rng(3)
        for j in rng.choice(case.n_voxels, 500, replace=False):
            gi, gv = col[rp[j]:rp[j + 1]], val[rp[j]:rp[j + 1]]
            oi, ov = D.indices[D.indptr[j]:D.indptr[j + 1]], D.data[D.indptr[j]:D.indptr[j + 1]]
            if np.array_equal(gi, oi):
                assert np.all(np.abs(gv.astype(np.float64) - ov) <= 2.0 ** -23 * np.abs(ov)), j
        import scipy.sparse as sp
        G = sp.csr_matrix((val.astype(np.float64), col, rp), shape=ref.shape)
        cs_g, cs_o = np.asarray(G.sum(axis=0)).ravel(), np.asarray(D.sum(axis=0)).ravel()
        assert np.all(np.abs(cs_g - cs_o) <= 1e-6 * np.abs(cs_o) + 1e-9)
        return
    only, ulps = _compare(rp, col, val, ref, spec)
    print(f"\n{name}/{profile}: nnz {len(col)} (oracle {ref.nnz}), entries on one side only {len(only)}, "
          f"largest value difference {ulps} FP32 ulp")
    assert ulps <= 1
    assert len(only) <= 1e-6 * ref.nnz + 2


def test_generated_equals_the_host_generator_bitwise_on_the_small_box(torch):
    """On the small box the device's D and the input generator's FP32 D are the
    same bits, so plans on either are the same plan."""
    from paper_1003_5402_gb300 import binding
    spec, case, a, ref = _workload("tiny")
    rp, col, val = binding.pencil_generate(a)
    assert np.array_equal(rp, case.indptr) and np.array_equal(col, case.indices) and np.array_equal(val, case.data)
    with _plan(case, torch, pencil=a) as p1, _plan(case, torch) as p2:
        r1, r2 = p1.solve(20), p2.solve(20)
        assert np.array_equal(r1[2], r2[2])
        assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(p1.apertures(), p2.apertures()))


@pytest.mark.parametrize("name,K", [("tiny", 20), ("prostate", 30)])
def test_plan_on_generated_matrix_against_the_oracle(torch, name, K):
    """A plan whose D was generated on the device, at every round against the
    oracle on the oracle's own matrix of the model."""
    spec, case, a, ref = _workload(name)
    ocase = copy.copy(case)
    r = ref.tocsr()
    ocase.indptr, ocase.indices, ocase.data = r.indptr.astype(np.int64), r.indices.astype(np.int32), \
        r.data.astype(np.float32)
    out = _free_running_checked(case, K, torch, plan_kw={"pencil": a}, ref_case=ocase)
    print(f"\n{name} on the generated D: ties {out['ties']}, max objective rel {out['worst_F_rel']:.2e}, "
          f"max dose diff {out['worst_dose']:.2e}")


def test_pencil_argument_checks(torch):
    from paper_1003_5402_gb300 import DaoError, binding
    spec, case, a, ref = _workload("micro")
    for bad in (dict(sigma_mm=0.0), dict(cols=33), dict(cutoff=1.0), dict(profile="gauss", sigma_mm=30.0)):
        b = dict(a)
        b.update(bad)
        with pytest.raises(DaoError) as e:
            binding.pencil_generate(b)
        assert e.value.status == -1
