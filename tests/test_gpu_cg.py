"""End-to-end column generation on the GPU against the FP64 oracle.

Bars: chosen leaves identical to the oracle's except near-ties (the oracle's
FP64 reduced cost of the GPU's choice within the window that the two masters'
differing duals allow), objective within 1e-5 relative, dose within 1e-4 of
the prescription per voxel, KKT of the GPU's master solution.
"""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import need_cuda

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5
DOSE_TOL = 1e-4          # times the prescription (1.0 in every workload)


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _plan(case, torch, **kw):
    from paper_1003_5402_gb300 import Plan
    return Plan(case, stream=torch.cuda.current_stream().cuda_stream, **kw)


def _tie_window(case, D, pi_gpu, pi_ref, apertures):
    """Largest change of an aperture's reduced cost between the GPU's and the
    oracle's duals, summed over the apertures compared, plus 1e-9 relative."""
    dpi = np.abs(pi_gpu.astype(np.float64) - pi_ref)
    absD = abs(D)
    tot = 0.0
    for b, lv in apertures:
        m = O.aperture_mask(case, b, lv)
        tot += float(np.abs(absD @ m) @ dpi) + float((absD @ m) @ np.abs(pi_ref)) * 4 * 2.0 ** -24
    return tot


def _teacher_forced(case, K, torch, plan_kw=None, ref_case=None):
    """Teacher-forced column generation: the GPU prices from its own state, and
    the oracle's aperture is added on both sides.  ``ref_case`` (default: case)
    is the matrix the oracle sees: the dequantised D for 16-bit storage."""
    gpu_case, case = case, (case if ref_case is None else ref_case)
    D = O.csr64(case)
    steps = []
    ref = O.column_generation(case, K, callback=lambda k, pr, m: steps.append((pr, m)))
    out = {"F_gpu": [], "F_ref": list(ref.objective), "ties": 0, "exact": 0}
    with _plan(gpu_case, torch, **(plan_kw or {})) as plan:
        zbuf = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        pbuf = torch.empty_like(zbuf)
        for k, (b_ref, lv_ref) in enumerate(ref.apertures):
            st, b, lv, rc = plan.price()
            pr_ref = steps[k][0]
            if b == b_ref and np.array_equal(lv, lv_ref):
                out["exact"] += 1
            else:
                plan.k_state(zbuf, pbuf)
                pi_gpu = pbuf.cpu().numpy()
                pi_ref = O.gradient(ref_z_before(ref, steps, k, case), O.voxel_terms(case))
                w_ref = O.beamlet_prices(D, pi_ref)
                v_gpu_choice = O.aperture_value(case, w_ref, b, lv)
                win = max(1e-9 * abs(pr_ref.reduced_cost),
                          _tie_window(case, D, pi_gpu, pi_ref, [(b, lv), (b_ref, lv_ref)]))
                assert abs(v_gpu_choice - pr_ref.reduced_cost) <= win, (k, v_gpu_choice, pr_ref.reduced_cost, win)
                out["ties"] += 1
            out["F_gpu"].append(plan.add_aperture(b_ref, lv_ref))
        out["y_gpu"] = plan.intensities()
        out["z_gpu"], out["F_dose"] = plan.dose()
        plan.k_state(zbuf, pbuf)
        out["pi_gpu"] = pbuf.cpu().numpy()
    out["ref"] = ref
    return out


def ref_z_before(ref, steps, k, case):
    """Oracle dose before pricing step k (z = 0 before the first aperture)."""
    if k == 0:
        return np.zeros(case.n_voxels)
    return steps[k - 1][1].z


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("name,K", [("micro", 12), ("tiny", 20)])
def test_teacher_forced_parity(torch, name, K, persistent):
    """Both master implementations: one persistent cooperative kernel per solve,
    and one launch per evaluation kernel."""
    case = P.make_case(P.CONFIGS[name]())
    r = _teacher_forced(case, K, torch, plan_kw={"master_persistent": persistent})
    Fg, Fr = np.array(r["F_gpu"]), np.array(r["F_ref"])
    rel = np.abs(Fg - Fr) / np.abs(Fr)
    assert np.all(rel <= RTOL_F), rel
    assert r["exact"] >= K - 2, r
    # dose of the GPU's own intensities: FP32 SpMV against the FP64 oracle
    D = O.csr64(case)
    ref = r["ref"]
    z_ref_gpu_y = O.dose(D, O.fluence(case, ref.apertures, r["y_gpu"]))
    assert np.max(np.abs(r["z_gpu"] - z_ref_gpu_y)) <= DOSE_TOL
    # against the oracle's own optimum (well-posed here: both masters are KKT points
    # of the same strictly convex-on-targets problem up to flat OAR regions)
    dz = np.abs(r["z_gpu"] - ref.z)
    assert np.max(dz) <= DOSE_TOL * 10, float(np.max(dz))
    assert abs(r["F_dose"] - Fr[-1]) <= RTOL_F * Fr[-1]


@pytest.mark.parametrize("name,K", [("micro", 12), ("tiny", 20)])
def test_free_running_matches_oracle(torch, name, K):
    case = P.make_case(P.CONFIGS[name]())
    ref = O.column_generation(case, K)
    with _plan(case, torch) as plan:
        st, n, trace = plan.solve(K)
        aps = plan.apertures()
    assert n == K
    same = 0
    for k in range(K):
        if aps[k][0] == ref.apertures[k][0] and np.array_equal(aps[k][1], ref.apertures[k][1]):
            same += 1
        else:
            break
    # the sequences agree until a near-tie; the objectives agree where they agree
    assert same >= min(K, 8), same
    rel = np.abs(trace[:same] - np.array(ref.objective[:same])) / np.array(ref.objective[:same])
    assert np.all(rel <= RTOL_F), rel
    # after any divergence the plan quality stays within the tolerance band of the oracle's
    assert trace[-1] <= ref.objective[-1] * (1 + 1e-3)


@pytest.mark.parametrize("persistent", [1, 0])
def test_master_kkt_on_gpu_solution(torch, persistent):
    case = P.make_case(P.spec_tiny())
    with _plan(case, torch, master_persistent=persistent) as plan:
        plan.solve(15)
        aps = plan.apertures()
        y = plan.intensities()
    D = O.csr64(case)
    vt = O.voxel_terms(case)
    S = np.column_stack([O.aperture_column(D, case, b, lv) for b, lv in aps])
    g = S.T @ O.gradient(S @ y, vt)
    scale = np.max(np.abs(S.T @ O.gradient(np.zeros(case.n_voxels), vt)))
    assert np.all(y >= 0)
    pos = y > 1e-6 * np.max(y)
    assert np.all(np.abs(g[pos]) <= 1e-4 * scale), np.max(np.abs(g[pos])) / scale
    assert np.all(g[~pos] >= -1e-4 * scale)


def test_optimal_termination_micro(torch):
    """Column generation run to its end on the micro case: the GPU stops with no
    negative reduced cost (status optimal or a duplicate at the FP32 floor) at an
    objective equal to the beamlet FMO optimum within the FP32 tolerance."""
    case = P.make_case(P.spec_micro())
    f = O.fmo(case)
    with _plan(case, torch) as plan:
        st, n, trace = plan.solve(64)
        _, F = plan.dose()
    assert st in (1, 2) or n == 64
    assert abs(F - f.F) <= 1e-4 * f.F, (F, f.F, n, st)


def test_reset_reproduces_bitwise(torch):
    case = P.make_case(P.spec_micro())
    with _plan(case, torch) as plan:
        _, _, t1 = plan.solve(8)
        z1, F1 = plan.dose()
        plan.reset()
        _, _, t2 = plan.solve(8)
        z2, F2 = plan.dose()
    assert np.array_equal(t1, t2) and np.array_equal(z1, z2) and F1 == F2


def test_add_aperture_validation_and_pool_limit(torch):
    from paper_1003_5402_gb300 import DaoError
    case = P.make_case(P.spec_micro())
    with _plan(case, torch, k_max=2) as plan:
        with pytest.raises(DaoError):
            plan.add_aperture(7, np.zeros((4, 2), np.int32))
        with pytest.raises(DaoError):
            plan.add_aperture(0, np.array([[0, 9]] * 4, np.int32))
        full = np.array([[0, 6]] * 4, np.int32)
        plan.add_aperture(0, full)
        plan.add_aperture(1, full)
        with pytest.raises(DaoError) as e:
            plan.add_aperture(2, full)
        assert e.value.status == -6


@pytest.mark.parametrize("workload", ["prostate", "hn"])
def test_full_size_properties(torch, workload):
    """The benchmark workload (prostate-shaped, 50 apertures) in the launch
    configuration the benchmark times, and the H&N-shaped workload (280,699
    voxels, 4,500 beamlets, two targets) in FP32: objective non-increasing,
    dose at sampled voxels equal to the oracle's sum over the plan's
    beamlets, master KKT with the oracle's FP64 aperture columns, first
    apertures and objectives equal to the oracle's."""
    case = P.make_case(P.spec_prostate() if workload == "prostate" else P.spec_hn())
    K = 50
    with _plan(case, torch) as plan:
        st, n, trace = plan.solve(K)
        aps = plan.apertures()
        y = plan.intensities()
        z, F = plan.dose()
    assert n == K
    assert np.all(np.diff(trace) <= 1e-6 * trace[:-1])
    D = O.csr64(case)
    x = O.fluence(case, aps, y)
    rng = np.random.default_rng(0)
    js = rng.choice(case.n_voxels, 2000, replace=False)
    zs = D[js] @ x
    assert np.max(np.abs(z[js] - zs)) <= DOSE_TOL
    vt = O.voxel_terms(case)
    S = np.column_stack([O.aperture_column(D, case, b, lv) for b, lv in aps])
    g = S.T @ O.gradient(S @ y, vt)
    scale = np.max(np.abs(S.T @ O.gradient(np.zeros(case.n_voxels), vt)))
    pos = y > 1e-6 * np.max(y)
    assert np.all(np.abs(g[pos]) <= 1e-4 * scale)
    assert np.all(g[~pos] >= -1e-4 * scale)
    ref = O.column_generation(case, 5)
    for k in range(5):
        assert aps[k][0] == ref.apertures[k][0] and np.array_equal(aps[k][1], ref.apertures[k][1]), k
    assert np.all(np.abs(trace[:5] - ref.objective) <= RTOL_F * np.array(ref.objective))


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("name,K,prec", [("micro", 30, 0), ("tiny", 20, 0), ("micro", 64, 0), ("micro", 30, 1),
                                         ("micro", 30, 2)], ids=["micro-30", "tiny-20", "micro-64", "micro-30-fp16",
                                                                 "micro-30-bf16"])
def test_graph_rounds_equal_host_driven_rounds(torch, name, K, prec, persistent):
    """dao_solve as CUDA graphs (no host synchronisation between rounds) gives
    bit-identical results to host-driven launches, for both master
    implementations and the three storage precisions; micro-64 runs until
    pricing stops the solve inside the graph's round loop."""
    case = P.make_case(P.CONFIGS[name]())
    out = []
    for g in (1, 0):
        with _plan(case, torch, use_graphs=g, master_persistent=persistent, precision=prec) as plan:
            st, n, trace = plan.solve(K)
            aps = plan.apertures()
            y = plan.intensities()
            z, F = plan.dose()
            ev, stt, kkt = plan.master_stats()
            out.append((st, n, trace, aps, y, z, F, ev, stt))
    a, b = out
    if K == 64:
        assert a[0] in (1, 2) and a[1] < 64  # stopped by pricing, not by the pool size
    assert a[0] == b[0] and a[1] == b[1]
    # trace entries after a pricing stop are NaN on both paths
    assert np.array_equal(a[2], b[2], equal_nan=True) and np.array_equal(a[4], b[4]) and np.array_equal(a[5], b[5])
    assert a[6] == b[6]
    assert all(x[0] == y_[0] and np.array_equal(x[1], y_[1]) for x, y_ in zip(a[3], b[3]))
    assert np.array_equal(a[7], b[7]) and np.array_equal(a[8], b[8])


def test_graph_solve_in_chunks_and_after_host_rounds(torch):
    """Rounds split across calls, and graph rounds after host-driven ones, continue
    the same column generation."""
    case = P.make_case(P.spec_micro())
    with _plan(case, torch) as plan:
        _, _, t_all = plan.solve(12)
        aps_all = plan.apertures()
    with _plan(case, torch) as plan:
        st, b, lv, rc = plan.price()
        plan.add_aperture(b, lv)
        _, _, t1 = plan.solve(4)
        _, _, t2 = plan.solve(7)
        aps = plan.apertures()
    assert len(aps) == 12
    assert all(x[0] == y_[0] and np.array_equal(x[1], y_[1]) for x, y_ in zip(aps, aps_all))
    assert np.array_equal(np.concatenate([t1, t2]), t_all[1:])
