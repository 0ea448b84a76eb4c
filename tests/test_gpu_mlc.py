"""MLC-constrained pricing on the GPU (Sec. 4: interdigitation, connectedness,
jaws-only) against the FP64 oracle (``oracle.mlc``).

Lockstep: the GPU prices a given FP32 w (dao_k_price) and must equal the
oracle on the same w bit for bit: the beam, every row's leaves and the FP64
reduced cost, on seeded continuous w and on integer-valued w (many exact
ties), over geometries of several beams with ragged row and column counts (up
to 64 rows and 32 columns).  Column generation with each constraint, teacher-
forced and free-running, meets the bars of the unconstrained plans at every
round, and every aperture the GPU adds is deliverable under the constraint.
"""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import need_cuda, random_case
from test_gpu_cg import RTOL_F, _free_running_checked, _plan, _teacher_forced

pytestmark = pytest.mark.gpu

MODES = ["interdigitation", "connected", "jaws"]


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _geoms():
    yield "micro", P.make_case(P.spec_micro())
    yield "ragged", random_case(41, 1500, rows=[3, 7, 1, 12], cols=[5, 32, 9, 17], mean_row=8.0)
    yield "wide", random_case(42, 900, rows=[64, 20], cols=[32, 30], mean_row=12.0)
    yield "hn_shape", random_case(43, 600, rows=[30] * 5, cols=[30] * 5, mean_row=6.0)


GEOMS = list(_geoms())


def _w_draws(N, seed):
    rng = np.random.default_rng(seed)
    yield "normal", rng.normal(size=N).astype(np.float32)
    yield "integer", rng.integers(-3, 4, size=N).astype(np.float32)
    yield "mostly_positive", np.abs(rng.normal(size=N)).astype(np.float32) * np.where(rng.uniform(size=N) < 0.1, -1, 1).astype(np.float32)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,case", GEOMS, ids=[g[0] for g in GEOMS])
def test_mlc_pricing_lockstep_bit_exact(torch, mode, name, case):
    from paper_1003_5402_gb300 import binding
    with _plan(case, torch, mlc_constraint=binding.MLC[mode]) as plan:
        for kind, w in _w_draws(case.n_beamlets, 60 + MODES.index(mode)):
            st, b, lv, rc, rv, rl = plan.k_price(torch.from_numpy(w).cuda())
            pr = O.price(case, w.astype(np.float64), mode)
            assert b == pr.beam, (kind, b, pr.beam)
            assert rc == pr.reduced_cost, (kind, rc, pr.reduced_cost)
            assert np.array_equal(lv, pr.leaves), (kind, lv, pr.leaves)
            g0 = 0
            for bb in range(case.n_beams):
                R = int(case.rows[bb])
                assert rv[g0] == pr.row_values[bb][0] and np.all(rv[g0 + 1:g0 + R] == 0.0), (kind, bb)
                assert np.array_equal(rl[g0:g0 + R], pr.row_leaves[bb]), (kind, bb)
                g0 += R


def _deliverable(lv, mode, C):
    R = len(lv)
    opn = [r for r in range(R) if lv[r][0] < lv[r][1]]
    if not opn:
        return True
    if mode == "connected":
        return opn == list(range(opn[0], opn[-1] + 1))
    if mode == "jaws":
        return opn == list(range(opn[0], opn[-1] + 1)) and len({tuple(lv[r]) for r in opn}) == 1
    # interdigitation: a parking position for every closed row, scanned row by row
    reach = {(int(lv[0][0]), int(lv[0][1]))} if 0 in opn else {(p, p) for p in range(C + 1)}
    for r in range(1, R):
        cand = [(int(lv[r][0]), int(lv[r][1]))] if r in opn else [(p, p) for p in range(C + 1)]
        reach = {s for s in cand if any(s[0] <= t[1] and t[0] <= s[1] for t in reach)}
        if not reach:
            return False
    return True


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,K", [("micro", 12), ("tiny", 16)])
def test_mlc_teacher_forced(torch, mode, name, K):
    from paper_1003_5402_gb300 import binding
    case = P.make_case(P.CONFIGS[name]())
    r = _teacher_forced(case, K, torch, plan_kw={"mlc_constraint": binding.MLC[mode]}, mlc=mode)
    Fg, Fr = np.array(r["F_gpu"]), np.array(r["F_ref"])
    assert len(Fg) == len(Fr) and np.all(np.abs(Fg - Fr) <= RTOL_F * np.abs(Fr))
    assert r["exact"] >= len(Fr) - 2, r
    for b, lv in r["ref"].apertures:
        assert _deliverable(lv, mode, int(case.cols[b]))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name,K", [("tiny", 16), ("prostate", 20)])
def test_mlc_free_running(torch, mode, name, K):
    """The device-driven graph path (the constrained pricing kernel between the
    D^T kernel and the beam decision) at every round against the oracle."""
    from paper_1003_5402_gb300 import binding
    case = P.make_case(P.CONFIGS[name]())
    r = _free_running_checked(case, K, torch, plan_kw={"mlc_constraint": binding.MLC[mode]}, mlc=mode)
    for b, lv in r["apertures"]:
        assert _deliverable(lv, mode, int(case.cols[b]))
    print(f"\n{mode} {name}: ties {r['ties']}, max objective rel {r['worst_F_rel']:.2e}, "
          f"max dose diff {r['worst_dose']:.2e}")


@pytest.mark.parametrize("mode", MODES)
def test_mlc_graph_rounds_equal_host_driven(torch, mode):
    from paper_1003_5402_gb300 import binding
    case = P.make_case(P.spec_micro())
    out = []
    for g, persistent in ((1, 1), (0, 1), (1, 0)):
        with _plan(case, torch, use_graphs=g, master_persistent=persistent, mlc_constraint=binding.MLC[mode]) as p:
            st, n, trace = p.solve(20)
            out.append((st, n, trace, p.apertures(), p.intensities()))
    for o in out[1:2]:
        assert o[0] == out[0][0] and o[1] == out[0][1]
        assert np.array_equal(o[2], out[0][2], equal_nan=True) and np.array_equal(o[4], out[0][4])
        assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(o[3], out[0][3]))
    # the per-kernel master reaches the same plan up to its own rounding
    a, c = out[0], out[2]
    assert a[1] == c[1]
    assert np.all(np.abs(a[2][:a[1]] - c[2][:c[1]]) <= RTOL_F * np.abs(a[2][:a[1]]))


def test_mlc_rejects_too_many_rows(torch):
    from paper_1003_5402_gb300 import DaoError, binding
    case = random_case(44, 300, rows=[65], cols=[4], mean_row=4.0)
    with pytest.raises(DaoError) as e:
        _plan(case, torch, mlc_constraint=binding.DAO_MLC_JAWS)
    assert e.value.status == -1
    with pytest.raises(DaoError):
        _plan(P.make_case(P.spec_micro()), torch, mlc_constraint=7)
