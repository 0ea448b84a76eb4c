"""Pins of the oracle's re-optimisation mode (Sec. 4: Eqs. 3-4 with
alpha_j = beta_j = 1 and T_j the planned dose deformed onto the day's anatomy)
against results fixed by mathematics or by independent library routines:

  - with both terms on every voxel F(z) is the squared distance ||z - T||^2 and
    its gradient 2 (z - T) (closed form);
  - with Eq. 3 on the target voxels only, a hand-worked four-voxel case;
  - the master problem with both terms on every voxel is non-negative least
    squares, min ||S y - T||^2 over y >= 0: scipy.optimize.nnls (Lawson-Hanson)
    gives y and F independently;
  - D = I with a uniform T on a full field: one full-field aperture, y = T,
    F = 0, column generation stops;
  - the per-voxel form equals the per-structure expansion when the thresholds
    and unit weights are constant per structure.
"""
import numpy as np
import pytest
import scipy.optimize as so

import oracle as O
import phantom as P


@pytest.fixture(scope="module")
def micro():
    return P.make_case(P.spec_micro())


def test_reopt_objective_is_squared_distance():
    rng = np.random.default_rng(3)
    T = rng.uniform(0.0, 1.2, 50)
    z = rng.uniform(0.0, 1.2, 50)
    vt = O.reoptimisation_terms(T)
    d = z - T
    assert abs(O.objective(z, vt) - float(d @ d)) <= 1e-14 * float(d @ d)
    assert np.allclose(O.gradient(z, vt), 2.0 * d, rtol=0, atol=1e-15)
    assert np.array_equal(O.curvature(z, vt), 2.0 * (z != T))


def test_reopt_objective_target_mask_by_hand():
    """Voxels 0, 1 targets (Eq. 3 and 4), voxels 2, 3 not (Eq. 4 only):
    z = (0.5, 1.5, 0.25, 2.0), T = (1, 1, 1, 1): under-dose 0.5^2 on voxel 0,
    over-dose 0.5^2 on voxel 1 and 1.0^2 on voxel 3, voxel 2's under-dose not
    counted: F = 0.25 + 0.25 + 1.0 = 1.5; gradient (-1, 1, 0, 2)."""
    vt = O.reoptimisation_terms(np.ones(4), target_mask=[True, True, False, False])
    z = np.array([0.5, 1.5, 0.25, 2.0])
    assert O.objective(z, vt) == 1.5
    assert np.array_equal(O.gradient(z, vt), np.array([-1.0, 1.0, 0.0, 2.0]))


def test_reopt_master_is_nonnegative_least_squares(micro):
    D = O.csr64(micro)
    rng = np.random.default_rng(8)
    cols = []
    for b in range(micro.n_beams):
        R, Cn = int(micro.rows[b]), int(micro.cols[b])
        for _ in range(3):
            lv = np.zeros((R, 2), np.int32)
            for r in range(R):
                L = int(rng.integers(0, Cn))
                lv[r] = (L, int(rng.integers(L + 1, Cn + 1)))
            cols.append(O.aperture_column(D, micro, b, lv))
    S = np.column_stack(cols)
    # a target that no non-negative combination reaches exactly: some bounds active
    y_true = rng.uniform(-0.5, 1.0, S.shape[1])
    T = S @ y_true + 0.05 * rng.standard_normal(S.shape[0])
    vt = O.reoptimisation_terms(T)
    m = O.solve_master(S, vt, np.zeros(S.shape[1]))
    y_ls, rnorm = so.nnls(S, T, maxiter=10000)
    assert np.any(y_ls == 0.0) and np.any(y_ls > 0.0)
    assert abs(m.F - rnorm ** 2) <= 1e-10 * rnorm ** 2
    assert np.max(np.abs(m.y - y_ls)) <= 1e-7 * max(1.0, np.max(y_ls))


def test_reopt_identity_dose_full_field():
    rows, cols, T = 3, 4, 0.7

    class C:
        pass
    c = C()
    N = rows * cols
    c.indptr = np.arange(N + 1, dtype=np.int64)
    c.indices = np.arange(N, dtype=np.int32)
    c.data = np.ones(N, dtype=np.float32)
    c.rows = np.array([rows], dtype=np.int32)
    c.cols = np.array([cols], dtype=np.int32)
    c.voxel_struct = np.zeros(N, dtype=np.int32)
    c.is_target = np.array([0], dtype=np.uint8)
    c.under_w = c.under_t = c.over_w = c.over_t = np.zeros(1)
    res = O.column_generation(c, 10, vt=O.reoptimisation_terms(np.full(N, T)))
    assert len(res.apertures) == 1 and res.status == "optimal"
    b, lv = res.apertures[0]
    assert b == 0 and np.all(lv[:, 0] == 0) and np.all(lv[:, 1] == cols)
    assert abs(res.y[0] - T) <= 1e-15 and res.objective[0] <= 1e-30


def test_reopt_form_equals_structure_expansion(micro):
    """Every voxel a target of its structure, thresholds T_s on both sides,
    unit weights, no volume division: the per-structure expansion of Eqs. 9-10
    and the per-voxel form give identical terms and an identical plan."""
    import copy
    c = copy.copy(micro)
    S = len(c.under_w)
    Ts = np.linspace(0.3, 1.0, S)
    c.is_target = np.ones(S, np.uint8)
    c.under_w = np.ones(S)
    c.over_w = np.ones(S)
    c.under_t = Ts.copy()
    c.over_t = Ts.copy()
    a = O.voxel_terms(c, normalize_by_volume=False)
    b = O.reoptimisation_terms(Ts[np.asarray(c.voxel_struct)])
    for f in ("alpha", "t_under", "beta", "t_over"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    r1 = O.column_generation(c, 4, normalize_by_volume=False)
    r2 = O.column_generation(c, 4, vt=b)
    assert r1.objective == r2.objective
    assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(r1.apertures, r2.apertures))
