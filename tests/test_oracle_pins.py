"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-worked
traces of the pricing loop (Sec. 2.3), brute-force enumeration of every leaf
setting, closed forms of Eqs. 3-5/9-10, central finite differences, the
adjoint identity of the two SpMVs, an independent library optimiser
(scipy L-BFGS-B) for the master problem, and the equality of the
column-generation optimum with beamlet-level FMO.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import oracle as O
import phantom as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def micro():
    return P.make_case(P.spec_micro())


@pytest.fixture(scope="module")
def tiny():
    return P.make_case(P.spec_tiny())


# ---------------------------------------------------------------------------
# Pricing loop (Sec. 2.3)
# ---------------------------------------------------------------------------

def _golden_rows():
    out = []
    with open(os.path.join(GOLDEN, "kadane_rows.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            left, right = line.split("|")
            w = [float(t) for t in left.split()]
            v, L, R = right.split()
            out.append((w, float(v), int(L), int(R)))
    return out


@pytest.mark.parametrize("w,v,L,R", _golden_rows())
def test_kadane_hand_worked(w, v, L, R):
    assert O.kadane_row(np.array(w)) == (v, L, R)


def _brute_row(w):
    """Every half-open [L, R) of the row; the most negative sum wins, ties go to the
    smallest R, then the smallest L (the strict comparisons of the loop)."""
    best = (0.0, 0, 0)
    n = len(w)
    cands = []
    for L in range(n):
        for R in range(L + 1, n + 1):
            cands.append((float(sum(w[L:R])), R, L))
    if not cands:
        return best
    s, R, L = min(cands)
    if s < 0:
        return (s, L, R)
    return best


def test_kadane_brute_force_integer_ties():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        n = int(rng.integers(0, 10))
        w = rng.integers(-3, 4, size=n).astype(np.float64)
        assert O.kadane_row(w) == _brute_row(list(w)), w


def test_kadane_brute_force_continuous():
    rng = np.random.default_rng(6)
    for _ in range(1000):
        n = int(rng.integers(1, 33))
        w = rng.normal(size=n) + 0.3
        v, L, R = O.kadane_row(w)
        bv, bL, bR = _brute_row(list(w))
        assert (L, R) == (bL, bR)
        assert abs(v - bv) <= 1e-12 * (1 + np.sum(np.abs(w)))


def test_kadane_is_negated_maximum_subarray():
    """Bentley's maximum-subarray value on -w (with the empty subarray allowed) is -v*."""
    rng = np.random.default_rng(7)
    for _ in range(500):
        w = rng.normal(size=int(rng.integers(1, 20)))
        best = cur = 0.0
        for t in -w:                       # textbook scan, separate from the oracle's loop
            cur = max(0.0, cur + t)
            best = max(best, cur)
        assert abs(O.kadane_row(w)[0] + best) <= 1e-12 * (1 + np.sum(np.abs(w)))


class _Geo:
    def __init__(self, rows, cols):
        self.rows = np.array(rows, dtype=np.int32)
        self.cols = np.array(cols, dtype=np.int32)


def _row_settings(n):
    return [(0, 0)] + [(L, R) for L in range(n) for R in range(L + 1, n + 1)]


def test_pricing_brute_force_all_leaf_settings():
    """On fields of <= 3 rows x 4 columns every aperture (each row closed or open on one
    consecutive range) is enumerated; the oracle's beam sums and chosen aperture must be
    the minimum of Eq. 8, lowest beam on equal sums."""
    rng = np.random.default_rng(8)
    for trial in range(60):
        B = int(rng.integers(1, 4))
        rows = [int(rng.integers(1, 4)) for _ in range(B)]
        cols = [int(rng.integers(1, 5)) for _ in range(B)]
        geo = _Geo(rows, cols)
        N = int(np.sum(np.array(rows) * np.array(cols)))
        w = rng.integers(-3, 3, size=N).astype(np.float64)
        pr = O.price(geo, w)
        off = 0
        best_vals = []
        for b in range(B):
            bm = np.inf
            for setting in itertools.product(_row_settings(cols[b]), repeat=rows[b]):
                s = 0.0
                for r, (L, R) in enumerate(setting):
                    s += np.sum(w[off + r * cols[b] + L: off + r * cols[b] + R])
                bm = min(bm, s)
            best_vals.append(bm)
            assert pr.beam_values[b] == bm
            off += rows[b] * cols[b]
        assert pr.beam == int(np.argmin(best_vals))          # argmin: first on ties
        assert O.aperture_value(geo, w, pr.beam, pr.leaves) == min(best_vals)
        assert pr.reduced_cost == min(best_vals)


def test_pricing_all_nonnegative_closes_everything():
    geo = _Geo([3, 2], [4, 5])
    w = np.abs(np.random.default_rng(9).normal(size=22))
    pr = O.price(geo, w)
    assert pr.reduced_cost == 0.0 and pr.beam == 0
    assert np.all(pr.leaves == 0)


# ---------------------------------------------------------------------------
# Dose and pricing weights (Eqs. 1, 2, 7, 8)
# ---------------------------------------------------------------------------

def _dense(case):
    V = len(case.indptr) - 1
    N = case.n_beamlets
    A = np.zeros((V, N))
    rows = np.repeat(np.arange(V), np.diff(case.indptr))
    np.add.at(A, (rows, case.indices.astype(np.int64)), case.data.astype(np.float64))
    return A


def test_unit_beamlet_dose_is_column(micro):
    D = O.csr64(micro)
    A = _dense(micro)
    for i in [0, 1, 17, micro.n_beamlets - 1]:
        e = np.zeros(micro.n_beamlets)
        e[i] = 1.0
        assert np.array_equal(O.dose(D, e), A[:, i])


def test_dose_and_prices_match_dense(micro):
    D = O.csr64(micro)
    A = _dense(micro)
    rng = np.random.default_rng(10)
    x = rng.uniform(size=micro.n_beamlets)
    g = rng.normal(size=micro.n_voxels)
    np.testing.assert_allclose(O.dose(D, x), A @ x, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(O.beamlet_prices(D, g), A.T @ g, rtol=1e-12, atol=1e-12)


def test_adjoint_identity(tiny):
    D = O.csr64(tiny)
    rng = np.random.default_rng(11)
    x = rng.uniform(size=tiny.n_beamlets)
    g = rng.normal(size=tiny.n_voxels)
    lhs = np.dot(O.dose(D, x), g)
    rhs = np.dot(x, O.beamlet_prices(D, g))
    assert abs(lhs - rhs) <= 1e-12 * np.dot(np.abs(O.dose(D, x)), np.abs(g))


def test_aperture_column_and_fluence(micro):
    """Eq. 2 column of an aperture equals the dense sum of its beamlet columns, and the
    dose of Eq. 1 through the aperture columns equals D x with x from Eq. 7."""
    D = O.csr64(micro)
    A = _dense(micro)
    aps = [(0, np.array([[0, 3], [1, 6], [0, 0], [2, 4]])), (2, np.array([[0, 6]] * 4))]
    y = np.array([0.7, 1.3])
    cols = [O.aperture_column(D, micro, b, lv) for b, lv in aps]
    m0 = np.zeros(micro.n_beamlets)
    off0 = 0
    for r, (L, R) in enumerate(aps[0][1]):
        m0[off0 + r * 6 + L: off0 + r * 6 + R] = 1
    np.testing.assert_allclose(cols[0], A @ m0, rtol=1e-13, atol=1e-15)
    z1 = sum(yk * c for yk, c in zip(y, cols))
    z2 = O.dose(D, O.fluence(micro, aps, y))
    np.testing.assert_allclose(z1, z2, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# Objective (Eqs. 3-5, 9-10)
# ---------------------------------------------------------------------------

def test_objective_closed_form_uniform_underdose(tiny):
    """All voxels of each target at T^- - delta, everything else below its over-threshold:
    Eq. 9 gives alpha_s * delta^2 per target (the 1/|v_s| cancels the voxel count)."""
    vt = O.voxel_terms(tiny)
    delta = 0.125
    z = np.zeros(tiny.n_voxels)
    tgt = tiny.is_target[tiny.voxel_struct].astype(bool)
    z[tgt] = tiny.under_t[tiny.voxel_struct[tgt]] - delta
    # targets' own over-threshold equals T^-, so they are below it; others sit at 0
    expect = sum(tiny.under_w[s] * delta ** 2 for s in range(len(tiny.names)) if tiny.is_target[s])
    assert abs(O.objective(z, vt) - expect) <= 1e-14


def test_objective_closed_form_uniform_overdose(tiny):
    """Every voxel of structure s at T_s^+ + delta (targets at their prescription plus
    delta): Eq. 10 gives beta_s * delta^2 per structure and Eq. 9 gives 0."""
    vt = O.voxel_terms(tiny)
    delta = 0.25
    z = tiny.over_t[tiny.voxel_struct] + delta
    expect = float(np.sum(tiny.over_w))
    expect *= delta ** 2
    assert abs(O.objective(z, vt) - expect) <= 1e-13


def test_objective_unnormalised_is_eqs_3_4():
    class C:
        voxel_struct = np.array([0, 0, 1])
        is_target = np.array([1, 0], dtype=np.uint8)
        under_w = np.array([2.0, 0.0])
        under_t = np.array([1.0, 0.0])
        over_w = np.array([3.0, 5.0])
        over_t = np.array([1.2, 0.5])
    vt = O.voxel_terms(C, normalize_by_volume=False)
    z = np.array([0.5, 1.5, 0.7])
    expect = 2.0 * 0.5 ** 2 + 3.0 * 0.3 ** 2 + 5.0 * 0.2 ** 2
    assert abs(O.objective(z, vt) - expect) <= 1e-14


def test_gradient_and_curvature_finite_differences(micro):
    """Central differences of each voxel's own term F_j (a one-voxel objective, so the
    difference quotient is not swamped by the other voxels' rounding)."""
    vt = O.voxel_terms(micro)
    rng = np.random.default_rng(12)
    z = rng.uniform(0.0, 1.5, size=micro.n_voxels)
    g = O.gradient(z, vt)
    h = O.curvature(z, vt)
    checked = 0
    for j in rng.choice(micro.n_voxels, 60, replace=False):
        # stay away from the kinks at T^- and T^+
        if min(abs(z[j] - vt.t_under[j]), abs(z[j] - vt.t_over[j])) < 1e-3:
            continue
        one = O.VoxelTerms(vt.alpha[j:j + 1], vt.t_under[j:j + 1], vt.beta[j:j + 1], vt.t_over[j:j + 1])
        e = 1e-5
        zp, zm = z[j:j + 1] + e, z[j:j + 1] - e
        fd = (O.objective(zp, one) - O.objective(zm, one)) / (2 * e)
        assert abs(fd - g[j]) <= 1e-8 * max(abs(g[j]), abs(vt.alpha[j]) + abs(vt.beta[j])) + 1e-18
        fd2 = (O.gradient(zp, one)[0] - O.gradient(zm, one)[0]) / (2 * e)
        assert abs(fd2 - h[j]) <= 1e-8 * max(abs(h[j]), abs(vt.alpha[j]) + abs(vt.beta[j])) + 1e-18
        checked += 1
    assert checked > 30


def test_chain_rule_in_aperture_intensities(micro):
    """d F(S y) / d y_k by central differences equals S^T grad F (the master gradient)."""
    D = O.csr64(micro)
    vt = O.voxel_terms(micro)
    rng = np.random.default_rng(13)
    aps = []
    for b in range(micro.n_beams):
        lv = np.array([[int(rng.integers(0, 3)), int(rng.integers(3, 7))] for _ in range(4)])
        aps.append((b, lv))
    S = np.column_stack([O.aperture_column(D, micro, b, lv) for b, lv in aps])
    y = rng.uniform(0.2, 1.0, size=S.shape[1])
    g = S.T @ O.gradient(S @ y, vt)
    for k in range(S.shape[1]):
        e = 1e-6
        yp, ym = y.copy(), y.copy()
        yp[k] += e
        ym[k] -= e
        fd = (O.objective(S @ yp, vt) - O.objective(S @ ym, vt)) / (2 * e)
        assert abs(fd - g[k]) <= 1e-5 * abs(g[k]) + 1e-9


# ---------------------------------------------------------------------------
# Master problem (Sec. 2.3: non-negative intensities, convex objective)
# ---------------------------------------------------------------------------

def test_master_one_voxel_one_beamlet_closed_form():
    """One target voxel (T = 1, alpha = 1), one aperture with D = 0.5: y* = T / D = 2, F = 0."""
    vt = O.VoxelTerms(alpha=np.array([1.0]), t_under=np.array([1.0]), beta=np.array([0.0]),
                      t_over=np.array([1.0]))
    m = O.solve_master(np.array([[0.5]]), vt, np.zeros(1))
    assert abs(m.y[0] - 2.0) <= 4e-16 * 2.0 and m.F <= 1e-30       # a few rounding steps of the solve


def test_identity_dose_full_field_single_aperture():
    """D = I over a full rectangular field with a uniform target prescription T: the
    first priced aperture opens every row completely, y_1 = T, F = 0 and column
    generation stops at K = 1 with no negative reduced cost."""
    rows, cols, T = 3, 4, 0.8

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
    c.is_target = np.array([1], dtype=np.uint8)
    c.under_w = np.array([1.0])
    c.under_t = np.array([T])
    c.over_w = np.array([1.0])
    c.over_t = np.array([T])
    res = O.column_generation(c, 10)
    assert len(res.apertures) == 1 and res.status == "optimal"
    b, lv = res.apertures[0]
    assert b == 0 and np.all(lv[:, 0] == 0) and np.all(lv[:, 1] == cols)
    assert abs(res.y[0] - T) <= 1e-15 and res.objective[0] <= 1e-30


def _lbfgsb_master(S, vt):
    f = lambda y: O.objective(S @ y, vt)
    # gradient by central differences: independent of the oracle's gradient formula
    def fg(y):
        g = np.zeros_like(y)
        for k in range(len(y)):
            e = 1e-7 * max(1.0, abs(y[k]))
            yp, ym = y.copy(), y.copy()
            yp[k] += e
            ym[k] -= e
            g[k] = (f(yp) - f(ym)) / (2 * e)
        return f(y), g
    r = so.minimize(fg, np.full(S.shape[1], 0.1), jac=True, method="L-BFGS-B",
                    bounds=[(0, None)] * S.shape[1], options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    return r.fun


def test_master_matches_independent_lbfgsb(micro):
    D = O.csr64(micro)
    vt = O.voxel_terms(micro)
    rng = np.random.default_rng(14)
    for trial in range(3):
        aps = []
        for k in range(5):
            b = int(rng.integers(0, micro.n_beams))
            lv = np.array([[int(rng.integers(0, 3)), int(rng.integers(3, 7))] for _ in range(4)])
            aps.append((b, lv))
        S = np.column_stack([O.aperture_column(D, micro, b, lv) for b, lv in aps])
        m = O.solve_master(S, vt, np.zeros(S.shape[1]))
        ref = _lbfgsb_master(S, vt)
        assert m.F <= ref * (1 + 1e-7) + 1e-15
        assert m.F >= ref * (1 - 1e-6) - 1e-15


def test_master_kkt_by_finite_differences(micro):
    """At the oracle's optimum, a finite-difference gradient satisfies y >= 0, g >= 0 where
    y = 0 and g = 0 where y > 0 (to finite-difference accuracy)."""
    D = O.csr64(micro)
    vt = O.voxel_terms(micro)
    res = O.column_generation(micro, 12)
    S = np.column_stack([O.aperture_column(D, micro, b, lv) for b, lv in res.apertures])
    y = res.y
    f = lambda yy: O.objective(S @ yy, vt)
    scale = np.max(np.abs(S.T @ np.abs(O.gradient(np.zeros(micro.n_voxels), vt))))
    assert np.all(y >= 0)
    for k in range(len(y)):
        e = 1e-6
        yp = y.copy()
        yp[k] += e
        if y[k] > 2 * e:
            ym = y.copy()
            ym[k] -= e
            fd = (f(yp) - f(ym)) / (2 * e)
            assert abs(fd) <= 1e-6 * scale
        else:
            fd = (f(yp) - f(y)) / e
            assert fd >= -1e-6 * scale


# ---------------------------------------------------------------------------
# Column generation (Sec. 2.2-2.3)
# ---------------------------------------------------------------------------

def test_cg_objective_non_increasing_and_reduced_costs_negative(tiny):
    res = O.column_generation(tiny, 20)
    F = np.array(res.objective)
    assert len(F) == 20
    assert np.all(np.diff(F) <= 1e-12 * F[:-1])
    assert np.all(np.array(res.reduced_cost) < 0)
    assert max(res.kkt) <= 1e-10 * abs(res.reduced_cost[0])


def test_cg_to_optimality_equals_fmo_and_certificate(micro):
    """Run to termination: no aperture (checked by enumerating every row setting) has a
    negative reduced cost, and the objective equals the beamlet-level FMO optimum."""
    res = O.column_generation(micro, 400)
    assert res.status == "optimal"
    f = O.fmo(micro)
    assert f.status == "kkt"
    assert abs(res.objective[-1] - f.F) <= 1e-8 * f.F
    assert all(Fk >= f.F * (1 - 1e-12) for Fk in res.objective)
    D = O.csr64(micro)
    w = O.beamlet_prices(D, res.pi)
    off = 0
    tau = O.pricing_tolerance(D, O.gradient(np.zeros(micro.n_voxels), O.voxel_terms(micro)))
    for b in range(micro.n_beams):
        R, C = int(micro.rows[b]), int(micro.cols[b])
        total = 0.0
        for r in range(R):
            seg = w[off + r * C: off + (r + 1) * C]
            total += min([0.0] + [float(np.sum(seg[L:Rr])) for L, Rr in _row_settings(C)[1:]])
        assert total >= -tau * 10
        off += R * C


def test_fmo_matches_independent_lbfgsb():
    c = P.make_case(P.spec_micro(seed=3, n_beams=2, rows=2, cols=3, grid=(12, 12, 4)))
    f = O.fmo(c)
    D = O.csr64(c)
    ref = _lbfgsb_master(D.toarray(), O.voxel_terms(c))
    assert abs(f.F - ref) <= 1e-7 * ref


def test_teacher_forcing_reproduces_free_run(micro):
    free = O.column_generation(micro, 8)
    forced = O.column_generation(micro, 8, teacher=free.apertures)
    np.testing.assert_allclose(forced.objective, free.objective, rtol=1e-12)


# ---------------------------------------------------------------------------
# Small definitions: the aperture indicator (Eq. 2), the KKT residual of the
# master's bound-constrained optimality and the pricing tolerance
# ---------------------------------------------------------------------------

class _Geometry:
    """Two beams: 2 rows x 3 beamlets, then 3 rows x 2 beamlets (N = 12)."""
    rows = np.array([2, 3])
    cols = np.array([3, 2])


def test_aperture_mask_by_hand():
    g = _Geometry()
    # beam 1 starts at beamlet 6; row r covers beamlets 6 + 2r .. 6 + 2r + 1
    m = O.aperture_mask(g, 1, [(0, 2), (1, 1), (1, 2)])
    want = np.zeros(12)
    want[[6, 7, 11]] = 1.0
    assert np.array_equal(m, want)
    # beam 0, row 0 open on [1, 3), row 1 closed
    m0 = O.aperture_mask(g, 0, [(1, 3), (0, 0)])
    want0 = np.zeros(12)
    want0[[1, 2]] = 1.0
    assert np.array_equal(m0, want0)


def test_aperture_value_is_sum_of_open_prices():
    g = _Geometry()
    w = np.arange(12, dtype=np.float64) - 5.0
    assert O.aperture_value(g, w, 1, [(0, 2), (1, 1), (1, 2)]) == w[6] + w[7] + w[11]


@pytest.mark.parametrize("y,g,res", [
    ([0.0, 2.0, 1.0], [3.0, 0.0, -1.0], 1.0),   # bound active with g > 0: 0; free with g = 0: 0; free with g != 0: |g|
    ([0.0], [-2.5], 2.5),                        # at the bound, descent into the feasible set
    ([0.4], [1.0], 0.4),                         # the projected step stops at the bound: |y - 0|
    ([], [], 0.0),
])
def test_kkt_residual_of_the_bound_constrained_problem(y, g, res):
    assert O.kkt_residual(np.array(y), np.array(g)) == res


def test_pricing_tolerance_is_rel_max_d_times_l1_of_pi():
    D = sp.csr_matrix(np.array([[0.5, 0.0, 2.0], [0.0, 1.5, 0.25]]))
    pi = np.array([-3.0, 4.0])
    assert O.pricing_tolerance(D, pi, rel=1e-3) == pytest.approx(1e-3 * 2.0 * 7.0, rel=0, abs=1e-18)
    assert O.pricing_tolerance(sp.csr_matrix((2, 3)), pi) == 0.0


def test_fluence_of_overlapping_apertures_by_hand():
    """Eq. 7: a beamlet's fluence is the sum of the intensities of the apertures
    that leave it open."""
    g = _Geometry()
    aps = [(1, [(0, 2), (1, 1), (1, 2)]),   # beamlets 6, 7, 11
           (1, [(1, 2), (0, 2), (0, 0)]),   # beamlets 7, 8, 9
           (0, [(0, 3), (0, 0)])]           # beamlets 0, 1, 2
    x = O.fluence(g, aps, [0.5, 2.0, 1.25])
    want = np.zeros(12)
    want[[0, 1, 2]] = 1.25
    want[6] = 0.5
    want[7] = 0.5 + 2.0
    want[[8, 9]] = 2.0
    want[11] = 0.5
    assert np.array_equal(x, want)
    assert np.array_equal(O.fluence(g, [], []), np.zeros(12))


def test_curvature_on_each_side_of_the_thresholds():
    """The generalised second derivative of one voxel's penalty: 2 alpha below
    T^-, 2 beta above T^+, 0 between them and at either kink (strict
    inequalities), both terms at once when T^+ < T^-."""
    vt = O.VoxelTerms(alpha=np.full(6, 3.0), t_under=np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0]),
                      beta=np.full(6, 0.5), t_over=np.array([1.2, 1.2, 1.2, 1.2, 1.2, 0.4]))
    z = np.array([0.9, 1.0, 1.1, 1.2, 1.3, 0.6])
    assert np.array_equal(O.curvature(z, vt), [6.0, 0.0, 0.0, 0.0, 1.0, 7.0])
