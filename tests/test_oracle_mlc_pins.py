"""Pins of the oracle's MLC-constrained pricing (Sec. 4: interdigitation,
connectedness, jaws-only) against brute-force enumeration of every
deliverable aperture on small fields, hand-worked cases, and the ordering the
constraints impose on the optimal values (each constraint only removes
apertures: consecutive <= interdigitation, connected <= jaws)."""
import itertools

import numpy as np
import pytest

import oracle as O
from oracle import mlc as M


def _I(w_row, L, R):
    P = M.row_prefix(w_row)
    return P[R] - P[L]


def _brute(w, R, C, mode):
    """(optimal value, [optimal apertures as tuples of (L, R) per row, closed
    rows as (p, p)]) over every aperture the constraint allows."""
    w = np.asarray(w, np.float64).reshape(R, C)
    states = M.interval_states(C)
    best, arg = 0.0, []
    if mode == "interdigitation":
        for seq in itertools.product(states, repeat=R):
            if any(not (seq[r][0] <= seq[r + 1][1] and seq[r + 1][0] <= seq[r][1]) for r in range(R - 1)):
                continue
            acc = _I(w[0], *seq[0])
            for r in range(1, R):
                acc = _I(w[r], *seq[r]) + acc
            if acc < best:
                best, arg = acc, [seq]
            elif acc == best and acc < 0:
                arg.append(seq)
    elif mode == "connected":
        opts = [(0, 0)] + [(L, Rr) for L in range(C) for Rr in range(L + 1, C + 1)]
        for seq in itertools.product(opts, repeat=R):
            open_rows = [r for r in range(R) if seq[r][0] < seq[r][1]]
            if not open_rows or open_rows != list(range(open_rows[0], open_rows[-1] + 1)):
                continue
            acc = sum(_I(w[r], *seq[r]) for r in open_rows)
            if acc < best:
                best, arg = acc, [seq]
            elif acc == best and acc < 0:
                arg.append(seq)
    elif mode == "jaws":
        for L in range(C):
            for Rr in range(L + 1, C + 1):
                for a in range(R):
                    for b in range(a + 1, R + 1):
                        acc = sum(_I(w[r], L, Rr) for r in range(a, b))
                        seq = tuple((L, Rr) if a <= r < b else (0, 0) for r in range(R))
                        if acc < best:
                            best, arg = acc, [seq]
                        elif acc == best and acc < 0:
                            arg.append(seq)
    return best, arg


def _norm(seq):
    return np.array([(L, R) if L < R else (0, 0) for L, R in seq], np.int32)


def _feasible(lv, mode, C):
    """An aperture (closed rows (0, 0)) meets the constraint, a closed row free
    to park its leaves anywhere."""
    R = len(lv)
    opn = [r for r in range(R) if lv[r][0] < lv[r][1]]
    if mode == "connected":
        return not opn or opn == list(range(opn[0], opn[-1] + 1))
    if mode == "jaws":
        return not opn or (opn == list(range(opn[0], opn[-1] + 1)) and len({tuple(lv[r]) for r in opn}) == 1)
    # interdigitation: closed rows choose a parking position p
    choices = [[(int(lv[r][0]), int(lv[r][1]))] if r in opn else [(p, p) for p in range(C + 1)] for r in range(R)]
    for seq in itertools.product(*choices):
        if all(seq[r][0] <= seq[r + 1][1] and seq[r + 1][0] <= seq[r][1] for r in range(R - 1)):
            return True
    return False


MODES = ["interdigitation", "connected", "jaws"]
SHAPES = [(1, 4), (2, 3), (3, 3), (2, 4), (3, 4)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("R,C", SHAPES)
def test_brute_force_integer_prices(mode, R, C):
    """Integer prices (many exact ties): the optimal value is exact, the
    aperture returned is deliverable and attains it."""
    rng = np.random.default_rng(100 * R + C)
    fn = M.MODES[mode]
    for trial in range(25):
        w = rng.integers(-3, 4, size=R * C).astype(np.float64)
        v, lv = fn(w, R, C)
        best, arg = _brute(w, R, C, mode)
        assert v == best, (trial, v, best)
        assert _feasible(lv, mode, C)
        got = sum(_I(w.reshape(R, C)[r], *lv[r]) for r in range(R))
        assert got == v
        if v < 0:
            assert any(np.array_equal(_norm(a), lv) for a in arg)
        else:
            assert np.all(lv == 0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("R,C", SHAPES)
def test_brute_force_continuous_prices(mode, R, C):
    rng = np.random.default_rng(7 * R + C)
    fn = M.MODES[mode]
    for trial in range(20):
        w = rng.normal(size=R * C).astype(np.float32).astype(np.float64)
        v, lv = fn(w, R, C)
        best, arg = _brute(w, R, C, mode)
        assert abs(v - best) <= 1e-12 * max(1.0, abs(best))
        assert _feasible(lv, mode, C)
        if best < -1e-9:
            assert np.array_equal(_norm(arg[0]), lv)


@pytest.mark.parametrize("R,C", SHAPES)
def test_interdigitation_tie_rule_is_reverse_lexicographic(R, C):
    """Among optimal state sequences the programme returns the one that is
    smallest read from the last row to the first (state index order)."""
    rng = np.random.default_rng(900 + R * C)
    states = M.interval_states(C)
    for trial in range(25):
        w = rng.integers(-2, 3, size=R * C).astype(np.float64)
        v, lv = M.price_interdigitation(w, R, C)
        best, arg = _brute(w, R, C, "interdigitation")
        if best < 0:
            key = lambda seq: tuple(states.index(seq[r]) for r in range(R - 1, -1, -1))
            assert np.array_equal(_norm(min(arg, key=key)), lv), trial


def test_interdigitation_by_hand():
    """Row 0 alone would open [0, 1) (price -3), row 1 alone [3, 4) (price -3);
    the two leaves would cross.  Opening both (row 1 from 1) costs
    -3 + (4 + 4 - 3) = 2; the best deliverable aperture opens one row (-3).
    The smallest final state is row 1 closed at 0, so row 0 opens [0, 1)."""
    w = np.array([-3, 4, 4, 4, 4, 4, 4, -3], np.float64)
    v, lv = M.price_interdigitation(w, 2, 4)
    assert v == -3.0 and np.array_equal(lv, [[0, 1], [0, 0]])
    # consecutiveness alone takes both rows: -6
    assert sum(O.kadane_row(w[r * 4:(r + 1) * 4])[0] for r in range(2)) == -6.0


def test_connected_by_hand():
    """Rows 0 and 2 are cheap, row 1 only costs: connectedness must open row 1
    too (its best non-empty interval, its first beamlet at +1) or take one
    row.  Rows' best non-empty values: -5, +1, -5: the block 0..2 gives -9."""
    w = np.array([-5, 2, 1, 3, -5, 2], np.float64)
    v, lv = M.price_connected(w, 3, 2)
    assert v == -9.0 and np.array_equal(lv, [[0, 1], [0, 1], [0, 1]])


def test_jaws_by_hand():
    """A rectangle: columns [1, 3) over rows 0..1 gives -2 - 2 - 2 - 2 = -8
    (a third row adds +10)."""
    w = np.array([5, -2, -2, 5,
                  5, -2, -2, 5,
                  5, 5, 5, 5], np.float64)
    v, lv = M.price_jaws(w, 3, 4)
    assert v == -8.0 and np.array_equal(lv, [[1, 3], [1, 3], [0, 0]])


def test_constraints_only_remove_apertures():
    rng = np.random.default_rng(55)
    for trial in range(40):
        R, C = int(rng.integers(1, 6)), int(rng.integers(1, 9))
        w = rng.normal(size=R * C)
        cons = sum(O.kadane_row(w[r * C:(r + 1) * C])[0] for r in range(R))
        vi = M.price_interdigitation(w, R, C)[0]
        vc = M.price_connected(w, R, C)[0]
        vj = M.price_jaws(w, R, C)[0]
        tol = 1e-12 * (1 + np.sum(np.abs(w)))
        assert cons <= vi + tol and cons <= vc + tol
        assert vi <= vj + tol and vc <= vj + tol
        if R == 1:
            assert abs(vi - cons) <= tol and abs(vc - cons) <= tol and abs(vj - cons) <= tol


def test_price_dispatch_and_beam_argmin():
    """price(case, w, mode): each beam priced under the constraint, the beam
    value at its first row, the lowest-value beam chosen (lowest index on ties)."""
    class C_:
        pass
    c = C_()
    c.rows = np.array([2, 3], np.int32)
    c.cols = np.array([4, 3], np.int32)
    rng = np.random.default_rng(3)
    w = rng.integers(-3, 4, size=8 + 9).astype(np.float64)
    for mode in MODES:
        pr = O.price(c, w, mode)
        v0, l0 = M.MODES[mode](w[:8], 2, 4)
        v1, l1 = M.MODES[mode](w[8:], 3, 3)
        assert list(pr.beam_values) == [v0, v1]
        assert pr.beam == (1 if v1 < v0 else 0)
        assert np.array_equal(pr.leaves, l1 if v1 < v0 else l0)
        assert pr.row_values[0][0] == v0 and np.all(pr.row_values[0][1:] == 0)
