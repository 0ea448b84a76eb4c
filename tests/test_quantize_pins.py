"""Pins of the test-side 16-bit quantiser of D (per-beamlet scale + RN16), which
the mixed-precision GPU tests use as the definition of the stored matrix: the
rounding of known bfloat16 ties and halfway cases, the scale mapping each
beamlet's largest entry to exactly 1, and the relative error bounds of the two
formats (unit roundoff 2^-8 for bfloat16 and 2^-11 for FP16 on quotients in
[2^-14, 1], each plus the FP32 quotient's 2^-24)."""
import numpy as np
import pytest

import phantom as P
from _helpers import bf16_round, beamlet_scale, quantized_case, random_case


def test_bf16_rounding_known_values():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)                   # bfloat16 spacing in [1, 2)
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                      # halfway, even neighbour is 1.0
        1.0 + 3 * 2.0 ** -8: 1.0 + 2 * 2.0 ** -7,  # halfway, rounds up to even
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,  # above halfway
        0.5 + 2.0 ** -10: 0.5,                     # below halfway
        3.140625: 3.140625,                        # exactly representable
        -1.0 - 3 * 2.0 ** -8: -(1.0 + 2 * 2.0 ** -7),
    }
    x = np.array(list(cases), np.float32)
    got = bf16_round(x)
    assert np.array_equal(got, np.array(list(cases.values()), np.float32))
    assert float(ulp) == float(one) * 2.0 ** -7


@pytest.mark.parametrize("prec,rel", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_quantised_matrix_error_bounds(prec, rel):
    case = P.make_case(P.spec_micro())
    q = quantized_case(case, prec)
    d = np.asarray(case.data, np.float64)
    s = beamlet_scale(case).astype(np.float64)[np.asarray(case.indices)]
    err = np.abs(q.data - d)
    # RN16 of a quotient r in (0, 1]: |RN16(r) - r| <= u |r| in the normal range
    # (u = 2^-p, p the significand bits); the FP32 quotient adds 2^-24 |r|; both
    # scaled back by s_i
    normal = d / s >= 2.0 ** -14
    assert np.all(err[normal] <= (rel + 2.0 ** -24) * d[normal] * (1 + 1e-12))
    assert np.all(err <= (rel + 2.0 ** -24) * s)  # absolute bound everywhere (values <= s_i)
    # and the bound is nearly attained: the rounding really is to 11 / 8 bits
    assert np.max(err[normal] / d[normal]) > rel / 4
    # per-beamlet maximum maps to exactly 1: dequantised equals the FP32 maximum
    for i in np.unique(case.indices)[:50]:
        m = case.indices == i
        j = np.argmax(np.abs(case.data[m]))
        assert q.data[m][j] == float(case.data[m][j])


def test_scale_of_empty_beamlet_is_one_and_structure_is_kept():
    case = random_case(5, 300, rows=[2, 3], cols=[4, 5], mean_row=3.0)
    s = beamlet_scale(case)
    present = np.zeros(case.n_beamlets, bool)
    present[np.unique(case.indices)] = True
    assert np.all(s[~present] == 1.0)
    q = quantized_case(case, "fp16")
    assert np.array_equal(q.indices, case.indices) and np.array_equal(q.indptr, case.indptr)
    assert q.data.dtype == np.float64 and case.data.dtype == np.float32
