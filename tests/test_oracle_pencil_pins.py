"""Pins of the oracle's pencil-beam coefficients (oracle.pencil) against closed
forms and against the input generator's windowed implementation
(phantom.make_case), an independent restatement of the same model."""
import math

import numpy as np
import pytest

import oracle.pencil as PB
import phantom as P


def _args(spec, case):
    return dict(xyz=case.voxel_xyz, iso=case.iso, B=spec.n_beams, R=spec.rows, C=spec.cols, w=spec.beamlet_mm,
                sigma=spec.sigma_mm, mu=spec.mu_per_mm, cutoff=spec.cutoff, profile=spec.profile,
                body_kind=spec.body.kind, body_center=spec.body.center[:2], body_size=spec.body.size[:2],
                jitter=spec.jitter, jitter_stream=(spec.seed * 0x100000001 + 0x5EED) & 0xFFFFFFFFFFFFFFFF)


def test_splitmix_matches_published_first_outputs():
    """SplitMix64 seeded with 0: the first outputs of the reference generator
    (next() = mix(state += gamma)) are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4."""
    u = PB.splitmix_uniform(0, np.arange(2))
    assert np.array_equal((u * 2 ** 53).astype(np.uint64),
                          np.array([0xE220A8397B1DCDAF >> 11, 0x6E789E6AA1B965F4 >> 11], np.uint64))
    assert np.array_equal(PB.splitmix_uniform(12345, np.arange(100)), P.uniform(12345, np.arange(100)))


def test_on_axis_voxel_is_pure_attenuation():
    """A voxel on the central axis of a beamlet at depth t: D = exp(-mu t) for
    the Gaussian profile; one sigma off axis in u: times exp(-1/2)."""
    xyz = np.array([[0.0, 20.0, 0.0], [3.0, 20.0, 0.0]])   # beam 0 points along -y from +y; body box 50 mm
    blk = PB.beam_coefficients(xyz, np.zeros(3), 0, 4, 2, 2, 5.0, 3.0, 0.01, "gauss", "box", (0.0, 0.0),
                               (50.0, 50.0))
    # beamlet (r=0, c=1) centre at u = +2.5, v = -2.5: voxel 0 at u = 0, v = 0
    t = 50.0 - 20.0
    d_u, d_v = -2.5, 2.5
    expect = math.exp(-0.01 * t) * math.exp(-d_v ** 2 / 18.0) * math.exp(-d_u ** 2 / 18.0)
    assert abs(blk[0, 1] - expect) <= 1e-15 * expect
    # voxel 1 at u = 3: one sigma from voxel 0's u-offset to beamlet c=1 is d_u = 0.5
    expect1 = math.exp(-0.01 * t) * math.exp(-d_v ** 2 / 18.0) * math.exp(-0.25 / 18.0)
    assert abs(blk[1, 1] - expect1) <= 1e-15 * expect1


def test_depth_through_an_elliptic_cylinder():
    """Entry parameter of a ray from the centre of a circle of radius 100: -100
    whatever the direction; from (60, 0) along -x (entering at x = 100): -40."""
    s = PB.entry_parameter("ecyl", (0.0, 0.0), (100.0, 100.0), np.array([0.0, 60.0]), np.array([0.0, 0.0]),
                           -1.0, 0.0)
    assert abs(s[0] + 100.0) <= 1e-12 and abs(s[1] + 40.0) <= 1e-12


def test_strip_profile_is_one_at_the_centre():
    assert abs(PB.lateral("strip", np.array(0.0), 3.0, 5.0) - 1.0) <= 1e-15
    a = PB.lateral("strip", np.array([-4.0, 4.0]), 3.0, 5.0)
    assert abs(a[0] - a[1]) <= 1e-15


@pytest.mark.parametrize("profile", ["gauss", "strip"])
@pytest.mark.parametrize("name", ["micro", "tiny"])
def test_matches_the_windowed_generator(name, profile):
    """Every voxel against every beamlet (here) and the generator's search window
    (phantom) give the same sparsity pattern and the same FP32 values."""
    from dataclasses import replace
    spec = replace(P.CONFIGS[name](), profile=profile)
    case = P.make_case(spec)
    D = PB.pencil_matrix(**_args(spec, case))
    assert D.nnz == case.nnz
    assert np.array_equal(D.indptr, case.indptr) and np.array_equal(D.indices, case.indices)
    assert np.array_equal(D.data.astype(np.float32), case.data)
