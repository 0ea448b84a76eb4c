"""Host-side checks of the seeded input generator (no method arithmetic lives there)."""
import numpy as np

import phantom as P


def test_splitmix64_published_vector():
    """SplitMix64 (Steele, Lea & Flood 2014) from seed 1234567: the reference
    implementation's first five outputs."""
    seed = np.uint64(1234567)
    with np.errstate(over="ignore"):
        states = seed + np.arange(1, 6, dtype=np.uint64) * P.GAMMA
    out = [int(v) for v in P.splitmix64(states)]
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_is_counter_based():
    a = P.uniform(42, np.arange(100))
    b = P.uniform(42, np.arange(100)[::-1])[::-1]
    assert np.array_equal(a, b)
    assert np.all((a >= 0) & (a < 1))


def test_micro_case_structure():
    c = P.make_case(P.spec_micro())
    V, N = c.n_voxels, c.n_beamlets
    assert c.indptr[0] == 0 and np.all(np.diff(c.indptr) >= 0)
    assert c.indices.dtype == np.int32 and c.data.dtype == np.float32
    for j in range(0, V, 97):
        seg = c.indices[c.indptr[j]:c.indptr[j + 1]]
        assert np.all(np.diff(seg) > 0)
    assert c.indices.min() >= 0 and c.indices.max() < N
    assert np.all(c.data > 0)
    # priority resolution gives one label per voxel; every structure is present
    assert set(np.unique(c.voxel_struct)) == set(range(len(c.names)))


def test_case_is_deterministic():
    a = P.make_case(P.spec_micro(seed=5))
    b = P.make_case(P.spec_micro(seed=5))
    assert np.array_equal(a.indptr, b.indptr) and np.array_equal(a.data, b.data)
    c = P.make_case(P.spec_micro(seed=6))
    assert not (a.data.shape == c.data.shape and np.array_equal(a.data, c.data))


def test_tiny_shapes():
    c = P.make_case(P.spec_tiny())
    assert c.n_voxels == 40 * 40 * 12 and c.n_beamlets == 500 and c.n_beams == 5
    assert 300_000 < c.nnz < 2_000_000


def test_downsampling_counts():
    spec = P.spec_micro(grid=(24, 24, 10), downsample=True)
    c = P.make_case(spec)
    full = P.make_case(P.spec_micro(grid=(24, 24, 10), downsample=False))
    # structure voxels are kept at full resolution, unspecified tissue is 8x coarser
    for k, nm in enumerate(c.names[:-1]):
        assert np.sum(c.voxel_struct == k) == np.sum(full.voxel_struct == k)
    assert c.n_voxels < full.n_voxels


def test_perturb_changes_anatomy():
    s = P.spec_micro()
    p = P.perturb(s, 4001)
    assert p.structures[0].shape.center != s.structures[0].shape.center
    assert p.seed == 4001


def test_random_csr_ragged():
    ip, ix, d = P.random_csr(3, 500, 300, 12.0)
    L = np.diff(ip)
    assert L.min() == 0 and L.max() > 60
    for r in range(0, 500, 37):
        seg = ix[ip[r]:ip[r + 1]]
        assert np.all(np.diff(seg) > 0) and (seg.size == 0 or seg.max() < 300)
