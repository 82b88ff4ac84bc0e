"""Properties of the seeded input instances (no GPU)."""
import numpy as np
import pytest

import instances

N, P = 1 << 16, 64
W = (2**64 - 1) // P


def _part(n, p):
    return (np.arange(n, dtype=np.uint64) * np.uint64(p)) // np.uint64(n)


def test_deterministic_and_seeded():
    a = instances.generate("uniform", 1000, seed=1)
    b = instances.generate("uniform", 1000, seed=1)
    c = instances.generate("uniform", 1000, seed=2)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()


def test_chunking_does_not_change_values(monkeypatch):
    a = instances.generate("gaussian", 5000, seed=3)
    monkeypatch.setattr(instances, "_CHUNK", 777)
    b = instances.generate("gaussian", 5000, seed=3)
    np.testing.assert_array_equal(a, b)


def test_slices():
    part = _part(N, P)
    bs = instances.generate("bucket_sorted", N, p=P)
    assert ((bs // np.uint64(W)) == part).all()
    at = instances.generate("all_to_one", N, p=P)
    assert ((at // np.uint64(W)) == 0).all()
    st = instances.generate("staggered", N, p=P)
    expect = np.where(part < P // 2, 2 * part + 1, 2 * (part - P // 2))
    assert ((st // np.uint64(W)) == expect).all()
    gg = instances.generate("g_group", N, p=P, g=8)
    sl = gg // np.uint64(W)
    # every partition of group G draws from the 8 slices (8G + 32 + t) mod 64
    for i in range(P):
        s = set(np.unique(sl[part == i]).tolist())
        g = i // 8
        assert s <= {(8 * g + 32 + t) % 64 for t in range(8)}


def test_reverse_strictly_descending():
    r = instances.generate("reverse", N)
    assert (np.diff(r.astype(object)) < 0).all()


def test_mirrored_and_dupl():
    m = instances.generate("mirrored", 1001)
    np.testing.assert_array_equal(m, m[::-1])
    rd = instances.generate("rand_dupl", N)
    assert rd.max() < 16
    dd = instances.generate("deter_dupl", N, p=P)
    assert set(np.unique(dd).tolist()) == set(range(7))
    assert (np.diff(dd.astype(np.int64)) >= 0).all()


def test_gaussian_moments():
    g = instances.generate("gaussian", 1 << 18).astype(np.float64)
    z = (g - 2.0**63) / 2.0**60
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_segmented_f64_shape():
    keys, offs = instances.segmented_f64(1000, 10, seed=2)
    sizes = np.diff(offs.astype(np.int64))
    assert sizes.min() >= 1 and sizes.max() <= 1024
    x = keys.view(np.float64)
    assert np.isfinite(x).all()
    # about 10% exact duplicates created inside segments
    assert 0.05 < 1 - np.unique(x).shape[0] / x.shape[0] < 0.15


@pytest.mark.parametrize("name", instances.NAMES)
def test_all_names_small_sizes(name):
    for n in (0, 1, 2, 3, 100):
        a = instances.generate(name, n, p=8)
        assert a.shape == (n,) and a.dtype == np.uint64


@pytest.mark.parametrize("name", instances.NAMES)
@pytest.mark.parametrize("n,p", [(1, 1024), (3, 2), (1000, 7), (65537, 1024), (40000, 1)])
def test_torch_generator_matches_numpy(name, n, p):
    """The torch generator (used on the GPU for full-size inputs) draws the
    same keys as the numpy one; the Gaussian instance may differ in the last
    bits of the rounding (at most a few units of 2^11, the spacing of float64
    values near 2^63)."""
    import torch  # noqa: F401
    a = instances.generate(name, n, p=p, seed=3)
    b = instances.generate_torch(name, n, p=p, seed=3).numpy().view(np.uint64)
    if name == "gaussian":
        assert np.abs(a.astype(np.float64) - b.astype(np.float64)).max() <= 4096
        assert np.count_nonzero(a != b) <= max(1, n // 1000)
    else:
        np.testing.assert_array_equal(a, b)


def test_torch_segmented_matches_numpy():
    """The device generator of the batched instance draws the same segment
    sizes and duplicate choices as the numpy one, and keys equal up to the
    last bits of log / sqrt / cos."""
    import torch  # noqa: F401
    for ns, ml, cap in [(700, 16, None), (50, 20, 1 << 21), (1, 3, None)]:
        a, oa = instances.segmented_f64(ns, ml, seed=3, total_cap=cap)
        b, ob = instances.segmented_f64_torch(ns, ml, seed=3, total_cap=cap)
        np.testing.assert_array_equal(oa.astype(np.int64), ob.numpy())
        av, bv = a.view(np.float64), b.numpy()
        assert np.abs(av - bv).max() <= 4e-15 * max(1.0, np.abs(av).max())
        # exact duplicates sit at the same positions
        np.testing.assert_array_equal(av[1:] == av[:-1], bv[1:] == bv[:-1])
