"""Buckets that are still larger than one SM's capacity (4096 keys) after the
last partition level: one CTA merge-sorts them through global memory.

With three levels the sampling makes such buckets vanishingly rare, so the
tunable max_levels (1..3) caps the recursion to force them: with one level
and p = 4, every bucket holds ~n/4 keys.  The result is still the unique
(key, position) order, compared bit for bit with the oracle, and the
statistics must show elements in the oversize class.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu

EINVAL = -1
BIG = 4  # size class of the oversize buckets in Stats.class_elems


def _ctx(levels: int, target: int = 0):
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    c.set_tunable("max_levels", levels)
    if target:
        c.set_tunable("target_bucket", target)
    return c


@pytest.fixture(scope="module")
def ctx1():
    c = _ctx(1)
    assert c.get_tunable("max_levels") == 1
    yield c
    c.close()


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def _eq(ko, po, rk, rp):
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)


@pytest.mark.parametrize("name", ["uniform", "zero", "rand_dupl", "deter_dupl", "reverse",
                                  "mirrored"])
def test_one_level_four_buckets(ctx1, oracle_mod, name):
    # ~65k keys per bucket: 17 runs of 4096 (the last one ragged), 5 merge rounds
    n = (1 << 18) + 333
    x = instances.generate(name, n, p=16, seed=2)
    ko, po, st = ctx1.sort(_dev(x), p=4, seed=5, stats=True)
    _eq(ko, po, *oracle_mod.sort(x))
    assert st.levels == 1
    assert st.class_elems[BIG] > 0
    assert sum(st.class_elems) == n
    ctx1.check()


def test_one_level_automatic_fanout(ctx1, oracle_mod):
    # 512 buckets of ~4096 keys: the ones just above 4096 take the oversize
    # path with one full run and one ragged run
    n = 1 << 21
    x = instances.generate("gaussian", n, p=16, seed=3)
    ko, po, st = ctx1.sort(_dev(x), p=1, seed=1, stats=True)
    _eq(ko, po, *oracle_mod.sort(x))
    assert st.class_elems[BIG] > 0
    assert sum(st.class_elems) == n


def test_one_level_f64(ctx1, oracle_mod):
    keys, _ = instances.segmented_f64(64, 14, seed=7)
    x = keys.view(np.float64).copy()
    assert x.shape[0] > 100_000
    x[:6] = [-0.0, 0.0, np.inf, -np.inf, -1e-310, 1e-310]
    ko, po, st = ctx1.sort(torch.from_numpy(x).cuda(), p=2, seed=1, stats=True)
    rk, rp = oracle_mod.sort(x, oracle_mod.KEY_F64)
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert st.class_elems[BIG] > 0


def test_one_level_in_place(ctx1, oracle_mod):
    # output aliasing the input: the oversize merge uses the output range of
    # its bucket as scratch only after the level has consumed the input
    x = instances.generate("uniform", 100_000, seed=9)
    rk, rp = oracle_mod.sort(x)
    t = _dev(x)
    ko, po = ctx1.sort(t, p=3, keys_out=t)
    assert ko.data_ptr() == t.data_ptr()
    _eq(ko, po, rk, rp)


def test_one_level_segmented(oracle_mod):
    # segments of 5k..70k keys, fan-out aimed at 4096-key buckets: many
    # buckets land just above 4096
    c = _ctx(1, target=4096)
    try:
        rng = np.random.default_rng(4)
        sizes = rng.integers(5000, 70_000, 40)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
        x = instances.generate("rand_dupl", int(off[-1]), p=64, seed=4)
        ko, po = c.segmented(_dev(x), torch.from_numpy(off.view(np.int64)).cuda())
        _eq(ko, po, *oracle_mod.segmented(x, off))
        c.check()
    finally:
        c.close()


def test_two_levels(oracle_mod):
    # level 1 splits 2^22 keys in two, level 2 into <= 512 buckets of ~4096
    c = _ctx(2)
    try:
        n = 1 << 22
        x = instances.generate("staggered", n, p=64, seed=6)
        ko, po, st = c.sort(_dev(x), p=2, seed=2, stats=True)
        _eq(ko, po, *oracle_mod.sort(x))
        assert st.levels == 2
        assert sum(st.class_elems) == n
    finally:
        c.close()


def test_max_levels_invalid():
    from paper_1606_08766_gb300 import Context
    from paper_1606_08766_gb300.binding import RsortError
    with Context(0) as c:
        assert c.get_tunable("max_levels") == 3
        for v in (0, 4, -1):
            with pytest.raises(RsortError) as e:
                c.set_tunable("max_levels", v)
            assert e.value.status == EINVAL
        assert c.get_tunable("max_levels") == 3
        assert c.get_tunable("deep_levels_stable") == 0
        for v in (2, -1):
            with pytest.raises(RsortError) as e:
                c.set_tunable("deep_levels_stable", v)
            assert e.value.status == EINVAL


@pytest.mark.parametrize("stable", [0, 1])
@pytest.mark.parametrize("name", ["zero", "deter_dupl", "rand_dupl", "uniform"])
def test_third_level_after_unordered_level(oracle_mod, name, stable):
    # 4096-key targets leave many level-2 buckets above 4096 keys, so a third
    # level partitions them.  With deep_levels_stable = 0 the level-2 scatter
    # ranks by atomics: level 3 then samples segments that are not in
    # position order (all-equal ones included), and equality buckets are
    # sorted by position instead of copied.
    c = _ctx(3, target=4096)
    try:
        c.set_tunable("deep_levels_stable", stable)
        n = (1 << 22) + 19
        x = instances.generate(name, n, p=64, seed=8)
        ko, po, st = c.sort(_dev(x), p=64, seed=4, stats=True)
        _eq(ko, po, *oracle_mod.sort(x))
        assert sum(st.class_elems) == n
        if name != "zero":
            assert st.levels == 3
        c.check()
    finally:
        c.close()
