"""Level 1's order decided on the device (tunable level1_stable = 2, the
default).

With many copies of a key, equality buckets (both bounding splitters hold one
key) make up a large share of level 1's buckets; kept in position order such
a bucket is final at once, so level 1 keeps input order.  On distinct keys it
ranks by shared-memory atomics.  Either way the result is the oracle's.  The
copy class of the in-SM stage (Stats.class_elems[0]) shows which way level 1
went: equality buckets in position order are copied, unordered ones sorted.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu

N = 1 << 22


@pytest.fixture(scope="module")
def ctx():
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


def _sort(ctx, keys, mode):
    ctx.set_tunable("level1_stable", mode)
    try:
        ko, po, st = ctx.sort(_dev(keys), p=1024, seed=4, stats=True)
        torch.cuda.synchronize()
        ctx.check()
    finally:
        ctx.set_tunable("level1_stable", 2)
    return ko.cpu().numpy().view(np.uint64), po.cpu().numpy().view(np.uint32), st


def test_default_is_device_decision(ctx):
    assert ctx.get_tunable("level1_stable") == 2


def test_tunable_range(ctx):
    for v in (0, 1, 2):
        ctx.set_tunable("level1_stable", v)
        assert ctx.get_tunable("level1_stable") == v
    with pytest.raises(RuntimeError):
        ctx.set_tunable("level1_stable", 3)
    ctx.set_tunable("level1_stable", 2)


@pytest.mark.parametrize("name", ["zero", "deter_dupl", "rand_dupl"])
def test_duplicates_keep_order_and_copy(ctx, oracle_mod, name):
    keys = instances.generate(name, N, p=1024, seed=3)
    rk, rp = oracle_mod.sort(keys)
    ko, po, st = _sort(ctx, keys, 2)
    np.testing.assert_array_equal(po, rp)
    np.testing.assert_array_equal(ko, rk)
    # most elements sit in equality buckets that leave level 1 in position
    # order and are copied
    assert st.class_elems[0] >= N // 2, st.class_elems
    # forced unordered: the same result, the equality buckets sorted instead
    ko0, po0, st0 = _sort(ctx, keys, 0)
    np.testing.assert_array_equal(po0, rp)
    np.testing.assert_array_equal(ko0, rk)
    assert st0.class_elems[0] < N // 16, st0.class_elems
    # forced stable: copied as in the automatic choice
    ko1, po1, st1 = _sort(ctx, keys, 1)
    np.testing.assert_array_equal(po1, rp)
    np.testing.assert_array_equal(ko1, rk)
    assert st1.class_elems[0] == st.class_elems[0]


@pytest.mark.parametrize("name", ["uniform", "gaussian", "staggered"])
def test_distinct_keys_rank_unordered(ctx, oracle_mod, name):
    keys = instances.generate(name, N, p=1024, seed=3)
    rk, rp = oracle_mod.sort(keys)
    ko, po, st = _sort(ctx, keys, 2)
    np.testing.assert_array_equal(po, rp)
    np.testing.assert_array_equal(ko, rk)
    assert st.class_elems[0] < N // 64, st.class_elems
