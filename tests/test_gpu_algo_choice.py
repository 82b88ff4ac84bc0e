"""Which in-SM algorithm finishes a bucket (the size-dependent choice of
Section 6 and Appendix "Bitonic Sort", applied per bucket): the counters in
rsort_stats.algo_elems show that every branch runs on inputs built to reach
it, and the result stays bit-exact with the oracle each time.

Inputs:
* tiny buckets (at most 64 keys): rank-by-counting;
* distinct keys: equal-width bins;
* a few distinct keys far apart (every bin that holds keys is crowded):
  bitonic, both through the direct path and after two partition levels;
* all keys equal, in position order: nothing to do;
* the opt-in quicksort and the oversize merge sort.
Copy-through buckets are not sorted, so the counters add up to the elements
outside class 0.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu

RANK, BINS, BITONIC, QUICK, MERGE, IN_ORDER = range(6)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64).copy()).cuda()


def _sort_and_check(ctx, oracle_mod, keys, p):
    rk, rp = oracle_mod.sort(keys)
    ko, po, st = ctx.sort(_dev(keys), p=p, seed=3, stats=True)
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert sum(st.algo_elems) + st.class_elems[0] == keys.shape[0]
    ctx.check()
    return st


@pytest.fixture(scope="module")
def ctx():
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _few_far_values(n, nvals, seed):
    """Keys drawn from nvals values spread over the whole u64 range, so that
    every bin of a bucket that holds keys holds many copies."""
    rng = np.random.default_rng(seed)
    vals = np.sort(rng.integers(0, 2**64 - 1, nvals, dtype=np.uint64))
    return vals[rng.integers(0, nvals, n)]


def test_rank_by_counting_tiny(ctx, oracle_mod):
    keys = instances.generate("uniform", 50, p=1, seed=1)
    st = _sort_and_check(ctx, oracle_mod, keys, 1)
    assert st.algo_elems[RANK] == 50


def test_bins_on_distinct_keys(ctx, oracle_mod):
    keys = instances.generate("uniform", 3000, p=1, seed=2)
    st = _sort_and_check(ctx, oracle_mod, keys, 1)
    assert st.algo_elems[BINS] == 3000


def test_bitonic_on_clustered_bucket(ctx, oracle_mod):
    keys = _few_far_values(3001, 3, seed=4)
    st = _sort_and_check(ctx, oracle_mod, keys, 1)
    assert st.algo_elems[BITONIC] == 3001


@pytest.mark.parametrize("p", [64, 1024])
def test_bitonic_after_partition_levels(ctx, oracle_mod, p):
    # 32 distinct keys over 2^20 + 5 positions: the buckets that straddle two
    # keys hold two far-apart keys, each many times
    keys = _few_far_values((1 << 20) + 5, 32, seed=p)
    st = _sort_and_check(ctx, oracle_mod, keys, p)
    # p = 64 leaves 16K-key buckets for a second level; p = 1024 leaves
    # buckets that one CTA sorts
    assert st.levels == (2 if p == 64 else 1)
    assert st.algo_elems[BITONIC] > 0


def test_in_order_equal_keys(ctx, oracle_mod):
    keys = np.full(2500, 77, dtype=np.uint64)
    st = _sort_and_check(ctx, oracle_mod, keys, 1)
    assert st.algo_elems[IN_ORDER] == 2500


def test_quicksort_when_selected(oracle_mod):
    from paper_1606_08766_gb300 import Context
    with Context(0) as c:
        c.set_tunable("medium_sort", 1)
        keys = instances.generate("gaussian", 3500, p=1, seed=5)
        st = _sort_and_check(c, oracle_mod, keys, 1)
        assert st.algo_elems[QUICK] == 3500


def test_merge_for_oversize_buckets(oracle_mod):
    from paper_1606_08766_gb300 import Context
    with Context(0) as c:
        c.set_tunable("max_levels", 1)
        keys = instances.generate("uniform", 40_000, p=2, seed=6)
        st = _sort_and_check(c, oracle_mod, keys, 2)
        assert st.algo_elems[MERGE] > 0
