"""Pins of the oracle's partition-step variants (CPU only).

oracle.partition_ex adds two switches to the robust partition step:
  * tie_break=False -- the NTB ablation of Section 6 (classification by key
    only, so every copy of a key lands in one partition);
  * over=b > 1      -- AMS-sort overpartitioning: b*k fine partitions whose
    exact sizes are grouped into k outputs by an in-order greedy scan with the
    smallest bound that needs at most k groups.
Each pin checks it against something other than its own formula: the full
sort's ranks, numpy's searchsorted, brute force over every contiguous grouping,
closed forms, and the balance bound of the greedy scan.
"""
import itertools

import numpy as np
import pytest

import instances


def _ranks(oracle_mod, keys):
    _, perm = oracle_mod.sort(keys)
    rank = np.empty(keys.shape[0], np.int64)
    rank[perm.astype(np.int64)] = np.arange(keys.shape[0])
    return rank


def _fine_splitter_positions(oracle_mod, keys, k, over, seed):
    """Fine splitter j (j = 1..K-1) is sorted sample floor(j*S/K); the sample
    and its positions come from the pinned plain partition step."""
    plain = oracle_mod.partition(keys, k, seed)
    sp = plain["sample_pos"].astype(np.int64)
    S = sp.shape[0]
    K = k * over
    sorted_pos = sp[np.lexsort((sp, keys[sp]))]
    r = (np.arange(1, K, dtype=np.int64) * S) // K
    return sorted_pos[r]


def _check_layout(oracle_mod, keys, res, k):
    n = keys.shape[0]
    off = res["offsets"].astype(np.int64)
    assert off[0] == 0 and off[-1] == n and (np.diff(off) >= 0).all()
    pos = res["pos_out"].astype(np.int64)
    np.testing.assert_array_equal(np.sort(pos), np.arange(n))
    np.testing.assert_array_equal(res["keys_out"], keys[pos])
    rank = _ranks(oracle_mod, keys)
    prev_max = -1
    for g in range(k):
        seg = pos[off[g]:off[g + 1]]
        assert (np.diff(seg) > 0).all()          # increasing position inside an output
        if seg.shape[0]:
            assert rank[seg].min() > prev_max    # outputs are ordered
            prev_max = rank[seg].max()


@pytest.mark.parametrize("name", ["uniform", "zero", "rand_dupl", "staggered"])
def test_plain_switches_reproduce_the_partition_step(oracle_mod, name):
    keys = instances.generate(name, 20_000, p=32, seed=4)
    a = oracle_mod.partition(keys, 32, seed=9)
    b = oracle_mod.partition_ex(keys, 32, seed=9, tie_break=True, over=1)
    for f in ("keys_out", "pos_out", "offsets"):
        np.testing.assert_array_equal(a[f], b[f])


def test_ntb_equals_robust_step_on_distinct_keys(oracle_mod):
    # with distinct keys no element can tie with a splitter it is not, so the
    # position never decides
    keys = instances.generate("uniform", 30_000, p=16, seed=5)
    assert np.unique(keys).shape[0] == keys.shape[0]
    for over in (1, 3):
        a = oracle_mod.partition_ex(keys, 48, seed=2, tie_break=True, over=over)
        b = oracle_mod.partition_ex(keys, 48, seed=2, tie_break=False, over=over)
        for f in ("fine_sizes", "pos_out", "offsets"):
            np.testing.assert_array_equal(a[f], b[f])


def test_ntb_zero_input_collapses_into_the_first_partition(oracle_mod):
    # every splitter key is 0 and no key is smaller than 0
    n, k = 5000, 16
    res = oracle_mod.partition_ex(np.zeros(n, np.uint64), k, seed=1, tie_break=False)
    np.testing.assert_array_equal(res["offsets"], np.array([0] + [n] * k, np.uint64))


@pytest.mark.parametrize("name", ["deter_dupl", "rand_dupl", "gaussian"])
def test_ntb_partition_is_searchsorted_over_splitter_keys(oracle_mod, name):
    keys = instances.generate(name, 25_000, p=64, seed=6)
    k = 40
    plain = oracle_mod.partition(keys, k, seed=3)
    res = oracle_mod.partition_ex(keys, k, seed=3, tie_break=False)
    want = np.searchsorted(plain["spl_key"], keys, side="left")   # #{splitter keys < x}
    off = res["offsets"].astype(np.int64)
    pos = res["pos_out"].astype(np.int64)
    for b in range(k):
        np.testing.assert_array_equal(np.sort(pos[off[b]:off[b + 1]]), np.flatnonzero(want == b))
    _check_layout(oracle_mod, keys, res, k)


@pytest.mark.parametrize("tie_break", [True, False])
@pytest.mark.parametrize("name", ["uniform", "deter_dupl", "zero"])
def test_fine_sizes_match_full_sort_ranks(oracle_mod, name, tie_break):
    keys = instances.generate(name, 12_000, p=16, seed=7)
    k, over = 24, 4
    res = oracle_mod.partition_ex(keys, k, seed=5, tie_break=tie_break, over=over)
    fine = res["fine_sizes"].astype(np.int64)
    assert fine.sum() == keys.shape[0]
    fpos = _fine_splitter_positions(oracle_mod, keys, k, over, seed=5)
    cum = np.cumsum(fine)[:-1]
    if tie_break:
        # elements up to and including fine splitter j in (key, position) order
        np.testing.assert_array_equal(cum, _ranks(oracle_mod, keys)[fpos] + 1)
    else:
        # elements whose key is at most the splitter's key
        np.testing.assert_array_equal(cum, np.searchsorted(np.sort(keys), keys[fpos], "right"))


def _best_max_group(fine, k):
    """Brute force: smallest possible largest group over every way to cut the
    fine sequence into k contiguous (possibly empty) groups."""
    K = fine.shape[0]
    cum = np.concatenate([[0], np.cumsum(fine)])
    best = None
    for cuts in itertools.combinations_with_replacement(range(K + 1), k - 1):
        edges = (0,) + cuts + (K,)
        m = max(cum[edges[g + 1]] - cum[edges[g]] for g in range(k))
        best = m if best is None else min(best, m)
    return best


@pytest.mark.parametrize("seed", range(12))
def test_greedy_grouping_is_optimal_by_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 90))
    k = int(rng.integers(2, 5))
    over = int(rng.integers(2, 4))
    name = ["uniform", "rand_dupl", "zero", "deter_dupl"][seed % 4]
    keys = instances.generate(name, n, p=4, seed=seed)
    res = oracle_mod.partition_ex(keys, k, seed=seed, over=over)
    sizes = np.diff(res["offsets"].astype(np.int64))
    assert sizes.max() == _best_max_group(res["fine_sizes"].astype(np.int64), k)
    _check_layout(oracle_mod, keys, res, k)


@pytest.mark.parametrize("name", instances.NAMES)
def test_overpartitioning_bounds_the_imbalance(oracle_mod, name):
    # l = 1 level, eps = 0.2: b = 2 / ((1 + eps) - 1) = 10 (Appendix
    # "Implementation Details").  The greedy scan never needs a bound above
    # ceil(n/k) + the largest fine partition.
    n, k, over = 1 << 15, 32, 10
    keys = instances.generate(name, n, p=k, seed=3)
    res = oracle_mod.partition_ex(keys, k, seed=8, over=over)
    sizes = np.diff(res["offsets"].astype(np.int64))
    fine = res["fine_sizes"].astype(np.int64)
    first = res["group_first"].astype(np.int64)
    L = sizes.max()
    assert L <= -(-n // k) + fine.max()
    assert L / (n / k) <= 1.2, name
    # groups are the contiguous fine ranges [first[g], first[g+1])
    assert first[0] == 0 and first[k] == over * k and (np.diff(first) >= 0).all()
    cum = np.concatenate([[0], np.cumsum(fine)])
    np.testing.assert_array_equal(sizes, cum[first[1:]] - cum[first[:-1]])
    # greedy: a group is closed only when the next fine partition would not fit
    for g in range(k - 1):
        if first[g + 1] < over * k and sizes[g + 1] > 0:
            assert sizes[g] + fine[first[g + 1]] > L
    _check_layout(oracle_mod, keys, res, k)


def test_overpartitioning_with_ntb_keeps_keys_together(oracle_mod):
    keys = instances.generate("deter_dupl", 20_000, p=64, seed=2)
    res = oracle_mod.partition_ex(keys, 16, seed=4, tie_break=False, over=5)
    off = res["offsets"].astype(np.int64)
    ko = res["keys_out"]
    for g in range(15):
        if off[g + 1] > off[g] and off[g + 2] > off[g + 1]:
            assert ko[off[g + 1] - 1] < ko[off[g + 1]]   # no key spans two outputs
    _check_layout(oracle_mod, keys, res, 16)


@pytest.mark.parametrize("n,k,over", [(0, 4, 3), (1, 4, 3), (7, 8, 10), (100, 1, 5),
                                      (3000, 37, 2)])
def test_variant_edge_shapes(oracle_mod, n, k, over):
    keys = instances.generate("uniform", n, p=8, seed=3)
    res = oracle_mod.partition_ex(keys, k, seed=5, over=over)
    assert res["fine_sizes"].sum() == n
    _check_layout(oracle_mod, keys, res, k)


def test_single_output_has_no_sample_and_one_fine_partition(oracle_mod):
    # k = 1: the sample-size rule 16 * ceil(log2 k) * k draws no sample, so no
    # fine splitter exists and everything is in fine partition 0
    keys = instances.generate("uniform", 1000, p=4, seed=1)
    res = oracle_mod.partition_ex(keys, 1, seed=2, over=7)
    np.testing.assert_array_equal(res["fine_sizes"], np.array([1000, 0, 0, 0, 0, 0, 0], np.uint64))
    np.testing.assert_array_equal(res["group_first"], np.array([0, 7], np.uint32))
    np.testing.assert_array_equal(res["pos_out"], np.arange(1000, dtype=np.uint32))
