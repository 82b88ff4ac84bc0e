"""Pins for the CPU oracle (no GPU).

Each test ties an oracle function to something other than itself: brute force
on tiny inputs, a library routine that computes a special case of the same
definition, closed forms of the input instances, published known-answer values,
or invariants that the paper's partition step must satisfy.  A plausible slip
anywhere in the oracle (a flipped comparison, a dropped tie-break, an
off-by-one splitter, a wrong stratum) fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import instances

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute_force_perm(keys_rank):
    """The unique permutation with (key[pi[j]], pi[j]) strictly increasing."""
    n = len(keys_rank)
    found = []
    for pi in itertools.permutations(range(n)):
        seq = [(keys_rank[i], i) for i in pi]
        if all(seq[j] < seq[j + 1] for j in range(n - 1)):
            found.append(pi)
    assert len(found) == 1
    return np.array(found[0], dtype=np.uint32)


@pytest.mark.parametrize("n", range(0, 7))
def test_sort_brute_force_all_ternary_inputs(oracle_mod, n):
    # Section 2: output sorted; ties broken by the unique position identifier.
    for vec in itertools.product(range(3), repeat=n):
        keys = np.array(vec, dtype=np.uint64)
        ko, po = oracle_mod.sort(keys)
        expect = _brute_force_perm(vec)
        np.testing.assert_array_equal(po, expect)
        np.testing.assert_array_equal(ko, keys[expect])


def _golden_f64():
    rows = []
    with open(os.path.join(GOLDEN, "f64_order.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(int(line.split()[0], 16))
    return np.array(rows, dtype=np.uint64)


def test_f64_order_matches_ieee_golden_list(oracle_mod):
    order = _golden_f64()
    rng = np.random.default_rng(7)
    for _ in range(20):
        shuffled = order[rng.permutation(order.shape[0])]
        ko, po = oracle_mod.sort(shuffled, oracle_mod.KEY_F64)
        np.testing.assert_array_equal(ko, order)


@pytest.mark.parametrize("n", range(0, 6))
def test_f64_brute_force_small(oracle_mod, n):
    # keys drawn from {-1.0, -0.0, +0.0, 1.0}; their hand-written ranks give the order
    vals = np.array([-1.0, -0.0, 0.0, 1.0])
    for vec in itertools.product(range(4), repeat=n):
        keys = vals[list(vec)] if n else np.empty(0)
        ko, po = oracle_mod.sort(keys.astype(np.float64), oracle_mod.KEY_F64)
        expect = _brute_force_perm(vec)
        np.testing.assert_array_equal(po, expect)


@pytest.mark.parametrize("n,universe", [(1000, 2**64), (50_000, 2**64), (50_000, 7),
                                        (1 << 18, 2**20), (3, 2)])
def test_sort_matches_numpy_stable_argsort(oracle_mod, n, universe):
    rng = np.random.default_rng(n + universe % 1000)
    keys = rng.integers(0, universe, size=n, dtype=np.uint64, endpoint=False) \
        if universe < 2**64 else rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64)
    ko, po = oracle_mod.sort(keys)
    expect = np.argsort(keys, kind="stable").astype(np.uint32)
    np.testing.assert_array_equal(po, expect)
    np.testing.assert_array_equal(ko, keys[expect])


def test_f64_matches_numpy_for_finite_values_without_negative_zero(oracle_mod):
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_000)
    x[::7] = x[rng.integers(0, x.shape[0], x[::7].shape[0])]  # exact duplicates
    x[x == 0.0] = 1.0
    ko, po = oracle_mod.sort(x, oracle_mod.KEY_F64)
    expect = np.argsort(x, kind="stable").astype(np.uint32)
    np.testing.assert_array_equal(po, expect)
    np.testing.assert_array_equal(ko.view(np.float64), x[expect])


def test_sort_matches_counting_sort_small_universe(oracle_mod):
    keys = instances.generate("rand_dupl", 200_000, p=64, seed=5)
    ko, po = oracle_mod.sort(keys)
    # stable counting sort over the 16-value universe
    counts = np.bincount(keys.astype(np.int64), minlength=16)
    start = np.concatenate([[0], np.cumsum(counts)[:-1]])
    expect = np.empty(keys.shape[0], np.uint32)
    for v in range(16):
        pos = np.nonzero(keys == v)[0]
        expect[start[v]:start[v] + pos.shape[0]] = pos
    np.testing.assert_array_equal(po, expect)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 65_537])
def test_closed_forms(oracle_mod, n):
    ident = np.arange(n, dtype=np.uint32)
    _, po = oracle_mod.sort(instances.generate("zero", n, p=64))
    np.testing.assert_array_equal(po, ident)
    _, po = oracle_mod.sort(instances.generate("deter_dupl", n, p=64))
    np.testing.assert_array_equal(po, ident)
    _, po = oracle_mod.sort(instances.generate("reverse", n, p=64))
    np.testing.assert_array_equal(po, ident[::-1])
    if n >= 64:
        _, po = oracle_mod.sort(instances.generate("bucket_sorted", n, p=64))
        part = (ident.astype(np.uint64) * 64) // n
        np.testing.assert_array_equal((po.astype(np.uint64) * 64) // n, part)


@pytest.mark.parametrize("n", [2, 10, 4096, 10_001])
def test_mirrored_closed_form(oracle_mod, n):
    keys = instances.generate("mirrored", n, p=64, seed=9)
    half = n // 2
    assert np.unique(keys[: n - half]).shape[0] == n - half  # first half unique
    ko, po = oracle_mod.sort(keys)
    if n % 2 == 0:
        a, b = po[0::2].astype(np.int64), po[1::2].astype(np.int64)
        np.testing.assert_array_equal(ko[0::2], ko[1::2])
        np.testing.assert_array_equal(a + b, np.full(half, n - 1))
        assert (a < half).all()


def test_segmented_is_per_segment_sort(oracle_mod):
    keys, offs = instances.segmented_f64(200, 12, seed=4)
    ko, po = oracle_mod.segmented(keys, offs, oracle_mod.KEY_F64)
    x = keys.view(np.float64)
    for s in range(offs.shape[0] - 1):
        a, b = int(offs[s]), int(offs[s + 1])
        seg = x[a:b].copy()
        neg0 = np.signbit(seg) & (seg == 0.0)
        assert not neg0.any()
        expect = np.argsort(seg, kind="stable").astype(np.uint32)
        np.testing.assert_array_equal(po[a:b], expect)
        np.testing.assert_array_equal(ko[a:b], keys[a:b][expect])


# --------------------------------------------------------------------------
# splitmix64 and the partition step
# --------------------------------------------------------------------------

def test_splitmix64_known_answers(oracle_mod):
    with open(os.path.join(GOLDEN, "splitmix64_kat.txt")) as fh:
        rows = [line.split() for line in fh if line.strip() and not line.startswith("#")]
    assert len(rows) == 5
    for s, c, out in rows:
        assert oracle_mod.splitmix64_at(int(s), int(c)) == int(out)
        assert instances.splitmix64_scalar(int(s), int(c)) == int(out)


def _lex_less(ka, pa, kb, pb):
    return (ka < kb) | ((ka == kb) & (pa < pb))


def _check_partition(oracle_mod, keys, k, seed, key_type=0):
    n = keys.shape[0]
    res = oracle_mod.partition(keys, k, seed, key_type)
    S = res["sample_pos"].shape[0]
    # stratified sampling: sample j lies in stratum j, all distinct
    if S:
        j = np.arange(S, dtype=np.uint64)
        assert (res["sample_pos"] >= (j * np.uint64(n)) // np.uint64(S)).all()
        assert (res["sample_pos"] < ((j + np.uint64(1)) * np.uint64(n)) // np.uint64(S)).all()
    bits = keys.view(np.uint64)
    mapped = bits if key_type == 0 else np.where(bits >> np.uint64(63) == 1, ~bits,
                                                 bits | np.uint64(1 << 63))
    # splitters are every S/k-th element of the lexicographically sorted sample
    if S and k > 1:
        sp = res["sample_pos"]
        order = np.lexsort((sp, mapped[sp]))
        sorted_pos = sp[order]
        r = (np.arange(1, k, dtype=np.uint64) * np.uint64(S)) // np.uint64(k)
        np.testing.assert_array_equal(res["spl_pos"], sorted_pos[r].astype(np.uint32))
        np.testing.assert_array_equal(res["spl_key"], mapped[sorted_pos[r]])
    off = res["offsets"].astype(np.int64)
    assert off[0] == 0 and off[-1] == n and (np.diff(off) >= 0).all()
    # cumulative size up to bucket b equals the full-sort rank of splitter b, plus 1
    _, perm = oracle_mod.sort(keys, key_type)
    rank = np.empty(n, np.int64)
    rank[perm.astype(np.int64)] = np.arange(n)
    if S and k > 1:
        np.testing.assert_array_equal(off[1:k], rank[res["spl_pos"].astype(np.int64)] + 1)
    # every bucket holds (lo-splitter, hi-splitter] in increasing position
    pos = res["pos_out"].astype(np.int64)
    np.testing.assert_array_equal(np.sort(pos), np.arange(n))
    np.testing.assert_array_equal(res["keys_out"], bits[pos])
    for b in range(k):
        seg = pos[off[b]:off[b + 1]]
        assert (np.diff(seg) > 0).all()
        if seg.shape[0] == 0:
            continue
        np.testing.assert_array_equal(res["bucket"][seg], np.full(seg.shape[0], b))
        if b > 0:
            assert _lex_less(res["spl_key"][b - 1], res["spl_pos"][b - 1],
                             mapped[seg], seg).all()
        if b < k - 1:
            assert (~_lex_less(res["spl_key"][b], res["spl_pos"][b], mapped[seg], seg)).all()
    return res


@pytest.mark.parametrize("name", ["uniform", "zero", "deter_dupl", "rand_dupl", "staggered",
                                  "gaussian", "all_to_one", "mirrored"])
def test_partition_invariants(oracle_mod, name):
    keys = instances.generate(name, 40_000, p=64, seed=2)
    _check_partition(oracle_mod, keys, 64, seed=11)


@pytest.mark.parametrize("n,k", [(0, 4), (1, 4), (5, 8), (100, 1), (100, 2), (3000, 37),
                                 (17, 64)])
def test_partition_edge_shapes(oracle_mod, n, k):
    keys = instances.generate("uniform", n, p=8, seed=3)
    _check_partition(oracle_mod, keys, k, seed=5)


def test_partition_f64(oracle_mod):
    keys, _ = instances.segmented_f64(1, 14, seed=8)
    _check_partition(oracle_mod, keys.view(np.float64), 32, seed=3, key_type=1)


def test_partition_zero_boundaries_by_hand(oracle_mod):
    # all keys equal: bucket b is exactly the positions (spl_pos[b-1], spl_pos[b]]
    n, k = 10_000, 16
    res = oracle_mod.partition(np.zeros(n, np.uint64), k, seed=99)
    np.testing.assert_array_equal(res["offsets"][1:k], res["spl_pos"].astype(np.uint64) + 1)


def test_partition_balance_is_robust_to_duplicates(oracle_mod):
    # Appendix "Robust Multi-Level Sample Sort": tie-broken partitioning splits
    # duplicate-heavy input as evenly as input with unique keys.
    n, k = 1 << 16, 64
    def imbalance(name):
        res = oracle_mod.partition(instances.generate(name, n, p=k, seed=1), k, seed=1)
        sizes = np.diff(res["offsets"].astype(np.int64))
        return sizes.max() / (n / k)
    uni = imbalance("uniform")
    assert uni < 1.5
    for name in ("zero", "deter_dupl", "rand_dupl"):
        assert imbalance(name) <= 1.1 * uni, name


@pytest.mark.parametrize("threads", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("n", range(0, 6))
def test_parallel_sort_brute_force_ternary(oracle_mod, n, threads):
    # the all-core timing oracle meets the same brute-force pin as the serial
    # one, for thread counts below, at and above n
    for vec in itertools.product(range(3), repeat=n):
        keys = np.array(vec, dtype=np.uint64)
        ko, po = oracle_mod.sort_parallel(keys, threads=threads)
        expect = _brute_force_perm(vec)
        np.testing.assert_array_equal(po, expect)
        np.testing.assert_array_equal(ko, keys[expect])


@pytest.mark.parametrize("threads", [2, 3, 7, 16])
@pytest.mark.parametrize("n,universe", [(100_003, 2**64), (100_003, 5), (1, 2)])
def test_parallel_sort_matches_numpy_stable_argsort(oracle_mod, n, universe, threads):
    rng = np.random.default_rng(n + threads)
    keys = rng.integers(0, universe, size=n, dtype=np.uint64) if universe < 2**64 \
        else rng.integers(0, 2**64 - 1, size=n, dtype=np.uint64)
    ko, po = oracle_mod.sort_parallel(keys, threads=threads)
    expect = np.argsort(keys, kind="stable").astype(np.uint32)
    np.testing.assert_array_equal(po, expect)
    np.testing.assert_array_equal(ko, keys[expect])


def test_parallel_sort_f64(oracle_mod):
    order = _golden_f64()
    rng = np.random.default_rng(11)
    shuffled = np.tile(order, 50)[rng.permutation(order.shape[0] * 50)]
    ko, po = oracle_mod.sort_parallel(shuffled, oracle_mod.KEY_F64, threads=6)
    np.testing.assert_array_equal(ko, np.repeat(order, 50))
    # ties keep position order
    assert all(po[j] < po[j + 1] for j in range(po.shape[0] - 1) if ko[j] == ko[j + 1])
