"""Pins of the oracle's binary-tree median approximation (Section 3,
"Approximate Median Selection with a Single Reduction"; Appendix
"Experimental Comparison of Median Approximation Trees").

* A worked example, derived by hand for every coin combination (n = 2, k = 2).
* Comparison-only: a strictly increasing map of the keys chooses the same
  element, and equal keys are told apart by position.
* A truthful estimator: the mean signed rank error over many seeds is ~0.
* The paper's measured quality: over 2000 runs on uniform random 32-bit keys
  the largest rank error |r/(n-1) - 1/2| stays below 1.44 n^-0.39 (window
  k = 16; the paper does not state k, and 16 is the smallest power of two
  whose maximum meets the bound at every size tested here).
"""
import numpy as np
import pytest


def _coins(oracle_mod, seed, P):
    return [oracle_mod.splitmix64_at(seed, i) & 1 for i in range(P + 1)]


def test_worked_example_two_elements(oracle_mod):
    # keys [5, 3], k = 2.  A leaf forwards [-inf, x] (coin 0) or [x, +inf]
    # (coin 1); the root keeps entries 2..3 of the 4 merged entries and
    # returns its entry 1 (root coin 0) or 2 (root coin 1), moving to the
    # nearest element when that entry is undefined.
    #   leaves 0,0: merged [-inf,-inf,3,5] -> window [-inf,3] -> 3 either way
    #   leaves 0,1 or 1,0: merged [-inf,3,5,+inf] -> window [3,5] -> 3 or 5
    #   leaves 1,1: merged [3,5,+inf,+inf] -> window [5,+inf] -> 5 either way
    keys = np.array([5, 3], np.uint64)
    want = {(0, 0, 0): 1, (0, 0, 1): 1, (0, 1, 0): 1, (0, 1, 1): 0,
            (1, 0, 0): 1, (1, 0, 1): 0, (1, 1, 0): 0, (1, 1, 1): 0}
    seen = set()
    for seed in range(200):
        c = tuple(_coins(oracle_mod, seed, 2))
        assert oracle_mod.tree_median(keys, 2, seed) == want[c], (seed, c)
        seen.add(c)
    assert seen == set(want)


def test_single_element(oracle_mod):
    for k in (2, 8, 16):
        assert oracle_mod.tree_median(np.array([42], np.uint64), k, seed=9) == 0


@pytest.mark.parametrize("n", [7, 64, 1000])
def test_comparison_only(oracle_mod, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 2**40, n, dtype=np.uint64)
    y = x * np.uint64(3) + np.uint64(17)          # strictly increasing map
    for seed in range(20):
        assert oracle_mod.tree_median(x, 16, seed) == oracle_mod.tree_median(y, 16, seed)
    # all keys equal: the choice follows positions, which are distinct
    z = np.zeros(n, np.uint64)
    r = [oracle_mod.tree_median(z, 16, s) for s in range(20)]
    assert all(0 <= v < n for v in r)


def test_truthful_estimator(oracle_mod):
    n, runs = 1 << 10, 2000
    errs = []
    for run in range(runs):
        x = np.random.default_rng(run).integers(0, 2**32, n, dtype=np.uint64)
        r = oracle_mod.tree_median(x, 16, seed=run)
        rank = int((x < x[r]).sum())
        errs.append(rank / (n - 1) - 0.5)
    errs = np.array(errs)
    assert abs(errs.mean()) < 4 * errs.std() / np.sqrt(runs)


@pytest.mark.parametrize("log_n", [6, 8, 10, 12, 14])
def test_max_rank_error_within_paper_bound(oracle_mod, log_n):
    n, runs = 1 << log_n, 2000
    worst = 0.0
    for run in range(runs):
        x = np.random.default_rng(run * 7919 + log_n).integers(0, 2**32, n, dtype=np.uint64)
        r = oracle_mod.tree_median(x, 16, seed=run)
        rank = int((x < x[r]).sum())
        worst = max(worst, abs(rank / (n - 1) - 0.5))
    assert worst <= 1.44 * n ** -0.39, worst
