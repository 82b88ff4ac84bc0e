"""The binary-tree median approximation on the GPU (rsort_approx_median) and
the in-SM quicksort that takes its pivots from it (tunable medium_sort = 1).

rsort_approx_median must choose exactly the element the oracle chooses for
the same keys, window and seed (same tree, same coins).  The quicksort's
pivots are free, but its output is the unique sorted order, compared bit for
bit with the oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu

EINVAL = -1


@pytest.fixture(scope="module")
def ctx():
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(a.view(np.int64).copy()).cuda()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 64, 1000, 65537, 1 << 18])
@pytest.mark.parametrize("k", [2, 4, 16, 32])
def test_approx_median_matches_oracle(ctx, oracle_mod, n, k):
    rng = np.random.default_rng(n * 31 + k)
    x = rng.integers(0, 2**64, n, dtype=np.uint64)
    t = _dev(x)
    for seed in (1, 2, 3):
        want = oracle_mod.tree_median(x, k, seed)
        got = int(ctx.approx_median(t, k, seed).item())
        assert got == want, (n, k, seed)


@pytest.mark.parametrize("name", ["zero", "rand_dupl", "deter_dupl", "reverse", "g_group"])
def test_approx_median_duplicates_and_orders(ctx, oracle_mod, name):
    x = instances.generate(name, 30_001, p=64, seed=5)
    t = _dev(x)
    for seed in range(4):
        assert int(ctx.approx_median(t, 16, seed).item()) == oracle_mod.tree_median(x, 16, seed)


def test_approx_median_f64(ctx, oracle_mod):
    keys, _ = instances.segmented_f64(1, 15, seed=2)
    keys = keys[:20_000]
    t = torch.from_numpy(keys.view(np.float64).copy()).cuda()
    for seed in range(3):
        want = oracle_mod.tree_median(keys, 8, seed, key_type=oracle_mod.KEY_F64)
        assert int(ctx.approx_median(t, 8, seed).item()) == want


def test_approx_median_invalid(ctx):
    from paper_1606_08766_gb300.binding import _ptr
    t = _dev(np.arange(10, dtype=np.uint64))
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    lib = ctx._lib
    for n, k in ((10, 3), (10, 0), (10, 64), (0, 16)):
        assert lib.rsort_approx_median(ctx._ctx, 0, _ptr(t), n, k, 1, _ptr(out), None) == EINVAL


@pytest.fixture(scope="module")
def ctx_qs():
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    c.set_tunable("medium_sort", 1)
    assert c.get_tunable("medium_sort") == 1
    yield c
    c.close()


@pytest.mark.parametrize("name", ["uniform", "zero", "rand_dupl", "deter_dupl", "reverse",
                                  "mirrored", "all_to_one"])
def test_quicksort_medium_class_matches_oracle(ctx_qs, oracle_mod, name):
    # segments of 1025..4096 keys go straight to the medium in-SM class
    rng = np.random.default_rng(7)
    sizes = rng.integers(1025, 4097, 120)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    x = instances.generate(name, n, p=64, seed=3)
    ko, po = ctx_qs.segmented(_dev(x), torch.from_numpy(off.view(np.int64)).cuda())
    rk, rp = oracle_mod.segmented(x, off)
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)
    ctx_qs.check()


def test_quicksort_in_full_sorts(ctx_qs, oracle_mod):
    for name in ("uniform", "gaussian", "rand_dupl"):
        x = instances.generate(name, (1 << 18) + 77, p=16, seed=9)
        ko, po = ctx_qs.sort(_dev(x), p=16)
        rk, rp = oracle_mod.sort(x)
        np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
        np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)
