"""Parity of rsort_partition_ex (NTB ablation, AMS overpartitioning) with the
oracle, bit for bit: output keys, positions, offsets, fine partition sizes
and group boundaries.  Larger cases are checked through the properties that
the greedy grouping guarantees at any size.
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


def _compare(got, ref, k, over):
    ko, po, off, fine, first = got
    torch.cuda.synchronize()
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), ref["offsets"])
    np.testing.assert_array_equal(fine.cpu().numpy().astype(np.uint64), ref["fine_sizes"])
    np.testing.assert_array_equal(first.cpu().numpy().astype(np.uint32), ref["group_first"])
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), ref["pos_out"])
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), ref["keys_out"])


NTB_CASES = [("uniform", 64), ("zero", 64), ("deter_dupl", 64), ("rand_dupl", 100),
             ("gaussian", 37), ("all_to_one", 16)]


@pytest.mark.parametrize("name,k", NTB_CASES)
def test_ntb_matches_oracle(ctx, oracle_mod, name, k):
    n = (1 << 17) + 1237
    keys = instances.generate(name, n, p=64, seed=7)
    ref = oracle_mod.partition_ex(keys, k, seed=5, tie_break=False)
    _compare(ctx.partition_ex(_dev(keys), k, seed=5, tie_break=False), ref, k, 1)
    ctx.check()


OVER_CASES = [("uniform", 64, 10, True), ("uniform", 37, 3, True), ("zero", 64, 10, True),
              ("deter_dupl", 32, 4, True), ("deter_dupl", 32, 4, False),
              ("rand_dupl", 100, 2, True), ("rand_dupl", 50, 5, False),
              ("staggered", 128, 8, True), ("all_to_one", 16, 10, True),
              ("gaussian", 200, 10, False), ("bucket_sorted", 1000, 10, True)]


@pytest.mark.parametrize("name,k,over,tb", OVER_CASES)
def test_overpartition_matches_oracle(ctx, oracle_mod, name, k, over, tb):
    n = (1 << 17) + 4099
    keys = instances.generate(name, n, p=64, seed=11)
    ref = oracle_mod.partition_ex(keys, k, seed=3, tie_break=tb, over=over)
    _compare(ctx.partition_ex(_dev(keys), k, seed=3, tie_break=tb, overpartition=over), ref, k,
             over)
    ctx.check()


@pytest.mark.parametrize("k,over", [(1024, 10), (2048, 5), (1, 7), (3, 3413)])
def test_overpartition_largest_fan_outs(ctx, oracle_mod, k, over):
    n = (1 << 16) + 17
    keys = instances.generate("uniform", n, p=8, seed=2)
    ref = oracle_mod.partition_ex(keys, k, seed=1, over=over)
    _compare(ctx.partition_ex(_dev(keys), k, seed=1, overpartition=over), ref, k, over)


def test_overpartition_f64(ctx, oracle_mod):
    keys, _ = instances.segmented_f64(1, 17, seed=5)
    keys = keys[:90_000]
    ref = oracle_mod.partition_ex(keys, 40, seed=4, key_type=oracle_mod.KEY_F64, over=4)
    t = torch.from_numpy(keys.view(np.float64).copy()).cuda()
    ko, po, off, fine, first = ctx.partition_ex(t, 40, seed=4, overpartition=4)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), ref["offsets"])
    np.testing.assert_array_equal(fine.cpu().numpy().astype(np.uint64), ref["fine_sizes"])
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), ref["pos_out"])
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), ref["keys_out"])


@pytest.mark.parametrize("n", [0, 1, 5, 4096])
@pytest.mark.parametrize("over", [1, 3])
def test_variants_small_and_empty(ctx, oracle_mod, n, over):
    keys = instances.generate("rand_dupl", n, seed=1)
    for tb in (True, False):
        ref = oracle_mod.partition_ex(keys, 8, seed=2, tie_break=tb, over=over)
        ko, po, off, fine, first = ctx.partition_ex(_dev(keys), 8, seed=2, tie_break=tb,
                                                    overpartition=over)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(off.cpu().numpy().astype(np.uint64), ref["offsets"])
        np.testing.assert_array_equal(fine.cpu().numpy().astype(np.uint64), ref["fine_sizes"])
        np.testing.assert_array_equal(first.cpu().numpy().astype(np.uint32), ref["group_first"])
        if n:
            np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), ref["pos_out"])


def test_variants_with_tree_classifier(oracle_mod):
    from paper_1606_08766_gb300 import Context
    keys = instances.generate("rand_dupl", (1 << 16) + 5, p=64, seed=9)
    with Context(0) as c:
        c.set_tunable("classifier", 0)
        for tb, over in ((False, 1), (True, 6), (False, 6)):
            ref = oracle_mod.partition_ex(keys, 64, seed=8, tie_break=tb, over=over)
            _compare(c.partition_ex(_dev(keys), 64, seed=8, tie_break=tb, overpartition=over),
                     ref, 64, over)


def test_invalid_variant_arguments(ctx):
    from paper_1606_08766_gb300.binding import _PartOpts, _ptr
    keys = _dev(instances.generate("uniform", 1000, seed=1))
    ko = torch.empty_like(keys)
    po = torch.empty(1000, dtype=torch.int32, device="cuda")
    off = torch.empty(2049, dtype=torch.int64, device="cuda")
    lib = ctx._lib
    for tb, over, k in ((2, 1, 8), (1, 0, 8), (1, 11, 1024), (0, 6, 2048)):
        opts = _PartOpts(tb, over)
        rc = lib.rsort_partition_ex(ctx._ctx, 0, _ptr(keys), 1000, k, 1, ctypes.byref(opts),
                                    _ptr(ko), _ptr(po), _ptr(off), None, None, None)
        assert rc == EINVAL, (tb, over, k)
    # NULL options: the plain robust step
    rc = lib.rsort_partition_ex(ctx._ctx, 0, _ptr(keys), 1000, 8, 1, None, _ptr(ko), _ptr(po),
                                _ptr(off), None, None, None)
    assert rc == 0
    k2, p2, o2 = ctx.partition(keys, 8, seed=1)
    assert torch.equal(ko, k2) and torch.equal(po, p2) and torch.equal(off[:9], o2)


@pytest.mark.parametrize("name", ["uniform", "zero", "rand_dupl", "deter_dupl"])
def test_overpartition_bound_at_2p24(ctx, name):
    # the launch configuration of a large step: k = 1024 outputs from 10240
    # fine partitions (eps = 0.2 with one level)
    n, k, over = 1 << 24, 1024, 10
    keys = instances.generate(name, n, p=k, seed=4)
    ko, po, off, fine, first = ctx.partition_ex(_dev(keys), k, seed=6, overpartition=over)
    torch.cuda.synchronize()
    off = off.cpu().numpy().astype(np.int64)
    fine = fine.cpu().numpy().astype(np.int64)
    first = first.cpu().numpy().astype(np.int64)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == n and fine.sum() == n
    cum = np.concatenate([[0], np.cumsum(fine)])
    np.testing.assert_array_equal(sizes, cum[first[1:]] - cum[first[:-1]])
    L = sizes.max()
    assert L <= -(-n // k) + fine.max()
    assert L / (n / k) <= 1.2, name
    for g in range(k - 1):   # greedy: a group closes only when the next would not fit
        if first[g + 1] < over * k and sizes[g + 1] > 0:
            assert sizes[g] + fine[first[g + 1]] > L
    # layout: a permutation, keys_out = keys[pos], increasing positions per output,
    # outputs ordered by (key, position)
    pos = po.cpu().numpy().view(np.uint32).astype(np.int64)
    kb = keys.view(np.uint64)
    assert np.bincount(pos, minlength=n).max() == 1
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), kb[pos])
    d = np.diff(pos)
    inner = np.ones(n - 1, bool)
    inner[off[1:-1][(off[1:-1] > 0) & (off[1:-1] < n)] - 1] = False
    assert (d[inner] > 0).all()
    for g in range(1, k):
        a, b = off[g] - 1, off[g]
        if 0 <= a and b < n and off[g] > 0:
            assert (kb[pos[a]], pos[a]) < (kb[pos[b]], pos[b])
