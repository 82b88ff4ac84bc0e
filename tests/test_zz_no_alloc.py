"""rsort_partition_noalloc, the allocation-free partition entry point.

Some callers cannot allocate device memory when they need to partition:
frameworks whose device memory must all come from their own allocator, and
real-time loops that forbid allocation after start-up.  This entry point takes
its scratch from a fixed static device array inside librsort.

The tests call it through the C ABI:
* twice in a row, on different inputs, each result bit for bit against
  rsort_partition (the allocating entry point), with no allocation through
  torch's allocator during the call;
* against the CPU oracle's partition step directly, at k = 1, 64 and 1024
  (the documented limit), for float64 keys and for n = 0;
* with outputs of the wrong dtype, size or device, which the binding refuses
  on the host before any kernel runs.
This file sorts last so a stop-at-first-failure run has already run every
other test.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu


def _outputs(n, k, dtype=torch.int64):
    return (torch.empty(n, dtype=dtype, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(k + 1, dtype=torch.int64, device="cuda"))


def test_noalloc_matches_partition_on_two_calls_in_a_row():
    from paper_1606_08766_gb300 import Context, RsortError, partition_noalloc
    cases = [("rand_dupl", 300_001, 1000, 3), ("uniform", (1 << 20) + 17, 64, 9)]
    with Context(0) as ctx:
        for name, n, k, seed in cases:
            keys = torch.from_numpy(instances.generate(name, n, p=64, seed=seed)
                                    .view(np.int64).copy()).cuda()
            ref_k, ref_p, ref_o = ctx.partition(keys, k, seed=seed)
            ko, po, oo = _outputs(n, k)
            torch.cuda.synchronize()
            # torch's count of allocations ever made (frees by garbage
            # collection do not change it)
            before = torch.cuda.memory_stats()["allocation.all.allocated"]
            partition_noalloc(keys, k, seed, ko, po, oo)
            torch.cuda.synchronize()
            assert torch.cuda.memory_stats()["allocation.all.allocated"] == before
            assert torch.equal(oo, ref_o)
            assert torch.equal(po, ref_p)
            assert torch.equal(ko, ref_k)
        t = torch.zeros(8, dtype=torch.int64, device="cuda")
        with pytest.raises(RsortError):
            partition_noalloc(t, 1025, 1, *_outputs(8, 1025))


@pytest.mark.parametrize("name,n,k", [("uniform", 200_003, 1), ("zero", 150_001, 64),
                                      ("deter_dupl", 262_147, 1024),
                                      ("rand_dupl", (1 << 19) + 9, 1024)])
def test_noalloc_matches_oracle(oracle_mod, name, n, k):
    from paper_1606_08766_gb300 import partition_noalloc
    keys = instances.generate(name, n, p=64, seed=11)
    ref = oracle_mod.partition(keys, k, seed=4)
    ko, po, oo = _outputs(n, k)
    partition_noalloc(torch.from_numpy(keys.view(np.int64).copy()).cuda(), k, 4, ko, po, oo)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oo.cpu().numpy().astype(np.uint64), ref["offsets"])
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), ref["pos_out"])
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), ref["keys_out"])


def test_noalloc_f64_matches_oracle(oracle_mod):
    from paper_1606_08766_gb300 import partition_noalloc
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100_003)
    x[::7] = x[5]                      # exact duplicates
    x[:4] = [0.0, -0.0, np.inf, -np.inf]
    bits = x.view(np.uint64)
    ref = oracle_mod.partition(bits, 100, seed=2, key_type=oracle_mod.KEY_F64)
    ko, po, oo = _outputs(x.shape[0], 100, torch.float64)
    partition_noalloc(torch.from_numpy(x.copy()).cuda(), 100, 2, ko, po, oo)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oo.cpu().numpy().astype(np.uint64), ref["offsets"])
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), ref["pos_out"])
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), ref["keys_out"])


def test_noalloc_empty_input():
    from paper_1606_08766_gb300 import partition_noalloc
    keys = torch.empty(0, dtype=torch.int64, device="cuda")
    ko, po, oo = _outputs(0, 16)
    oo.fill_(-1)
    partition_noalloc(keys, 16, 1, ko, po, oo)
    torch.cuda.synchronize()
    assert bool((oo == 0).all())


def test_noalloc_refuses_bad_outputs_on_the_host():
    from paper_1606_08766_gb300 import partition_noalloc
    keys = torch.zeros(64, dtype=torch.int64, device="cuda")
    ko, po, oo = _outputs(64, 8)
    bad = [
        (ko, po, oo.to(torch.int32)),                       # offsets too narrow
        (ko, po.to(torch.int64), oo),                       # positions too wide
        (ko.to(torch.float64), po, oo),                     # keys_out of another dtype
        (ko, po, torch.empty(8, dtype=torch.int64, device="cuda")),   # k + 1 entries missing
        (torch.empty(128, dtype=torch.int64, device="cuda")[::2], po, oo),  # not contiguous
        (ko.cpu(), po, oo),                                 # not on the device
    ]
    for a, b, c in bad:
        with pytest.raises(ValueError):
            partition_noalloc(keys, 8, 1, a, b, c)
