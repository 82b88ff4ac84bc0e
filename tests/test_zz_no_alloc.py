"""rsort_partition_noalloc, the allocation-free partition entry point.

Some callers cannot allocate device memory when they need to partition: code
running inside a strict-mode CUDA graph capture, frameworks whose device memory
must all come from their own allocator, real-time loops that forbid allocation
after start-up.  This entry point takes its scratch from a fixed static device
array inside librsort.  The test calls it through the C ABI twice in a row, on
different inputs, and checks each result bit for bit against rsort_partition
(the allocating entry point), and that the call makes no allocation through
torch's allocator.  This file sorts last so a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu


def test_noalloc_matches_partition_on_two_calls_in_a_row():
    from paper_1606_08766_gb300 import Context, RsortError, partition_noalloc
    cases = [("rand_dupl", 300_001, 1000, 3), ("uniform", (1 << 20) + 17, 64, 9)]
    with Context(0) as ctx:
        for name, n, k, seed in cases:
            keys = torch.from_numpy(instances.generate(name, n, p=64, seed=seed)
                                    .view(np.int64).copy()).cuda()
            ref_k, ref_p, ref_o = ctx.partition(keys, k, seed=seed)
            ko = torch.empty_like(keys)
            po = torch.empty(n, dtype=torch.int32, device="cuda")
            oo = torch.empty(k + 1, dtype=torch.int64, device="cuda")
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
            partition_noalloc(t, 1025, 1, torch.empty_like(t),
                              torch.empty(8, dtype=torch.int32, device="cuda"),
                              torch.empty(1026, dtype=torch.int64, device="cuda"))
