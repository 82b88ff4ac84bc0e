"""Serving runtime: continuous batching with admission by HBM budget.

Each request's result must be the same as sorting it alone (bit for bit,
against the oracle or a standalone rsort_sort), whatever it was batched with;
cancellation, the budget check and bounded waits are exercised on the host
side (no request is made to fail on the device).
"""
import threading

import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu

OK, PENDING, EINVAL, ENOMEM, ETIMEOUT, ECANCELLED = 0, 1, -1, -2, -4, -5


def _mixed_requests(count, seed, max_log2=21):
    rng = np.random.default_rng(seed)
    names = instances.NAMES
    reqs = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(16), np.log(2 ** max_log2))))
        name = names[i % len(names)]
        if i % 2:
            keys = instances.generate(name, n, p=16, seed=seed + i)
            t = torch.from_numpy(keys.view(np.int64).copy()).cuda()
            kt = 0
        else:
            x = instances.generate(name, n, p=16, seed=seed + i).astype(np.float64) - 2.0**63
            keys = x.view(np.uint64)
            t = torch.from_numpy(x.copy()).cuda()
            kt = 1
        reqs.append((keys, t, kt))
    return reqs


def test_served_results_equal_alone(oracle_mod):
    from paper_1606_08766_gb300 import Context
    reqs = _mixed_requests(120, seed=3)
    outs = [(torch.empty_like(t), torch.empty(t.numel(), dtype=torch.int32, device="cuda"))
            for _, t, _ in reqs]
    torch.cuda.synchronize()
    tickets = [None] * len(reqs)
    with Context(0) as ctx:
        def submit(lo, hi):
            for i in range(lo, hi):
                _, t, kt = reqs[i]
                tickets[i] = ctx.submit(t, outs[i][0], outs[i][1], p=0, seed=i, key_type=kt)
        th = [threading.Thread(target=submit, args=(0, 60)),
              threading.Thread(target=submit, args=(60, 120))]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for i, t in enumerate(tickets):
            assert ctx.wait(t, timeout_s=120) == OK, i
            st, lat = ctx.poll(t)
            assert st == OK and lat > 0
        stats = ctx.serve_stats()
        assert stats["completed"] == len(reqs) and stats["failed"] == 0
        assert stats["batches"] < len(reqs)  # small requests were batched together
        assert stats["p99_us"] >= stats["p50_us"] > 0
        for i, (keys, t, kt) in enumerate(reqs):
            ko, po = outs[i]
            if keys.shape[0] <= (1 << 17):
                rk, rp = oracle_mod.sort(keys, kt)
            else:  # larger requests: the same sort alone through rsort_sort
                k1, p1 = ctx.sort(t, p=1, key_type=kt)
                rk, rp = k1.cpu().numpy().view(np.uint64), p1.cpu().numpy().view(np.uint32)
            np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
            np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)


def test_cancel_before_start_leaves_buffers_untouched():
    from paper_1606_08766_gb300 import Context
    with Context(0) as ctx:
        big = torch.from_numpy(instances.generate("uniform", 1 << 24, seed=1).view(np.int64)).cuda()
        big_o = torch.empty_like(big)
        big_p = torch.empty(big.numel(), dtype=torch.int32, device="cuda")
        small = [torch.from_numpy(instances.generate("uniform", 5000, seed=s).view(np.int64)).cuda()
                 for s in range(40)]
        outs = [(torch.full_like(t, 7), torch.full((t.numel(),), 9, dtype=torch.int32,
                                                   device="cuda")) for t in small]
        torch.cuda.synchronize()
        tb = ctx.submit(big, big_o, big_p)
        ts = [ctx.submit(t, o, p) for t, (o, p) in zip(small, outs)]
        cancelled = [i for i, t in enumerate(ts) if i % 3 == 0 and ctx.cancel(t) == OK]
        assert ctx.wait(tb, timeout_s=120) == OK
        for i, t in enumerate(ts):
            st = ctx.wait(t, timeout_s=120)
            if i in cancelled:
                assert st == ECANCELLED
                assert bool((outs[i][0] == 7).all()) and bool((outs[i][1] == 9).all())
            else:
                assert st == OK
                k1, p1 = ctx.sort(small[i], p=1)
                assert torch.equal(k1, outs[i][0]) and torch.equal(p1, outs[i][1])
        assert ctx.cancel(tb) == EINVAL  # finished requests cannot be cancelled
        stats = ctx.serve_stats()
        assert stats["cancelled"] == len(cancelled)


def test_budget_admission_and_bounded_wait():
    from paper_1606_08766_gb300 import Context, RsortError
    with Context(0, hbm_budget_bytes=256 << 20) as ctx:
        huge = torch.zeros(1 << 26, dtype=torch.int64, device="cuda")
        with pytest.raises(RsortError) as ei:
            ctx.submit(huge, torch.empty_like(huge),
                       torch.empty(huge.numel(), dtype=torch.int32, device="cuda"))
        assert ei.value.status == ENOMEM
        keys = torch.from_numpy(instances.generate("gaussian", 1 << 21, seed=4)
                                .view(np.int64)).cuda()
        ko = torch.empty_like(keys)
        po = torch.empty(keys.numel(), dtype=torch.int32, device="cuda")
        t = ctx.submit(keys, ko, po)
        st = ctx.wait(t, timeout_s=1e-9)
        assert st in (ETIMEOUT, OK)
        assert ctx.wait(t, timeout_s=120) == OK
        k1, p1 = ctx.sort(keys, p=1)
        assert torch.equal(k1, ko) and torch.equal(p1, po)
        assert ctx.poll(123456789)[0] == EINVAL


def test_finished_records_are_bounded_by_serve_history():
    """Only the last serve_history finished requests keep their record: an
    older ticket reads as unknown, the newer ones keep status and latency,
    the latency percentiles cover the kept completions, and every result is
    still the sort of that request alone."""
    from paper_1606_08766_gb300 import Context, RsortError
    with Context(0) as ctx:
        assert ctx.get_tunable("serve_history") == 1 << 20
        ctx.set_tunable("serve_history", 4)
        keys = [torch.from_numpy(instances.generate("uniform", 3000 + 17 * s, seed=s)
                                 .view(np.int64)).cuda() for s in range(10)]
        outs = [(torch.empty_like(k), torch.empty(k.numel(), dtype=torch.int32, device="cuda"))
                for k in keys]
        torch.cuda.synchronize()
        tickets = []
        for k, (o, p) in zip(keys, outs):
            tickets.append(ctx.submit(k, o, p))
            assert ctx.wait(tickets[-1], timeout_s=120) == OK  # one finishes before the next
        for t in tickets[:6]:
            assert ctx.poll(t)[0] == EINVAL and ctx.wait(t, timeout_s=1) == EINVAL
        for t in tickets[6:]:
            st, lat = ctx.poll(t)
            assert st == OK and lat > 0
        stats = ctx.serve_stats()
        assert stats["completed"] == 10 and stats["failed"] == 0
        assert stats["p99_us"] >= stats["p50_us"] > 0
        # n = 0 finishes at submit and counts as a finished request too
        empty = torch.empty(0, dtype=torch.int64, device="cuda")
        t0 = ctx.submit(empty, torch.empty_like(empty),
                        torch.empty(0, dtype=torch.int32, device="cuda"))
        assert ctx.poll(t0)[0] == OK and ctx.poll(tickets[6])[0] == EINVAL
        with pytest.raises(RsortError):
            ctx.set_tunable("serve_history", 8)  # fixed once the runtime has started
        for k, (o, p) in zip(keys, outs):
            k1, p1 = ctx.sort(k, p=1)
            assert torch.equal(k1, o) and torch.equal(p1, p)
