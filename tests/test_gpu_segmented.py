"""Batched segmented sort (one launch sequence for all segments) against the
oracle, against one plain rsort_sort per segment, under CUDA-graph replay,
and with invalid offsets (reported as a device error, never followed)."""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _mixed_u64_segments(seed=3):
    """Segments of several instances and sizes: empty, 1, tiny, medium, >4096,
    and one large enough for two sample-sort levels."""
    sizes = [0, 1, 2, 17, 64, 65, 300, 4096, 4097, 0, 9000, 70_000, 3, 1 << 18, 5]
    names = ["uniform", "zero", "rand_dupl", "reverse", "gaussian", "staggered", "deter_dupl"]
    parts = [instances.generate(names[i % len(names)], m, p=16, seed=seed + i)
             for i, m in enumerate(sizes)]
    keys = np.concatenate(parts).astype(np.uint64)
    offs = np.zeros(len(sizes) + 1, np.uint64)
    offs[1:] = np.cumsum(sizes)
    return keys, offs


def test_segmented_u64_matches_oracle(ctx, oracle_mod):
    keys, offs = _mixed_u64_segments()
    rk, rp = oracle_mod.segmented(keys, offs)
    ko, po = ctx.segmented(torch.from_numpy(keys.view(np.int64)).cuda(),
                           torch.from_numpy(offs.view(np.int64)).cuda())
    np.testing.assert_array_equal(_u32(po), rp)
    np.testing.assert_array_equal(_u64(ko), rk)
    ctx.check()


@pytest.mark.parametrize("nseg,maxlog", [(3000, 12), (500, 17)])
def test_segmented_f64_matches_oracle(ctx, oracle_mod, nseg, maxlog):
    keys, offs = instances.segmented_f64(nseg, maxlog, seed=nseg)
    rk, rp = oracle_mod.segmented(keys, offs, oracle_mod.KEY_F64)
    ko, po = ctx.segmented(torch.from_numpy(keys.view(np.float64).copy()).cuda(),
                           torch.from_numpy(offs.view(np.int64)).cuda())
    np.testing.assert_array_equal(_u32(po), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)


def test_segmented_equals_plain_per_segment(ctx):
    keys, offs = instances.segmented_f64(200, 15, seed=11)
    x = torch.from_numpy(keys.view(np.float64).copy()).cuda()
    ko, po = ctx.segmented(x, torch.from_numpy(offs.view(np.int64)).cuda())
    for s in range(0, 200, 7):
        a, b = int(offs[s]), int(offs[s + 1])
        k1, p1 = ctx.sort(x[a:b].contiguous(), p=1)
        assert torch.equal(k1, ko[a:b]) and torch.equal(p1, po[a:b])


def test_segmented_bad_offsets_reported(ctx):
    from paper_1606_08766_gb300 import RsortError
    keys = torch.from_numpy(instances.generate("uniform", 1000).view(np.int64)).cuda()
    offs = torch.tensor([0, 500, 400, 1000], dtype=torch.int64, device="cuda")  # decreasing
    ctx.segmented(keys, offs)
    with pytest.raises(RsortError) as ei:
        ctx.check()
    assert ei.value.status == -7
    offs = torch.tensor([0, 10, 2000], dtype=torch.int64, device="cuda")  # beyond n
    ctx.segmented(keys, offs)
    with pytest.raises(RsortError):
        ctx.check()
    ctx.check()  # the error was cleared by the read


def test_segmented_cuda_graph_replay(ctx, oracle_mod):
    keys, offs = instances.segmented_f64(400, 14, seed=21)
    x = torch.from_numpy(keys.view(np.float64).copy()).cuda()
    o = torch.from_numpy(offs.view(np.int64)).cuda()
    ko = torch.empty_like(x)
    po = torch.empty(x.numel(), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.segmented(x, o, keys_out=ko, perm_out=po)  # sizes the scratch outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.segmented(x, o, keys_out=ko, perm_out=po, stream=s)
    keys2, _ = instances.segmented_f64(400, 14, seed=22)
    keys2 = keys2[: keys.shape[0]] if keys2.shape[0] >= keys.shape[0] else np.resize(keys2, keys.shape[0])
    x.copy_(torch.from_numpy(keys2.view(np.float64).copy()))
    g.replay()
    torch.cuda.synchronize()
    rk, rp = oracle_mod.segmented(keys2, offs, oracle_mod.KEY_F64)
    np.testing.assert_array_equal(_u32(po), rp)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint64), rk)
    ctx.check()
