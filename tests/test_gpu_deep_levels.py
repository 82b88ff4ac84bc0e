"""Levels after the first rank by shared-memory atomics (tunable
deep_levels_stable = 0, the default): buckets of level 2 come out in no
particular order, equality buckets there are sorted instead of copied, and
the in-SM sort restores the unique (key, position) order.  Float64 keys and
segmented inputs with heavy duplicates through two levels, bit-exact against
the oracle, in both settings of the tunable.
"""
import numpy as np
import pytest
import torch

import instances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1])
def ctx_deep(request):
    from paper_1606_08766_gb300 import Context
    c = Context(0)
    c.set_tunable("deep_levels_stable", request.param)
    yield c
    c.close()


def _u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def test_f64_two_levels_with_duplicates(ctx_deep, oracle_mod):
    # 16 level-1 buckets of ~135k keys each: level 2 partitions them
    keys, _ = instances.segmented_f64(200, 17, seed=11)
    x = keys.view(np.float64).copy()
    n = x.shape[0]
    assert n > 1_000_000
    rng = np.random.default_rng(3)
    x[rng.integers(0, n, n // 4)] = -0.0        # a quarter of the keys tie
    x[rng.integers(0, n, n // 8)] = np.inf
    ko, po, st = ctx_deep.sort(torch.from_numpy(x).cuda(), p=16, seed=2, stats=True)
    rk, rp = oracle_mod.sort(x, oracle_mod.KEY_F64)
    assert st.levels >= 2
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(_u64(ko), rk)
    ctx_deep.check()


def test_segmented_two_levels_with_duplicates(ctx_deep, oracle_mod):
    # segments of up to ~1.3M keys (level 2 needed), mostly zeros
    sizes = [1_300_000, 5_000, 900_000, 1, 0, 2_100_000]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    n = int(off[-1])
    x = instances.generate("zero", n, p=16, seed=1)
    rng = np.random.default_rng(5)
    x[rng.integers(0, n, n // 10)] = rng.integers(0, 7, n // 10, dtype=np.uint64)
    ko, po = ctx_deep.segmented(torch.from_numpy(x.view(np.int64)).cuda(),
                                torch.from_numpy(off.view(np.int64)).cuda())
    rk, rp = oracle_mod.segmented(x, off)
    np.testing.assert_array_equal(po.cpu().numpy().view(np.uint32), rp)
    np.testing.assert_array_equal(_u64(ko), rk)
    ctx_deep.check()
