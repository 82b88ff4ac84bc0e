"""Host logic of the autotuner (no GPU): the synthetic segment batches, the
choice rule (fastest candidate, ties to the default) and the table format
that rsort_create reads ("name value" lines, '#' comments)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_segment_batch_shapes():
    from paper_1606_08766_gb300 import autotune
    keys, offs = autotune.segment_batch(2048, 4096, 1 << 16, seed=1, device="cpu")
    o = offs.numpy()
    sizes = np.diff(o)
    assert o[0] == 0 and o[-1] == keys.numel()
    assert sizes.min() > 2048 and sizes.max() <= 4096
    assert keys.dtype == torch.float64
    # about 10 % of the keys repeat another key of the same segment
    k = keys.numpy()
    dup = sum(len(k[a:b]) - len(np.unique(k[a:b])) for a, b in zip(o[:-1], o[1:]))
    assert 0.05 * k.size < dup < 0.15 * k.size


class _FakeCtx:
    def __init__(self, times):
        self.times = times
        self.cur = None
        self.set = []

    def set_tunable(self, name, v):
        self.cur = v
        self.set.append((name, v))


def test_choice_rule_fastest_beyond_noise(monkeypatch):
    from paper_1606_08766_gb300 import autotune
    times = {0: 2.0, 16: 1.5, 32: 1.5, 64: 1.7}
    monkeypatch.setattr(autotune, "_time_batches", lambda ctx, batches, reps: times[ctx.cur])
    ctx = _FakeCtx(times)
    # a tie between 16 and 32: the search stays where it stands (32)
    r = autotune._tune_knob(ctx, "rank_max", (0, 16, 32, 64), [], 1, 64, 32, "w")
    assert r.chosen == 32 and ctx.set[-1] == ("rank_max", 32)
    # 16 faster than 32, but within 1 %: stays at 32
    times[16] = 1.49
    r = autotune._tune_knob(ctx, "rank_max", (0, 16, 32, 64), [], 1, 64, 32, "w")
    assert r.chosen == 32
    # 16 more than 1 % faster: moves
    times[16] = 1.4
    r = autotune._tune_knob(ctx, "rank_max", (0, 16, 32, 64), [], 1, 64, 32, "w")
    assert r.chosen == 16 and ctx.set[-1] == ("rank_max", 16)
    # the current value not among the candidates: the fastest wins
    r = autotune._tune_knob(ctx, "rank_max", (0, 64), [], 1, 64, 32, "w")
    assert r.chosen == 64


def test_table_format(tmp_path):
    from paper_1606_08766_gb300 import autotune
    res = autotune.TuneResult(0, [autotune.KnobResult("target_bucket@18", "w", {1024: 2.0, 1536: 1.0},
                                                      1536, 0),
                                  autotune.KnobResult("sort_mid", "w", {0: 1.0, 2: 3.0}, 0, 0)])
    p = autotune.write_table(res, str(tmp_path / "t.tune"))
    lines = [ln.split() for ln in open(p) if not ln.startswith("#")]
    assert lines == [["target_bucket@18", "1536"], ["sort_mid", "0"]]
