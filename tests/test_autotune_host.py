"""The autotuner's composed mode on the host: coordinate descent over the
patch-area buckets that hold sources, with the timing replaced by a known
cost function (no GPU)."""
import numpy as np

import fields
from paper_1803_00113_gb300 import autotune as AT


class _Dev:
    def __init__(self, problem):
        self.host = problem


def test_composed_mode_finds_the_coordinate_minimum(monkeypatch):
    p = fields.batched(seed=21, n_sources=40, min_side=15, max_side=101, max_images_per_band=1)
    used = sorted({AT.source_bucket(p, s) for s in range(p.n_sources)})
    assert len(used) >= 2
    best = {0: 512, 1: 128, 2: 1024, 3: 256}
    calls = []

    def fake(ctx, dprob, groups, tiles, reps):
        calls.append(tuple(tiles))
        # separable cost with its minimum at `best` in every used bucket;
        # unused buckets must stay 0
        assert all(tiles[b] == 0 for b in range(4) if b not in used)
        return sum(abs(np.log2(tiles[b]) - np.log2(best[b])) for b in used) + 1.0

    monkeypatch.setattr(AT, "_composed_ms", fake)
    groups = [np.arange(0, 20), np.arange(20, 40)]
    tiles, report = AT.autotune(None, _Dev(p), range(p.n_sources), groups=groups, reps=1)
    for b in range(4):
        assert tiles[b] == (best[b] if b in used else 0)
    # each distinct configuration is timed once
    assert len(calls) == len(set(calls)) == len(report["composed_ms"])
    assert len(calls) <= len(used) * len(AT.CANDIDATES)
