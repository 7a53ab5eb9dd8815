"""Autotuner search and cache logic on the CPU: a stand-in batch whose step time is a
known function of the knobs replaces the GPU timing."""
import json
import types

import pytest

pytest.importorskip("torch")

from paper_2604_10377_gb300 import _lib, autotune  # noqa: E402


class FakeBatch:
    def __init__(self):
        self.layout = types.SimpleNamespace(ns=[100, 200], ks=[30, 30], ds=[64, 64], feat_dtype="bf16")
        self.pairs = [(0, 1, 1e-3)]
        self.dfeat = object()
        self.device = "cpu"
        self._t = {f: 0 for f in _lib.TUNING_FIELDS}
        self.retunes = 0

    @property
    def tuning(self):
        return dict(self._t)

    def retune(self, t):
        self._t = {f: int(t.get(f, 0)) for f in _lib.TUNING_FIELDS}
        self.retunes += 1


def fake_time(batch):
    # fastest at bwd_chunk_v = 4096 and proj_max_stages = 4; solve knobs make no difference
    t = batch.tuning
    ms = 10.0
    ms -= {0: 0.0, 2048: 0.5, 4096: 1.0, 16384: 0.2}[t["bwd_chunk_v"]]
    ms -= {0: 0.0, 4: 0.6, 3: 0.1}[t["proj_max_stages"]]
    ms -= 0.01 if t["solve_threads_k64"] == 128 else 0.0     # below the 1% threshold
    return ms


def test_coordinate_descent_and_cache(tmp_path, monkeypatch):
    b = FakeBatch()
    monkeypatch.setattr(autotune, "time_step", lambda step, dev, iters=3, reps=3: fake_time(b))
    cache = str(tmp_path / "tune.json")
    res = autotune.autotune(b, lambda: None, cache_path=cache)
    assert not res["cached"]
    assert res["tuning"]["bwd_chunk_v"] == 4096 and res["tuning"]["proj_max_stages"] == 4
    assert res["tuning"]["solve_threads_k64"] == 0          # 0.1% gain: kept the built-in choice
    assert b.tuning == res["tuning"]                         # the batch is left re-planned
    assert res["baseline_ms"] == 10.0 and abs(res["ms"] - 8.4) < 1e-9
    n_trials = sum(len([v for v in vals if v != 0]) for vals in autotune.CANDIDATES.values())
    assert len(res["trials"]) == 1 + n_trials
    for knob in autotune.CANDIDATES:
        assert res["tuning"][knob] in autotune.CANDIDATES[knob]
    assert res["tuning"]["proj_ctas"] == 0 and res["tuning"]["bwd_ctas"] == 0   # not searched here
    with open(cache) as fh:
        assert autotune.batch_signature(b) in json.load(fh)

    # a second batch of the same signature takes the cached choice without timing anything
    b2 = FakeBatch()
    monkeypatch.setattr(autotune, "time_step", lambda *a, **k: pytest.fail("timed a cached batch"))
    res2 = autotune.autotune(b2, lambda: None, cache_path=cache)
    assert res2["cached"] and b2.tuning == res["tuning"]


def test_signature_depends_on_the_batch_shape():
    a, b = FakeBatch(), FakeBatch()
    assert autotune.batch_signature(a) == autotune.batch_signature(b)
    b.layout.ks = [50, 50]
    assert autotune.batch_signature(a) != autotune.batch_signature(b)
