"""Autotuner of the tiling knobs of a batch.

The library plans every launch (projection work items and pipeline depth, backward-
projection feature groups and vertex chunks, row-solve block sizes) from a handful of
knobs in `fmap_options` (0 = its built-in choice). Which values are fastest depends on the
batch: vertex counts, spectral sizes, feature width. `autotune` times the caller's own step
(for instance project + solve + loss + backward) on the real batch for the candidate values
of one knob at a time, keeps the fastest, and moves on (coordinate descent from the
built-in choice). Re-planning only rebuilds the library's work lists: inputs, outputs and
results stay in place, and every candidate computes the same outputs up to the order of
partial sums.

Results can be cached in a JSON file keyed by a signature of the batch (sizes, spectral
sizes, feature widths, precision), so that the search runs once per batch shape.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from typing import Callable, Dict, Iterable, Optional

import torch

# Candidate values per knob (0 = the library's built-in choice), in search order.
CANDIDATES: Dict[str, tuple] = {
    "bwd_group_features": (0, 64),
    "bwd_chunk_v": (0, 2048, 4096, 16384),
    "proj_max_stages": (0, 4, 3),
    "proj_seg_max_v": (0, 4096, 16384),
    "solve_threads_k64": (0, 128),
    "solve_threads_k128": (0, 256),
    "solve_no_g_copy": (0, 1),
    "adjoint_kernel": (0, 1, 2),
    "adjoint_features": (0, 64, 128, 256),
    "adjoint_stages": (0, 1, 2),
}


def batch_signature(batch) -> str:
    lay = batch.layout
    key = json.dumps({"n": lay.ns, "k": lay.ks, "d": lay.ds, "feat": lay.feat_dtype,
                      "pairs": [(x, y) for (x, y, _) in batch.pairs], "grad": batch.dfeat is not None})
    return hashlib.sha256(key.encode()).hexdigest()[:24]


def time_step(step: Callable[[], None], device, iters: int = 3, reps: int = 3) -> float:
    """Median over `reps` of the mean CUDA-event time (ms) of `iters` calls, after one
    untimed call."""
    step()
    torch.cuda.synchronize(device)
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            step()
        e1.record()
        torch.cuda.synchronize(device)
        out.append(e0.elapsed_time(e1) / iters)
    out.sort()
    return out[len(out) // 2]


def autotune(batch, step: Callable[[], None], knobs: Optional[Iterable[str]] = None, iters: int = 3,
             reps: int = 3, min_gain: float = 0.01, cache_path: Optional[str] = None) -> dict:
    """Tune `batch` (an api.FmapBatch) for `step`; leaves the batch re-planned with the best
    knobs found and returns {"tuning", "ms", "baseline_ms", "trials", "seconds", "cached"}.
    A candidate replaces the current best only when it is at least `min_gain` faster."""
    t0 = time.time()
    sig = batch_signature(batch)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
    if sig in cache:
        batch.retune(cache[sig]["tuning"])
        return {"tuning": batch.tuning, "ms": cache[sig]["ms"], "baseline_ms": cache[sig]["baseline_ms"],
                "trials": [], "seconds": time.time() - t0, "cached": True}

    dev = batch.device
    best = batch.tuning
    best_ms = time_step(step, dev, iters, reps)
    baseline_ms = best_ms
    trials = [{"tuning": dict(best), "ms": best_ms}]
    for knob in (knobs or CANDIDATES.keys()):
        for val in CANDIDATES[knob]:
            if val == best[knob]:
                continue
            cand = dict(best, **{knob: val})
            batch.retune(cand)
            ms = time_step(step, dev, iters, reps)
            trials.append({"tuning": dict(cand), "ms": ms})
            if ms < best_ms * (1.0 - min_gain):
                best, best_ms = cand, ms
        batch.retune(best)
    if cache_path:
        cache[sig] = {"tuning": best, "ms": best_ms, "baseline_ms": baseline_ms}
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return {"tuning": best, "ms": best_ms, "baseline_ms": baseline_ms, "trials": trials,
            "seconds": time.time() - t0, "cached": False}
