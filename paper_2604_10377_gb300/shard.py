"""Sharding a batch of shape pairs over several GPUs (one process per GPU).

Every pair's functional map depends on its own two shapes only (Eq. 4 is solved
per pair), so the batch partitions into independent pairs: each rank runs the
whole path on its own pairs and no tensor of the data path crosses ranks. The
only cross-rank traffic is the timing reduction of a benchmark (the slowest rank
sets the step time) and the count of pairs all ranks processed.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def pair_cost(n_x: int, n_y: int, k: int, d: int, feat_bytes: int, k_y: int = None) -> float:
    """Estimated GPU time of one pair's forward+backward step, in microseconds:
    the bytes the projections stream (basis, mass and features of both shapes,
    read forward and backward, feature gradients written) at ~6.5 TB/s plus the
    row-wise solves (k_y systems of size k = k_x, O(k_y k^3 / 3) flops forward and
    adjoint) at ~6 TFLOP/s. k_y defaults to k (square maps). Only the ratio between
    pairs matters."""
    ky = k if k_y is None else k_y
    stream = n_x * (2 * 4 * k + 2 * 4 + 3 * feat_bytes * d) + n_y * (2 * 4 * ky + 2 * 4 + 3 * feat_bytes * d)
    solve = 2.0 * ky * k ** 3 / 3.0
    return stream / 6.5e6 + solve / 6.0e6


def partition_pairs(costs: Sequence[float], world: int) -> List[List[int]]:
    """Split pair indices over `world` ranks, balancing the summed cost.

    Longest-processing-time first: pairs in order of decreasing cost (ties by
    index) each go to the rank with the smallest load so far (ties to the lower
    rank). Deterministic, so every rank computes the same partition without
    communicating. Each rank's list is returned in increasing pair order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def job_throughput(units_local: float, ms_local: float, group=None) -> Tuple[float, float, float]:
    """Whole-job throughput of one timed step: (units of all ranks) / (slowest rank's
    time). Returns (units per second, max ms over ranks, total units). Uses the
    default process group when torch.distributed is initialised (any backend; the
    tensors live on the device that backend needs), else the local values."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return units_local / (ms_local / 1000.0), ms_local, units_local
    dev = torch.device("cpu")
    if dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    ms = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    units = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(units, op=dist.ReduceOp.SUM, group=group)
    ms_max, total = float(ms.item()), float(units.item())
    return total / (ms_max / 1000.0), ms_max, total
