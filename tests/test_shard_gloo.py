"""Multi-rank path on CPU: two `gloo` ranks shard a batch of pairs.

Pairs are independent (Eq. 4 is solved per pair), so sharding needs no exchange
of data: the ranks agree on the partition without communicating, the union of
their shards is the batch, each rank's results equal the whole batch's results
for its pairs, and the benchmark's job throughput is (units of all ranks) /
(slowest rank's time)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2604_10377_gb300 import shard, synth  # noqa: E402

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    return synth.make_small(77, 6, (60, 400), [5, 8, 12], 32, feat_dtype="bf16")


def _costs(wl):
    fb = 2 if wl.feat_dtype == "bf16" else 4
    return [shard.pair_cost(wl.shapes[p.x].n, wl.shapes[p.y].n, wl.shapes[p.x].k, wl.shapes[p.x].d, fb)
            for p in wl.pairs]


def _sub_workload(wl, idx):
    shapes, pairs = [], []
    for i in idx:
        p = wl.pairs[i]
        shapes += [wl.shapes[p.x], wl.shapes[p.y]]
        pairs.append(synth.Pair(x=len(shapes) - 2, y=len(shapes) - 1, lam=p.lam, mask=p.mask, c_gt=p.c_gt))
    return synth.Workload(name=wl.name, shapes=shapes, pairs=pairs, feat_dtype=wl.feat_dtype)


def _rank_main(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from oracle import fmap_oracle as orc
        from tests._bridge import oracle_inputs

        wl = _workload()
        parts = shard.partition_pairs(_costs(wl), WORLD)
        mine = parts[rank]
        # forward + backward of this rank's pairs only
        sub = _sub_workload(wl, mine)
        shapes, pairs = oracle_inputs(sub)
        fwd = orc.forward_batch(shapes, pairs)
        d_c = [np.ones_like(c) for c in fwd["C"]]
        bwd = orc.backward_batch(shapes, pairs, fwd, d_c)
        res = {i: (fwd["C"][j], bwd["dF"][2 * j], bwd["dF"][2 * j + 1]) for j, i in enumerate(mine)}
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, {"parts": parts, "res": res})
        # slowest rank sets the step time: rank r takes 10 (r + 1) ms
        value, ms_max, total = shard.job_throughput(float(len(mine)), 10.0 * (rank + 1))
        torch.save({"gathered": gathered, "tp": (value, ms_max, total)}, os.path.join(out_dir, f"r{rank}.pt"))
    finally:
        dist.destroy_process_group()


def test_partition_is_balanced_and_complete():
    costs = [5.0, 1.0, 4.0, 4.0, 2.0, 3.0, 3.0]
    parts = shard.partition_pairs(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    # LPT bound: max load <= 4/3 OPT; here the optimum 22/3 -> 8 is reachable
    assert max(loads) <= 8.0
    assert shard.partition_pairs(costs, 1) == [list(range(len(costs)))]
    assert shard.partition_pairs([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard.partition_pairs(costs, 0)


def test_job_throughput_single_process():
    v, ms, tot = shard.job_throughput(256.0, 16.0)
    assert (ms, tot) == (16.0, 256.0) and abs(v - 16000.0) < 1e-9


def test_two_gloo_ranks_shard_without_exchange(tmp_path):
    from oracle import fmap_oracle as orc
    from tests._bridge import oracle_inputs

    port = _free_port()
    mp.start_processes(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True, start_method="spawn")
    outs = [torch.load(os.path.join(tmp_path, f"r{r}.pt"), weights_only=False) for r in range(WORLD)]

    wl = _workload()
    gathered = outs[0]["gathered"]
    # both ranks derived the same partition, and it covers the batch exactly once
    assert gathered[0]["parts"] == gathered[1]["parts"]
    parts = gathered[0]["parts"]
    assert sorted(parts[0] + parts[1]) == list(range(len(wl.pairs)))
    assert parts[0] and parts[1]

    # per-rank results equal the whole-batch results (no cross-pair coupling)
    shapes, pairs = oracle_inputs(wl)
    fwd = orc.forward_batch(shapes, pairs)
    bwd = orc.backward_batch(shapes, pairs, fwd, [np.ones_like(c) for c in fwd["C"]])
    merged = {}
    for g in gathered:
        merged.update(g["res"])
    assert sorted(merged) == list(range(len(wl.pairs)))
    for i, p in enumerate(wl.pairs):
        c, dfx, dfy = merged[i]
        np.testing.assert_array_equal(c, fwd["C"][i])
        # every shape belongs to exactly one pair in this batch
        np.testing.assert_array_equal(dfx, bwd["dF"][p.x])
        np.testing.assert_array_equal(dfy, bwd["dF"][p.y])

    # job throughput: all ranks' pairs over the slowest rank's time, same on every rank
    for o in outs:
        value, ms_max, total = o["tp"]
        assert ms_max == 20.0 and total == float(len(wl.pairs))
        assert abs(value - len(wl.pairs) / 0.020) < 1e-9


def test_pair_cost_rectangular():
    """k_y systems of size k_x: the solve term scales with k_y k_x^3 and each shape streams
    its own basis; the square case is unchanged."""
    from paper_2604_10377_gb300 import shard
    sq = shard.pair_cost(1000, 2000, 50, 128, 2)
    assert shard.pair_cost(1000, 2000, 50, 128, 2, k_y=50) == sq
    assert shard.pair_cost(1000, 2000, 50, 128, 2, k_y=100) > sq
    # solve term only (no vertices): ratio k_y / k_x
    assert abs(shard.pair_cost(0, 0, 40, 16, 2, k_y=80) / shard.pair_cost(0, 0, 40, 16, 2) - 2.0) < 1e-12
