"""Host-side helpers of bench.py on the CPU: the DRAM-traffic profile is reported only
for the kernel sources it was captured on, and the algorithmic work per step follows the
sizes of the batch."""
import hashlib
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2604_10377_gb300", "csrc")


def _sha(src):
    h = hashlib.sha256()
    for f in (src, "fmap_internal.cuh", "tc_ptx.cuh"):
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()


def test_traffic_is_reported_only_for_matching_sources(tmp_path, monkeypatch):
    prof = tmp_path / "traffic.txt"
    prof.write_text("# header\n"
                    f"solve k_chol.cu {_sha('k_chol.cu')} 1234\n"
                    f"project k_project_tc.cu {'0' * 64} 999\n"
                    "not a data line\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILES", {7: str(prof)})
    got = bench.load_traffic(7)
    assert got == {"solve": 1234}          # the stale SHA gives no number
    assert bench.load_traffic(5) == {}     # no profile for that workload


def test_committed_traffic_profile_parses():
    rel = bench.TRAFFIC_FILES[4]
    lines = [l.split() for l in open(os.path.join(ROOT, rel)) if l.strip() and not l.startswith("#")]
    assert lines and all(len(p) == 4 and len(p[2]) == 64 and int(p[3]) > 0 for p in lines)
    assert {p[0] for p in lines} >= {"project", "project_bwd", "solve", "adj_solve"}


def _wl(shapes, pairs, feat="bf16"):
    return types.SimpleNamespace(shapes=[types.SimpleNamespace(n=n, k=k, d=d) for (n, k, d) in shapes],
                                 pairs=[types.SimpleNamespace(x=x, y=y) for (x, y) in pairs], feat_dtype=feat)


def test_algorithmic_work_counts():
    wl = _wl([(1000, 30, 256), (2000, 30, 256), (500, 200, 128), (700, 200, 128)], [(0, 1), (2, 3)])
    w = bench.algorithmic_work(wl, ir_steps=1, saved_k_max=304)
    # projection: Phi (4k), mass (4), BF16 features (2d) per vertex, A (4kd) per shape
    want = sum(n * (4 * k + 4 + 2 * d) + 4 * k * d for (n, k, d) in [(1000, 30, 256), (2000, 30, 256),
                                                                      (500, 200, 128), (700, 200, 128)])
    assert w["project"]["bytes"] == want == w["project_bwd"]["bytes"]
    assert w["project"]["flops"] == 2.0 * (1000 * 30 * 256 + 2000 * 30 * 256 + 500 * 200 * 128 + 700 * 200 * 128)
    # row solves: k factorisations of k^3/3 flops plus substitutions and one refinement
    assert w["solve"]["flops"] == sum(k ** 4 / 3.0 + 6.0 * k ** 3 for k in (30, 200))
    # saved factors: k systems of 32Q(Q+2) + 64Q floats (Q = ceil(k/8)), written and read back
    fac = sum(4 * k * (32 * q * (q + 2) + 64 * q) for k, q in ((30, 4), (200, 25)))
    assert w["solve"]["bytes"] == sum(12 * k * k for k in (30, 200)) + fac
    assert w["adj_solve"]["bytes"] == sum(8 * k * k for k in (30, 200)) + fac
    # without saved factors the adjoint refactors (k^4/3 more flops) and moves no factors
    w0 = bench.algorithmic_work(wl, ir_steps=1, saved_k_max=0)
    assert w0["adj_solve"]["flops"] == sum(k ** 4 / 3.0 + 2.0 * k ** 3 for k in (30, 200))
    assert w0["adj_solve"]["bytes"] == sum(8 * k * k for k in (30, 200))
    # FP32 features stream twice the feature bytes
    w32 = bench.algorithmic_work(_wl([(1000, 30, 256)], [], feat="fp32"), 1, 304)
    assert w32["project"]["bytes"] == 1000 * (4 * 30 + 4 + 4 * 256) + 4 * 30 * 256


def test_algorithmic_work_rectangular():
    """A k_Y x k_X map has k_Y row systems of size k_X."""
    wl = _wl([(1000, 30, 64), (2000, 50, 64)], [(0, 1)])
    w = bench.algorithmic_work(wl, ir_steps=1, saved_k_max=304)
    assert w["solve"]["flops"] == 50 * 30 ** 3 / 3.0 + 6.0 * 50 * 30 ** 2
    q = 4
    assert w["solve"]["bytes"] == 4 * (30 * 30 + 2 * 50 * 30) + 4 * 50 * (32 * q * (q + 2) + 64 * q)


def test_oracle_pool_times_every_step_on_the_requested_workers():
    """The CPU baseline's process pool (spawn, single-threaded BLAS per worker) returns one
    wall time per step and never uses more workers than pairs."""
    import bench
    times, used = bench.oracle_pool_steps(0, [0], 2, 4)
    assert used == 1 and len(times) == 2 and all(t > 0 for t in times)
    times, used = bench.oracle_pool_steps(1, [0, 1, 2], 1, 2)
    assert used == 2 and len(times) == 1


def test_config_sizes_match_the_drawn_shapes():
    from paper_2604_10377_gb300 import synth
    sizes = synth.config_sizes(1)
    wl = synth.make_config(1, pairs=[0, 5, 31], n_scale=1.0)
    for j, p in enumerate([0, 5, 31]):
        assert sizes[p] == (wl.shapes[2 * j].n, wl.shapes[2 * j + 1].n, wl.shapes[2 * j].k)
