"""Benchmark of the functional-map hot path on GB300.

One step = one pass of the whole hot path over the ragged batch: fmap_project,
fmap_solve, the training loss and fmap_solve_backward (projection backward
included). The default workload is the ragged mixed batch: 256 shape pairs, n
log-uniform in 1k..100k, k drawn from {30, 50, 100, 200}, d = 256 BF16 features
(about 10 GB of inputs per step, so every step streams from HBM, not L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun every rank runs its own batch of
pairs (weak scaling, no collective on the data path); the time is the max over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fmap solves/sec (fwd+bwd, pairs/s) vs plain fwd solve; % of tensor/HBM roofline"
WORKLOADS = {
    4: "ragged mixed batch: 256 pairs, n log-uniform 1k-100k, k in {30,50,100,200}, d=256 BF16 features",
    3: "large spectrum: 4 pairs, n=200k, k=200, d=512 BF16 features, FP64 Gram, factors recomputed",
    2: "differentiable: 8 pairs, n=20k, k=100, d=384 BF16 features",
    1: "batched: 32 pairs, n log-uniform 5k-50k, k=50, d=256 FP32 features",
    0: "single pair: n=5000, k=30, d=128 FP32 features",
}
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return dict(hbm_gbs=float(p["hbm_gbs"]), bf16_tflops=float(p["bf16_tflops"]),
                    bf16_tflops_sustained=float(p.get("bf16_tflops_sustained", p["bf16_tflops"])),
                    sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0, sm_max_mhz=2070.0,
                    source="fallback")


# DRAM traffic per step of each kernel kind, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum), committed with the SHA-256 of the kernel source it was taken
# on (the kernel's file followed by the two shared headers); a kind whose source changed
# since reports null.
TRAFFIC_FILES = {4: "profiles/traffic_ragged256_k30-200_d256.txt"}
KIND_SOURCES = {"project": "k_project_tc.cu", "project_bwd": "k_project_bwd_tc.cu", "solve": "k_chol.cu",
                "adj_solve": "k_chol.cu"}


def load_traffic(workload: int) -> dict:
    import hashlib
    out = {}
    rel = TRAFFIC_FILES.get(workload)
    if not rel or not os.path.exists(os.path.join(ROOT, rel)):
        return out
    csrc = os.path.join(ROOT, "paper_2604_10377_gb300", "csrc")
    for line in open(os.path.join(ROOT, rel)):
        parts = line.split()
        if len(parts) != 4 or line.startswith("#"):
            continue
        kind, src, sha, nbytes = parts
        try:
            h = hashlib.sha256()
            for f in (src, "fmap_internal.cuh", "tc_ptx.cuh"):
                h.update(open(os.path.join(csrc, f), "rb").read())
            cur = h.hexdigest()
        except OSError:
            continue
        if cur == sha:
            out[kind] = int(nbytes)
    return out


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------- clocks sampler
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--id={self.uuid}", "--query-gpu=" + ",".join(self.FIELDS),
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- measured peaks
PEAK_KINDS = {"fp32_fma": 0, "fp64_fma": 1, "tf32_mma": 2, "bf16_mma": 3, "fp32x2_fma": 4}


def measure_peaks(dev, target_s: float = 0.25, reps: int = 3):
    """The library's peak loops (fmap_peak_loop): FP32 and FP64 FMA chains on every SM,
    tcgen05 kind::tf32 and kind::f16 (BF16) MMA loops with one CTA per SM. Each launch is
    scaled to about `target_s` seconds; the best of `reps` CUDA-event timed launches is
    kept. Returns TFLOP/s per kind, with the SM clock sampled while they ran."""
    import ctypes
    import torch
    from paper_2604_10377_gb300 import _lib
    L = _lib.lib()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(4 * sms, dtype=torch.int32, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    out = {}
    for name, kind in PEAK_KINDS.items():
        blocks = sms if "mma" in name else 4 * sms
        fl = ctypes.c_double(0.0)

        def launch(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _lib.check(L.fmap_peak_loop(kind, blocks, int(iters), ctypes.c_void_p(sink.data_ptr()),
                                        ctypes.byref(fl), st), "fmap_peak_loop")
            e1.record()
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1) / 1000.0

        iters = 1000
        t = launch(iters)
        while t < 0.02:
            iters *= 8
            t = launch(iters)
        iters = max(1, int(iters * target_s / t))
        best = 0.0
        for _ in range(reps):
            t = launch(iters)
            best = max(best, fl.value / t / 1e12)
        out[name] = best
    if int(sink[0].item()) != 0:
        raise RuntimeError("an MMA peak loop reported a timed-out wait")
    return out


# ---------------------------------------------------------------- algorithmic work
def algorithmic_work(wl, ir_steps, saved_k_max):
    """Bytes (HBM) and flops per launch of each kernel kind, from the sizes alone."""
    fsz = 2 if wl.feat_dtype == "bf16" else 4
    proj_bytes = sum(s.n * (4 * s.k + 4 + fsz * s.d) + 4 * s.k * s.d for s in wl.shapes)
    proj_flops = sum(2.0 * s.n * s.k * s.d for s in wl.shapes)
    bwd_bytes = sum(s.n * (4 * s.k + 4 + fsz * s.d) + 4 * s.k * s.d for s in wl.shapes)
    solve_flops, adj_flops, loss_flops, gemm_flops = 0.0, 0.0, 0.0, 0.0
    solve_bytes, adj_bytes = 0, 0
    da_tiles = 0
    for p in wl.pairs:
        # C is ky x k: ky row systems of size k (square maps: ky == k)
        k, ky = wl.shapes[p.x].k, wl.shapes[p.y].k
        kp = (k + 7) // 8 * 8
        q = kp // 8
        fac = 4 * ky * (32 * q * (q + 2) + 64 * q) if k <= saved_k_max else 0
        solve_flops += ky * k ** 3 / 3.0 + (2.0 + 4.0 * ir_steps) * ky * k ** 2
        adj_flops += (0.0 if k <= saved_k_max else ky * k ** 3 / 3.0) + 2.0 * ky * k ** 2
        loss_flops += 2.0 * ky * ky * k + 2.0 * ky * ky * k
        # adjoint GEMMs: W = Gamma^T C + C^T Gamma, dA_y = Gamma A_x, dA_x = Gamma^T A_y - W A_x
        d = wl.shapes[p.x].d
        gemm_flops += 4.0 * k * k * ky + 2.0 * ky * k * d + 2.0 * k * (ky + k) * d
        da_tiles += -(-k // 128) * -(-d // 128)
        # G, R and C move once each, saved factors written (forward) / read (adjoint)
        solve_bytes += 4 * (k * k + 2 * ky * k) + fac
        adj_bytes += 4 * 2 * ky * k + fac
    return dict(project=dict(bytes=proj_bytes, flops=proj_flops), project_bwd=dict(bytes=bwd_bytes, flops=proj_flops),
                solve=dict(flops=solve_flops, bytes=solve_bytes), adj_solve=dict(flops=adj_flops, bytes=adj_bytes),
                loss=dict(flops=loss_flops), adj_gemm=dict(flops=gemm_flops, da_tiles=da_tiles))


# ---------------------------------------------------------------- oracle timing
# The CPU baseline and the reference arm time the FP64 oracle, as it stands, on the host
# cores: a pool of single-threaded worker processes (started with "spawn", BLAS limited to
# one thread each), one per core of the affinity mask, over a fixed sample of the
# workload's pairs shared out by estimated cost. Every worker draws its own pairs from the
# seeds first (not timed); then each step is one pass of fwd + loss + bwd over the sample,
# with a barrier between steps, and its wall time is the step time.
ORACLE_SAMPLE_PAIRS = 32
THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
               "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_pair_fwd_bwd(orc, s_x, s_y, lam, c_gt):
    """Oracle fwd + training loss + bwd of one pair (inputs already FP64)."""
    ax = orc.project(s_x["phi"], s_x["mass"], s_x["feat"])
    ay = orc.project(s_y["phi"], s_y["mass"], s_y["feat"])
    dm = orc.mask_from_evals(s_x["evals"], s_y["evals"])
    c = orc.solve(ax, ay, dm, lam)
    _, dc = orc.loss_orth_gt(c, c_gt)
    g = orc.solve_backward(ax, ay, c, dm, lam, dc)
    return c, orc.project_backward(s_x["phi"], s_x["mass"], g["dA"]), orc.project_backward(s_y["phi"], s_y["mass"],
                                                                                          g["dB"])


def _f64_shape(s):
    import numpy as np
    return dict(phi=s.phi.astype(np.float64), mass=s.mass.astype(np.float64), feat=s.feat_f64(),
                evals=s.evals.astype(np.float64))


def _oracle_worker(config, replica, pair_ids, n_steps, barrier, queue):
    import numpy as np
    from oracle import fmap_oracle as orc
    from paper_2604_10377_gb300 import synth
    try:
        wl = synth.make_config(config, pairs=pair_ids, replica=replica) if pair_ids else None
        work = []
        if wl is not None:
            for p in wl.pairs:
                work.append((_f64_shape(wl.shapes[p.x]), _f64_shape(wl.shapes[p.y]), float(np.float32(p.lam)),
                             p.c_gt))
        barrier.wait(timeout=1800)
        for _ in range(n_steps):
            for sx, sy, lam, gt in work:
                oracle_pair_fwd_bwd(orc, sx, sy, lam, gt)
            barrier.wait(timeout=1800)
        queue.put(("ok", len(work)))
    except Exception as e:   # reported to the parent; the barrier is broken for everyone
        queue.put(("error", repr(e)))
        barrier.abort()


def oracle_pool_steps(config, pair_ids, n_steps, workers, replica=0):
    """Wall time (s) of each of n_steps oracle passes over `pair_ids`, on `workers`
    single-threaded processes. Returns (step times, workers used)."""
    import multiprocessing as mp
    from paper_2604_10377_gb300 import synth
    sizes = synth.config_sizes(config, replica)
    workers = max(1, min(workers, len(pair_ids)))
    # longest-processing-time first over an estimate of each pair's oracle cost
    cost = {p: (sizes[p][0] + sizes[p][1]) * sizes[p][2] * 4.0 + sizes[p][2] ** 4 / 3.0 for p in pair_ids}
    shares, load = [[] for _ in range(workers)], [0.0] * workers
    for p in sorted(pair_ids, key=lambda q: (-cost[q], q)):
        w = min(range(workers), key=lambda i: (load[i], i))
        shares[w].append(p)
        load[w] += cost[p]
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers + 1)
    queue = ctx.Queue()
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    for k in THREAD_VARS:
        os.environ[k] = "1"
    try:
        procs = [ctx.Process(target=_oracle_worker, args=(config, replica, sorted(shares[w]), n_steps, barrier, queue),
                             daemon=True) for w in range(workers)]
        for pr in procs:
            pr.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    times = []
    try:
        barrier.wait(timeout=1800)          # every worker has drawn its pairs
        for _ in range(n_steps):
            t0 = time.perf_counter()
            barrier.wait(timeout=1800)
            times.append(time.perf_counter() - t0)
    except threading.BrokenBarrierError:
        pass
    results = [queue.get(timeout=60) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    errs = [r[1] for r in results if r[0] != "ok"]
    if errs or len(times) != n_steps:
        raise RuntimeError(f"oracle worker failed: {errs}")
    return times, workers


# ---------------------------------------------------------------- plain PyTorch comparator
def torch_restatement(lay, b, wl, gt_host_list, dev, steps: int, warmup: int):
    """The method written with plain PyTorch FP32 ops on the same GPU and the same
    resident inputs: A = Phi^T (M F), G = A A^T and R = B A^T per pair, the k row
    systems G + lambda diag(D_i) stacked with diag_embed and handed to
    torch.linalg.solve, the orthogonality + ground-truth loss, and autograd for the
    backward. Pairs of equal k are batched. A comparator only: none of this runs on
    the library's path. Returns (fwd+bwd pairs/s, fwd pairs/s, ms fwd+bwd, ms fwd)."""
    import numpy as np
    import torch

    views = []
    for s in range(lay.n_shapes):
        n, k, ld = lay.ns[s], lay.ks[s], lay.ld_phi[s]
        phi = b.phi[lay.phi_off[s]:lay.phi_off[s] + n * ld].view(n, ld)[:, :k]
        mass = b.mass[lay.mass_off[s]:lay.mass_off[s] + n]
        ev = b.evals[lay.evals_off[s]:lay.evals_off[s] + k]
        views.append((phi, mass, lay.feat_view(b.feat, s), ev))
    groups = {}
    for pi, p in enumerate(wl.pairs):
        groups.setdefault(lay.ks[p.x], []).append(pi)
    gts = {k: torch.from_numpy(np.stack([gt_host_list[pi] for pi in pl])).to(dev) for k, pl in groups.items()}
    lams = {k: torch.tensor([float(np.float32(wl.pairs[pi].lam)) for pi in pl], device=dev)
            for k, pl in groups.items()}

    def step(with_bwd: bool):
        feats = [v[2].float().requires_grad_(with_bwd) for v in views]
        a = [v[0].t() @ (v[1][:, None] * f) for v, f in zip(views, feats)]
        loss = 0.0
        for k, pl in groups.items():
            ax = torch.stack([a[wl.pairs[pi].x] for pi in pl])
            ay = torch.stack([a[wl.pairs[pi].y] for pi in pl])
            ex = torch.stack([views[wl.pairs[pi].x][3] for pi in pl])
            ey = torch.stack([views[wl.pairs[pi].y][3] for pi in pl])
            g = ax @ ax.transpose(1, 2)
            r = ay @ ax.transpose(1, 2)
            dmask = (ey[:, :, None] - ex[:, None, :]) ** 2
            sysm = g[:, None] + lams[k][:, None, None, None] * torch.diag_embed(dmask)
            c = torch.linalg.solve(sysm, r.unsqueeze(-1)).squeeze(-1)
            eye = torch.eye(k, device=dev)
            loss = loss + ((c @ c.transpose(1, 2) - eye) ** 2).sum() + ((c - gts[k]) ** 2).sum()
        if with_bwd:
            loss.backward()
        return loss

    out = []
    for with_bwd in (True, False):
        with torch.set_grad_enabled(with_bwd):
            for _ in range(warmup):
                step(with_bwd)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                step(with_bwd)
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1) / steps)
    npairs = len(wl.pairs)
    return npairs / (out[0] / 1000.0), npairs / (out[1] / 1000.0), out[0], out[1]


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the FP64 oracle (the paper's method written plainly), as it
    stands, on the host cores; each step is one pass over the first ORACLE_SAMPLE_PAIRS
    pairs of the workload (the same sample as our arm's cpu_baseline)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2604_10377_gb300 import synth
    npairs = synth.CONFIGS[args.workload]["pairs"]
    sample = list(range(min(ORACLE_SAMPLE_PAIRS, npairs)))
    times, used = oracle_pool_steps(args.workload, sample, args.warmup + args.steps, cpu_cores())
    timed = times[args.warmup:]
    tot = sum(timed)
    value = len(sample) * len(timed) / tot
    ks = [synth.config_sizes(args.workload)[p][2] for p in sample]
    what = (f"fwd+loss+bwd of pairs 0..{len(sample) - 1} of the workload (k={ks}) per step, on {used} "
            f"single-threaded processes, NumPy FP64")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "pairs_per_step": len(sample)},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": used, "kind": "oracle", "sample": what},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def bench_workload(wid, args, dev, peaks, measured, uuid, rank, world, full):
    """Time one workload: the whole step (project, solve, loss, backward) and the plain
    forward (project + solve), each as one CUDA graph, plus an eager pass with the
    library's per-kind event timing. `full` adds the end-to-end loop, the autotuner, the
    PyTorch comparator and the CPU baseline (the main workload of the line). Returns the
    fields of the JSON line for this workload."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2604_10377_gb300 import api, shard, synth

    # the large-spectrum workload runs as its config states: factors recomputed in the
    # backward pass, none stored
    store_max_k = 0 if wid == 3 else args.store_factors_max_k
    t_gen = time.time()
    wl = synth.make_config(wid, replica=rank, pairs=range(args.pairs) if args.pairs else None)
    t_gen = time.time() - t_gen
    lay = api.BatchLayout([s.n for s in wl.shapes], [s.k for s in wl.shapes], [s.d for s in wl.shapes], wl.feat_dtype)
    host = lay.pack_host(wl.shapes)
    fixed_tuning = json.loads(args.tuning) if args.tuning else {}
    b = api.FmapBatch(lay, [(p.x, p.y, p.lam) for p in wl.pairs], device=dev, precision=wl.feat_dtype,
                      with_grad=True, masks=[p.mask for p in wl.pairs], ir_steps=args.ir_steps,
                      store_factors_max_k=store_max_k, tuning=fixed_tuning)
    b.upload(host)
    gt_host = np.zeros(int(b.c_off[-1]), np.float32)
    for p, pr in enumerate(wl.pairs):
        gt_host[b.c_off[p]:b.c_off[p + 1]] = pr.c_gt.reshape(-1)
    gt = torch.from_numpy(gt_host).to(dev)
    loss = torch.empty(len(wl.pairs), dtype=torch.float32, device=dev)
    dc = torch.empty_like(b.C)
    npairs = len(wl.pairs)

    def step():
        a = b.project()
        c = b.solve(a)
        b.loss_orth(c, gt, loss=loss, d_c=dc)
        b.solve_backward(dc, a, c)

    def fwd_step():
        a = b.project()
        b.solve(a)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps, timing=False):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(); barrier(); torch.cuda.synchronize()
        if timing:
            b.set_timing(True)
        st = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        kt = b.read_timing() if timing else None
        if timing:
            b.set_timing(False)
        barrier()
        # whole job: pairs of all ranks over the slowest rank's time
        rate, ms, _ = shard.job_throughput(float(npairs), e0.elapsed_time(e1) / steps)
        return ms, None, kt, rate

    # tile shapes / launch plans picked by the project's autotuner on this batch (outside
    # every timed region)
    tune = None
    if full and not args.no_autotune and not fixed_tuning:
        from paper_2604_10377_gb300 import autotune as at
        res = at.autotune(b, step)
        tune = {"tuning": res["tuning"], "tuned_ms": res["ms"], "default_ms": res["baseline_ms"],
                "trials": len(res["trials"]), "seconds": round(res["seconds"], 1)}

    sampler = ClockSampler(uuid) if uuid else None
    if sampler:
        sampler.start()
    # eager pass with the library's per-kind event timing (the kernel breakdown)
    ms_eager, _, ktime, rate_eager = timed(step, args.steps, timing=True)
    if args.no_graph:
        ms_step, rate_step = ms_eager, rate_eager
        ms_fwd, _, _, rate_fwd = timed(fwd_step, args.steps)
    else:
        # the step as one CUDA graph: every C-ABI call only enqueues, so it captures
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            step()
            fwd_step()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize()
        g_step, g_fwd = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_step):
            step()
        with torch.cuda.graph(g_fwd):
            fwd_step()
        torch.cuda.synchronize()
        ms_step, _, _, rate_step = timed(g_step.replay, args.steps)
        ms_fwd, _, _, rate_fwd = timed(g_fwd.replay, args.steps)
        # leave the last timed results of the whole step in the buffers (accuracy below)
        g_step.replay()
        torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    status = b.status[:npairs].cpu().numpy()

    # ---- end to end: host inputs -> device, step, loss and C back to the host
    e2e = None
    if full and not args.no_e2e:
        pinned = {k: api.host_to_torch(v).pin_memory() for k, v in host.items()}
        gt_pin = torch.from_numpy(gt_host).pin_memory()
        loss_host = torch.empty(npairs, dtype=torch.float32).pin_memory()
        c_host = torch.empty(b.C.numel(), dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in pinned.values()) + gt_pin.numel() * 4
        d2h = loss_host.numel() * 4 + c_host.numel() * 4

        def e2e_step():
            b.upload(pinned, non_blocking=True, copy_streams=args.copy_streams)
            gt.copy_(gt_pin, non_blocking=True)
            step()
            loss_host.copy_(loss, non_blocking=True)
            c_host.copy_(b.C, non_blocking=True)

        e2e_steps = max(1, args.steps // 2)
        ms_serial, _, _, rate_serial = timed(e2e_step, e2e_steps)
        e2e = {"value": rate_serial, "unit": "pairs/s", "ms_per_step": ms_serial, "copy_streams": args.copy_streams,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "pipeline": "none"}
        if not args.no_pipeline:
            # the same steps through api.UploadPipeline: two input buffers, the upload of
            # step i+1 (copy stream) overlaps the compute of step i; every step's inputs
            # still cross the host link inside the timed region
            b2 = api.FmapBatch(lay, [(p.x, p.y, p.lam) for p in wl.pairs], device=dev, precision=wl.feat_dtype,
                               with_grad=True, masks=[p.mask for p in wl.pairs], ir_steps=args.ir_steps,
                               store_factors_max_k=store_max_k, tuning=b.tuning)
            pipe = api.UploadPipeline([b, b2])
            gts = [gt, torch.empty_like(gt)]

            def pipelined(nsteps):
                j = pipe.next_buffer
                pipe.prefetch(pinned, [(gts[j], gt_pin)])
                for s_ in range(nsteps):
                    j = pipe.acquire()
                    if s_ + 1 < nsteps:
                        jn = pipe.next_buffer
                        pipe.prefetch(pinned, [(gts[jn], gt_pin)])
                    bb = pipe.batches[j]
                    a_ = bb.project()
                    c_ = bb.solve(a_)
                    bb.loss_orth(c_, gts[j], loss=loss, d_c=dc)
                    bb.solve_backward(dc, a_, c_)
                    loss_host.copy_(loss, non_blocking=True)
                    c_host.copy_(bb.C, non_blocking=True)
                    pipe.release()

            pipelined(args.warmup)
            torch.cuda.synchronize(); barrier(); torch.cuda.synchronize()
            st_ = torch.cuda.current_stream(dev)
            e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0_.record(st_)
            pipelined(e2e_steps)
            e1_.record(st_)
            torch.cuda.synchronize()
            barrier()
            rate_p, ms_p, _ = shard.job_throughput(float(npairs), e0_.elapsed_time(e1_) / e2e_steps)
            # the pipelined loop must give the serial loop's results
            same = bool(torch.equal(b2.C, b.C))
            e2e = {"value": rate_p, "unit": "pairs/s", "ms_per_step": ms_p, "copy_streams": 1,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "pipeline": "api.UploadPipeline, 2 input buffers (upload of step i+1 overlaps step i)",
                   "buffers_agree": same,
                   "serial": {"value": rate_serial, "ms_per_step": ms_serial, "copy_streams": args.copy_streams}}
            del pipe, b2

    # ---- roofline of every kernel kind, and of the dominant one
    work = algorithmic_work(wl, args.ir_steps, store_max_k)
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
               for k, v in ktime.items() if v[1] > 0}
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    launches_total = sum(v[1] for v in ktime.values())
    if measured:
        fp32_peak_tflops = measured["fp32_fma"]
        fp32_peak_source = "measured FP32 FMA loop on this GPU (fmap_peak_loop)"
    else:
        fp32_peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        fp32_peak_source = "derived: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock"

    traffic = load_traffic(wid)

    def roof_for(kind):
        # the launches of one kind in one step process the batch once: the unit is the step
        per_step_ms = ktime[kind][0] / args.steps
        if kind in ("project", "project_bwd"):
            ach = work[kind]["bytes"] / (per_step_ms / 1000.0) / 1e9
            r = {"kernel": kind, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / peaks["hbm_gbs"], "traffic": traffic.get(kind),
                 "peak_source": f"{peaks['source']} HBM copy bandwidth"}
            if measured:
                # tensor pipe: algorithmic flops over the measured MMA peak of the dtype the MMAs run in
                # (BF16 features: kind::f16 forward, kind::tf32 backward; FP32 features: kind::tf32)
                tflops = work[kind]["flops"] / (per_step_ms / 1000.0) / 1e12
                mma = "bf16_mma" if (kind == "project" and wl.feat_dtype == "bf16") else "tf32_mma"
                r["tensor"] = {"achieved_tflops": tflops, "peak_tflops": measured[mma], "peak": mma,
                               "frac": tflops / measured[mma]}
            return r
        if kind == "adj_gemm":
            # tensor cores when the knob says so, or by the library's built-in choice
            # (fmap_options.adjoint_kernel = 0): at least two 128-column dA_x tiles per SM
            ach = work[kind]["flops"] / (per_step_ms / 1000.0) / 1e12
            ak = fixed_tuning.get("adjoint_kernel", 0)
            if ak == 1 or (ak == 0 and work[kind]["da_tiles"] >= 2 * SM_COUNT):
                pk = measured["tf32_mma"] / 3.0 if measured else None
                return {"kernel": kind, "bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                        "frac": ach / pk if pk else None, "traffic": None,
                        "peak_source": "measured TF32 MMA peak / 3 (three TF32 passes per FP32-class product)"
                        if pk else "TF32 peak not measured (--no-peaks)"}
            return {"kernel": kind, "bound": "alu", "achieved": ach, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak_tflops, "traffic": None, "peak_source": fp32_peak_source}
        flops = work.get(kind, {}).get("flops")
        if flops is None:
            return {"kernel": kind, "bound": "alu", "achieved": None, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "frac": None, "traffic": None}
        ach = flops / (per_step_ms / 1000.0) / 1e12
        return {"kernel": kind, "bound": "alu", "achieved": ach, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": ach / fp32_peak_tflops, "traffic": traffic.get(kind),
                "algorithmic_bytes": work.get(kind, {}).get("bytes"),
                "peak_source": fp32_peak_source}

    roofline = roof_for(dom)
    others = {k: roof_for(k) for k in ("project", "project_bwd", "solve", "adj_solve", "adj_gemm")
              if k in kernels and k != dom}

    # ---- accuracy against the FP64 oracle on sampled pairs (two of every k), last timed step
    accuracy = None
    if rank == 0 and not args.no_accuracy:
        from oracle import fmap_oracle as orc
        ks = wl.k_of_pair
        sample = []
        for kk in sorted(set(ks)):
            sample += [p for p in range(npairs) if ks[p] == kk][:2]
        ec, ef = [], []
        for pi in sample:
            pr = wl.pairs[pi]
            sx, sy = _f64_shape(wl.shapes[pr.x]), _f64_shape(wl.shapes[pr.y])
            c_ref, dfx, dfy = oracle_pair_fwd_bwd(orc, sx, sy, float(np.float32(pr.lam)), pr.c_gt)
            c_gpu = b.c_view(b.C, pi).double().cpu().numpy()
            ec.append(float(np.linalg.norm(c_gpu - c_ref) / np.linalg.norm(c_ref)))
            for sidx, dref in ((pr.x, dfx), (pr.y, dfy)):
                dg = lay.feat_view(b.dfeat, sidx).double().cpu().numpy()
                ef.append(float(np.linalg.norm(dg - dref) / np.linalg.norm(dref)))
        accuracy = {"pairs": len(ec), "pairs_sampled": sample, "C_rel_fro_max": max(ec),
                    "C_rel_fro_mean": float(np.mean(ec)), "dF_rel_fro_max": max(ef),
                    "dF_rel_fro_mean": float(np.mean(ef)),
                    "tolerance": 3e-3 if wl.feat_dtype == "bf16" else 1e-5,
                    "dF_storage": wl.feat_dtype,
                    "reference": "FP64 oracle on the same inputs"}

    cpu = None
    if full and rank == 0 and not args.no_cpu_baseline:
        sample = list(range(min(ORACLE_SAMPLE_PAIRS, npairs)))
        times, used = oracle_pool_steps(wid, sample, 3, cpu_cores(), replica=rank)
        v = len(sample) * 2 / sum(times[1:])
        t1, _ = oracle_pool_steps(0, [0], 3, 1)
        cpu = {"value": v, "unit": "pairs/s", "cores": used, "kind": "oracle",
               "sample": (f"fwd+loss+bwd of pairs 0..{len(sample) - 1} of the same workload (k="
                          f"{[wl.shapes[wl.pairs[p].x].k for p in sample]}), {used} single-threaded processes, "
                          f"one untimed pass then two timed passes, NumPy FP64"),
               "single_pair_1thread_s": min(t1[1:]),
               "single_pair_1thread": "the single-pair workload (n=5000, k=30, d=128) fwd+loss+bwd on one "
                                      "single-threaded process (best of two passes after one untimed)"}

    torch_cmp = None
    if full and rank == 0 and not args.no_torch_compare:
        v_fb, v_f, ms_fb, ms_f = torch_restatement(lay, b, wl, [p.c_gt for p in wl.pairs], dev, 3, 1)
        torch_cmp = {"value": v_fb, "unit": "pairs/s", "ms_per_step": ms_fb,
                     "fwd_only": {"value": v_f, "unit": "pairs/s", "ms_per_step": ms_f},
                     "what": "plain PyTorch FP32 ops on the same GPU (diag_embed + torch.linalg.solve, autograd)"}

    out = {
        "value": rate_step, "ms_per_step": ms_step,
        "config": {"workload": WORKLOADS[wid] + (f" (first {npairs} pairs only)" if args.pairs else ""),
                   "pairs_per_gpu": npairs, "global_batch": world * npairs,
                   "parallelism": f"pairs sharded over {world} GPU(s), no collective",
                   "l2": "inputs larger than L2 (%.2f GB streamed per step)" % (work["project"]["bytes"] / 1e9)
                   if work["project"]["bytes"] > 129e6 else
                   "inputs smaller than L2 (%.3f GB per step): steps replay from a warm L2"
                   % (work["project"]["bytes"] / 1e9)},
        "fwd_only": {"value": rate_fwd, "unit": "pairs/s", "ms_per_step": ms_fwd},
        "tuning": fixed_tuning or None,
        "launch": "eager" if args.no_graph else "one CUDA graph per step",
        "eager": {"value": rate_eager, "unit": "pairs/s", "ms_per_step": ms_eager},
        "roofline": roofline,
        "roofline_other": others,
        "kernels": kernels,
        "gpu_launches": int(launches_total),
        "accuracy": accuracy,
        "clocks": clocks,
        "status_ok": bool((status == 0).all()),
        "gen_s": round(t_gen, 1),
    }
    if wid == 3:
        out["config"]["factors"] = "recomputed in the backward pass (none stored)"
    if full:
        out.update({"cpu_baseline": cpu, "torch_restatement": torch_cmp, "autotune": tune, "e2e": e2e})
    b.close()
    del b
    torch.cuda.empty_cache()
    return out


GRADFEAT_WORKLOAD = ("spatial gradient features (DiffusionNet, Sec. 'Learned Scaling and Rotation'): 64 shapes, "
                     "n log-uniform 1k-100k, D=128 channels, one block-diagonal complex gradient operator "
                     "(7 entries per row), BF16 features out")


def bench_gradient_features(args, dev, peaks, measured, uuid):
    """fmap_gradient_features over a batch of 64 shapes stored as one block-diagonal CSR
    operator (n log-uniform in 1k..100k per shape, D = 128), variants A and B, BF16 output
    rows of width D: vertices/s and the roofline of the kernel (HBM bytes: X read once, the
    CSR read once, F written once; tensor flops: 2 n (2D)^2)."""
    import numpy as np
    import torch
    from paper_2604_10377_gb300 import api, synth
    rng = np.random.Generator(np.random.PCG64(synth.BASE_SEED + 7000))
    dim = 128
    ns = [int(round(np.exp(rng.uniform(np.log(1000), np.log(100000))))) for _ in range(64)]
    t_gen = time.time()
    parts = [synth.make_gradient_input(synth.BASE_SEED + 7001 + i, n, dim) for i, n in enumerate(ns)]
    off = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    row_ptr = [np.zeros(1, np.int64)]
    eoff = 0
    for p_, o in zip(parts, off[:-1]):
        row_ptr.append(p_.row_ptr[1:] + eoff)
        eoff += int(p_.row_ptr[-1])
    row_ptr = torch.from_numpy(np.concatenate(row_ptr)).to(dev)
    col = torch.from_numpy(np.concatenate([p_.col_idx + np.int32(o) for p_, o in zip(parts, off[:-1])])).to(dev)
    vals = torch.from_numpy(np.concatenate([np.stack([p_.g_re, p_.g_im], 1) for p_ in parts])).to(dev)
    x = torch.from_numpy(np.concatenate([p_.feat for p_ in parts])).to(dev)
    a_re, a_im = torch.from_numpy(parts[0].a_re).to(dev), torch.from_numpy(parts[0].a_im).to(dev)
    t_gen = time.time() - t_gen
    n = int(off[-1])
    nnz = int(col.numel())
    out = torch.empty((n, dim), dtype=torch.bfloat16, device=dev)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    res = {}
    sampler = ClockSampler(uuid) if uuid else None
    if sampler:
        sampler.start()
    for variant in ("A", "B"):
        for _ in range(max(3, args.warmup)):
            api.gradient_features(row_ptr, col, vals, x, a_re, a_im, variant=variant, out=out, ws=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            _, status = api.gradient_features(row_ptr, col, vals, x, a_re, a_im, variant=variant, out=out, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[variant] = {"ms_per_call": ms, "vertices_per_s": n / (ms * 1e-3), "status": int(status.item())}
    clocks = sampler.stop() if sampler else None
    nbytes = n * dim * 4 + (n + 1) * 8 + nnz * 12 + n * dim * 2 + (2 * dim) ** 2 * 4
    flops = 2.0 * n * (2 * dim) ** 2
    ms = min(r["ms_per_call"] for r in res.values())
    gbs = nbytes / (ms * 1e-3) / 1e9
    tfl = flops / (ms * 1e-3) / 1e12
    tf32 = measured["tf32_mma"] if measured else None
    hbm_frac = gbs / peaks["hbm_gbs"]
    ten_frac = tfl / tf32 if tf32 else None
    bound = "tensor" if (ten_frac is not None and (flops / (tf32 * 1e12)) > nbytes / (peaks["hbm_gbs"] * 1e9)) else "hbm"
    # accuracy: the first shape's rows against the FP64 oracle (variant B ran last)
    from oracle import fmap_oracle as orc
    p0 = parts[0]
    gx, gy = orc.gradient_apply(p0.row_ptr, p0.col_idx, p0.g_re, p0.g_im, p0.feat)
    ref = orc.spatial_gradient_features(gx, gy, p0.a_re, p0.a_im, "B")
    got = out[:p0.n].float().cpu().numpy()
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"workload": GRADFEAT_WORKLOAD, "vertices": n, "nnz": nnz, "variants": res,
            "roofline": {"bound": bound, "achieved": gbs if bound == "hbm" else tfl,
                         "peak": peaks["hbm_gbs"] if bound == "hbm" else tf32,
                         "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
                         "frac": hbm_frac if bound == "hbm" else ten_frac,
                         "hbm": {"achieved_gbs": gbs, "frac": hbm_frac, "algorithmic_bytes": nbytes},
                         "tensor": {"achieved_tflops": tfl, "frac": ten_frac, "algorithmic_flops": flops,
                                    "peak": "measured tf32_mma"}},
            "accuracy": {"rows": p0.n, "rel_fro": err, "tolerance": 3e-3, "reference": "FP64 oracle, BF16 output"},
            "clocks": clocks, "gen_s": round(t_gen, 1)}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", ""))
    if uuid and not uuid.startswith("GPU-"):
        uuid = "GPU-" + uuid

    # measured peaks (the roofline denominators), with the clocks seen while they ran
    measured = None
    if not args.no_peaks:
        psamp = ClockSampler(uuid) if uuid else None
        if psamp:
            psamp.start()
        measured = measure_peaks(dev)
        measured["clocks"] = psamp.stop() if psamp else None
        measured["how"] = ("fmap_peak_loop: FP32/FP64 FMA chains (4 x SMs CTAs of 512 threads), tcgen05 "
                           "kind::tf32 / kind::f16 M=128 N=256 MMA loops (one CTA per SM); ~0.25 s launches, "
                           "best of 3, CUDA events")

    main = bench_workload(args.workload, args, dev, peaks, measured, uuid, rank, world, full=True)
    gradfeat = None
    if world == 1 and not args.no_sub_workloads:
        gradfeat = bench_gradient_features(args, dev, peaks, measured, uuid)
    subs = None
    if world == 1 and not args.no_sub_workloads:
        # the other workloads of the hot path, each timed the same way (one line, one key)
        subs = {}
        for wid in sorted(WORKLOADS):
            if wid != args.workload:
                subs[str(wid)] = bench_workload(wid, args, dev, peaks, measured, uuid, rank, world, full=False)

    if rank == 0:
        line = {
            "metric": METRIC, "value": main["value"], "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32",
            "data": "synthetic",
        }
        line.update({k: v for k, v in main.items() if k not in ("value", "ms_per_step")})
        line["peaks_measured"] = measured
        line["workloads"] = subs
        line["gradient_features"] = gradfeat
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- spectral-resolution sweep
# Fig. 1 of the paper: runtime of the functional-map solve against the number of
# eigenfunctions k for one shape pair. The paper's numbers for its batched PyTorch solver
# (another GPU; context, not a target), in ms.
PAPER_FIG1_MS = {20: 1.98, 30: 1.11, 40: 1.98, 50: 1.82, 60: 1.90, 70: 2.79, 80: 2.65, 90: 2.37, 100: 2.59,
                 110: 2.80, 120: 2.96, 130: 3.89, 140: 3.85, 150: 4.33, 160: 4.45, 170: 5.23, 180: 5.57,
                 190: 6.03, 200: 7.05, 210: 7.86, 220: 8.39, 230: 9.28, 240: 9.54, 250: 10.94, 260: 12.29,
                 270: 13.47, 280: 14.66, 290: 16.53, 300: 17.46}


def run_ksweep(args):
    """One pair per k (n = 5000 vertices per shape, d = 256 BF16 features, mask from the
    eigenvalues): the solve alone (Gram + row solves from resident A, B), the whole
    forward (projection + solve) and forward + loss + backward, each timed with CUDA
    events over `steps` launches after `warmup`; beside them the same solve written with
    plain PyTorch FP32 ops (G + lambda diag_embed(D), torch.linalg.solve) on this GPU."""
    import numpy as np
    import torch

    from paper_2604_10377_gb300 import api, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def time_ms(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    rows = []
    for k in sorted(PAPER_FIG1_MS):
        wl = synth.make_small(1000 + k, 1, (5000, 5000), [k], 256, feat_dtype="bf16", lam_range=(1e-3, 1e-3))
        b = api.batch_from_workload(wl, device=dev, with_grad=True)
        gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
        loss = torch.empty(1, device=dev)
        dc = torch.empty_like(b.C)
        a = b.project()

        def fwd_bwd():
            aa = b.project()
            cc = b.solve(aa)
            b.loss_orth(cc, gt, loss=loss, d_c=dc)
            b.solve_backward(dc, aa, cc)

        t_solve = time_ms(lambda: b.solve(a))
        t_fwd = time_ms(lambda: b.solve(b.project()))
        t_fb = time_ms(fwd_bwd)
        ax, ay = b.a_view(a, 0).clone(), b.a_view(a, 1).clone()
        lay = b.layout
        ex = b.evals[lay.evals_off[0]:lay.evals_off[0] + k]
        ey = b.evals[lay.evals_off[1]:lay.evals_off[1] + k]
        lam = float(np.float32(wl.pairs[0].lam))

        def torch_solve():
            g = ax @ ax.t()
            r = ay @ ax.t()
            sysm = g[None] + lam * torch.diag_embed((ey[:, None] - ex[None, :]) ** 2)
            return torch.linalg.solve(sysm, r.unsqueeze(-1)).squeeze(-1)

        t_torch = time_ms(torch_solve)
        c_ref = torch_solve()
        err = float((b.c_view(b.solve(a), 0) - c_ref).norm() / c_ref.norm())
        rows.append({"k": k, "solve_ms": t_solve, "fwd_ms": t_fwd, "fwd_bwd_ms": t_fb, "torch_solve_ms": t_torch,
                     "rel_diff_vs_torch_fp32": err, "paper_fig1_ms": PAPER_FIG1_MS[k]})
        b.close()
        del b
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "spectral resolution k (Fig. 1), one pair, n = 5000, d = 256 BF16",
                      "steps": args.steps, "warmup": args.warmup, "rows": rows,
                      "paper_fig1_ms": "the paper's batched PyTorch solver on its own GPU (context only)"}),
          flush=True)


def run_overlap(args):
    """Overlap-prediction metrics (IoU, balanced accuracy, ...) over 4096 segments with
    n log-uniform in [1k, 100k] vertices (the shape-size recipe of the ragged workload;
    ~0.45 GB of scores and labels, above L2), threshold 0.5, labels Bernoulli(r) with r
    uniform per segment. One JSON line: vertices/s and the HBM roofline of the count pass
    (5 bytes per vertex)."""
    import numpy as np
    import torch

    from paper_2604_10377_gb300 import api

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = load_peaks()
    rng = np.random.default_rng(20260410)
    lens = np.exp(rng.uniform(np.log(1000), np.log(100000), 4096)).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    scores = torch.rand(n, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    ratio = torch.from_numpy(np.repeat(rng.uniform(0.0, 1.0, len(lens)), lens).astype(np.float32)).to(dev)
    labels = (torch.rand(n, device=dev, generator=torch.Generator(device=dev).manual_seed(2)) < ratio).to(torch.uint8)
    del ratio
    for _ in range(max(3, args.warmup)):
        api.overlap_metrics(scores, labels, off)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        api.overlap_metrics(scores, labels, off)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    counts, metrics = api.overlap_metrics(scores, labels, off)
    torch.cuda.synchronize()
    assert int(counts.sum().item()) == n
    gbs = 5.0 * n / (ms * 1e-3) / 1e9
    line = {"metric": "overlap metrics (vertices/s)", "value": n / (ms * 1e-3), "unit": "vertices/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 scores, u8 labels, i64 counts, f64 metrics",
            "data": "synthetic",
            "config": {"workload": f"{len(lens)} segments, n log-uniform 1k-100k ({n} vertices), threshold 0.5",
                       "l2": "inputs larger than L2 (%.2f GB per pass)" % (5.0 * n / 1e9)},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                         "peak_source": "measured HBM copy bandwidth" if peaks["source"] == "measured" else "fallback"},
            "note": "per call: counts zeroed, one count launch over all segments, one metrics launch; the timed "
                    "region includes the host-to-device copy of the segment offsets made by api.overlap_metrics"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=4, choices=sorted(WORKLOADS))
    ap.add_argument("--ir-steps", type=int, default=1)
    ap.add_argument("--store-factors-max-k", type=int, default=304)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="end to end: upload then compute each step (no overlap of the next upload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-torch-compare", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time eager launches instead of one CUDA graph per step")
    ap.add_argument("--k-sweep", action="store_true", help="spectral-resolution sweep (Fig. 1) instead of the step")
    ap.add_argument("--overlap", action="store_true", help="overlap-prediction metrics instead of the step")
    ap.add_argument("--gradfeat", action="store_true",
                    help="spatial gradient features (DiffusionNet variants A and B) instead of the step")
    ap.add_argument("--copy-streams", type=int, default=4, help="side streams of the end-to-end host-to-device copies")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's built-in tiling choices")
    ap.add_argument("--tuning", default="",
                    help='fixed tuning knobs as JSON (fmap_options names, e.g. {"adjoint_kernel": 1}); no autotuner')
    ap.add_argument("--no-peaks", action="store_true", help="derive the FP32 peak instead of measuring it")
    ap.add_argument("--no-sub-workloads", action="store_true",
                    help="time only the main workload (not the other four as sub-results)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the oracle check of sampled pairs")
    ap.add_argument("--pairs", type=int, default=0,
                    help="first N pairs of the workload only (small cases for ncu captures; not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.overlap:
        run_overlap(args)
        return
    if args.gradfeat:
        import torch
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        measured = None if args.no_peaks else measure_peaks(dev)
        print(json.dumps(bench_gradient_features(args, dev, load_peaks(), measured, None)), flush=True)
        return
    if args.k_sweep:
        run_ksweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
