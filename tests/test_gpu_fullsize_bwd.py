"""Forward and backward at the full sizes of the differentiable workloads, against the
FP64 oracle (GPU).

* 8 pairs, n = 20k, k = 100, d = 384 BF16 (the differentiable workload): every pair's C,
  dA and dF (the BF16 gradient and its FP32 copy before rounding) against the oracle
  gradient, and directional derivatives against central finite differences (h = 1e-3)
  of the FP64 pipeline along seeded random directions.
* 4 pairs, n = 200k, k = 200, d = 512 BF16 (the large-spectrum workload) with the
  factors recomputed in the backward pass (none stored), as that workload runs; two of
  its pairs are recomputed by the oracle.
* The ragged 256-pair batch fwd + bwd; eight sampled pairs (two per k) recomputed by the
  oracle one by one.
Tolerances as in test_gpu_parity: C and the BF16 dF within 3e-3, the FP32 copy of dF
within 1e-3 (TF32 operands of the backward projection).
"""
import numpy as np
import pytest

from oracle import fmap_oracle as orc
from paper_2604_10377_gb300 import synth
from _bridge import oracle_inputs, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 3e-3
GTOL = 3e-3
GTOL_F32_COPY = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    import os
    from paper_2604_10377_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _lib.lib()


def _run_gpu(wl, **kw):
    """Whole batch: project, solve, training loss, backward (FP32 dF copy on)."""
    from paper_2604_10377_gb300 import api
    b = api.batch_from_workload(wl, with_grad=True, grad_f32_copy=True, **kw)
    a = b.project()
    c = b.solve(a)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    loss, dc = b.loss_orth(c, gt)
    b.solve_backward(dc, a, c)
    torch.cuda.synchronize()
    return b, a, c


def _oracle_pair(shapes, pr, c_gt):
    """Oracle fwd + loss + bwd of one pair whose shapes belong to no other pair."""
    sx, sy = shapes[pr["x"]], shapes[pr["y"]]
    ax = orc.project(sx["phi"], sx["mass"], sx["feat"])
    ay = orc.project(sy["phi"], sy["mass"], sy["feat"])
    dm = orc.pair_mask(sx, sy, pr.get("mask"))
    c = orc.solve(ax, ay, dm, pr["lam"])
    loss, dc = orc.loss_orth_gt(c, c_gt)
    g = orc.solve_backward(ax, ay, c, dm, pr["lam"], dc)
    dfx = orc.project_backward(sx["phi"], sx["mass"], g["dA"])
    dfy = orc.project_backward(sy["phi"], sy["mass"], g["dB"])
    return dict(c=c, loss=loss, dA=g["dA"], dB=g["dB"], dFx=dfx, dFy=dfy, dm=dm)


def _check_pair(b, c_flat, p, pr, ref):
    lay = b.layout
    assert rel_fro(b.c_view(c_flat, p).cpu().numpy(), ref["c"]) <= TOL
    for s, da, df in ((pr["x"], ref["dA"], ref["dFx"]), (pr["y"], ref["dB"], ref["dFy"])):
        assert rel_fro(b.a_view(b.dA, s).cpu().numpy(), da) <= GTOL
        f32 = lay.feat_view(b.dfeat32, s)
        e32 = rel_fro(f32.cpu().numpy(), df)
        assert e32 <= GTOL_F32_COPY, (p, s, e32)
        assert rel_fro(lay.feat_view(b.dfeat, s).float().cpu().numpy(), df) <= GTOL
        assert torch.equal(f32.to(torch.bfloat16).view(torch.int16), lay.feat_view(b.dfeat, s).view(torch.int16))


def test_differentiable_workload_full_size():
    """8 pairs, n = 20k, k = 100, d = 384 BF16: all pairs against the oracle gradient, and
    the GPU gradient's directional derivatives against central differences (h = 1e-3) of
    the FP64 pipeline. The oracle's own analytic gradient is pinned at this size too: to
    1e-5 of the h = 1e-3 difference (its O(h^2) truncation) and to 1e-8 of the Richardson
    extrapolation of the h and h/2 differences (O(h^4))."""
    wl = synth.make_config(2)
    b, a, c = _run_gpu(wl)
    assert np.all(b.status[:len(wl.pairs)].cpu().numpy() == 0)
    shapes, pairs = oracle_inputs(wl)
    refs = []
    for p, pr in enumerate(pairs):
        ref = _oracle_pair(shapes, pr, wl.pairs[p].c_gt)
        _check_pair(b, c, p, pr, ref)
        refs.append(ref)

    rng = np.random.default_rng(20260410)
    h = 1e-3
    for p in (0, 5):
        pr = pairs[p]
        for s, key in ((pr["x"], "dFx"), (pr["y"], "dFy")):
            g_gpu = b.layout.feat_view(b.dfeat32, s).cpu().numpy().astype(np.float64)
            g_ref = refs[p][key]
            for _ in range(3):
                v = rng.standard_normal(g_ref.shape)

                def loss_at(sign):
                    sh = [dict(x) for x in shapes]
                    sh[s] = dict(shapes[s], feat=shapes[s]["feat"] + sign * h * v)
                    ax = orc.project(sh[pr["x"]]["phi"], sh[pr["x"]]["mass"], sh[pr["x"]]["feat"])
                    ay = orc.project(sh[pr["y"]]["phi"], sh[pr["y"]]["mass"], sh[pr["y"]]["feat"])
                    cc = orc.solve(ax, ay, refs[p]["dm"], pr["lam"])
                    return orc.loss_orth_gt(cc, wl.pairs[p].c_gt)[0]

                fd = (loss_at(1.0) - loss_at(-1.0)) / (2 * h)
                fd_half = (loss_at(0.5) - loss_at(-0.5)) / h
                fd_rich = (4.0 * fd_half - fd) / 3.0
                an_ref = float(np.sum(g_ref * v))
                an_gpu = float(np.sum(g_gpu * v))
                scale = max(abs(fd), float(np.linalg.norm(g_ref)))
                assert abs(an_ref - fd) <= 1e-5 * scale, (p, s, an_ref, fd)
                assert abs(an_ref - fd_rich) <= 1e-8 * scale, (p, s, an_ref, fd_rich)
                assert abs(an_gpu - fd) <= GTOL_F32_COPY * scale, (p, s, an_gpu, fd)


def test_large_spectrum_workload_recomputed_factors():
    """4 pairs, n = 200k, k = 200, d = 512 BF16, double-float Gram, no stored factors (the
    backward pass refactors every row system): pairs 0 and 3 against the oracle."""
    wl = synth.make_config(3)
    b, a, c = _run_gpu(wl, store_factors_max_k=0)
    assert b.saved is None or b.sizes.saved_bytes == 0
    assert np.all(b.status[:len(wl.pairs)].cpu().numpy() == 0)
    shapes, pairs = oracle_inputs(wl)
    for p in (0, 3):
        _check_pair(b, c, p, pairs[p], _oracle_pair(shapes, pairs[p], wl.pairs[p].c_gt))


def test_ragged_batch_sampled_pairs_backward():
    """The ragged 256-pair batch, fwd + loss + bwd on the GPU; two pairs of every k
    recomputed by the oracle (C, dA, dF and its FP32 copy)."""
    wl = synth.make_config(4)
    b, a, c = _run_gpu(wl)
    assert np.all(b.status[:len(wl.pairs)].cpu().numpy() == 0)
    shapes, pairs = oracle_inputs(wl)
    ks = wl.k_of_pair
    for kk in (30, 50, 100, 200):
        for p in [q for q in range(len(ks)) if ks[q] == kk][:2]:
            _check_pair(b, c, p, pairs[p], _oracle_pair(shapes, pairs[p], wl.pairs[p].c_gt))
