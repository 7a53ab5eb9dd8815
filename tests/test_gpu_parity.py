"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the GPU.

Tolerances (relative Frobenius error per shape / pair):
  FP32 features: A, C within 1e-5; dL/dF within 1e-4.
  BF16 features: A, C within 3e-3; dL/dF (stored in BF16) within 3e-3; the FP32 copy of
  dL/dF taken before that rounding within GTOL_F32_COPY = 1e-3.
"""
import dataclasses

import numpy as np
import pytest

from oracle import fmap_oracle as orc
from paper_2604_10377_gb300 import synth
from _bridge import gpu_forward, oracle_inputs, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16": 3e-3}
GTOL = {"fp32": 1e-4, "bf16": 3e-3}
# BF16 batches, dL/dF before its BF16 rounding: the backward projection multiplies TF32
# operands (Phi truncated by the MMA, relative error in [0, 2^-10) with mean 2^-11 ~ 4.9e-4,
# a common scale of every output; dA rounded to TF32 when its image is built, ~2^-12 on
# average) after the adjoint's own FP32 error (~1e-4): about 6e-4 expected.
GTOL_F32_COPY = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    import os
    from paper_2604_10377_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _lib.lib()


def _check_forward(wl, tol=None, **kw):
    tol = tol or TOL[wl.feat_dtype]
    b, a_gpu, c_gpu, status = gpu_forward(wl, **kw)
    shapes, pairs = oracle_inputs(wl)
    ref = orc.forward_batch(shapes, pairs)
    assert np.all(status == 0), status
    ea = [rel_fro(x, r) for x, r in zip(a_gpu, ref["A"])]
    ec = [rel_fro(x, r) for x, r in zip(c_gpu, ref["C"])]
    assert max(ea) <= tol, ea
    assert max(ec) <= tol, ec
    return b, ea, ec


def _shape(rng, n, k, d, feat_dtype="fp32", orthonormal=False):
    phi = rng.standard_normal((n, k))
    mass = rng.uniform(0.5, 1.5, n) / n
    if orthonormal:
        phi = synth.m_orthonormalize(phi, mass)
    else:
        phi = phi / np.sqrt(n * mass.mean())
    feat = rng.standard_normal((n, d), dtype=np.float32)
    if feat_dtype == "bf16":
        feat = synth.f32_to_bf16_bits(feat)
    return synth.Shape(n=n, k=k, d=d, phi=phi.astype(np.float32), mass=mass.astype(np.float32),
                       evals=np.sort(rng.uniform(0, 100, k)).astype(np.float32), feat=feat, feat_dtype=feat_dtype)


# ------------------------------------------------------------------ forward
@pytest.mark.parametrize("feat_dtype", ["fp32", "bf16"])
def test_small_ragged_batch(feat_dtype):
    """Several tiles and ragged tails in every dimension: n across chunk edges, k not a
    multiple of the tile, mixed k in one batch."""
    wl = synth.make_small(1, 6, (300, 9000), [3, 17, 30, 50, 64, 100], 256, feat_dtype=feat_dtype)
    _check_forward(wl)


def test_edge_sizes():
    """n = 1 and n just past a chunk edge, k = 1 and k = 256, d = 16 and a large d
    (d >= 2k throughout, so that the FP32 solve is well conditioned)."""
    rng = np.random.default_rng(5)
    shapes = [
        _shape(rng, 1, 1, 16), _shape(rng, 1, 1, 16),
        _shape(rng, 4097, 256, 512), _shape(rng, 4095, 256, 512),
        _shape(rng, 129, 5, 1040), _shape(rng, 64, 5, 1040),
        _shape(rng, 8193, 8, 16), _shape(rng, 333, 8, 16),
    ]
    pairs = [synth.Pair(x=0, y=1, lam=0.5), synth.Pair(x=2, y=3, lam=1e-3),
             synth.Pair(x=4, y=5, lam=1e-2), synth.Pair(x=6, y=7, lam=1e-1)]
    wl = synth.Workload("edges", shapes, pairs, "fp32")
    _check_forward(wl)


def test_identity_case_gives_identity():
    wl = synth.make_small(2, 3, (2000, 6000), [30, 50, 100], 256, identity=True)
    b, a_gpu, c_gpu, status = gpu_forward(wl)
    for c in c_gpu:
        assert rel_fro(c, np.eye(c.shape[0])) < 1e-5


def test_explicit_mask():
    wl = synth.make_small(3, 4, (500, 3000), [8, 40], 128, with_mask=True)
    _check_forward(wl)


def test_shared_shape_and_self_pair():
    """A shape used by several pairs, and a pair mapping a shape onto itself."""
    rng = np.random.default_rng(11)
    shapes = [_shape(rng, 700, 20, 64, orthonormal=True) for _ in range(3)]
    pairs = [synth.Pair(0, 1, 1e-3), synth.Pair(1, 2, 1e-2), synth.Pair(2, 0, 1e-1), synth.Pair(1, 1, 1e-3)]
    _check_forward(synth.Workload("shared", shapes, pairs, "fp32"))


def test_not_spd_reports_row_and_nan():
    """A negative mask entry makes row system 3 of pair 1 indefinite: status NOT_SPD | 3 << 8,
    its row of C is NaN, and the other pair is unaffected."""
    wl = synth.make_small(4, 2, (400, 800), [10], 32, with_mask=True)
    wl.pairs[1].mask[3, 4] = -1e9
    b, a_gpu, c_gpu, status = gpu_forward(wl)
    assert status[0] == 0
    assert status[1] == (4 | (3 << 8)), hex(int(status[1]))
    assert np.all(np.isnan(c_gpu[1][3]))
    assert np.all(np.isfinite(np.delete(c_gpu[1], 3, axis=0)))
    shapes, pairs = oracle_inputs(wl)
    ref = orc.forward_batch(shapes, pairs[:1])
    assert rel_fro(c_gpu[0], ref["C"][0]) < 1e-5


def test_not_spd_in_a_256_thread_system():
    """A row system of the 256-thread class (k = 150) meets an indefinite pivot in a late
    panel (mask entry 140 of row system 5 of pair 1): status NOT_SPD | 5 << 8, that row of
    C is NaN, the other rows and pair 0 match the oracle."""
    wl = synth.make_small(5, 2, (3000, 3500), [150], 448, with_mask=True)
    shapes, pairs = oracle_inputs(wl)
    ref = orc.forward_batch(shapes, pairs)   # row systems other than 5 do not see its mask entry
    wl.pairs[1].mask[5, 140] = -1e12
    b, a_gpu, c_gpu, status = gpu_forward(wl)
    assert status[0] == 0
    assert status[1] == (4 | (5 << 8)), hex(int(status[1]))
    assert np.all(np.isnan(c_gpu[1][5]))
    assert rel_fro(c_gpu[0], ref["C"][0]) < 1e-5
    assert rel_fro(np.delete(c_gpu[1], 5, axis=0), np.delete(ref["C"][1], 5, axis=0)) < 1e-5


def test_empty_batch():
    from paper_2604_10377_gb300 import api
    lay = api.BatchLayout([100], [10], [16], "fp32")
    b = api.FmapBatch(lay, [], with_grad=True)
    b.project(); b.solve(); b.solve_backward(torch.zeros(1, device="cuda"))
    torch.cuda.synchronize()


def test_ir_steps_and_hi_gram():
    """FP64 Gram (hi_gram_min_k low) and 0..2 refinement steps all meet the FP32 tolerance."""
    wl = synth.make_small(6, 3, (1000, 4000), [20, 60, 120], 256)
    for ir in (0, 1, 2):
        _check_forward(wl, ir_steps=ir, hi_gram_min_k=50)


@pytest.mark.parametrize("ks,hi_min,ir", [((129, 150, 199), 200, 1), ((150, 256), 1000, 2), ((136, 256), 1000, 0)])
def test_refinement_with_fp32_gram_from_global(ks, hi_min, ir):
    """Row systems above the shared-memory copy of G (k > 128) with the FP32 Gram: the
    refinement residual reads the lower triangle of G from global memory, for one and two
    refinement steps (d >= 2k, well-conditioned FP32 systems); forward only (no saved
    factors)."""
    rng = np.random.default_rng(17)
    shapes, pairs = [], []
    for i, k in enumerate(ks):
        shapes += [_shape(rng, 3000 + 7 * i, k, 512), _shape(rng, 2500 + 5 * i, k, 512)]
        pairs.append(synth.Pair(x=2 * i, y=2 * i + 1, lam=1e-2))
    wl = synth.Workload("gram_global", shapes, pairs, "fp32")
    _check_forward(wl, ir_steps=ir, hi_gram_min_k=hi_min, with_grad=False)


@pytest.mark.parametrize("feat_dtype,hi_min", [("fp32", 1000), ("fp32", 150), ("bf16", 200)])
def test_row_solve_sizes_129_to_200(feat_dtype, hi_min):
    """Row systems of the 256-thread launches (128 < k <= 200) at sizes where the trailing
    update's tile counts change shape (k = 129: one padded row past a block; 144, 152, 184,
    200), with the FP32 and the double-float Gram, forward against the oracle at the
    mode's tolerance (d = 448, well-conditioned systems)."""
    rng = np.random.default_rng(23)
    shapes, pairs = [], []
    for i, k in enumerate((129, 144, 152, 184, 200)):
        shapes += [_shape(rng, 2600 + 9 * i, k, 448, feat_dtype), _shape(rng, 2400 + 7 * i, k, 448, feat_dtype)]
        pairs.append(synth.Pair(x=2 * i, y=2 * i + 1, lam=1e-3))
    wl = synth.Workload("tc_trailing", shapes, pairs, feat_dtype)
    _check_forward(wl, hi_gram_min_k=hi_min)


@pytest.mark.parametrize("ir", [1, 2])
def test_refinement_residual_without_the_shared_memory_copy_of_g(ir):
    """Row systems of k <= 128 with solve_no_g_copy = 1: the refinement residual reads G from
    L2 instead of a shared-memory copy; forward against the oracle at the FP32 tolerance."""
    wl = synth.make_small(19, 4, (1000, 6000), [20, 60, 100, 128], 320)
    _check_forward(wl, ir_steps=ir, tuning={"solve_no_g_copy": 1})


def test_bitwise_reproducible():
    wl = synth.make_small(7, 3, (3000, 20000), [30, 64, 100], 64)
    from paper_2604_10377_gb300 import api
    b = api.batch_from_workload(wl)
    a1 = b.project().clone(); c1 = b.solve(a1).clone()
    a2 = b.project().clone(); c2 = b.solve(a2).clone()
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(c1, c2)


# ------------------------------------------------------------------ backward
def _gpu_backward(wl, use_saved=True, **kw):
    from paper_2604_10377_gb300 import api
    b = api.batch_from_workload(wl, with_grad=True, **kw)
    a = b.project()
    c = b.solve(a)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    loss, dc = b.loss_orth(c, gt)
    d_mask = torch.empty_like(c)
    d_lam = torch.empty(len(wl.pairs), device=b.device)
    b.solve_backward(dc, a, c, use_saved=use_saved, d_mask=d_mask, d_lambda=d_lam)
    torch.cuda.synchronize()
    out = dict(
        loss=loss[:len(wl.pairs)].cpu().numpy(),
        dC=[b.c_view(dc, p).cpu().numpy() for p in range(len(wl.pairs))],
        dA=[b.a_view(b.dA, s).cpu().numpy() for s in range(len(wl.shapes))],
        dF=[b.layout.feat_view(b.dfeat, s).float().cpu().numpy() for s in range(len(wl.shapes))],
        dD=[b.c_view(d_mask, p).cpu().numpy() for p in range(len(wl.pairs))],
        dlam=d_lam.cpu().numpy(),
        C=[b.c_view(c, p).cpu().numpy() for p in range(len(wl.pairs))],
        status=b.status[:len(wl.pairs)].cpu().numpy(),
        dlam_rows=[None if b.dlam_rows_view(p) is None else b.dlam_rows_view(p).cpu().numpy()
                   for p in range(len(wl.pairs))],
    )
    if b.dfeat32 is not None:
        out["dF32"] = [b.layout.feat_view(b.dfeat32, s).cpu().numpy() for s in range(len(wl.shapes))]
        # the BF16 gradient is the round-to-nearest-even of the FP32 copy, bit for bit
        out["bf16_is_rounded_copy"] = all(
            torch.equal(b.layout.feat_view(b.dfeat32, s).to(torch.bfloat16).view(torch.int16),
                        b.layout.feat_view(b.dfeat, s).view(torch.int16)) for s in range(len(wl.shapes)))
    return out


def _oracle_backward(wl):
    shapes, pairs = oracle_inputs(wl)
    fwd = orc.forward_batch(shapes, pairs)
    losses, dcs = [], []
    for c, p in zip(fwd["C"], wl.pairs):
        l, dc = orc.loss_orth_gt(c, p.c_gt)
        losses.append(l); dcs.append(dc)
    g = orc.backward_batch(shapes, pairs, fwd, dcs)
    return shapes, pairs, fwd, losses, dcs, g


@pytest.mark.parametrize("feat_dtype,use_saved", [("fp32", True), ("fp32", False), ("bf16", True)])
def test_rectangular_maps(feat_dtype, use_saved):
    """Pairs whose bases differ in size (C is k_Y x k_X: k_Y row systems of size k_X):
    k_Y above and below k_X, system sizes on both sides of the 64/128/256 block classes,
    the double-float Gram (k_X >= 200), an explicit k_Y x k_X mask, a shape shared by a
    rectangular and a square pair. Forward and backward against the oracle."""
    rng = np.random.default_rng(29)
    ks = [30, 50, 60, 20, 130, 100, 210, 70, 40]
    shapes = [_shape(rng, 600 + 37 * i, k, 448, feat_dtype) for i, k in enumerate(ks)]
    pairs = [synth.Pair(x=0, y=1, lam=1e-2), synth.Pair(x=2, y=3, lam=1e-3), synth.Pair(x=4, y=5, lam=1e-2),
             synth.Pair(x=6, y=7, lam=1e-3), synth.Pair(x=1, y=8, lam=1e-2), synth.Pair(x=8, y=8, lam=1e-2)]
    mrng = np.random.default_rng(3)
    pairs[1].mask = mrng.uniform(0.0, 50.0, (ks[3], ks[2])).astype(np.float32)
    for i, p in enumerate(pairs):
        p.c_gt = (mrng.standard_normal((ks[p.y], ks[p.x])) / np.sqrt(ks[p.x])).astype(np.float32)
    wl = synth.Workload("rect", shapes, pairs, feat_dtype)
    out = _gpu_backward(wl, use_saved=use_saved)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    tol, gtol = TOL[feat_dtype], GTOL[feat_dtype]
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert out["C"][p].shape == (ks[wl.pairs[p].y], ks[wl.pairs[p].x])
        assert rel_fro(out["C"][p], fwd["C"][p]) <= tol
        assert abs(out["loss"][p] - losses[p]) <= tol * max(1.0, abs(losses[p]))
        assert rel_fro(out["dD"][p], g["pair"][p]["dD"]) <= gtol
        assert abs(out["dlam"][p] - g["pair"][p]["dlam"]) <= gtol * max(1.0, abs(g["pair"][p]["dlam"]))
    for s_ in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s_], g["dA"][s_]) <= gtol
        assert rel_fro(out["dF"][s_], g["dF"][s_]) <= gtol


@pytest.mark.parametrize("feat_dtype,use_saved", [("fp32", True), ("fp32", False), ("bf16", True)])
def test_row_weights(feat_dtype, use_saved):
    """A weight per row of C (lambda_rows: row i solves (G + lambda_i diag(D_i)) c_i = R_i):
    square and rectangular pairs with row weights beside pairs with a scalar lambda, one
    with an explicit mask, k across the 64 / 128 / 256-thread row-solve classes; C, dA, dF,
    dD, the per-pair dlambda (the sum over rows) and dL/dlambda_i per row against the
    oracle."""
    rng = np.random.default_rng(47)
    ks = [40, 40, 90, 60, 150, 150, 20, 30]
    shapes = [_shape(rng, 900 + 31 * i, k, 320, feat_dtype) for i, k in enumerate(ks)]
    wr = np.random.default_rng(9)
    pairs = [synth.Pair(x=0, y=1, lam=1e-2, lam_rows=wr.uniform(1e-3, 5e-2, ks[1]).astype(np.float32)),
             synth.Pair(x=2, y=3, lam=1e-3, lam_rows=wr.uniform(1e-4, 1e-2, ks[3]).astype(np.float32)),
             synth.Pair(x=4, y=5, lam=1e-2),
             synth.Pair(x=4, y=5, lam=1e-2, lam_rows=wr.uniform(1e-3, 3e-2, ks[5]).astype(np.float32)),
             synth.Pair(x=6, y=7, lam=1e-2, lam_rows=wr.uniform(1e-3, 3e-2, ks[7]).astype(np.float32))]
    pairs[4].mask = wr.uniform(0.0, 40.0, (ks[7], ks[6])).astype(np.float32)
    for p in pairs:
        p.c_gt = (wr.standard_normal((ks[p.y], ks[p.x])) / np.sqrt(ks[p.x])).astype(np.float32)
    wl = synth.Workload("row_weights", shapes, pairs, feat_dtype)
    out = _gpu_backward(wl, use_saved=use_saved)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    tol, gtol = TOL[feat_dtype], GTOL[feat_dtype]
    assert np.all(out["status"] == 0)
    for p, pr in enumerate(wl.pairs):
        assert rel_fro(out["C"][p], fwd["C"][p]) <= tol
        assert rel_fro(out["dD"][p], g["pair"][p]["dD"]) <= gtol
        dl = g["pair"][p]["dlam"]
        if pr.lam_rows is None:
            assert out["dlam_rows"][p] is None
            assert abs(out["dlam"][p] - dl) <= gtol * max(1.0, abs(dl))
        else:
            assert rel_fro(out["dlam_rows"][p], dl) <= gtol
            assert abs(out["dlam"][p] - np.sum(dl)) <= gtol * max(1.0, np.sum(np.abs(dl)))
    for s_ in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s_], g["dA"][s_]) <= gtol
        assert rel_fro(out["dF"][s_], g["dF"][s_]) <= gtol


@pytest.mark.parametrize("use_saved,adj_ir", [(True, 0), (False, 0), (True, 1), (False, 1)])
@pytest.mark.parametrize("ks", [(129, 136), (160, 200), (231, 256)])
def test_backward_256_thread_class(ks, use_saved, adj_ir):
    """Backward through row systems of 128 < k <= 256: the adjoint solves on saved factors,
    or refactoring in the adjoint pass, with and without adjoint refinement; FP32 and
    double-float Gram sizes; dA, dF, dD against the oracle."""
    rng = np.random.default_rng(31)
    shapes, pairs = [], []
    for i, k in enumerate(ks):
        shapes += [_shape(rng, 1800 + 13 * i, k, 512), _shape(rng, 1700 + 11 * i, k, 512)]
        pairs.append(synth.Pair(x=2 * i, y=2 * i + 1, lam=1e-2, c_gt=synth.random_orthogonal(60 + i, k)))
    wl = synth.Workload("bwd_256", shapes, pairs, "fp32")
    out = _gpu_backward(wl, use_saved=use_saved, adjoint_ir_steps=adj_ir)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert rel_fro(out["C"][p], fwd["C"][p]) <= TOL["fp32"]
        assert rel_fro(out["dD"][p], g["pair"][p]["dD"]) <= GTOL["fp32"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= GTOL["fp32"]
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["fp32"]


@pytest.mark.parametrize("use_saved,adj_ir", [(True, 1), (False, 1), (True, 2)])
def test_backward_with_adjoint_refinement(use_saved, adj_ir):
    """Refinement steps in the adjoint row solves (off by default): k below and above the
    shared-memory Gram copy, FP32 and double-float Gram, saved or recomputed factors."""
    rng = np.random.default_rng(23)
    shapes, pairs = [], []
    for i, k in enumerate((60, 150, 210)):
        shapes += [_shape(rng, 2000 + 11 * i, k, 448), _shape(rng, 1800 + 13 * i, k, 448)]
        pairs.append(synth.Pair(x=2 * i, y=2 * i + 1, lam=1e-2,
                                c_gt=synth.random_orthogonal(40 + i, k)))
    wl = synth.Workload("adj_ir", shapes, pairs, "fp32")
    out = _gpu_backward(wl, use_saved=use_saved, adjoint_ir_steps=adj_ir)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert rel_fro(out["C"][p], fwd["C"][p]) <= TOL["fp32"]
        assert rel_fro(out["dD"][p], g["pair"][p]["dD"]) <= GTOL["fp32"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= GTOL["fp32"]
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["fp32"]


@pytest.mark.parametrize("feat_dtype,use_saved", [("fp32", True), ("fp32", False), ("bf16", True)])
def test_backward_against_oracle(feat_dtype, use_saved):
    wl = synth.make_small(8, 4, (500, 6000), [12, 30, 64, 100], 256, feat_dtype=feat_dtype)
    out = _gpu_backward(wl, use_saved=use_saved)
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    tol, gtol = TOL[feat_dtype], GTOL[feat_dtype]
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert abs(out["loss"][p] - losses[p]) <= tol * max(1.0, abs(losses[p]))
        assert rel_fro(out["dC"][p], dcs[p]) <= 10 * tol
        assert rel_fro(out["dD"][p], g["pair"][p]["dD"]) <= gtol
        assert abs(out["dlam"][p] - g["pair"][p]["dlam"]) <= gtol * max(1.0, abs(g["pair"][p]["dlam"]))
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= gtol
        assert rel_fro(out["dF"][s], g["dF"][s]) <= gtol


@pytest.mark.parametrize("d,ks", [(16, [4, 8]), (64, [20, 30]), (384, [64, 100]), (256, [200, 230])])
def test_backward_fp32_feature_groups(d, ks):
    """FP32 backward projection on the tensor cores (three TF32 passes): feature groups of
    64 (32 when the basis needs more than six 32-blocks), partial last groups, vertex
    counts ending inside a tile; gradients within the FP32-mode tolerance."""
    wl = synth.make_small(15, 2 * len(ks), (260, 3000), ks, d, feat_dtype="fp32")
    out = _gpu_backward(wl)
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["fp32"]


@pytest.mark.parametrize("d", [16, 48, 384, 640])
def test_backward_bf16_feature_groups(d):
    """BF16 backward projection with feature counts that leave the second group of a
    cluster empty (16), uneven (48), split into four groups (384) or into six (640),
    and vertex counts that end inside the second 64-row half of a tile."""
    wl = synth.make_small(11, 4, (66, 3000), [7, 30, 64, 64], d, feat_dtype="bf16")
    out = _gpu_backward(wl)
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= GTOL["bf16"]
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["bf16"]


@pytest.mark.parametrize("d,ks,n_range", [(16, [7, 12], (66, 3000)), (48, [7, 30], (66, 3000)),
                                         (256, [30, 100, 200], (300, 5000)), (384, [100, 200], (300, 5000))])
def test_backward_bf16_fp32_copy(d, ks, n_range):
    """The BF16 backward projection checked before its rounding: the optional FP32 copy of
    dL/dF against the oracle gradient within GTOL_F32_COPY, and the BF16 gradient equal to
    the round-to-nearest-even of that copy bit for bit. k on both sides of the 32-blocks of
    the basis, up to the double-float Gram (k = 200); one or two feature groups per CTA pair
    (d = 16 leaves the second group empty); vertex counts ending inside a tile (n >= k, as
    the M-orthonormal basis needs)."""
    wl = synth.make_small(21, 2 * len(ks), n_range, ks, d, feat_dtype="bf16")
    out = _gpu_backward(wl, grad_f32_copy=True)
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    assert out["bf16_is_rounded_copy"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dF32"][s], g["dF"][s]) <= GTOL_F32_COPY, (s, rel_fro(out["dF32"][s], g["dF"][s]))
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["bf16"]


@pytest.mark.parametrize("feat_dtype", ["fp32", "bf16"])
def test_split_backward_and_projection_cta_counts(feat_dtype):
    """fmap_adjoint followed by fmap_project_backward writes the same dL/dA and dL/dF as
    fmap_solve_backward, bit for bit; with the projections on fewer persistent CTAs
    (proj_ctas = 48, bwd_ctas = 38) A, C and dL/dF still match the oracle."""
    import torch
    from paper_2604_10377_gb300 import api
    wl = synth.make_small(33, 4, (700, 9000), [30, 64, 100, 200], 256, feat_dtype=feat_dtype)
    b = api.batch_from_workload(wl, with_grad=True)
    a = b.project(); c = b.solve(a)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    _, dc = b.loss_orth(c, gt)
    da1 = b.solve_backward(dc, a, c).clone(); df1 = b.dfeat.clone()
    b.dfeat.zero_()
    da2 = b.adjoint(dc, a, c, d_a=torch.empty_like(da1))
    b.project_backward(da2)
    torch.cuda.synchronize()
    assert torch.equal(da1, da2) and torch.equal(df1, b.dfeat)

    b2 = api.batch_from_workload(wl, with_grad=True, tuning={"proj_ctas": 48, "bwd_ctas": 38})
    a2 = b2.project(); c2 = b2.solve(a2)
    _, dc2 = b2.loss_orth(c2, api.flat_c(b2, [p.c_gt for p in wl.pairs]))
    b2.solve_backward(dc2, a2, c2)
    torch.cuda.synchronize()
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    tol, gtol = TOL[feat_dtype], GTOL[feat_dtype]
    assert np.all(b2.status[:len(wl.pairs)].cpu().numpy() == 0)
    for s in range(len(wl.shapes)):
        assert rel_fro(b2.a_view(a2, s).cpu().numpy(), fwd["A"][s]) <= tol
        dfs = b2.layout.feat_view(b2.dfeat, s).float().cpu().numpy()
        assert rel_fro(dfs, g["dF"][s]) <= gtol
    for p in range(len(wl.pairs)):
        assert rel_fro(b2.c_view(c2, p).cpu().numpy(), fwd["C"][p]) <= tol


@pytest.mark.parametrize("feat_dtype,use_saved", [("fp32", True), ("bf16", True), ("bf16", False)])
def test_large_spectral_sizes(feat_dtype, use_saved):
    """k above 256 up to the 304 limit: the tensor-core projection splits the basis into
    two ranges, the solve runs 320-thread blocks with one system per SM; forward and
    backward (saved or recomputed factors) against the oracle."""
    wl = synth.make_small(12, 3, (400, 1500), [257, 300, 304], 320, feat_dtype=feat_dtype)
    out = _gpu_backward(wl, use_saved=use_saved)
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    tol, gtol = TOL[feat_dtype], GTOL[feat_dtype]
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert rel_fro(out["C"][p], fwd["C"][p]) <= tol
        assert abs(out["loss"][p] - losses[p]) <= tol * max(1.0, abs(losses[p]))
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= gtol
        assert rel_fro(out["dF"][s], g["dF"][s]) <= gtol


@pytest.mark.parametrize("tuning", [{"adjoint_kernel": 1, "adjoint_stages": 1, "adjoint_features": 256},
                                    {"adjoint_kernel": 1, "adjoint_stages": 2, "adjoint_features": 256},
                                    {"adjoint_kernel": 1, "adjoint_stages": 1, "adjoint_features": 128},
                                    {"adjoint_kernel": 1, "adjoint_stages": 2, "adjoint_features": 64},
                                    {"adjoint_kernel": 1}, {"adjoint_kernel": 2}])
@pytest.mark.parametrize("d", [16, 272, 448])
def test_adjoint_gemm_kernels(tuning, d):
    """dA_x = Gamma^T A_y - W A_x and dA_y = Gamma A_x on the tensor cores (one or two
    shared-memory stages, 64 to 256 columns per CTA) and on the CUDA cores, W = Gamma^T C +
    C^T Gamma with them (the tensor-core kernel's first launch): square and
    rectangular pairs with k from 3 to 304 (one to three 128-row tiles, reductions
    k_Y + k_X up to 608 with ragged 32-wide tails), d of one partial feature tile (16), a
    full and a 16-wide one (272) and a full and a 192-wide one (448); dA against the
    oracle, and each tensor-core variant against the CUDA-core kernel at the FP32
    accumulation level. k stays at or below d so that every Gram matrix has full rank."""
    rng = np.random.default_rng(41)
    ks = {16: [5, 8, 12, 16, 3, 10, 7, 14], 272: [5, 33, 129, 260, 270, 96, 200, 257],
          448: [5, 33, 129, 300, 304, 96, 200, 257]}[d]
    shapes = [_shape(rng, 500 + 41 * i, k, d) for i, k in enumerate(ks)]
    pairs = [synth.Pair(x=0, y=1, lam=1e-2), synth.Pair(x=3, y=4, lam=1e-3), synth.Pair(x=2, y=5, lam=1e-2),
             synth.Pair(x=6, y=7, lam=1e-3), synth.Pair(x=7, y=2, lam=1e-2), synth.Pair(x=4, y=4, lam=1e-2)]
    mrng = np.random.default_rng(5)
    for p in pairs:
        p.c_gt = (mrng.standard_normal((ks[p.y], ks[p.x])) / np.sqrt(ks[p.x])).astype(np.float32)
    wl = synth.Workload("adjoint_gemm", shapes, pairs, "fp32")
    out = _gpu_backward(wl, tuning=tuning)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    # the training loss and dL/dC run on the same kernel (E = C C^T - I, then 4 E C + 2 (C - C_gt));
    # odd k put the pairs' dL/dC at offsets that are not 16-byte aligned
    for p in range(len(wl.pairs)):
        assert abs(out["loss"][p] - losses[p]) <= TOL["fp32"] * max(1.0, abs(losses[p]))
        assert rel_fro(out["dC"][p], dcs[p]) <= 10 * TOL["fp32"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= GTOL["fp32"]
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["fp32"]
    if tuning.get("adjoint_kernel") != 2:
        # two FP32-class accumulations of sums of length up to k_Y + k_X = 608 differ by a few
        # 2^-24 sqrt(K) ~ 1.5e-6 relative per element, more where Gamma^T A_y and W A_x cancel
        ref = _gpu_backward(wl, tuning={"adjoint_kernel": 2})
        for s in range(len(wl.shapes)):
            assert rel_fro(out["dA"][s], ref["dA"][s]) <= 1e-5


def test_adjoint_default_on_a_batch_that_fills_the_sms():
    """160 pairs (k = 30, d = 256: 320 dA_x tiles of 128 columns, two per SM on 152 SMs):
    the built-in choice runs the adjoint GEMMs and the training loss's GEMMs on the tensor
    cores; the loss, dC, dA and dF against the oracle, and dA against the FP32 FMA tiles."""
    wl = synth.make_small(43, 160, (300, 600), [30], 256)
    out = _gpu_backward(wl)
    shapes_o, pairs_o, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert abs(out["loss"][p] - losses[p]) <= TOL["fp32"] * max(1.0, abs(losses[p]))
        assert rel_fro(out["dC"][p], dcs[p]) <= 10 * TOL["fp32"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], g["dA"][s]) <= GTOL["fp32"]
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["fp32"]
    ref = _gpu_backward(wl, tuning={"adjoint_kernel": 2})
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dA"][s], ref["dA"][s]) <= 1e-5


def test_timeout_after_the_row_solves_reaches_every_pair():
    """A bounded wait that gave up after the row solves (adjoint GEMMs, backward projection)
    leaves FMAP_ERR_TIMEOUT in the workspace's control word; the backward entry points turn
    it into every pair's status. The failure is made on the host: the test writes the code
    into the control word (no GPU wait runs out), and a clean control word leaves the status
    at 0."""
    from paper_2604_10377_gb300 import _lib, api
    wl = synth.make_small(51, 3, (500, 1500), [20, 40, 70], 64, feat_dtype="bf16")
    b = api.batch_from_workload(wl, with_grad=True)
    a = b.project(); c = b.solve(a)
    dc = torch.randn_like(c) * 1e-3
    b.adjoint(dc, a, c)
    b.status.zero_()
    b.project_backward()
    torch.cuda.synchronize()
    assert np.all(b.status[:3].cpu().numpy() == 0)
    b.ws[:4].view(torch.int32).fill_(_lib.FMAP_ERR_TIMEOUT)
    b.status.zero_()
    b.status[1] = _lib.FMAP_ERR_NOT_SPD | (2 << 8)   # an earlier error is kept
    b.project_backward()
    torch.cuda.synchronize()
    st = b.status[:3].cpu().numpy()
    assert st[0] == _lib.FMAP_ERR_TIMEOUT and st[2] == _lib.FMAP_ERR_TIMEOUT
    assert st[1] == _lib.FMAP_ERR_NOT_SPD | (2 << 8)
    b.ws[:256].zero_()


def _tuning_cases():
    from paper_2604_10377_gb300.autotune import CANDIDATES
    return [(knob, v) for knob, vals in CANDIDATES.items() for v in vals if v != 0]


@pytest.mark.parametrize("knob,value", _tuning_cases())
def test_every_tuning_candidate_matches_the_oracle(knob, value):
    """Each value the autotuner may pick re-plans the launches without changing the
    results beyond the order of partial sums: forward and backward stay within tolerance."""
    wl = synth.make_small(13, 4, (300, 9000), [30, 64, 100, 128], 256, feat_dtype="bf16")
    out = _gpu_backward(wl, tuning={knob: value})
    shapes, pairs, fwd, losses, dcs, g = _oracle_backward(wl)
    assert np.all(out["status"] == 0)
    for p in range(len(wl.pairs)):
        assert rel_fro(out["C"][p], fwd["C"][p]) <= TOL["bf16"]
    for s in range(len(wl.shapes)):
        assert rel_fro(out["dF"][s], g["dF"][s]) <= GTOL["bf16"]


def test_autotune_picks_a_candidate_and_keeps_results():
    from paper_2604_10377_gb300 import api, autotune
    wl = synth.make_small(14, 6, (2000, 30000), [30, 50, 100], 256, feat_dtype="bf16")
    b = api.batch_from_workload(wl, with_grad=True)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    loss = torch.empty(len(wl.pairs), device=b.device)
    dc = torch.empty_like(b.C)

    def step():
        a = b.project()
        c = b.solve(a)
        b.loss_orth(c, gt, loss=loss, d_c=dc)
        b.solve_backward(dc, a, c)

    res = autotune.autotune(b, step, iters=1, reps=1)
    for knob in autotune.CANDIDATES:
        assert res["tuning"][knob] in autotune.CANDIDATES[knob]
    assert res["ms"] <= res["baseline_ms"]
    step()
    torch.cuda.synchronize()
    shapes, pairs = oracle_inputs(wl)
    fwd = orc.forward_batch(shapes, pairs)
    for p in range(len(wl.pairs)):
        assert rel_fro(b.c_view(b.C, p).cpu().numpy(), fwd["C"][p]) <= TOL["bf16"]


def test_gradient_against_finite_differences():
    """GPU dL/dF (FP32 mode) against central differences (h = 1e-3) of the FP64
    pipeline along 8 seeded random directions per shape."""
    wl = synth.make_small(9, 2, (300, 900), [10, 24], 64)
    out = _gpu_backward(wl)
    shapes, pairs, *_ = _oracle_backward(wl)
    gts = [p.c_gt for p in wl.pairs]

    def total_loss(sh):
        f = orc.forward_batch(sh, pairs)
        return sum(orc.loss_orth_gt(c, gt)[0] for c, gt in zip(f["C"], gts))

    rng = np.random.default_rng(0)
    h = 1e-3
    for s in range(len(shapes)):
        for _ in range(8):
            v = rng.standard_normal(shapes[s]["feat"].shape)
            sp = [dict(x) for x in shapes]; sp[s] = dict(shapes[s], feat=shapes[s]["feat"] + h * v)
            sm = [dict(x) for x in shapes]; sm[s] = dict(shapes[s], feat=shapes[s]["feat"] - h * v)
            fd = (total_loss(sp) - total_loss(sm)) / (2 * h)
            an = float(np.sum(out["dF"][s].astype(np.float64) * v))
            assert abs(an - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.linalg.norm(v)), (s, an, fd)


def test_autograd_function():
    from paper_2604_10377_gb300 import api
    wl = synth.make_small(10, 2, (400, 1200), [16], 32)
    b = api.batch_from_workload(wl, with_grad=True)
    feat = b.feat.clone().requires_grad_(True)
    c = api.FmapFunction.apply(feat, b)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    loss = 0
    for p in range(len(wl.pairs)):
        cp, gp = b.c_view(c, p), b.c_view(gt, p)
        e = cp @ cp.T - torch.eye(cp.shape[0], device=cp.device)
        loss = loss + (e * e).sum() + ((cp - gp) ** 2).sum()
    loss.backward()
    _, _, _, _, _, g = _oracle_backward(wl)
    for s in range(len(wl.shapes)):
        grad = b.layout.feat_view(feat.grad, s).cpu().numpy()
        assert rel_fro(grad, g["dF"][s]) <= 1e-4


# ------------------------------------------------------------------ full-size workloads
@pytest.mark.parametrize("config", [0, 1, 2])
def test_config_full_size(config):
    wl = synth.make_config(config)
    _check_forward(wl)


def test_config3_full_size():
    wl = synth.make_config(3)
    _check_forward(wl, hi_gram_min_k=200, store_factors_max_k=0)


def test_config4_sampled_pairs():
    """The 256-pair ragged batch runs whole on the GPU; 8 sampled pairs (covering every k)
    are recomputed by the oracle one by one."""
    wl = synth.make_config(4)
    b, a_gpu, c_gpu, status = gpu_forward(wl)
    assert np.all(status == 0)
    ks = wl.k_of_pair
    sample = []
    for kk in (30, 50, 100, 200):
        idx = [p for p in range(len(ks)) if ks[p] == kk]
        sample += idx[:2]
    shapes, pairs = oracle_inputs(wl)
    for p in sample:
        pr = pairs[p]
        sx, sy = shapes[pr["x"]], shapes[pr["y"]]
        ax = orc.project(sx["phi"], sx["mass"], sx["feat"])
        ay = orc.project(sy["phi"], sy["mass"], sy["feat"])
        c = orc.solve(ax, ay, orc.mask_from_evals(sx["evals"], sy["evals"]), pr["lam"])
        assert rel_fro(a_gpu[pr["x"]], ax) <= TOL["bf16"]
        assert rel_fro(c_gpu[p], c) <= TOL["bf16"], (p, ks[p])


def test_upload_pipeline_steps_match_serial_steps():
    """api.UploadPipeline (two input buffers, the next upload on a copy stream) gives every
    step exactly the results of the same step run serially; each step's inputs differ, so
    a step that computed on the wrong buffer would show."""
    from paper_2604_10377_gb300 import api
    wl = synth.make_small(31, 4, (2000, 20000), [30, 50], 64, feat_dtype="fp32")
    lay = api.BatchLayout([s.n for s in wl.shapes], [s.k for s in wl.shapes], [s.d for s in wl.shapes], "fp32")
    pairs = [(p.x, p.y, p.lam) for p in wl.pairs]
    base = lay.pack_host(wl.shapes)
    hosts = []
    for s in range(4):
        h = dict(base)
        h["feat"] = (base["feat"] * np.float32(1.0 + 0.25 * s)).astype(np.float32)
        hosts.append({k: api.host_to_torch(v).pin_memory() for k, v in h.items()})

    def mk():
        return api.FmapBatch(lay, pairs, device="cuda:0", precision="fp32", with_grad=True)

    def compute(bb):
        a = bb.project()
        c = bb.solve(a)
        dc = torch.ones_like(c)
        bb.solve_backward(dc, a, c)
        return c.clone(), bb.dfeat.clone()

    ref = mk()
    want = []
    for h in hosts:
        ref.upload(h)
        want.append(compute(ref))
    torch.cuda.synchronize()

    pipe = api.UploadPipeline([mk(), mk()])
    with pytest.raises(RuntimeError):
        pipe.acquire()
    with pytest.raises(RuntimeError):
        pipe.release()
    got = []
    pipe.prefetch(hosts[0])
    for s in range(len(hosts)):
        j = pipe.acquire()
        if s + 1 < len(hosts):
            pipe.prefetch(hosts[s + 1])
        got.append(compute(pipe.batches[j]))
        pipe.release()
    torch.cuda.synchronize()
    for (c, df), (c_ref, df_ref) in zip(got, want):
        assert torch.equal(c, c_ref)
        assert torch.equal(df, df_ref)
    assert not torch.equal(want[0][0], want[1][0])
    pipe.prefetch(hosts[0])
    pipe.prefetch(hosts[1])
    with pytest.raises(RuntimeError):
        pipe.prefetch(hosts[2])


def test_overlap_metrics_against_oracle():
    """Overlap counts (exact) and metrics (FP64, bitwise) per segment against the oracle:
    empty and one-vertex segments, lengths around the 4096-vertex block chunk, a long
    segment, scores equal to the threshold and NaN scores, overlap ratios from 0 to 1."""
    from paper_2604_10377_gb300 import api
    rng = np.random.default_rng(41)
    lens = [0, 1, 5, 4095, 4096, 4097, 250000, 33, 1000, 1000, 12288]
    ratios = [0.5, 0.3, 0.0, 0.02, 0.5, 0.98, 0.25, 1.0, 0.5, 0.0, 0.7]
    scores, labels = [], []
    for n, r in zip(lens, ratios):
        sc = rng.uniform(0, 1, n).astype(np.float32)
        if n > 10:
            sc[rng.integers(n, size=3)] = np.float32(0.25)
            sc[rng.integers(n, size=2)] = np.nan
        scores.append(sc)
        labels.append((rng.uniform(0, 1, n) < r).astype(np.uint8))
    scores[9][:] = 0.0                       # no predicted and no true positives: NaN ratios
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    s_all, l_all = np.concatenate(scores), np.concatenate(labels)
    counts, metrics = api.overlap_metrics(torch.from_numpy(s_all).cuda(), torch.from_numpy(l_all).cuda(), off,
                                          threshold=0.25)
    counts, metrics = counts.cpu().numpy(), metrics.cpu().numpy()
    for i in range(len(lens)):
        c = orc.overlap_counts(s_all[off[i]:off[i + 1]], l_all[off[i]:off[i + 1]], threshold=0.25)
        assert tuple(int(x) for x in counts[i]) == c, (i, counts[i], c)
        m = np.array(orc.overlap_metrics(*c))
        assert np.array_equal(np.isnan(m), np.isnan(metrics[i])), (i, m, metrics[i])
        ok = ~np.isnan(m)
        assert np.array_equal(m[ok], metrics[i][ok]), (i, m, metrics[i])
    c0, m0 = api.overlap_metrics(torch.from_numpy(s_all).cuda(), torch.from_numpy(l_all).cuda(), [0], 0.5)
    assert c0.shape == (0, 4) and m0.shape == (0, 7)
