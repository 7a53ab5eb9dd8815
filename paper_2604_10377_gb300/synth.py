"""Seeded synthetic inputs for the functional-map hot path.

This module only draws inputs; it contains none of the functional-map arithmetic
(no projection, no Gram matrix, no solve). Both the FP64 oracle and the CUDA path
are fed from it, so that they see bit-identical inputs.

Recipe (one generator per shape and one per batch, NumPy PCG64):

* ``seed(shape) = 20260410 + 1000*config + 2*pair + side`` (side 0 = source X,
  side 1 = target Y); ``seed(batch) = 20260410 + 1000*config + 999`` drives the
  per-pair spectral size k and weight lambda, drawn pair by pair in that order;
  ``seed(gt) = 20260410 + 1000*config + 500 + pair`` draws the target map C_gt.
* A shape draws, in order: n (log-uniform, when the config gives a range), the
  basis Phi (n x k Gaussian, FP64), the lumped mass M (uniform in [0.5, 1.5]/n),
  k eigenvalues (uniform in [0, 100], sorted ascending) and the features F
  (n x d, N(0, 1), FP32; rounded to BF16 for the BF16 configs).
* Phi is made M-orthonormal (Phi^T M Phi = I) by two passes of Cholesky-QR in
  the M inner product, in FP64, then stored as FP32. The stored FP32 values are
  the input of both sides.

The shapes stand in for the meshes of the paper's benchmarks (FAUST, SCAPE,
SMAL, ...), which are not used here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20260410

# Sizes of the five workloads of the functional-map hot path.
CONFIGS = {
    # single pair, plain forward, FP32 features
    0: dict(pairs=1, n=(5000, 5000), k=(30,), d=128, feat="fp32", lam=("fixed", 1e-3)),
    # 32 pairs, ragged n, FP32 features
    1: dict(pairs=32, n=(5000, 50000), k=(50,), d=256, feat="fp32", lam=("logu", 1e-4, 1e-1)),
    # differentiable, 8 pairs, BF16 features
    2: dict(pairs=8, n=(20000, 20000), k=(100,), d=384, feat="bf16", lam=("fixed", 1e-3)),
    # large spectrum, 4 pairs, BF16 features
    3: dict(pairs=4, n=(200000, 200000), k=(200,), d=512, feat="bf16", lam=("fixed", 1e-3)),
    # ragged mixed batch, 256 pairs, mixed k, BF16 features
    4: dict(pairs=256, n=(1000, 100000), k=(30, 50, 100, 200), d=256, feat="bf16",
            lam=("fixed", 1e-3)),
}


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round FP32 to BF16 (round to nearest even); returns the uint16 bit patterns."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((b >> 16) & 1) + np.uint32(0x7FFF)
    return ((b + r) >> 16).astype(np.uint16)


def bf16_bits_to_f32(u: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(u, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


@dataclasses.dataclass
class Shape:
    n: int
    k: int
    d: int
    phi: np.ndarray        # (n, k) float32, M-orthonormal up to FP32 rounding
    mass: np.ndarray       # (n,) float32
    evals: np.ndarray      # (k,) float32, ascending
    feat: np.ndarray       # (n, d) float32, or uint16 BF16 bit patterns
    feat_dtype: str        # "fp32" or "bf16"

    def feat_f64(self) -> np.ndarray:
        if self.feat_dtype == "bf16":
            return bf16_bits_to_f32(self.feat).astype(np.float64)
        return self.feat.astype(np.float64)


@dataclasses.dataclass
class Pair:
    x: int                  # index of the source shape
    y: int                  # index of the target shape
    lam: float              # stored as FP32 on both sides
    mask: Optional[np.ndarray] = None   # (k, k) float32 or None: use eigenvalues
    c_gt: Optional[np.ndarray] = None   # (k, k) float32 target map for the training loss
    lam_rows: Optional[np.ndarray] = None   # (k_Y,) float32 weight per row of C, or None: lam


@dataclasses.dataclass
class Workload:
    name: str
    shapes: List[Shape]
    pairs: List[Pair]
    feat_dtype: str

    @property
    def k_of_pair(self):
        return [self.shapes[p.x].k for p in self.pairs]


def _loguniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def m_orthonormalize(phi: np.ndarray, mass: np.ndarray, passes: int = 2) -> np.ndarray:
    """Cholesky-QR in the M inner product (input preparation, FP64)."""
    phi = np.array(phi, dtype=np.float64, copy=True)
    for _ in range(passes):
        s = phi.T @ (mass[:, None] * phi)
        l = np.linalg.cholesky(s)
        # phi <- phi L^{-T}
        phi = np.linalg.solve(l, phi.T).T
    return phi


def _draw_n(rng, n_range) -> int:
    lo, hi = n_range
    return lo if lo == hi else int(round(_loguniform(rng, lo, hi)))


def make_shape(seed: int, n_range, k: int, d: int, feat_dtype: str) -> Shape:
    rng = np.random.Generator(np.random.PCG64(seed))
    n = _draw_n(rng, n_range)
    phi = rng.standard_normal((n, k))
    mass = rng.uniform(0.5, 1.5, n) / n
    evals = np.sort(rng.uniform(0.0, 100.0, k))
    feat = rng.standard_normal((n, d), dtype=np.float32)
    phi = m_orthonormalize(phi, mass)
    if feat_dtype == "bf16":
        feat = f32_to_bf16_bits(feat)
    return Shape(n=n, k=k, d=d, phi=phi.astype(np.float32), mass=mass.astype(np.float32),
                 evals=evals.astype(np.float32), feat=feat, feat_dtype=feat_dtype)


def random_orthogonal(seed: int, k: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    q, r = np.linalg.qr(rng.standard_normal((k, k)))
    q = q * np.sign(np.diag(r))[None, :]
    return q.astype(np.float32)


def _config_draws(config: int, replica: int):
    cfg = CONFIGS[config]
    base = BASE_SEED + 1000000 * replica
    brng = np.random.Generator(np.random.PCG64(base + 1000 * config + 999))
    ks, lams = [], []
    for _ in range(cfg["pairs"]):
        kk = cfg["k"]
        ks.append(int(kk[0]) if len(kk) == 1 else int(kk[int(brng.integers(0, len(kk)))]))
        lam = cfg["lam"]
        lams.append(float(np.float32(lam[1] if lam[0] == "fixed" else _loguniform(brng, lam[1], lam[2]))))
    return cfg, base, ks, lams


def config_sizes(config: int, replica: int = 0):
    """(n_x, n_y, k) of every pair of workload `config`, drawn exactly as make_config draws
    them but without the arrays (for planning work, e.g. sharing pairs among processes)."""
    cfg, base, ks, _ = _config_draws(config, replica)
    out = []
    for p in range(cfg["pairs"]):
        ns = [_draw_n(np.random.Generator(np.random.PCG64(base + 1000 * config + 2 * p + side)), cfg["n"])
              for side in (0, 1)]
        out.append((ns[0], ns[1], ks[p]))
    return out


def make_config(config: int, pairs: Optional[Sequence[int]] = None, n_scale: float = 1.0,
                with_gt: bool = True, replica: int = 0) -> Workload:
    """Draw workload `config` (0..4). `pairs` selects a subset of pair indices
    (each pair's draws do not depend on the others, so a subset is identical to
    the same pairs of the full batch). `n_scale` < 1 shrinks every n for quick
    tests (the draws are otherwise unchanged). `replica` r > 0 draws an
    independent batch of the same recipe (all seeds shifted by 10^6 r), one per
    GPU when pairs are sharded over several GPUs."""
    cfg, base, ks, lams = _config_draws(config, replica)
    npairs = cfg["pairs"]
    sel = list(range(npairs)) if pairs is None else list(pairs)
    shapes: List[Shape] = []
    plist: List[Pair] = []
    lo, hi = cfg["n"]
    n_range = (max(8, int(lo * n_scale)), max(8, int(hi * n_scale)))
    for p in sel:
        sx = make_shape(base + 1000 * config + 2 * p + 0, n_range, ks[p], cfg["d"], cfg["feat"])
        sy = make_shape(base + 1000 * config + 2 * p + 1, n_range, ks[p], cfg["d"], cfg["feat"])
        shapes += [sx, sy]
        gt = random_orthogonal(base + 1000 * config + 500 + p, ks[p]) if with_gt else None
        plist.append(Pair(x=len(shapes) - 2, y=len(shapes) - 1, lam=lams[p], c_gt=gt))
    return Workload(name=f"config{config}", shapes=shapes, pairs=plist, feat_dtype=cfg["feat"])


def make_small(seed: int, npairs: int, n_range, ks, d: int, feat_dtype: str = "fp32",
               lam_range=(1e-4, 1e-1), identity: bool = False, with_mask: bool = False) -> Workload:
    """Small ragged batches for parity tests: n drawn log-uniform in n_range, k
    cycling through `ks`. identity=True makes each target a copy of its source
    (same basis, mass, eigenvalues and features), so the mask has a zero diagonal.
    with_mask=True gives every pair an explicit positive random mask instead of
    eigenvalues."""
    brng = np.random.Generator(np.random.PCG64(seed))
    shapes: List[Shape] = []
    pairs: List[Pair] = []
    for p in range(npairs):
        k = int(ks[p % len(ks)])
        lam = float(np.float32(_loguniform(brng, *lam_range)))
        sx = make_shape(seed * 7919 + 2 * p, n_range, k, d, feat_dtype)
        if identity:
            sy = dataclasses.replace(sx)
        else:
            sy = make_shape(seed * 7919 + 2 * p + 1, n_range, k, d, feat_dtype)
        shapes += [sx, sy]
        mask = None
        if with_mask:
            mask = brng.uniform(0.0, 50.0, (k, k)).astype(np.float32)
        gt = random_orthogonal(seed * 7919 + 100003 + p, k)
        pairs.append(Pair(x=len(shapes) - 2, y=len(shapes) - 1, lam=lam, mask=mask, c_gt=gt))
    return Workload(name=f"small{seed}", shapes=shapes, pairs=pairs, feat_dtype=feat_dtype)


# ---------------------------------------------------------------- spatial gradient inputs
@dataclasses.dataclass
class GradientInput:
    """Inputs of the spatial-gradient feature kernel for one shape: a sparse complex
    gradient operator in CSR form (n x n, values g_re + i g_im), FP32 features X (n x D)
    and a learned complex D x D matrix A = a_re + i a_im."""
    n: int
    dim: int
    row_ptr: np.ndarray    # (n + 1,) int64
    col_idx: np.ndarray    # (nnz,) int32, sorted within each row
    g_re: np.ndarray       # (nnz,) float32
    g_im: np.ndarray       # (nnz,) float32
    feat: np.ndarray       # (n, D) float32
    a_re: np.ndarray       # (D, D) float32
    a_im: np.ndarray       # (D, D) float32


def make_gradient_input(seed: int, n: int, dim: int, nbrs: int = 6, window: int = 64) -> GradientInput:
    """A random stand-in for a mesh gradient operator: every vertex has itself and up to
    `nbrs` distinct other vertices within +-`window` indices (the locality of a vertex
    ordering along a mesh; offsets that fall outside [0, n) are dropped), off-diagonal
    complex values N(0, 1) / sqrt(nbrs), and a diagonal value that makes every row sum to
    zero (the gradient of a constant field vanishes). X is N(0, 1); A has N(0, 1 / D)
    entries."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = np.concatenate([np.arange(-window, 0), np.arange(1, window + 1)])
    k = min(nbrs, len(pool))
    pick = np.argsort(rng.random((n, len(pool))), axis=1)[:, :k]
    cols = np.arange(n)[:, None] + pool[pick]
    cols = np.concatenate([cols, np.arange(n)[:, None]], axis=1)          # the vertex itself last
    valid = (cols >= 0) & (cols < n)
    cols = np.where(valid, cols, n)                                       # invalid entries sort to the end
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, axis=1)
    valid = np.take_along_axis(valid, order, axis=1)
    counts = valid.sum(axis=1)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    col = cols[valid].astype(np.int32)
    nnz = len(col)
    re = rng.standard_normal(nnz) / np.sqrt(max(nbrs, 1))
    im = rng.standard_normal(nnz) / np.sqrt(max(nbrs, 1))
    row = np.repeat(np.arange(n), counts)
    diag = col == row
    re[diag] = 0.0
    im[diag] = 0.0
    re[diag] = -np.bincount(row, weights=re, minlength=n)
    im[diag] = -np.bincount(row, weights=im, minlength=n)
    feat = rng.standard_normal((n, dim), dtype=np.float32)
    a_re = (rng.standard_normal((dim, dim)) / np.sqrt(dim)).astype(np.float32)
    a_im = (rng.standard_normal((dim, dim)) / np.sqrt(dim)).astype(np.float32)
    return GradientInput(n=n, dim=dim, row_ptr=ptr, col_idx=col, g_re=re.astype(np.float32),
                         g_im=im.astype(np.float32), feat=feat, a_re=a_re, a_im=a_im)
