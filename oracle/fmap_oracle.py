"""FP64 CPU oracle for the functional-map hot path.

TEST INFRASTRUCTURE ONLY. This module is imported by the tests, by
``__graft_entry__.smoke()`` and by the ``cpu_baseline`` / reference leg of
``bench.py``, and by nothing else. The CUDA path never imports, links or calls
it, and it shares no code, table or helper with the CUDA path.

Everything is plain NumPy in float64, written from the paper (DeepShapeMatchingKit,
arXiv 2604.10377, Sec. 3.1 "Batched Functional Map Solver"):

* Eq. 1: spectral descriptors A = Phi_X^+ F_X, B = Phi_Y^+ F_Y. The paper writes the
  Moore-Penrose pseudo-inverse Phi^+; for a basis that is orthonormal in the mass inner
  product (Phi^T M Phi = I) the inverse used here is the M-weighted left inverse
  Phi^+ = Phi^T M, which satisfies Phi^+ Phi = I and equals the Euclidean pseudo-inverse
  when M is a multiple of the identity (both are pinned in the tests).
* Eq. 2: the energy ||C A - B||^2 + lambda ||C Delta_X - Delta_Y C||^2.
* Eq. 3: with Delta diagonal in its eigenbasis, the commutativity term is the
  entry-wise weight D_ij = (Lambda_Y(i) - Lambda_X(j))^2.
* Eq. 4: normal equations C A A^T + lambda (D o C) = B A^T.
* Eq. 5-7: row i of C solves (A A^T + lambda diag(D_i)) c_i = (B A^T)_i. C maps the
  k_X coefficients of shape X to the k_Y of shape Y (k_Y x k_X); the paper's shapes share
  k, and with k_X != k_Y the same equations give k_Y row systems of size k_X.
* Eq. 8-9: the rows are independent, so all of them are solved as one batch.
* The paper's lambda is one scalar. A weight per row of C (lambda_i, the regulariser
  sum_i lambda_i sum_j D_ij C_ij^2) keeps every row system separate: row i solves
  (A A^T + lambda_i diag(D_i)) c_i = (B A^T)_i; a scalar lambda is the case of equal
  weights.

The solve uses a Cholesky factorisation written out below (the row systems are
symmetric positive definite when A A^T or every lambda D_ij is positive). If a
pivot is not positive the oracle raises ``NotSPD``.

The backward pass (not in the paper) is the adjoint of Eq. 5 derived by hand:
gamma_i = S_i^{-1} dL/dc_i, dB = Gamma A, dA = Gamma^T B - (Gamma^T C + C^T Gamma) A,
dD = -lambda Gamma o C, dlambda = -sum(D o Gamma o C), dF = M Phi dA (with row weights,
dD_ij = -lambda_i Gamma_ij C_ij and dlambda_i = -sum_j D_ij Gamma_ij C_ij).

Spatial gradient features (Sec. "Learned Scaling and Rotation in DiffusionNet"): the
complex per-vertex gradients z = G X of features X under a sparse complex gradient
operator G, a learned complex D x D matrix A, and the real features g = Re(conj(z) o Az),
in the paper's real decomposition; variant A (rotation and isotropic scaling) and
variant B (the other indexing of the imaginary part: fixed +-45 degree rotations and
anisotropic scaling).

Overlap metrics (Sec. "Overlap Prediction Metrics"): confusion counts of a thresholded
per-vertex overlap prediction against binary labels, and IoU, accuracy, precision,
recall, specificity, F1 and balanced accuracy from them.

Parity pins: every function here is checked against something other than itself
in tests/test_oracle_pins.py (Kronecker k^2 x k^2 solve, lambda = 0 closed form,
identity case, energy minimality, exact rational solve, Moore-Penrose inverse,
finite differences, LAPACK; for the overlap metrics the paper's closed forms for the
Zeros / Ones / Random predictors and brute-force counting; for the spatial gradient
features the complex form Re(conj(z) o Az), the paper's per-channel 2 x 2 block sums by
brute force, the diagonal closed form s |z|^2 cos(theta), invariance under a global
rotation of the tangent frames (variant A only) and the dense operator product). No
function is "parity unpinned".
"""
from __future__ import annotations

import numpy as np


class NotSPD(ArithmeticError):
    def __init__(self, row, column):
        super().__init__(f"row system {row}: pivot {column} is not positive")
        self.row = row
        self.column = column


# --------------------------------------------------------------------------
# Eq. 1 — spectral projection
# --------------------------------------------------------------------------
def project(phi, mass, feat):
    """A = Phi^T diag(M) F (Eq. 1 with Phi^+ = Phi^T M). phi (n, k), mass (n,), feat (n, d)."""
    phi = np.asarray(phi, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    feat = np.asarray(feat, dtype=np.float64)
    return phi.T @ (mass[:, None] * feat)


def project_backward(phi, mass, d_a):
    """dL/dF = diag(M) Phi dL/dA (chain rule of Eq. 1)."""
    phi = np.asarray(phi, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    return mass[:, None] * (phi @ np.asarray(d_a, dtype=np.float64))


# --------------------------------------------------------------------------
# Eq. 3 / Eq. 4 — the penalty mask
# --------------------------------------------------------------------------
def mask_from_evals(evals_x, evals_y):
    """D_ij = (Lambda_Y(i) - Lambda_X(j))^2: row i indexes the target basis."""
    ex = np.asarray(evals_x, dtype=np.float64)
    ey = np.asarray(evals_y, dtype=np.float64)
    return (ey[:, None] - ex[None, :]) ** 2


# --------------------------------------------------------------------------
# Eq. 2 — the energy the map minimises
# --------------------------------------------------------------------------
def energy(c, a, b, evals_x, evals_y, lam):
    """||C A - B||_F^2 + lambda ||C Delta_X - Delta_Y C||_F^2 with Delta = diag(eigenvalues)."""
    c = np.asarray(c, dtype=np.float64)
    dx = np.diag(np.asarray(evals_x, dtype=np.float64))
    dy = np.diag(np.asarray(evals_y, dtype=np.float64))
    r = c @ a - b
    s = c @ dx - dy @ c
    return float(np.sum(r * r) + lam * np.sum(s * s))


# --------------------------------------------------------------------------
# Cholesky factorisation and triangular solves (batched over leading axes)
# --------------------------------------------------------------------------
def cholesky(s):
    """Lower L with L L^T = S for every matrix of the batch s (..., k, k).

    Column by column (Cholesky-Crout): L_jj = sqrt(S_jj - sum_{m<j} L_jm^2),
    L_ij = (S_ij - sum_{m<j} L_im L_jm) / L_jj for i > j.
    """
    s = np.asarray(s, dtype=np.float64)
    batch_shape = s.shape[:-2]
    k = s.shape[-1]
    sf = s.reshape((-1, k, k))
    l = np.zeros_like(sf)
    for j in range(k):
        lj = l[:, j, :j]                                   # (b, j)
        piv = sf[:, j, j] - np.einsum("bm,bm->b", lj, lj)
        bad = ~(piv > 0.0)
        if np.any(bad):
            raise NotSPD(int(np.argmax(bad)), j)
        ljj = np.sqrt(piv)
        l[:, j, j] = ljj
        if j + 1 < k:
            below = sf[:, j + 1:, j] - np.einsum("bim,bm->bi", l[:, j + 1:, :j], lj)
            l[:, j + 1:, j] = below / ljj[:, None]
    return l.reshape(batch_shape + (k, k))


def cholesky_solve(l, rhs):
    """x with (L L^T) x = rhs, batched: l (..., k, k), rhs (..., k)."""
    l = np.asarray(l, dtype=np.float64)
    rhs = np.asarray(rhs, dtype=np.float64)
    k = l.shape[-1]
    lf = l.reshape((-1, k, k))
    bf = rhs.reshape((-1, k))
    y = np.zeros_like(bf)
    for i in range(k):                      # L y = b
        y[:, i] = (bf[:, i] - np.einsum("bm,bm->b", lf[:, i, :i], y[:, :i])) / lf[:, i, i]
    x = np.zeros_like(bf)
    for i in range(k - 1, -1, -1):          # L^T x = y
        x[:, i] = (y[:, i] - np.einsum("bm,bm->b", lf[:, i + 1:, i], x[:, i + 1:])) / lf[:, i, i]
    return x.reshape(rhs.shape)


# --------------------------------------------------------------------------
# Eq. 4-9 — the row-wise (batched) regularised solve
# --------------------------------------------------------------------------
def _row_weights(lam, ky):
    """lambda as a column of k_Y row weights: a scalar (the paper's single weight) or one
    weight per row of C (the regulariser sum_i lambda_i sum_j D_ij C_ij^2)."""
    lam = np.asarray(lam, dtype=np.float64)
    if lam.ndim == 0:
        return lam
    if lam.shape != (ky,):
        raise ValueError("per-row lambda needs one weight per row of C")
    return lam.reshape((ky, 1))


def row_systems(a, d_mask, lam):
    """S_i = A A^T + lambda_i diag(D_i) for every row i of C, stacked as (k_Y, k_X, k_X)
    (Eq. 5, Eq. 8; lambda_i = lambda for the paper's single weight). A is k_X x d; D is
    k_Y x k_X, one row per row of C, so a map between bases of different sizes (C of
    k_Y x k_X) has k_Y systems of size k_X."""
    a = np.asarray(a, dtype=np.float64)
    d_mask = np.asarray(d_mask, dtype=np.float64)
    g = a @ a.T
    kx = g.shape[0]
    ky = d_mask.shape[0]
    s = np.broadcast_to(g, (ky, kx, kx)).copy()
    idx = np.arange(kx)
    s[:, idx, idx] += _row_weights(lam, ky) * d_mask
    return s


def solve(a, b, d_mask, lam, return_factors=False):
    """C minimising Eq. 2 (with Eq. 3's weights): row i solves Eq. 5."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = row_systems(a, d_mask, lam)
    r = b @ a.T                              # right-hand sides, row i = (B A^T)_i
    l = cholesky(s)
    c = cholesky_solve(l, r)
    return (c, l) if return_factors else c


def solve_backward(a, b, c, d_mask, lam, d_c, factors=None):
    """Adjoint of the row-wise solve. Returns dict(gamma, dA, dB, dD, dlam); with one
    lambda per row of C, dD = -lambda_i Gamma_ij C_ij and dlam is the vector of
    dL/dlambda_i = -sum_j D_ij Gamma_ij C_ij."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    d_mask = np.asarray(d_mask, dtype=np.float64)
    d_c = np.asarray(d_c, dtype=np.float64)
    l = factors if factors is not None else cholesky(row_systems(a, d_mask, lam))
    gamma = cholesky_solve(l, d_c)           # row i: S_i gamma_i = dL/dc_i
    w = gamma.T @ c + c.T @ gamma
    d_a = gamma.T @ b - w @ a
    d_b = gamma @ a
    wts = _row_weights(lam, c.shape[0])
    d_d = -wts * gamma * c
    if np.ndim(wts) == 0:
        d_lam = float(-np.sum(d_mask * gamma * c))
    else:
        d_lam = -np.sum(d_mask * gamma * c, axis=1)
    return dict(gamma=gamma, dA=d_a, dB=d_b, dD=d_d, dlam=d_lam)


# --------------------------------------------------------------------------
# Training loss used by the differentiable workloads
# --------------------------------------------------------------------------
def loss_orth_gt(c, c_gt):
    """L = ||C C^T - I||_F^2 + ||C - C_gt||_F^2 and dL/dC = 4 (C C^T - I) C + 2 (C - C_gt)."""
    c = np.asarray(c, dtype=np.float64)
    c_gt = np.asarray(c_gt, dtype=np.float64)
    e = c @ c.T - np.eye(c.shape[0])
    r = c - c_gt
    return float(np.sum(e * e) + np.sum(r * r)), 4.0 * e @ c + 2.0 * r


# --------------------------------------------------------------------------
# Whole batches: lists of shapes and pairs
# --------------------------------------------------------------------------
def pair_mask(shape_x, shape_y, explicit_mask=None):
    if explicit_mask is not None:
        return np.asarray(explicit_mask, dtype=np.float64)
    return mask_from_evals(shape_x["evals"], shape_y["evals"])


def pair_lambda(p):
    """The pair's weight: its per-row vector when given (lam_rows), else the scalar lam."""
    return p["lam_rows"] if p.get("lam_rows") is not None else p["lam"]


def forward_batch(shapes, pairs):
    """shapes: list of dict(phi, mass, feat, evals); pairs: list of dict(x, y, lam, mask)
    (optionally lam_rows: one weight per row of C, used instead of lam).

    Returns dict(A=[per shape], C=[per pair])."""
    a_list = [project(s["phi"], s["mass"], s["feat"]) for s in shapes]
    c_list = []
    for p in pairs:
        sx, sy = shapes[p["x"]], shapes[p["y"]]
        dm = pair_mask(sx, sy, p.get("mask"))
        c_list.append(solve(a_list[p["x"]], a_list[p["y"]], dm, pair_lambda(p)))
    return dict(A=a_list, C=c_list)


def backward_batch(shapes, pairs, fwd, d_c_list):
    """Gradients of sum_p <dC_p, C_p> w.r.t. every A and F (shapes may be shared by pairs)."""
    d_a = [np.zeros_like(a) for a in fwd["A"]]
    extra = []
    for p, dc in zip(pairs, d_c_list):
        sx, sy = shapes[p["x"]], shapes[p["y"]]
        dm = pair_mask(sx, sy, p.get("mask"))
        g = solve_backward(fwd["A"][p["x"]], fwd["A"][p["y"]], fwd["C"][len(extra)], dm, pair_lambda(p), dc)
        d_a[p["x"]] += g["dA"]
        d_a[p["y"]] += g["dB"]
        extra.append(g)
    d_f = [project_backward(s["phi"], s["mass"], da) for s, da in zip(shapes, d_a)]
    return dict(dA=d_a, dF=d_f, pair=extra)


# --------------------------------------------------------------------------
# Spatial gradient features (Sec. "Learned Scaling and Rotation in DiffusionNet")
# --------------------------------------------------------------------------
def gradient_apply(row_ptr, col_idx, g_re, g_im, feat):
    """z = G X for a sparse complex gradient operator G (CSR: row_ptr, col_idx, values
    g_re + i g_im) and real features X (n x D). Returns (x, y) = (Re z, Im z), each n x D:
    x_v = sum_u Re(G_vu) X_u, y_v = sum_u Im(G_vu) X_u."""
    import scipy.sparse as sp
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = len(row_ptr) - 1
    feat = np.asarray(feat, dtype=np.float64)
    gx = sp.csr_matrix((np.asarray(g_re, np.float64), np.asarray(col_idx), row_ptr), shape=(n, feat.shape[0]))
    gy = sp.csr_matrix((np.asarray(g_im, np.float64), np.asarray(col_idx), row_ptr), shape=(n, feat.shape[0]))
    return np.asarray(gx @ feat), np.asarray(gy @ feat)


def spatial_gradient_features(x, y, a_re, a_im, variant="A"):
    """g (n x D) from the per-vertex tangent vectors z = x + i y (rows of x, y) and the
    learned complex matrix A = a_re + i a_im (D x D, (Az)_i = sum_j A_ij z_j):
      (Az)_re = A_re x - A_im y,
      (Az)_im = A_re y + A_im x   (variant A)   or   A_re x + A_im y   (variant B),
      g = x o (Az)_re + y o (Az)_im."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    a_re = np.asarray(a_re, dtype=np.float64)
    a_im = np.asarray(a_im, dtype=np.float64)
    az_re = x @ a_re.T - y @ a_im.T
    if variant == "A":
        az_im = y @ a_re.T + x @ a_im.T
    elif variant == "B":
        az_im = x @ a_re.T + y @ a_im.T
    else:
        raise ValueError("variant must be 'A' or 'B'")
    return x * az_re + y * az_im


# --------------------------------------------------------------------------
# Overlap-prediction metrics (Sec. "Overlap Prediction Metrics")
# --------------------------------------------------------------------------
def overlap_counts(scores, labels, threshold=0.5):
    """(TP, FP, FN, TN) of one segment: a vertex is predicted overlapping when its FP32
    score exceeds the FP32 threshold, truly overlapping when its label is nonzero."""
    pred = np.asarray(scores, dtype=np.float32) > np.float32(threshold)
    lab = np.asarray(labels) != 0
    tp = int(np.count_nonzero(pred & lab))
    fp = int(np.count_nonzero(pred & ~lab))
    fn = int(np.count_nonzero(~pred & lab))
    tn = int(np.count_nonzero(~pred & ~lab))
    return tp, fp, fn, tn


def _ratio(num, den):
    return num / den if den > 0 else float("nan")


def overlap_metrics(tp, fp, fn, tn):
    """IoU, balanced accuracy, accuracy, precision, recall, specificity, F1 (FP64); a
    ratio with a zero denominator is NaN. Balanced accuracy is the mean of sensitivity
    TP/(TP+FN) and specificity TN/(TN+FP)."""
    tp, fp, fn, tn = float(tp), float(fp), float(fn), float(tn)
    recall = _ratio(tp, tp + fn)
    spec = _ratio(tn, tn + fp)
    return (_ratio(tp, tp + fp + fn), (recall + spec) * 0.5, _ratio(tp + tn, tp + fp + fn + tn),
            _ratio(tp, tp + fp), recall, spec, _ratio(2.0 * tp, 2.0 * tp + fp + fn))
