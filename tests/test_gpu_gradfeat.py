"""Spatial gradient features (fmap_gradient_features) against the FP64 oracle, on the GPU.

The kernel multiplies TF32 operands (x and y truncated by the MMA: relative error in
[0, 2^-10), mean 2^-11; the complex matrix rounded to TF32) with FP32 accumulation, so
the FP32 output carries ~6e-4 relative error (a common scale of the outputs, plus noise):
the tolerance is 1.5e-3. A BF16 output adds its own rounding (2^-9 at most): 3e-3, the
BF16 budget of the hot path.
"""
import numpy as np
import pytest

from oracle import fmap_oracle as orc
from paper_2604_10377_gb300 import synth
from _bridge import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1.5e-3, "bf16": 3e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    import os
    from paper_2604_10377_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _lib.lib()


def _dev(gi, ld_in=None):
    dim = gi.dim
    ld = ld_in or dim
    x = np.zeros((gi.n, ld), np.float32)
    x[:, :dim] = gi.feat
    vals = np.stack([gi.g_re, gi.g_im], axis=1).astype(np.float32)
    return (torch.from_numpy(gi.row_ptr).cuda(), torch.from_numpy(gi.col_idx).cuda(), torch.from_numpy(vals).cuda(),
            torch.from_numpy(x).cuda(), torch.from_numpy(gi.a_re).cuda(), torch.from_numpy(gi.a_im).cuda())


def _oracle(gi, variant, row_ptr=None, col_idx=None, g_re=None, g_im=None):
    x, y = orc.gradient_apply(gi.row_ptr if row_ptr is None else row_ptr, gi.col_idx if col_idx is None else col_idx,
                              gi.g_re if g_re is None else g_re, gi.g_im if g_im is None else g_im,
                              gi.feat.astype(np.float64))
    return orc.spatial_gradient_features(x, y, gi.a_re, gi.a_im, variant)


@pytest.mark.parametrize("n,dim", [(1, 16), (127, 48), (128, 64), (129, 128), (1000, 80), (5000, 128), (3001, 32)])
@pytest.mark.parametrize("variant", ["A", "B"])
@pytest.mark.parametrize("out_dtype", ["fp32", "bf16"])
def test_gradient_features_against_oracle(n, dim, variant, out_dtype):
    """Tiles of 128 vertices with ragged last tiles, every supported width class (one to
    eight vertices per warp pass in the gather, one to eight K-blocks), both variants,
    both output types."""
    from paper_2604_10377_gb300 import api
    gi = synth.make_gradient_input(100 + n + dim, n, dim)
    tdt = torch.bfloat16 if out_dtype == "bf16" else torch.float32
    out, status = api.gradient_features(*_dev(gi), variant=variant, out_dtype=tdt)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    err = rel_fro(out.float().cpu().numpy(), _oracle(gi, variant))
    assert err <= TOL[out_dtype], (n, dim, variant, out_dtype, err)


def test_gradient_features_long_and_empty_rows_and_wide_layouts():
    """Rows with no entry (g = 0), rows longer than a warp (40 entries), input rows wider
    than D and an output written into the first D columns of wider rows (the columns past
    D keep their values)."""
    from paper_2604_10377_gb300 import api
    rng = np.random.default_rng(5)
    n, dim = 300, 64
    lens = rng.integers(0, 9, n)
    lens[[3, 77, 200]] = 40
    lens[[0, 10, 299]] = 0
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    gi = synth.GradientInput(n=n, dim=dim, row_ptr=ptr, col_idx=col,
                             g_re=rng.standard_normal(len(col)).astype(np.float32),
                             g_im=rng.standard_normal(len(col)).astype(np.float32),
                             feat=rng.standard_normal((n, dim)).astype(np.float32),
                             a_re=(rng.standard_normal((dim, dim)) / 8).astype(np.float32),
                             a_im=(rng.standard_normal((dim, dim)) / 8).astype(np.float32))
    out = torch.full((n, dim + 24), 7.0, dtype=torch.float32, device="cuda")
    row_ptr, col_idx, vals, x, are, aim = _dev(gi, ld_in=dim + 12)
    _, status = api.gradient_features(row_ptr, col_idx, vals, x, are, aim, variant="A", out=out)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = out.cpu().numpy()
    assert np.all(got[:, dim:] == 7.0)
    ref = _oracle(gi, "A")
    assert np.all(got[lens == 0, :dim] == 0.0)
    assert rel_fro(got[:, :dim], ref) <= TOL["fp32"]


def test_tiles_of_long_rows_beside_short_ones():
    """Whole 128-vertex tiles of long rows (24 entries per row: three rounds of eight loads
    per lane; 16 per row: two) beside tiles of short rows, in one call, against the oracle."""
    from paper_2604_10377_gb300 import api
    rng = np.random.default_rng(6)
    n, dim = 600, 32
    lens = rng.integers(0, 9, n)
    lens[:128] = 24
    lens[300:428] = 16   # 2048 entries: exactly the slice
    ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(n, size=l, replace=False)) for l in lens]).astype(np.int32)
    gi = synth.GradientInput(n=n, dim=dim, row_ptr=ptr, col_idx=col,
                             g_re=rng.standard_normal(len(col)).astype(np.float32),
                             g_im=rng.standard_normal(len(col)).astype(np.float32),
                             feat=rng.standard_normal((n, dim)).astype(np.float32),
                             a_re=(rng.standard_normal((dim, dim)) / 6).astype(np.float32),
                             a_im=(rng.standard_normal((dim, dim)) / 6).astype(np.float32))
    row_ptr, col_idx, vals, x, are, aim = _dev(gi)
    for variant in ("A", "B"):
        out, status = api.gradient_features(row_ptr, col_idx, vals, x, are, aim, variant=variant)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert rel_fro(out.cpu().numpy(), _oracle(gi, variant)) <= TOL["fp32"], variant


def test_out_of_range_column_is_reported_and_skipped():
    """A column index past the input rows sets the status word to INVALID_ARG and the entry
    is skipped (the kernel checks every index before it loads)."""
    from paper_2604_10377_gb300 import _lib, api
    gi = synth.make_gradient_input(9, 500, 32)
    bad = gi.col_idx.copy()
    bad[17] = 10 ** 6
    row_ptr, _, vals, x, are, aim = _dev(gi)
    out, status = api.gradient_features(row_ptr, torch.from_numpy(bad).cuda(), vals, x, are, aim, variant="B")
    torch.cuda.synchronize()
    assert int(status.item()) == _lib.FMAP_ERR_INVALID_ARG
    gre = gi.g_re.copy(); gre[17] = 0.0
    gim = gi.g_im.copy(); gim[17] = 0.0
    ref = _oracle(gi, "B", g_re=gre, g_im=gim)
    assert rel_fro(out.cpu().numpy(), ref) <= TOL["fp32"]


def test_features_feed_the_projection_in_place():
    """The kernel writes BF16 features straight into a batch's flat feature buffer; the
    projection and solve that follow match the oracle run on those same BF16 values."""
    from paper_2604_10377_gb300 import api
    from _bridge import oracle_inputs
    wl = synth.make_small(61, 2, (2000, 6000), [30, 50], 128, feat_dtype="bf16")
    b = api.batch_from_workload(wl, with_grad=False)
    for s, sh in enumerate(wl.shapes):
        gi = synth.make_gradient_input(300 + s, sh.n, 128)
        view = b.layout.feat_view(b.feat, s)
        _, status = api.gradient_features(*_dev(gi), variant="A" if s % 2 == 0 else "B", out=view)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ref = _oracle(gi, "A" if s % 2 == 0 else "B")
        assert rel_fro(view.float().cpu().numpy(), ref) <= TOL["bf16"]
        sh.feat = view.view(torch.int16).cpu().numpy().view(np.uint16).reshape(sh.n, 128).copy()
    a = b.project()
    c = b.solve(a)
    torch.cuda.synchronize()
    shapes, pairs = oracle_inputs(wl)
    fwd = orc.forward_batch(shapes, pairs)
    for p in range(len(wl.pairs)):
        assert rel_fro(b.c_view(c, p).cpu().numpy(), fwd["C"][p]) <= 3e-3
