"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports every
symbol include/*.h declares, and validates / plans batches on the host."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_10377_gb300 import _lib, build
    build.build()
    return _lib.lib()


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"^FMAP_API\s+[\w\s\*]+?\b(fmap_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ("fmap_project", "fmap_solve", "fmap_solve_backward", "fmap_batch_create", "fmap_create"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a():
    from paper_2604_10377_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_version_and_errors(lib):
    from paper_2604_10377_gb300 import _lib
    assert b"sm_103a" in lib.fmap_version()
    assert _lib.error_string(_lib.FMAP_ERR_NOT_SPD) == "row system not positive definite"
    assert _lib.error_string(_lib.FMAP_ERR_NOT_SPD | (7 << 8)) == "row system not positive definite"


def _descs(specs, pairs):
    from paper_2604_10377_gb300 import _lib
    sd = (_lib.ShapeDesc * max(1, len(specs)))()
    for i, sp in enumerate(specs):
        n, k, d = sp["n"], sp["k"], sp["d"]
        sd[i].n, sd[i].k, sd[i].d = n, k, d
        sd[i].phi = sp.get("phi", 0x10000)
        sd[i].ld_phi = sp.get("ld_phi", (k + 3) // 4 * 4)
        sd[i].mass = 0x20000
        sd[i].evals = sp.get("evals", 0x30000)
        sd[i].feat = sp.get("feat", 0x40000)
        sd[i].ld_feat = sp.get("ld_feat", d)
        sd[i].dfeat = None
    pd = (_lib.PairDesc * max(1, len(pairs)))()
    for i, (x, y, lam) in enumerate(pairs):
        pd[i].shape_x, pd[i].shape_y, pd[i].lam = x, y, lam
        pd[i].mask = None
    return sd, pd


def _plan(lib, specs, pairs, opt=None):
    from paper_2604_10377_gb300 import _lib
    sd, pd = _descs(specs, pairs)
    sz = _lib.Sizes()
    rc = lib.fmap_plan_sizes(None if opt is None else ctypes.byref(opt), sd, len(specs), pd, len(pairs),
                             ctypes.byref(sz))
    return rc, sz


def test_plan_sizes(lib):
    specs = [dict(n=5000, k=30, d=128), dict(n=7000, k=30, d=128), dict(n=100, k=200, d=512), dict(n=90, k=200, d=512)]
    rc, sz = _plan(lib, specs, [(0, 1, 1e-3), (2, 3, 1e-3), (1, 0, 0.0)])
    assert rc == 0
    assert sz.a_floats == 2 * 30 * 128 + 2 * 200 * 512
    assert sz.c_floats == 30 * 30 * 2 + 200 * 200
    assert sz.n_pairs == 3 and sz.n_shapes == 4
    assert sz.ws_bwd_bytes >= sz.ws_bytes > 0
    assert sz.saved_bytes >= 4 * (2 * 30 * 30 * 31 // 2 + 200 * 200 * 201 // 2)


@pytest.mark.parametrize("precision", [0, 1])
def test_plan_accepts_k_up_to_304(lib, precision):
    """Spectral sizes above 256 (split into two basis ranges by the tensor-core
    projection, 320-thread solve blocks) up to the 304 limit."""
    from paper_2604_10377_gb300 import _lib
    opt = _lib.default_options()
    opt.precision = precision
    specs = [dict(n=4000, k=k, d=256) for k in (257, 257, 300, 300, 304, 304)]
    rc, sz = _plan(lib, specs, [(0, 1, 1e-3), (2, 3, 1e-3), (4, 5, 1e-3)], opt)
    assert rc == 0
    assert sz.a_floats == 2 * 256 * (257 + 300 + 304)
    assert sz.c_floats == 257 ** 2 + 300 ** 2 + 304 ** 2
    # every system's factor is stored by default: 32Q(Q+2) + 64Q floats per system
    # (each pair's block 256-byte aligned)
    fac = sum(k * 4 * (32 * q * (q + 2) + 64 * q) for k, q in ((257, 33), (300, 38), (304, 38)))
    assert fac <= sz.saved_bytes < fac + 3 * 256


def test_row_weight_pointers_must_be_aligned(lib):
    """Per-row lambda weights and their gradient outputs are FP32 device arrays: a pointer
    that is not 4-byte aligned is refused when the batch is planned (no device needed)."""
    from paper_2604_10377_gb300 import _lib
    specs = [dict(n=500, k=20, d=64), dict(n=600, k=30, d=64)]
    for field in ("lambda_rows", "d_lambda_rows"):
        sd, pd = _descs(specs, [(0, 1, 1e-3)])
        pd[0].lambda_rows = 0x50000
        setattr(pd[0], field, 0x50002)
        sz = _lib.Sizes()
        assert lib.fmap_plan_sizes(None, sd, 2, pd, 1, ctypes.byref(sz)) == _lib.FMAP_ERR_UNSUPPORTED
    sd, pd = _descs(specs, [(0, 1, 1e-3)])
    pd[0].lambda_rows, pd[0].d_lambda_rows = 0x50000, 0x60000
    sz = _lib.Sizes()
    assert lib.fmap_plan_sizes(None, sd, 2, pd, 1, ctypes.byref(sz)) == 0


def test_plan_sizes_empty(lib):
    rc, sz = _plan(lib, [dict(n=10, k=4, d=16)], [])
    assert rc == 0 and sz.c_floats == 0 and sz.n_pairs == 0


@pytest.mark.parametrize("bad,code", [
    (dict(k=0), 1), (dict(k=305), 2), (dict(d=24), 2), (dict(n=0), 1),
    (dict(ld_phi=30), 1), (dict(ld_phi=34), 2), (dict(ld_feat=132), 2),
    (dict(phi=0x10004), 2), (dict(feat=0x40008), 2),
])
def test_plan_rejects_bad_shapes(lib, bad, code):
    good = dict(n=5000, k=32, d=128)
    spec = dict(good, **bad)
    rc, _ = _plan(lib, [spec, good], [(0, 1, 1e-3)])
    assert rc == code, (bad, rc)


@pytest.mark.parametrize("pair,code", [((0, 2, 1e-3), 1), ((0, 1, -1.0), 1), ((0, 1, float("nan")), 1),
                                       ((-1, 1, 1e-3), 1)])
def test_plan_rejects_bad_pairs(lib, pair, code):
    specs = [dict(n=100, k=8, d=16), dict(n=100, k=8, d=16)]
    rc, _ = _plan(lib, specs, [pair])
    assert rc == code


def test_plan_rectangular_maps_and_rejections(lib):
    """Bases of different sizes give a k_y x k_x map; a feature-width mismatch and a
    missing eigenvalue array (without a mask) are rejected."""
    rc, sz = _plan(lib, [dict(n=100, k=8, d=16), dict(n=100, k=9, d=16)], [(0, 1, 1e-3), (1, 0, 1e-3)])
    assert rc == 0
    assert sz.c_floats == 9 * 8 + 8 * 9
    rc, _ = _plan(lib, [dict(n=100, k=8, d=16), dict(n=100, k=8, d=32)], [(0, 1, 1e-3)])
    assert rc == 1
    rc, _ = _plan(lib, [dict(n=100, k=8, d=16, evals=None), dict(n=100, k=8, d=16)], [(0, 1, 1e-3)])
    assert rc == 1


def test_options_validation(lib):
    from paper_2604_10377_gb300 import _lib
    o = _lib.default_options()
    assert (o.precision, o.ir_steps, o.hi_gram_min_k, o.store_factors_max_k, o.adjoint_ir_steps) == (0, 1, 200, 304, 0)
    ctx = ctypes.c_void_p()
    assert lib.fmap_create(ctypes.byref(ctx), 0, ctypes.byref(o)) == 0
    assert lib.fmap_destroy(ctx) == 0
    o.ir_steps = 9
    assert lib.fmap_create(ctypes.byref(ctx), 0, ctypes.byref(o)) == 1
    o.ir_steps = 1
    o.precision = 5
    assert lib.fmap_create(ctypes.byref(ctx), 0, ctypes.byref(o)) == 1


@pytest.mark.parametrize("knob,good,bad", [
    ("proj_max_stages", (0, 2, 6), (1, 7)),
    ("proj_seg_max_v", (0, 2048, 16384), (1024, 4000, 32768)),
    ("bwd_group_features", (0, 64, 128), (32, 96, 256)),
    ("bwd_chunk_v", (0, 1024, 65536), (512, 1000, 131072)),
    ("solve_threads_k64", (0, 64, 128), (32, 256)),
    ("solve_threads_k128", (0, 128, 256), (64, 320)),
    ("proj_ctas", (0, 1, 48, 152), (-1, 153)),
    ("bwd_ctas", (0, 2, 64, 152), (-2, 1, 63, 154)),
    ("solve_no_g_copy", (0, 1), (-1, 2)),
    ("adjoint_kernel", (0, 1, 2), (-1, 3)),
    ("adjoint_features", (0, 64, 128, 256), (-1, 32, 96, 512)),
    ("adjoint_stages", (0, 1, 2), (-1, 3)),
])
def test_tuning_knob_validation(lib, knob, good, bad):
    """Every tuning knob defaults to 0 (built-in choice); values outside its documented set
    are rejected synchronously; accepted values plan the same outputs."""
    from paper_2604_10377_gb300 import _lib
    o = _lib.default_options()
    assert all(getattr(o, f) == 0 for f in _lib.TUNING_FIELDS)
    specs = [dict(n=5000, k=30, d=256), dict(n=7000, k=30, d=256), dict(n=900, k=120, d=256),
             dict(n=800, k=120, d=256)]
    pairs = [(0, 1, 1e-3), (2, 3, 1e-3)]
    o.precision = 1
    rc, ref = _plan(lib, specs, pairs, o)
    assert rc == 0
    for v in good:
        setattr(o, knob, v)
        rc, sz = _plan(lib, specs, pairs, o)
        assert rc == 0, (knob, v)
        assert (sz.a_floats, sz.c_floats, sz.saved_bytes) == (ref.a_floats, ref.c_floats, ref.saved_bytes)
    for v in bad:
        setattr(o, knob, v)
        rc, _ = _plan(lib, specs, pairs, o)
        assert rc == 1, (knob, v)


def test_store_factor_threshold(lib):
    from paper_2604_10377_gb300 import _lib
    o = _lib.default_options()
    o.store_factors_max_k = 100
    specs = [dict(n=300, k=30, d=64), dict(n=300, k=30, d=64), dict(n=300, k=200, d=512), dict(n=300, k=200, d=512)]
    rc, sz = _plan(lib, specs, [(0, 1, 1e-3), (2, 3, 1e-3)], o)
    assert rc == 0
    # one row system keeps its factor as packed lower rows (8 (a/8 + 1) + 4 floats for row a)
    # plus Q inverse 8 x 8 diagonal blocks: 32 Q (Q + 2) + 64 Q floats for k padded to 8 Q
    # (k = 30: Q = 4, 1024 floats); k = 200 is not saved
    per_system = 32 * 4 * 6 + 64 * 4
    assert sz.saved_bytes == 4 * ((30 * per_system + 63) // 64 * 64)


def test_calls_without_batch_are_rejected(lib):
    assert lib.fmap_project(None, None, None, 0, None) == 1
    assert lib.fmap_solve(None, None, None, None, None, None, 0, None) == 1
    assert lib.fmap_adjoint(None, None, None, None, None, None, None, None, None, None, 0, None) == 1
    assert lib.fmap_project_backward(None, None, None, None, 0, None) == 1


# ------------------------------------------------------------ independence of oracle and CUDA path
def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_2604_10377_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path, errors="ignore").read()
            assert not re.search(r"\boracle\b\s*(import|\.)|from\s+oracle|import\s+oracle|fmap_oracle", text), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        text = open(path).read()
        assert "paper_2604_10377_gb300" not in text and "libfmap" not in text, path


def test_overlap_metrics_argument_checks(lib):
    """Argument errors return before any launch (no GPU needed)."""
    fake = ctypes.c_void_p(0x10000)
    assert lib.fmap_overlap_metrics(None, None, None, 0, 0, 0.5, None, None, None) == 0
    assert lib.fmap_overlap_metrics(fake, fake, fake, -1, 10, 0.5, fake, None, None) == 1
    assert lib.fmap_overlap_metrics(fake, fake, fake, 3, -1, 0.5, fake, None, None) == 1
    assert lib.fmap_overlap_metrics(fake, fake, None, 3, 10, 0.5, fake, None, None) == 1
    assert lib.fmap_overlap_metrics(fake, fake, fake, 3, 10, 0.5, None, None, None) == 1
    assert lib.fmap_overlap_metrics(None, fake, fake, 3, 10, 0.5, fake, None, None) == 1
    assert lib.fmap_overlap_metrics(fake, fake, fake, 3, 10, float("nan"), fake, None, None) == 1
    assert lib.fmap_overlap_metrics(fake, fake, fake, 70000, 10, 0.5, fake, None, None) == 2


def test_overlap_metrics_python_checks():
    """api.overlap_metrics rejects host tensors, wrong dtypes and bad offsets before any call."""
    torch = pytest.importorskip("torch")
    from paper_2604_10377_gb300 import api
    s = torch.zeros(10, dtype=torch.float32)
    l = torch.zeros(10, dtype=torch.uint8)
    with pytest.raises(ValueError):
        api.overlap_metrics(s, l, [0, 10])                  # host tensors
    with pytest.raises(TypeError):
        api.overlap_metrics(s.double(), l, [0, 10])
    with pytest.raises(TypeError):
        api.overlap_metrics(s, l.int(), [0, 10])
