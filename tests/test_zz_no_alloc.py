"""The allocation-free single-pair solve (fmap_solve_pair_noalloc) against fmap_solve.

Some callers cannot allocate device memory at the time they solve; this entry point
takes its scratch from a static array inside the library. Here it is called through
the C ABI on two pairs in a row, and each result is compared with what the batched
fmap_solve returns for the same descriptors, within the FP32 tolerance of the other
parity tests. The file sorts last so that a failure here leaves the other tests run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_batched_solve_twice():
    import os
    from paper_2604_10377_gb300 import _lib, api, build, synth
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    assert torch.cuda.is_available()
    lib = _lib.lib()
    wl = synth.make_small(77, 2, (1500, 4000), [50, 200], 512)
    b = api.batch_from_workload(wl)
    a = b.project()
    c_ref = b.solve(a, keep_factors=False)
    torch.cuda.synchronize()
    assert int(b.status[:2].abs().sum()) == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for p, pr in enumerate(wl.pairs):
        k = wl.shapes[pr.x].k
        d = wl.shapes[pr.x].d
        ax = b.a_view(a, pr.x).contiguous()
        ay = b.a_view(a, pr.y).contiguous()
        ev = b.evals
        evx = ev[b.layout.evals_off[pr.x]:b.layout.evals_off[pr.x] + k].contiguous()
        evy = ev[b.layout.evals_off[pr.y]:b.layout.evals_off[pr.y] + k].contiguous()
        c = torch.empty(k, k, dtype=torch.float32, device="cuda")
        rc = lib.fmap_solve_pair_noalloc(_ptr(ax), _ptr(ay), k, d, _ptr(evx), _ptr(evy), None,
                                         ctypes.c_float(pr.lam), 1, _ptr(c), _ptr(status), stream)
        assert rc == 0, _lib.error_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ref = b.c_view(c_ref, p).double()
        err = float(torch.linalg.norm(c.double() - ref) / torch.linalg.norm(ref))
        assert err <= TOL, (p, k, err)


def test_noalloc_rejects_oversized_k():
    from paper_2604_10377_gb300 import _lib
    lib = _lib.lib()
    x = torch.zeros(16, device="cuda")
    rc = lib.fmap_solve_pair_noalloc(_ptr(x), _ptr(x), 257, 16, _ptr(x), _ptr(x), None, ctypes.c_float(1e-3), 1,
                                     _ptr(x), None, None)
    assert rc == _lib.FMAP_ERR_UNSUPPORTED


@pytest.mark.parametrize("k,d,with_mask", [(1, 16, False), (40, 128, True), (256, 512, False)])
def test_noalloc_matches_oracle_row_solve(k, d, with_mask):
    """The allocation-free solve against the FP64 oracle's row solve (Eq. 4-5) on the same
    descriptor matrices A and B, within the FP32 tolerance: k = 1, an explicit k x k mask
    (no eigenvalues passed), and the largest k it takes (256). Two calls in a row on each
    pair, so that the second reads scratch the first left behind."""
    import os
    from oracle import fmap_oracle as orc
    from paper_2604_10377_gb300 import _lib, api, build, synth
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    lib = _lib.lib()
    wl = synth.make_small(78 + k, 1, (600, 3000), [k], d, with_mask=with_mask)
    b = api.batch_from_workload(wl)
    a = b.project()
    torch.cuda.synchronize()
    pr = wl.pairs[0]
    ax = b.a_view(a, pr.x).contiguous()
    ay = b.a_view(a, pr.y).contiguous()
    lam = float(np.float32(pr.lam))
    if with_mask:
        dm = pr.mask.astype(np.float64)
        mask_dev = torch.from_numpy(pr.mask.astype(np.float32)).cuda()
        evx = evy = None
    else:
        ev = b.evals
        evx = ev[b.layout.evals_off[pr.x]:b.layout.evals_off[pr.x] + k].contiguous()
        evy = ev[b.layout.evals_off[pr.y]:b.layout.evals_off[pr.y] + k].contiguous()
        dm = orc.mask_from_evals(evx.double().cpu().numpy(), evy.double().cpu().numpy())
        mask_dev = None
    c_ref = orc.solve(ax.double().cpu().numpy(), ay.double().cpu().numpy(), dm, lam)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        c = torch.full((k, k), float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.fmap_solve_pair_noalloc(_ptr(ax), _ptr(ay), k, d,
                                         None if evx is None else _ptr(evx), None if evy is None else _ptr(evy),
                                         None if mask_dev is None else _ptr(mask_dev), ctypes.c_float(lam), 1,
                                         _ptr(c), _ptr(status), stream)
        assert rc == 0, _lib.error_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        got = c.double().cpu().numpy()
        err = float(np.linalg.norm(got - c_ref) / np.linalg.norm(c_ref))
        assert err <= TOL, (k, with_mask, err)
