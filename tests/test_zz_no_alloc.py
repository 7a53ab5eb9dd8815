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
