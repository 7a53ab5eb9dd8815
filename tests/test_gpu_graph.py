"""The whole fwd+bwd step captured in a CUDA graph: every C-ABI call only enqueues,
so it can be captured; replays give bitwise the same results as eager execution
(every reduction runs in a fixed order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_graph_replay_is_bitwise_identical():
    import os
    from paper_2604_10377_gb300 import _lib, api, build, synth
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    wl = synth.make_small(31, 4, (800, 9000), [30, 50, 100, 200], 256, feat_dtype="bf16")
    b = api.batch_from_workload(wl, with_grad=True)
    gt = api.flat_c(b, [p.c_gt for p in wl.pairs])
    loss = torch.empty(len(wl.pairs), device="cuda")
    dc = torch.empty_like(b.C)

    def step():
        a = b.project()
        c = b.solve(a)
        b.loss_orth(c, gt, loss=loss, d_c=dc)
        b.solve_backward(dc, a, c)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ref = [b.A.clone(), b.C.clone(), loss.clone(), b.dA.clone(), b.dfeat.clone()]

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        b.A.zero_(); b.C.zero_(); loss.zero_(); b.dA.zero_(); b.dfeat.zero_()
        g.replay()
        torch.cuda.synchronize()
        out = [b.A, b.C, loss, b.dA, b.dfeat]
        for r, o in zip(ref, out):
            assert torch.equal(r, o)
    assert int(b.status[:len(wl.pairs)].abs().sum()) == 0
