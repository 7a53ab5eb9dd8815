"""Test helpers: hand the same synthetic inputs to the oracle and to the CUDA path."""
import numpy as np

from paper_2604_10377_gb300 import synth


def oracle_inputs(wl: "synth.Workload"):
    shapes = [dict(phi=s.phi.astype(np.float64), mass=s.mass.astype(np.float64),
                   feat=s.feat_f64(), evals=s.evals.astype(np.float64)) for s in wl.shapes]
    pairs = [dict(x=p.x, y=p.y, lam=float(np.float32(p.lam)),
                  mask=None if p.mask is None else p.mask.astype(np.float64),
                  lam_rows=None if getattr(p, "lam_rows", None) is None
                  else np.asarray(p.lam_rows, np.float32).astype(np.float64)) for p in wl.pairs]
    return shapes, pairs


def rel_fro(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))


def gpu_forward(wl, **kw):
    """Run fmap_project + fmap_solve on the GPU; returns (batch, A list, C list, status)."""
    import torch
    from paper_2604_10377_gb300 import api
    b = api.batch_from_workload(wl, **kw)
    a = b.project()
    c = b.solve(a)
    torch.cuda.synchronize()
    a_list = [b.a_view(a, s).cpu().numpy().astype(np.float64) for s in range(len(wl.shapes))]
    c_list = [b.c_view(c, p).cpu().numpy().astype(np.float64) for p in range(len(wl.pairs))]
    return b, a_list, c_list, b.status[:len(wl.pairs)].cpu().numpy()
