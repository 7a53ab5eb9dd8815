"""Python front end of the functional-map library.

A batch of shape pairs lives in a handful of flat device buffers (bases, masses,
eigenvalues, features, feature gradients), laid out by :class:`BatchLayout`.
:class:`FmapBatch` binds those buffers to a C-ABI batch once; every later call
(project, solve, solve_backward, loss) only enqueues kernels of libfmap.so on the
current torch stream. Torch provides the memory and the stream, nothing else.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import FmapError, check


def _round_up(x: int, a: int) -> int:
    return (x + a - 1) // a * a


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class BatchLayout:
    """Offsets of every shape inside the flat buffers (128-byte aligned blocks).

    phi: n x ld_phi FP32 with ld_phi = k rounded up to 4; mass: n FP32; evals: k FP32;
    feat / dfeat: n x d in the feature dtype."""

    def __init__(self, ns: Sequence[int], ks: Sequence[int], ds: Sequence[int], feat_dtype: str):
        assert len(ns) == len(ks) == len(ds)
        self.ns, self.ks, self.ds = [int(x) for x in ns], [int(x) for x in ks], [int(x) for x in ds]
        self.feat_dtype = feat_dtype
        self.ld_phi = [_round_up(k, 4) for k in self.ks]
        self.phi_off, self.mass_off, self.evals_off, self.feat_off = [], [], [], []
        p = m = e = f = 0
        for n, k, d, ld in zip(self.ns, self.ks, self.ds, self.ld_phi):
            self.phi_off.append(p); p = _round_up(p + n * ld, 32)
            self.mass_off.append(m); m = _round_up(m + n, 32)
            self.evals_off.append(e); e = _round_up(e + k, 32)
            self.feat_off.append(f); f = _round_up(f + n * d, 64)
        self.phi_len, self.mass_len, self.evals_len, self.feat_len = p, m, e, f

    @property
    def n_shapes(self):
        return len(self.ns)

    def torch_feat_dtype(self):
        return torch.bfloat16 if self.feat_dtype == "bf16" else torch.float32

    def pack_host(self, shapes) -> dict:
        """Flat host arrays (NumPy) for a list of synth.Shape-like objects."""
        phi = np.zeros(self.phi_len, np.float32)
        mass = np.zeros(self.mass_len, np.float32)
        evals = np.zeros(self.evals_len, np.float32)
        fdt = np.uint16 if self.feat_dtype == "bf16" else np.float32
        feat = np.zeros(self.feat_len, fdt)
        for i, s in enumerate(shapes):
            n, k, d, ld = self.ns[i], self.ks[i], self.ds[i], self.ld_phi[i]
            blk = phi[self.phi_off[i]:self.phi_off[i] + n * ld].reshape(n, ld)
            blk[:, :k] = s.phi
            mass[self.mass_off[i]:self.mass_off[i] + n] = s.mass
            evals[self.evals_off[i]:self.evals_off[i] + k] = s.evals
            feat[self.feat_off[i]:self.feat_off[i] + n * d] = np.asarray(s.feat, dtype=fdt).reshape(-1)
        return dict(phi=phi, mass=mass, evals=evals, feat=feat)

    def feat_view(self, flat: torch.Tensor, s: int) -> torch.Tensor:
        o, n, d = self.feat_off[s], self.ns[s], self.ds[s]
        return flat[o:o + n * d].view(n, d)


def host_to_torch(arr: np.ndarray, dtype_name: str = "") -> torch.Tensor:
    t = torch.from_numpy(arr)
    if arr.dtype == np.uint16:
        t = t.view(torch.int16).view(torch.bfloat16)
    return t


class FmapBatch:
    """A ragged batch of shape pairs bound to flat device buffers.

    pairs: list of (x, y, lam); masks: optional list (per pair) of k_Y x k_X arrays or None
    (k_X = the basis size of shape x, k_Y of shape y; C_p is k_Y x k_X)."""

    def __init__(self, layout: BatchLayout, pairs, device="cuda:0", precision: str = "fp32",
                 with_grad: bool = True, masks=None, ir_steps: int = 1, hi_gram_min_k: int = 200,
                 store_factors_max_k: int = 304, adjoint_ir_steps: int = 0, tuning: Optional[dict] = None,
                 grad_f32_copy: bool = False, lambda_rows=None):
        self.layout = layout
        self.device = torch.device(device)
        self.precision = precision
        lay = layout
        dev = self.device
        self.phi = torch.zeros(lay.phi_len, dtype=torch.float32, device=dev)
        self.mass = torch.zeros(lay.mass_len, dtype=torch.float32, device=dev)
        self.evals = torch.zeros(lay.evals_len, dtype=torch.float32, device=dev)
        self.feat = torch.zeros(lay.feat_len, dtype=lay.torch_feat_dtype(), device=dev)
        self.dfeat = torch.zeros_like(self.feat) if with_grad else None
        # BF16 batches: optional FP32 copy of dL/dF before its rounding to BF16 (for checking)
        self.dfeat32 = (torch.zeros(lay.feat_len, dtype=torch.float32, device=dev)
                        if with_grad and grad_f32_copy and lay.feat_dtype == "bf16" else None)
        self.pairs = [(int(x), int(y), float(lam)) for (x, y, lam) in pairs]
        # C_p maps the k_X coefficients of shape x to the k_Y of shape y: k_Y x k_X
        self.ks = [lay.ks[x] for (x, _, _) in self.pairs]
        self.kys = [lay.ks[y] for (_, y, _) in self.pairs]
        self.c_off_host = np.concatenate([[0], np.cumsum([ky * k for k, ky in zip(self.ks, self.kys)])]).astype(np.int64)
        self.mask = None
        if masks is not None and any(m is not None for m in masks):
            host = np.zeros(int(self.c_off_host[-1]), np.float32)
            for p, m in enumerate(masks):
                if m is not None:
                    host[self.c_off_host[p]:self.c_off_host[p + 1]] = np.asarray(m, np.float32).reshape(-1)
            self.mask = torch.from_numpy(host).to(dev)
        self._masks_present = [m is not None for m in masks] if masks is not None else [False] * len(self.pairs)
        # optional weight per row of C (k_Y floats per pair, in place of lam) and, with
        # gradients, dL/dlambda_i per row; each pair's segment starts on a 16-byte boundary
        self.lam_rows = self.dlam_rows = None
        self._lr_off = None
        if lambda_rows is not None and any(v is not None for v in lambda_rows):
            offs, cur = [], 0
            for p, v in enumerate(lambda_rows):
                offs.append(cur if v is not None else -1)
                if v is not None:
                    if np.shape(v) != (self.kys[p],):
                        raise ValueError(f"pair {p}: lambda_rows needs {self.kys[p]} weights (one per row of C)")
                    cur += (self.kys[p] + 3) // 4 * 4
            host = np.zeros(max(cur, 4), np.float32)
            for p, v in enumerate(lambda_rows):
                if v is not None:
                    host[offs[p]:offs[p] + self.kys[p]] = np.asarray(v, np.float32)
            self._lr_off = offs
            self.lam_rows = torch.from_numpy(host).to(dev)
            if with_grad:
                self.dlam_rows = torch.zeros_like(self.lam_rows)

        L = _lib.lib()
        opt = _lib.default_options()
        opt.precision = _lib.FMAP_PREC_BF16 if precision == "bf16" else _lib.FMAP_PREC_FP32
        opt.ir_steps = ir_steps
        opt.hi_gram_min_k = hi_gram_min_k
        opt.store_factors_max_k = store_factors_max_k
        opt.adjoint_ir_steps = adjoint_ir_steps
        self.options = opt
        self._ctx = None
        self._batch = None
        self.ws = None
        self.saved = None
        self._apply_tuning(tuning or {})
        self._create()
        self._alloc_outputs()

    # ------------------------------------------------------------------ setup
    def _descs(self):
        lay = self.layout
        fel = 2 if lay.feat_dtype == "bf16" else 4
        sd = (_lib.ShapeDesc * max(1, lay.n_shapes))()
        for s in range(lay.n_shapes):
            d = sd[s]
            d.n, d.k, d.d = lay.ns[s], lay.ks[s], lay.ds[s]
            d.phi = self.phi.data_ptr() + 4 * lay.phi_off[s]
            d.ld_phi = lay.ld_phi[s]
            d.mass = self.mass.data_ptr() + 4 * lay.mass_off[s]
            d.evals = self.evals.data_ptr() + 4 * lay.evals_off[s]
            d.feat = self.feat.data_ptr() + fel * lay.feat_off[s]
            d.ld_feat = lay.ds[s]
            d.dfeat = (self.dfeat.data_ptr() + fel * lay.feat_off[s]) if self.dfeat is not None else None
            d.dfeat_f32 = (self.dfeat32.data_ptr() + 4 * lay.feat_off[s]) if self.dfeat32 is not None else None
        pd = (_lib.PairDesc * max(1, len(self.pairs)))()
        for p, (x, y, lam) in enumerate(self.pairs):
            pd[p].shape_x, pd[p].shape_y, pd[p].lam = x, y, lam
            pd[p].mask = (self.mask.data_ptr() + 4 * int(self.c_off_host[p])) if self._masks_present[p] else None
            lr = self._lr_off[p] if self._lr_off is not None else -1
            pd[p].lambda_rows = (self.lam_rows.data_ptr() + 4 * lr) if lr >= 0 else None
            pd[p].d_lambda_rows = (self.dlam_rows.data_ptr() + 4 * lr) if (lr >= 0 and self.dlam_rows is not None) else None
        return sd, pd

    def _apply_tuning(self, tuning: dict):
        for name in _lib.TUNING_FIELDS:
            setattr(self.options, name, int(tuning.get(name, 0)))

    @property
    def tuning(self) -> dict:
        """The tuning knobs of this batch (0 = the library's built-in choice)."""
        return {name: int(getattr(self.options, name)) for name in _lib.TUNING_FIELDS}

    def _create(self):
        """Context + batch handle for the current options over the same device buffers; the
        workspace and factor buffers are (re)allocated when their sizes change."""
        L = _lib.lib()
        ctx = ctypes.c_void_p()
        check(L.fmap_create(ctypes.byref(ctx), self.device.index or 0, ctypes.byref(self.options)), "fmap_create")
        self._ctx = ctx
        sd, pd = self._descs()
        b = ctypes.c_void_p()
        check(L.fmap_batch_create(self._ctx, sd, self.layout.n_shapes, pd, len(self.pairs), ctypes.byref(b)),
              "fmap_batch_create")
        self._batch = b
        sz = _lib.Sizes()
        check(L.fmap_batch_sizes(b, ctypes.byref(sz)), "fmap_batch_sizes")
        self.sizes = sz
        a_off = (ctypes.c_int64 * (self.layout.n_shapes + 1))()
        c_off = (ctypes.c_int64 * (len(self.pairs) + 1))()
        check(L.fmap_batch_offsets(b, a_off, c_off), "fmap_batch_offsets")
        self.a_off = np.array(a_off[:], dtype=np.int64)
        self.c_off = np.array(c_off[:], dtype=np.int64)
        dev = self.device
        if self.ws is None or self.ws.numel() < sz.ws_bwd_bytes:
            self.ws = torch.empty(max(256, sz.ws_bwd_bytes), dtype=torch.uint8, device=dev)
            self.ws[:256].zero_()   # control words (fmap_project clears them again each step)
        if sz.saved_bytes and (self.saved is None or self.saved.numel() < sz.saved_bytes):
            self.saved = torch.empty(max(256, sz.saved_bytes), dtype=torch.uint8, device=dev)

    def retune(self, tuning: dict):
        """Re-plan the batch with other tuning knobs (see fmap_options). Inputs, outputs and
        results stay where they are; only the library's work lists change."""
        torch.cuda.synchronize(self.device)
        self.close()
        self._apply_tuning(tuning)
        self._create()

    def _alloc_outputs(self):
        sz = self.sizes
        dev = self.device
        self.A = torch.empty(max(1, sz.a_floats), dtype=torch.float32, device=dev)
        self.C = torch.empty(max(1, sz.c_floats), dtype=torch.float32, device=dev)
        self.dA = torch.empty_like(self.A)
        self.status = torch.zeros(max(1, len(self.pairs)), dtype=torch.int32, device=dev)

    def close(self):
        L = _lib.lib()
        if self._batch is not None:
            L.fmap_batch_destroy(self._batch)
            self._batch = None
        if self._ctx is not None:
            L.fmap_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ instrumentation
    def set_timing(self, enable: bool):
        check(_lib.lib().fmap_batch_set_timing(self._batch, 1 if enable else 0), "fmap_batch_set_timing")

    def read_timing(self) -> dict:
        """{kernel kind: (total ms, launches)} since the last read (synchronises)."""
        n = len(_lib.KIND_NAMES)
        ms = (ctypes.c_float * n)()
        cnt = (ctypes.c_int32 * n)()
        check(_lib.lib().fmap_batch_read_timing(self._batch, ms, cnt, n), "fmap_batch_read_timing")
        return {name: (float(ms[i]), int(cnt[i])) for i, name in enumerate(_lib.KIND_NAMES)}

    # ------------------------------------------------------------------ data
    def upload(self, host: dict, non_blocking: bool = False, copy_streams: int = 1):
        """Copy flat host arrays (from BatchLayout.pack_host, or pinned torch tensors) to the device.

        With non_blocking and copy_streams > 1 the copies are cut into 64 MiB pieces spread
        over that many side streams (several copy engines at once); the side streams start
        after the current stream's earlier work and the current stream waits for them, so
        the call stays ordered like a single copy."""
        srcs = []
        for name in ("phi", "mass", "evals", "feat"):
            src = host[name]
            if isinstance(src, np.ndarray):
                src = host_to_torch(src)
            srcs.append((getattr(self, name), src))
        if copy_streams <= 1 or not non_blocking:
            for dst, src in srcs:
                dst.copy_(src, non_blocking=non_blocking)
            return
        if len(getattr(self, "_copy_streams", [])) != copy_streams:
            self._copy_streams = [torch.cuda.Stream(self.device) for _ in range(copy_streams)]
        cur = torch.cuda.current_stream(self.device)
        for st in self._copy_streams:
            st.wait_stream(cur)
        i = 0
        for dst, src in srcs:
            step = max(1, (64 << 20) // dst.element_size())
            for o in range(0, dst.numel(), step):
                with torch.cuda.stream(self._copy_streams[i % copy_streams]):
                    dst[o:o + step].copy_(src[o:o + step], non_blocking=True)
                i += 1
        for st in self._copy_streams:
            cur.wait_stream(st)

    def dlam_rows_view(self, p: int) -> Optional[torch.Tensor]:
        """dL/dlambda_i of pair p's row weights (written by solve_backward), or None."""
        if self.dlam_rows is None or self._lr_off[p] < 0:
            return None
        return self.dlam_rows[self._lr_off[p]:self._lr_off[p] + self.kys[p]]

    def a_view(self, flat: torch.Tensor, s: int) -> torch.Tensor:
        k, d = self.layout.ks[s], self.layout.ds[s]
        return flat[int(self.a_off[s]):int(self.a_off[s + 1])].view(k, d)

    def c_view(self, flat: torch.Tensor, p: int) -> torch.Tensor:
        """Pair p's k_Y x k_X block of a flat C-layout buffer."""
        return flat[int(self.c_off[p]):int(self.c_off[p + 1])].view(self.kys[p], self.ks[p])

    # ------------------------------------------------------------------ calls
    def project(self, a_out: Optional[torch.Tensor] = None) -> torch.Tensor:
        a = self.A if a_out is None else a_out
        check(_lib.lib().fmap_project(self._batch, _ptr(a), _ptr(self.ws), self.ws.numel(), _stream(self.device)),
              "fmap_project")
        return a

    def solve(self, a: Optional[torch.Tensor] = None, c_out: Optional[torch.Tensor] = None,
              keep_factors: bool = True) -> torch.Tensor:
        a = self.A if a is None else a
        c = self.C if c_out is None else c_out
        saved = self.saved if keep_factors else None
        check(_lib.lib().fmap_solve(self._batch, _ptr(a), _ptr(c), _ptr(saved), _ptr(self.status), _ptr(self.ws),
                                    self.ws.numel(), _stream(self.device)), "fmap_solve")
        return c

    def solve_backward(self, d_c: torch.Tensor, a: Optional[torch.Tensor] = None, c: Optional[torch.Tensor] = None,
                       use_saved: bool = True, d_a: Optional[torch.Tensor] = None, d_mask: Optional[torch.Tensor] = None,
                       d_lambda: Optional[torch.Tensor] = None):
        a = self.A if a is None else a
        c = self.C if c is None else c
        d_a = self.dA if d_a is None else d_a
        saved = self.saved if use_saved else None
        check(_lib.lib().fmap_solve_backward(self._batch, _ptr(d_c), _ptr(a), _ptr(c), _ptr(saved), _ptr(d_a),
                                             _ptr(d_mask), _ptr(d_lambda), _ptr(self.status), _ptr(self.ws),
                                             self.ws.numel(), _stream(self.device)), "fmap_solve_backward")
        return d_a

    def adjoint(self, d_c: torch.Tensor, a: Optional[torch.Tensor] = None, c: Optional[torch.Tensor] = None,
                use_saved: bool = True, d_a: Optional[torch.Tensor] = None, d_mask: Optional[torch.Tensor] = None,
                d_lambda: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The first half of solve_backward: dL/dA (and dL/dD, dL/dlambda), no dL/dF."""
        a = self.A if a is None else a
        c = self.C if c is None else c
        d_a = self.dA if d_a is None else d_a
        saved = self.saved if use_saved else None
        check(_lib.lib().fmap_adjoint(self._batch, _ptr(d_c), _ptr(a), _ptr(c), _ptr(saved), _ptr(d_a),
                                      _ptr(d_mask), _ptr(d_lambda), _ptr(self.status), _ptr(self.ws),
                                      self.ws.numel(), _stream(self.device)), "fmap_adjoint")
        return d_a

    def project_backward(self, d_a: Optional[torch.Tensor] = None):
        """The second half of solve_backward: dL/dF of every shape from dL/dA."""
        d_a = self.dA if d_a is None else d_a
        check(_lib.lib().fmap_project_backward(self._batch, _ptr(d_a), _ptr(self.status), _ptr(self.ws),
                                               self.ws.numel(), _stream(self.device)), "fmap_project_backward")

    def loss_orth(self, c: torch.Tensor, c_gt: torch.Tensor, loss: Optional[torch.Tensor] = None,
                  d_c: Optional[torch.Tensor] = None):
        if loss is None:
            loss = torch.empty(max(1, len(self.pairs)), dtype=torch.float32, device=self.device)
        if d_c is None:
            d_c = torch.empty_like(c)
        check(_lib.lib().fmap_loss_orth(self._batch, _ptr(c), _ptr(c_gt), _ptr(loss), _ptr(d_c), _ptr(self.ws),
                                        self.ws.numel(), _stream(self.device)), "fmap_loss_orth")
        return loss, d_c


class UploadPipeline:
    """Host -> device input staging that overlaps the upload of the next step with the
    compute of the current one.

    The pipeline owns two or more FmapBatch objects of one layout (buffers). `prefetch`
    enqueues the upload of one step's inputs into the next buffer on a copy stream, after
    the last step that computed on that buffer has finished; `acquire` makes the current
    stream wait for the oldest prefetched upload and returns its batch; `release` marks the
    end of the current stream's work on it. A loop of
        prefetch(step 0); for each step: acquire, prefetch(next step), compute, release
    moves every step's inputs from host to device once, and with two buffers the copy of
    step i+1 runs while step i computes. Buffers are named by index (`batches[j]`);
    `next_buffer` is the one the next prefetch fills, so that per-buffer extras (targets,
    labels) can be passed as `extra` pairs (device tensor, host tensor) copied with it.
    """

    def __init__(self, batches: Sequence[FmapBatch]):
        if len(batches) < 2:
            raise ValueError("an upload pipeline needs at least two batches")
        self.batches = list(batches)
        self.device = self.batches[0].device
        self.copy_stream = torch.cuda.Stream(self.device)
        n = len(self.batches)
        self._done: List[Optional[torch.cuda.Event]] = [None] * n
        self._ready: List[Optional[torch.cuda.Event]] = [None] * n
        self._next = 0
        self._queued: List[int] = []
        self._cur: Optional[int] = None

    def prefetch(self, host: dict, extra: Sequence = ()) -> int:
        """Enqueue the upload of `host` (pinned tensors, as for FmapBatch.upload) into the
        next buffer; returns the buffer's index."""
        if len(self._queued) >= len(self.batches):
            raise RuntimeError("every buffer already holds an upload that was not acquired")
        j = self._next
        self._next = (j + 1) % len(self.batches)
        cs = self.copy_stream
        if self._done[j] is not None:
            cs.wait_event(self._done[j])
        with torch.cuda.stream(cs):
            self.batches[j].upload(host, non_blocking=True)
            for dst, src in extra:
                dst.copy_(src, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(cs)
        self._ready[j] = ev
        self._queued.append(j)
        return j

    @property
    def next_buffer(self) -> int:
        return self._next

    def acquire(self) -> int:
        """Index of the buffer of the oldest prefetched upload; the current stream waits
        for that upload."""
        if not self._queued:
            raise RuntimeError("acquire without a prefetched upload")
        if self._cur is not None:
            raise RuntimeError("the previous batch was not released")
        j = self._queued.pop(0)
        torch.cuda.current_stream(self.device).wait_event(self._ready[j])
        self._cur = j
        return j

    def release(self) -> None:
        """End of the current stream's work on the acquired batch: the next upload into its
        buffer starts after this point."""
        if self._cur is None:
            raise RuntimeError("release without an acquired batch")
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(self.device))
        self._done[self._cur] = ev
        self._cur = None


OVERLAP_METRICS = ("iou", "balanced_accuracy", "accuracy", "precision", "recall", "specificity", "f1")


def overlap_metrics(scores: torch.Tensor, labels: torch.Tensor, seg_offsets, threshold: float = 0.5,
                    with_metrics: bool = True):
    """Overlap-prediction counts and metrics per segment (fmap_overlap_metrics).

    scores: device float32 (n,); labels: device uint8 (n,), nonzero = truly overlapping;
    seg_offsets: host sequence of n_seg + 1 non-decreasing offsets into them. Returns
    (counts int64 (n_seg, 4) = TP, FP, FN, TN, metrics float64 (n_seg, 7) in the order of
    OVERLAP_METRICS, or None), both on the scores' device; the call only enqueues."""
    if scores.dtype != torch.float32 or labels.dtype != torch.uint8:
        raise TypeError("scores must be float32 and labels uint8")
    if not (scores.is_cuda and labels.is_cuda) or scores.device != labels.device:
        raise ValueError("scores and labels must be CUDA tensors on the same device")
    if not (scores.is_contiguous() and labels.is_contiguous()) or scores.numel() != labels.numel():
        raise ValueError("scores and labels must be contiguous and of equal length")
    off = np.asarray(seg_offsets, dtype=np.int64)
    n_seg = len(off) - 1
    if n_seg < 0 or (n_seg > 0 and (off[0] < 0 or np.any(np.diff(off) < 0) or off[-1] > scores.numel())):
        raise ValueError("seg_offsets must be non-decreasing offsets within the arrays")
    dev = scores.device
    counts = torch.empty((max(n_seg, 1), 4), dtype=torch.int64, device=dev)
    metrics = torch.empty((max(n_seg, 1), 7), dtype=torch.float64, device=dev) if with_metrics else None
    off_dev = torch.from_numpy(off).to(dev)
    max_len = int(np.max(np.diff(off))) if n_seg > 0 else 0
    check(_lib.lib().fmap_overlap_metrics(_ptr(scores), _ptr(labels), _ptr(off_dev), n_seg, max_len,
                                          float(threshold), _ptr(counts), _ptr(metrics), _stream(dev)),
          "fmap_overlap_metrics")
    counts = counts[:n_seg]
    return counts, (metrics[:n_seg] if metrics is not None else None)


def gradient_features(row_ptr: torch.Tensor, col_idx: torch.Tensor, g_vals: torch.Tensor, x_in: torch.Tensor,
                      a_re: torch.Tensor, a_im: torch.Tensor, variant: str = "A", out: Optional[torch.Tensor] = None,
                      out_dtype=torch.float32, ws: Optional[torch.Tensor] = None):
    """Spatial gradient features (fmap_gradient_features): F = Re(conj(z) o Az) (variant A)
    or the variant-B form, z = G X, written into `out` (n x ld_out rows of out_dtype; a new
    n x D tensor when None). row_ptr int64 (n+1,), col_idx int32 (nnz,), g_vals float32
    (nnz, 2) = (Re, Im), x_in float32 (n_in, ld_in) with D = a_re.shape[0] used columns.
    Returns (out, status int32 (1,) device tensor); the call only enqueues."""
    dev = x_in.device
    n = row_ptr.numel() - 1
    dim = a_re.shape[0]
    if out is None:
        out = torch.empty((max(n, 0), dim), dtype=out_dtype, device=dev)
    bf16 = out.dtype == torch.bfloat16
    if out.dtype not in (torch.bfloat16, torch.float32):
        raise TypeError("out must be float32 or bfloat16")
    for t, dt in ((row_ptr, torch.int64), (col_idx, torch.int32), (g_vals, torch.float32), (x_in, torch.float32),
                  (a_re, torch.float32), (a_im, torch.float32)):
        if t.dtype != dt or t.device != dev or not t.is_contiguous():
            raise ValueError("gradient_features: wrong dtype, device or layout of an input")
    L = _lib.lib()
    need = int(L.fmap_gradient_features_ws_bytes(int(dim)))
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ld_in = x_in.stride(0) if x_in.dim() == 2 else dim
    ld_out = out.stride(0) if out.dim() == 2 else dim
    check(L.fmap_gradient_features(int(n), _ptr(row_ptr), _ptr(col_idx), _ptr(g_vals), int(col_idx.numel()),
                                   int(x_in.shape[0]), _ptr(x_in), int(ld_in), int(dim), _ptr(a_re), _ptr(a_im),
                                   0 if variant == "A" else 1, _ptr(out), int(ld_out),
                                   _lib.FMAP_PREC_BF16 if bf16 else _lib.FMAP_PREC_FP32, _ptr(status), _ptr(ws),
                                   ws.numel(), _stream(dev)), "fmap_gradient_features")
    return out, status


def batch_from_workload(wl, device="cuda:0", with_grad=True, **kw) -> FmapBatch:
    """Allocate a batch for a synth.Workload and upload its inputs."""
    lay = BatchLayout([s.n for s in wl.shapes], [s.k for s in wl.shapes], [s.d for s in wl.shapes], wl.feat_dtype)
    masks = [p.mask for p in wl.pairs]
    lam_rows = [getattr(p, "lam_rows", None) for p in wl.pairs]
    if "lambda_rows" not in kw and any(v is not None for v in lam_rows):
        kw["lambda_rows"] = lam_rows
    b = FmapBatch(lay, [(p.x, p.y, p.lam) for p in wl.pairs], device=device, precision=wl.feat_dtype,
                  with_grad=with_grad, masks=masks, **kw)
    b.upload(lay.pack_host(wl.shapes))
    return b


def flat_c(batch: FmapBatch, mats: List[np.ndarray]) -> torch.Tensor:
    """Pack per-pair k_Y x k_X matrices into the flat C layout of `batch`."""
    host = np.zeros(int(batch.c_off[-1]), np.float32)
    for p, m in enumerate(mats):
        host[batch.c_off[p]:batch.c_off[p + 1]] = np.asarray(m, np.float32).reshape(-1)
    return torch.from_numpy(host).to(batch.device)


class FmapFunction(torch.autograd.Function):
    """C = fmap(F) for a bound batch: forward runs fmap_project + fmap_solve, backward
    runs fmap_solve_backward and returns dL/dF in the batch's flat feature layout."""

    @staticmethod
    def forward(ctx, feat: torch.Tensor, batch: FmapBatch):
        if feat.data_ptr() != batch.feat.data_ptr():
            batch.feat.copy_(feat.reshape(-1))
        a = batch.project().clone()
        c = batch.solve(a)
        batch._gen = getattr(batch, "_gen", 0) + 1
        ctx.gen = batch._gen
        ctx.batch = batch
        c = c.clone()
        ctx.save_for_backward(a, c)
        return c

    @staticmethod
    def backward(ctx, d_c):
        a, c = ctx.saved_tensors
        batch = ctx.batch
        use_saved = getattr(batch, "_gen", 0) == ctx.gen
        batch.solve_backward(d_c.contiguous(), a, c, use_saved=use_saved)
        return batch.dfeat.clone(), None
