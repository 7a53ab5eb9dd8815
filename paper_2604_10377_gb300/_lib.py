"""ctypes binding of libfmap.so (the C ABI of include/fmap.h): argument marshalling only.

The library is loaded from the package directory. If it is missing the import
of any compute entry point fails loudly: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmap.so")

FMAP_OK = 0
FMAP_ERR_INVALID_ARG = 1
FMAP_ERR_UNSUPPORTED = 2
FMAP_ERR_CUDA = 3
FMAP_ERR_NOT_SPD = 4
FMAP_ERR_NONFINITE = 5
FMAP_ERR_TIMEOUT = 6
FMAP_ERR_WORKSPACE = 7

FMAP_PREC_FP32 = 0
FMAP_PREC_BF16 = 1


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("ir_steps", c_int32), ("hi_gram_min_k", c_int32),
                ("store_factors_max_k", c_int32), ("adjoint_ir_steps", c_int32),
                ("proj_max_stages", c_int32), ("proj_seg_max_v", c_int32), ("bwd_group_features", c_int32),
                ("bwd_chunk_v", c_int32), ("solve_threads_k64", c_int32), ("solve_threads_k128", c_int32),
                ("proj_ctas", c_int32), ("bwd_ctas", c_int32), ("solve_no_g_copy", c_int32),
                ("adjoint_kernel", c_int32),
                ("adjoint_features", c_int32), ("adjoint_stages", c_int32)]


TUNING_FIELDS = ("proj_max_stages", "proj_seg_max_v", "bwd_group_features", "bwd_chunk_v", "proj_ctas", "bwd_ctas",
                 "solve_threads_k64", "solve_threads_k128", "solve_no_g_copy", "adjoint_kernel",
                 "adjoint_features", "adjoint_stages")


class ShapeDesc(ctypes.Structure):
    _fields_ = [("n", c_int64), ("k", c_int32), ("d", c_int32), ("phi", c_void_p), ("ld_phi", c_int64),
                ("mass", c_void_p), ("evals", c_void_p), ("feat", c_void_p), ("ld_feat", c_int64),
                ("dfeat", c_void_p), ("dfeat_f32", c_void_p)]


class PairDesc(ctypes.Structure):
    _fields_ = [("shape_x", c_int32), ("shape_y", c_int32), ("lam", c_float), ("mask", c_void_p),
                ("lambda_rows", c_void_p), ("d_lambda_rows", c_void_p)]


class Sizes(ctypes.Structure):
    _fields_ = [("a_floats", c_int64), ("c_floats", c_int64), ("ws_bytes", c_int64), ("ws_bwd_bytes", c_int64),
                ("saved_bytes", c_int64), ("n_shapes", c_int32), ("n_pairs", c_int32)]


class FmapError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {error_string(code)} (code {code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


_lib = None

# name -> (restype, argtypes)
_PROTOS = {
    "fmap_version": (c_char_p, []),
    "fmap_error_string": (c_char_p, [c_int32]),
    "fmap_last_cuda_error": (c_char_p, []),
    "fmap_default_options": (c_int32, [POINTER(Options)]),
    "fmap_create": (c_int32, [POINTER(c_void_p), c_int32, POINTER(Options)]),
    "fmap_destroy": (c_int32, [c_void_p]),
    "fmap_plan_sizes": (c_int32, [POINTER(Options), POINTER(ShapeDesc), c_int32, POINTER(PairDesc), c_int32,
                                  POINTER(Sizes)]),
    "fmap_batch_create": (c_int32, [c_void_p, POINTER(ShapeDesc), c_int32, POINTER(PairDesc), c_int32,
                                    POINTER(c_void_p)]),
    "fmap_batch_destroy": (c_int32, [c_void_p]),
    "fmap_batch_sizes": (c_int32, [c_void_p, POINTER(Sizes)]),
    "fmap_batch_offsets": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int64)]),
    "fmap_project": (c_int32, [c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_solve": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_solve_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_adjoint": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_project_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_loss_orth": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "fmap_batch_set_timing": (c_int32, [c_void_p, c_int32]),
    "fmap_batch_read_timing": (c_int32, [c_void_p, POINTER(c_float), POINTER(c_int32), c_int32]),
    "fmap_solve_pair_noalloc": (c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                          c_float, c_int32, c_void_p, c_void_p, c_void_p]),
    "fmap_gradient_features_ws_bytes": (c_size_t, [c_int32]),
    "fmap_gradient_features": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_int64,
                                         c_int32, c_void_p, c_void_p, c_int32, c_void_p, c_int64, c_int32, c_void_p,
                                         c_void_p, c_size_t, c_void_p]),
    "fmap_peak_loop": (c_int32, [c_int32, c_int32, c_int64, c_void_p, POINTER(ctypes.c_double), c_void_p]),
    "fmap_overlap_metrics": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_float, c_void_p, c_void_p,
                                       c_void_p]),
}

KIND_NAMES = ["project", "project_reduce", "gram", "solve", "adj_solve", "adj_gemm", "gather", "project_bwd",
              "loss", "status"]


def lib():
    """Load libfmap.so (once). Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfmap.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                              "python paper_2604_10377_gb300/build.py")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def error_string(code: int) -> str:
    return lib().fmap_error_string(int(code)).decode()


def check(rc: int, where: str):
    if rc != FMAP_OK:
        detail = lib().fmap_last_cuda_error().decode() if rc == FMAP_ERR_CUDA else ""
        raise FmapError(rc, where, detail)


def default_options() -> Options:
    o = Options()
    check(lib().fmap_default_options(ctypes.byref(o)), "fmap_default_options")
    return o
