"""ctypes binding of libblockbp.so (include/blockbp.h); argument marshalling only.

Every step of the decoder runs in the library's CUDA kernels.  If the library
is missing this module raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libblockbp.so")

BBP_OK = 0
FP64, FP32 = 0, 1
ALG_MPS, ALG_FUSED = 0, 1
FLAG_UNTRUSTED, FLAG_OVERLAP, FLAG_BLOCK, FLAG_NONFINITE = 1, 2, 4, 8
FLAG_CAPACITY, FLAG_CHECK = 1 << 16, 1 << 17

# Exported symbols, as declared in include/blockbp.h.
SYMBOLS = ("bbp_workspace_bytes", "bbp_decode_batch", "bbp_decode_batch_host", "bbp_sample",
           "bbp_strerror", "bbp_version", "bbp_decode_batch_static", "bbp_message_count",
           "bbp_message_features", "bbp_warm_param_count", "bbp_warm_workspace_bytes", "bbp_warm_infer",
           "bbp_warm_train_step", "bbp_decode_batch_ex", "bbp_decode_mixed", "bbp_warm_infer_syndromes",
           "bbp_pure_error", "bbp_message_classes", "bbp_message_features_rows", "bbp_expand_rows",
           "bbp_decode_warm", "bbp_decode_warm_host", "bbp_decode_warm_workspace_bytes",
           "bbp_message_feature_bits_rows", "bbp_warm_infer_bits")
WARM_F, WARM_H, WARM_O, WARM_MAX_ROWS = 256, 256, 16, 4194240
WARM_STATUS_OFFSET = 270336       # int32 status word of bbp_warm_infer in its workspace
WARM_INFER_WS_BYTES = 270592      # workspace of bbp_warm_infer, for any N
# Compiled launch shapes (warps per CTA, cosets per CTA) of the fused kernel.
FUSED_SHAPES = {"fp32": ((8, 4), (8, 2), (4, 2), (4, 4), (16, 1), (8, 1), (4, 1)),
                "fp64": ((4, 2), (8, 2), (8, 1), (4, 4))}
# ... of which these also with their messages in workspace slots (messages=2)
FUSED_SHAPES_WS = {"fp32": ((8, 4), (8, 2)), "fp64": ((4, 2),)}
# ... of which these also in register-form-only variants (messages=3; k = 4
# with a one-node-wide last block, i.e. odd d), sized for more CTAs per SM.
FUSED_SHAPES_LEAN = {"fp32": ((8, 4), (8, 2)), "fp64": ((4, 2), (8, 2))}
# ... and for block sides 5 and 6 (one coset per CTA, messages in the workspace).
FUSED_SHAPES_K6 = {"fp32": ((6, 1), (4, 1), (2, 1)), "fp64": ((3, 1), (2, 1))}
BBP_ETOOLARGE = -5
STATIC_WORKSPACE_BYTES = 32 << 20


class BbpParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("k", ctypes.c_int32), ("D", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("p", ctypes.c_double), ("eta", ctypes.c_double),
                ("delta0", ctypes.c_double), ("delta1", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("precision", ctypes.c_int32), ("algorithm", ctypes.c_int32),
                ("launch_warps", ctypes.c_int32), ("launch_ctas_per_sm", ctypes.c_int32),
                ("launch_cosets", ctypes.c_int32), ("launch_messages", ctypes.c_int32)]


@dataclass
class DecoderParams:
    """Decoder parameters (Sec. III.E); defaults are the values of Sec. IV."""
    d: int
    k: int = 4
    D: int = 8
    p: float = 0.1
    max_iter: int = 20
    eta: float = 0.1
    delta0: float = 1e-4
    delta1: float = 1e-2
    cutoff: float | None = None
    precision: str = "fp64"
    algorithm: str = "mps"          # "mps" (Sec. III.D) or "fused" (Remark 9, k <= 6)
    warps: int = 0                  # fused launch shape (tuning only): warps per CTA
    ctas_per_sm: int = 0            # persistent mixed launch: resident CTAs per SM (0 = occupancy)
    cosets: int = 0                 # fused launch shape (tuning only): cosets per CTA (1, 2, 4)
    messages: int = 0               # fused (tuning only): 1 shared memory, 2 workspace slots, 3 register form only, 0 = default

    def c(self) -> BbpParams:
        prec = FP64 if self.precision == "fp64" else FP32
        cut = self.cutoff if self.cutoff is not None else (1e-13 if prec == FP64 else 1e-7)
        alg = ALG_MPS if self.algorithm == "mps" else ALG_FUSED
        return BbpParams(self.d, self.k, self.D, self.max_iter, self.p, self.eta, self.delta0,
                         self.delta1, cut, prec, alg, self.warps, self.ctas_per_sm, self.cosets, self.messages)

    @property
    def m(self) -> int:
        return 2 * self.d * (self.d - 1)


class BbpError(RuntimeError):
    pass


_lib = None
_lib_path = LIB_PATH


def use_library(path: str | None = None):
    """Make lib() load the library at ``path`` (None: the default build), e.g.
    the build with device bounds checks; returns the path used before."""
    global _lib, _lib_path
    prev = _lib_path
    path = path or LIB_PATH
    if path != _lib_path:
        _lib, _lib_path = None, path
    return prev


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_lib_path):
            raise BbpError(f"{_lib_path} is missing: build it with paper_2402_04834_gb300.build.build()")
        L = ctypes.CDLL(_lib_path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        P = ctypes.POINTER(BbpParams)
        L.bbp_workspace_bytes.argtypes = [P, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        L.bbp_workspace_bytes.restype = ctypes.c_int
        L.bbp_decode_batch.argtypes = [vp, i64, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bbp_decode_batch.restype = ctypes.c_int
        L.bbp_decode_batch_host.argtypes = [vp, i64, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bbp_decode_batch_host.restype = ctypes.c_int
        L.bbp_decode_batch_ex.argtypes = [vp, i64, P, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bbp_decode_mixed.argtypes = [vp, vp, vp, vp, i64, i32, P, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bbp_decode_mixed.restype = ctypes.c_int
        L.bbp_decode_batch_ex.restype = ctypes.c_int
        L.bbp_message_count.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        L.bbp_message_count.restype = ctypes.c_int
        L.bbp_message_features.argtypes = [vp, i64, P, vp, vp, vp]
        L.bbp_message_features.restype = ctypes.c_int
        L.bbp_warm_param_count.argtypes = []
        L.bbp_warm_param_count.restype = ctypes.c_int
        L.bbp_warm_workspace_bytes.argtypes = [i64, ctypes.POINTER(ctypes.c_size_t)]
        L.bbp_warm_workspace_bytes.restype = ctypes.c_int
        L.bbp_warm_infer.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp, ctypes.c_size_t, vp]
        L.bbp_warm_infer_syndromes.argtypes = [vp, vp, i64, P, ctypes.c_float, vp, vp, ctypes.c_size_t, vp]
        L.bbp_warm_infer_syndromes.restype = ctypes.c_int
        L.bbp_warm_infer.restype = ctypes.c_int
        L.bbp_warm_train_step.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp, vp, i64, vp, vp, vp,
                                          ctypes.c_size_t, vp]
        L.bbp_warm_train_step.restype = ctypes.c_int
        L.bbp_decode_batch_static.argtypes = [vp, i64, P, vp, vp, vp, vp, vp, vp]
        L.bbp_decode_batch_static.restype = ctypes.c_int
        L.bbp_sample.argtypes = [ctypes.c_uint64, i64, i64, i32, ctypes.c_double, vp, vp, vp, vp, vp]
        L.bbp_sample.restype = ctypes.c_int
        L.bbp_pure_error.argtypes = [i32, vp, i64, vp, vp, vp]
        L.bbp_pure_error.restype = ctypes.c_int
        L.bbp_message_classes.argtypes = [P, vp, vp, ctypes.POINTER(i32)]
        L.bbp_message_classes.restype = ctypes.c_int
        L.bbp_message_features_rows.argtypes = [vp, i64, P, vp, i32, vp, vp, vp]
        L.bbp_message_features_rows.restype = ctypes.c_int
        L.bbp_message_feature_bits_rows.argtypes = [vp, i64, P, vp, i32, vp, vp, vp]
        L.bbp_message_feature_bits_rows.restype = ctypes.c_int
        L.bbp_warm_infer_bits.argtypes = [vp, vp, vp, i64, ctypes.c_double, ctypes.c_float, vp, vp, ctypes.c_size_t,
                                          vp]
        L.bbp_warm_infer_bits.restype = ctypes.c_int
        L.bbp_expand_rows.argtypes = [vp, i64, i32, vp, i32, vp, vp]
        L.bbp_expand_rows.restype = ctypes.c_int
        L.bbp_decode_warm.argtypes = [vp, vp, i64, P, ctypes.c_float, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.bbp_decode_warm.restype = ctypes.c_int
        L.bbp_decode_warm_host.argtypes = [vp, vp, i64, P, ctypes.c_float, vp, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                           vp]
        L.bbp_decode_warm_host.restype = ctypes.c_int
        L.bbp_decode_warm_workspace_bytes.argtypes = [P, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
        L.bbp_decode_warm_workspace_bytes.restype = ctypes.c_int
        L.bbp_strerror.argtypes = [ctypes.c_int]
        L.bbp_strerror.restype = ctypes.c_char_p
        L.bbp_version.argtypes = []
        L.bbp_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(rc: int):
    if rc != BBP_OK:
        raise BbpError(f"blockbp error {rc}: {lib().bbp_strerror(rc).decode()}")


def workspace_bytes(prm: DecoderParams, B: int, include_io: bool = False) -> int:
    out = ctypes.c_size_t(0)
    cp = prm.c()
    check(lib().bbp_workspace_bytes(ctypes.byref(cp), B, int(include_io), ctypes.byref(out)))
    return int(out.value)
