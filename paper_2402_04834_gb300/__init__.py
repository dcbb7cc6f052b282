"""GB300 blockBP decoder for the planar surface code (arXiv:2402.04834).

The compute path is libblockbp.so (hand-written sm_103a CUDA, C ABI in
include/blockbp.h); this package only marshals arguments and provides
device memory and streams through PyTorch.
"""

from ._lib import (FP32, FP64, FUSED_SHAPES, FUSED_SHAPES_K6, FUSED_SHAPES_WS, BbpError, DecoderParams,  # noqa: F401
                   lib, workspace_bytes)
from .decoder import Workspace, decode, decode_host, pure_error, sample  # noqa: F401

__all__ = ["DecoderParams", "decode", "decode_host", "pure_error", "sample", "workspace_bytes", "Workspace",
           "lib", "BbpError", "FP32", "FP64"]
