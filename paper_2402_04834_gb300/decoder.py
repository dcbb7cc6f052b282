"""Python face of the blockBP decoder: device buffers from PyTorch, compute in libblockbp.

``decode`` takes a CUDA uint8 tensor of syndromes [B, m] and returns the
per-coset log-probabilities (Lemma 1), Delta, iteration counts, flags and the
decision of Algorithm 1.  ``decode_host`` takes host arrays and goes through
the library's host entry point (copies included).  ``sample`` draws seeded
depolarizing errors and syndromes on the device.
"""

from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from ._lib import DecoderParams, check, lib, workspace_bytes


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Workspace:
    """Device scratch for the decoder, grown on demand (256-byte aligned)."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != torch.device(device):
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        return self.buf


_default_ws = Workspace()


def decode(syndromes: torch.Tensor, prm: DecoderParams, workspace: Workspace | None = None,
           stream=None, out: dict | None = None) -> dict:
    """Decode syndromes [B, m] (CUDA uint8); all outputs stay on the device."""
    if not syndromes.is_cuda or syndromes.dtype != torch.uint8:
        raise ValueError("syndromes must be a CUDA uint8 tensor")
    syndromes = syndromes.contiguous()
    B = syndromes.shape[0]
    if syndromes.dim() != 2 or syndromes.shape[1] != prm.m:
        raise ValueError(f"syndromes must have shape [B, {prm.m}]")
    dev = syndromes.device
    if out is None:
        out = {
            "logp": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "delta": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "iters": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "flags": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "decision": torch.empty(B, dtype=torch.int8, device=dev),
        }
    ws = (workspace or _default_ws).get(workspace_bytes(prm, B), dev)
    cp = prm.c()
    check(lib().bbp_decode_batch(_ptr(syndromes), B, ctypes.byref(cp), _ptr(out["logp"]),
                                 _ptr(out["delta"]), _ptr(out["iters"]), _ptr(out["flags"]),
                                 _ptr(out["decision"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def decode_host(syndromes: np.ndarray, prm: DecoderParams, workspace: Workspace | None = None,
                stream=None, out: dict | None = None, device="cuda") -> dict:
    """Decode host syndromes [B, m]; the library copies in and out and syncs."""
    syndromes = np.ascontiguousarray(syndromes, dtype=np.uint8)
    B = syndromes.shape[0]
    if out is None:
        out = {"logp": np.empty((B, 4)), "delta": np.empty((B, 4)),
               "iters": np.empty((B, 4), dtype=np.int32), "flags": np.empty((B, 4), dtype=np.int32),
               "decision": np.empty(B, dtype=np.int8)}
    ws = (workspace or _default_ws).get(workspace_bytes(prm, B, include_io=True), device)
    cp = prm.c()

    def hp(a):
        return None if a is None else a.ctypes.data

    check(lib().bbp_decode_batch_host(syndromes.ctypes.data, B, ctypes.byref(cp), hp(out.get("logp")),
                                      hp(out.get("delta")), hp(out.get("iters")), hp(out.get("flags")),
                                      hp(out["decision"]), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def pure_error(syndromes: torch.Tensor, d: int, stream=None):
    """Pure error f_s of each syndrome on the device (Algorithm 1): (fx, fz), [B][n] uint8."""
    B = syndromes.shape[0]
    n = d * d + (d - 1) ** 2
    fx = torch.empty(B, n, dtype=torch.uint8, device=syndromes.device)
    fz = torch.empty(B, n, dtype=torch.uint8, device=syndromes.device)
    check(lib().bbp_pure_error(d, _ptr(syndromes), B, _ptr(fx), _ptr(fz), _stream(stream)))
    return fx, fz


def sample(seed: int, first_shot: int, B: int, d: int, p: float, device="cuda", with_errors=True,
           stream=None):
    """Seeded depolarizing errors and syndromes on the device (Sec. IV workload)."""
    n = d * d + (d - 1) ** 2
    m = 2 * d * (d - 1)
    ex = torch.empty(B, n, dtype=torch.uint8, device=device) if with_errors else None
    ez = torch.empty(B, n, dtype=torch.uint8, device=device) if with_errors else None
    s = torch.empty(B, m, dtype=torch.uint8, device=device)
    tc = torch.empty(B, dtype=torch.int8, device=device)
    check(lib().bbp_sample(seed, first_shot, B, d, p, _ptr(ex) if ex is not None else None,
                           _ptr(ez) if ez is not None else None, _ptr(s), _ptr(tc), _stream(stream)))
    return ex, ez, s, tc


def pack_mixed(syndromes_by_shot, device="cuda"):
    """Pack per-shot syndromes of different lengths: (packed, offsets, d_of)."""
    lens = [len(s) for s in syndromes_by_shot]
    d_of = []
    for m in lens:
        d = int(round((1 + (1 + 2 * m) ** 0.5) / 2))     # m = 2 d (d - 1)
        if 2 * d * (d - 1) != m:
            raise ValueError(f"syndrome length {m} is not 2d(d-1)")
        d_of.append(d)
    offsets = np.zeros(len(lens), dtype=np.int64)
    offsets[1:] = np.cumsum(lens)[:-1]
    packed = np.concatenate([np.asarray(s, dtype=np.uint8) for s in syndromes_by_shot])
    return (torch.from_numpy(packed).to(device), torch.from_numpy(offsets).to(device),
            torch.tensor(d_of, dtype=torch.int32, device=device))


def decode_mixed(packed, offsets, d_of, prm: DecoderParams, largest_first=True, stream=None, out=None,
                 counter=None, order=None, d_max=None):
    """Syndromes of different distances in one persistent launch (fused path).

    ``order`` and ``d_max`` may be passed precomputed (needed inside CUDA-graph
    capture, where they cannot be derived with a host synchronisation)."""
    B = d_of.shape[0]
    dev = d_of.device
    if out is None:
        out = {
            "logp": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "delta": torch.empty(B, 4, dtype=torch.float64, device=dev),
            "iters": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "flags": torch.empty(B, 4, dtype=torch.int32, device=dev),
            "decision": torch.empty(B, dtype=torch.int8, device=dev),
        }
    if order is None and largest_first:
        order = torch.argsort(d_of, descending=True, stable=True).to(torch.int32)
    if d_max is None:
        d_max = int(d_of.max().item())
    # The work counter, then the message slots when the launch shape keeps
    # its messages in the workspace (none otherwise).
    need = 256 + workspace_bytes(dataclasses.replace(prm, d=d_max), B)
    if counter is None or counter.numel() < need:
        counter = torch.empty(need, dtype=torch.uint8, device=dev)
    cp = prm.c()
    check(lib().bbp_decode_mixed(_ptr(packed), _ptr(offsets), _ptr(d_of), _ptr(order) if order is not None else None,
                                 B, d_max, ctypes.byref(cp), _ptr(out["logp"]), _ptr(out["delta"]),
                                 _ptr(out["iters"]), _ptr(out["flags"]), _ptr(out["decision"]), _ptr(counter),
                                 counter.numel(), _stream(stream)))
    return out
