"""Launch-shape autotuner of the fused decoder.

The results never depend on the launch shape; only the time does.  For a
given workload the tuner times every candidate (warps per CTA, and for
mixed batches resident CTAs per SM) with CUDA events and keeps the fastest,
caching the choice per workload signature for the life of the process.
"""

from __future__ import annotations

import dataclasses

import torch

from ._lib import DecoderParams
from .decoder import decode, decode_mixed

_cache: dict = {}


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_uniform(syndromes, prm: DecoderParams, warps=(4, 8, 16)):
    """Best warps per CTA for a same-distance batch; returns (params, table)."""
    key = ("uniform", prm.d, prm.k, prm.precision, prm.max_iter)
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    cands = warps if prm.precision == "fp32" else (8,)
    table = []
    for w in cands:
        p2 = dataclasses.replace(prm, warps=w)
        table.append(({"warps": w}, _time(lambda: decode(syndromes, p2))))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table


def tune_mixed(packed, offsets, d_of, prm: DecoderParams, warps=(4, 8, 16), ctas=(0, 1, 2, 3, 4)):
    """Best (warps, resident CTAs per SM) for a mixed batch; returns (params, table)."""
    sig = tuple(sorted(torch.unique(d_of).tolist()))
    key = ("mixed", sig, prm.k, prm.precision, prm.max_iter)
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    cands = warps if prm.precision == "fp32" else (8,)
    counter = torch.empty(256, dtype=torch.uint8, device=d_of.device)
    table = []
    for w in cands:
        for c in ctas:
            p2 = dataclasses.replace(prm, warps=w, ctas_per_sm=c)
            try:
                t = _time(lambda: decode_mixed(packed, offsets, d_of, p2, counter=counter))
            except RuntimeError:
                continue          # a shape the shared memory cannot hold
            table.append(({"warps": w, "ctas_per_sm": c}, t))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table
