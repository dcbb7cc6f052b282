"""Launch-shape autotuner of the fused decoder.

The results never depend on the launch shape; only the time does.  For a
given workload the tuner times every candidate (warps per CTA and cosets
per CTA, and for mixed batches resident CTAs per SM) with CUDA events and
keeps the fastest, caching the choice per workload signature for the life
of the process.  Shapes whose shared memory does not fit are skipped.
"""

from __future__ import annotations

import dataclasses

import torch

from ._lib import FUSED_SHAPES, FUSED_SHAPES_K6, BbpError, DecoderParams
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


def tune_uniform(syndromes, prm: DecoderParams, shapes=None):
    """Best (warps, cosets) per CTA for a same-distance batch; returns (params, table)."""
    shapes = tuple(shapes or (FUSED_SHAPES_K6 if prm.k > 4 else FUSED_SHAPES)[prm.precision])
    key = ("uniform", prm.d, prm.k, prm.precision, prm.max_iter, shapes)
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    table = []
    for w, c in shapes:
        p2 = dataclasses.replace(prm, warps=w, cosets=c)
        try:
            t = _time(lambda: decode(syndromes, p2))
        except BbpError:
            continue          # a shape the shared memory cannot hold
        table.append(({"warps": w, "cosets": c}, t))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table


def tune_mixed(packed, offsets, d_of, prm: DecoderParams, shapes=None, ctas=(0, 1, 2, 3, 4)):
    """Best (warps, cosets, resident CTAs per SM) for a mixed batch; returns (params, table)."""
    shapes = tuple(shapes or (FUSED_SHAPES_K6 if prm.k > 4 else FUSED_SHAPES)[prm.precision])
    sig = tuple(sorted(torch.unique(d_of).tolist()))
    key = ("mixed", sig, prm.k, prm.precision, prm.max_iter, shapes, tuple(ctas))
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    counter = torch.empty(256, dtype=torch.uint8, device=d_of.device)
    table = []
    for w, c in shapes:
        for n in ctas:
            p2 = dataclasses.replace(prm, warps=w, cosets=c, ctas_per_sm=n)
            try:
                t = _time(lambda: decode_mixed(packed, offsets, d_of, p2, counter=counter))
            except BbpError:
                continue
            table.append(({"warps": w, "cosets": c, "ctas_per_sm": n}, t))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table
