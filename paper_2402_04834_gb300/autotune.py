"""Launch-shape autotuner of the fused decoder.

The results never depend on the launch shape; only the time does.  For a
given workload the tuner times every candidate (warps per CTA, cosets per
CTA, messages in shared memory or in workspace slots, and for mixed batches
resident CTAs per SM) with CUDA events and
keeps the fastest, caching the choice per workload signature for the life
of the process.  Shapes whose shared memory does not fit are skipped.
"""

from __future__ import annotations

import dataclasses

import torch

from ._lib import FUSED_SHAPES, FUSED_SHAPES_K6, FUSED_SHAPES_LEAN, FUSED_SHAPES_WS, BbpError, DecoderParams
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


def candidates(prm: DecoderParams):
    """Compiled (warps, cosets, messages) of the fused kernel: messages 1 in
    shared memory, 2 in workspace slots (always for k = 5, 6), 3 every block
    update in register form (k = 4 at odd d)."""
    if prm.k > 4:
        return tuple((w, c, 2) for w, c in FUSED_SHAPES_K6[prm.precision])
    lean = ()
    if prm.k == 4 and prm.d % 2 == 1:
        lean = tuple((w, c, 3) for w, c in FUSED_SHAPES_LEAN[prm.precision])
    return (lean + tuple((w, c, 1) for w, c in FUSED_SHAPES[prm.precision]) +
            tuple((w, c, 2) for w, c in FUSED_SHAPES_WS[prm.precision]))


def tune_uniform(syndromes, prm: DecoderParams, shapes=None):
    """Best (warps, cosets, messages) for a same-distance batch; returns (params, table)."""
    shapes = tuple(shapes or candidates(prm))
    key = ("uniform", prm.d, prm.k, prm.precision, prm.max_iter, shapes)
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    table = []
    for w, c, mem in shapes:
        p2 = dataclasses.replace(prm, warps=w, cosets=c, messages=mem)
        try:
            t = _time(lambda: decode(syndromes, p2))
        except BbpError:
            continue          # a shape the shared memory cannot hold
        table.append(({"warps": w, "cosets": c, "messages": mem}, t))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table


def tune_mixed(packed, offsets, d_of, prm: DecoderParams, shapes=None, ctas=(0, 1, 2, 3, 4)):
    """Best (warps, cosets, messages, resident CTAs per SM) for a mixed batch; returns (params, table).
    The register-form-only shapes (messages 3) are candidates when every
    distance of the batch is odd (k = 4)."""
    sig = tuple(sorted(torch.unique(d_of).tolist()))
    if shapes is None:
        shapes = candidates(prm)
        if prm.k == 4 and all(d % 2 == 1 for d in sig):
            shapes = tuple((w, c, 3) for w, c in FUSED_SHAPES_LEAN[prm.precision]) + tuple(shapes)
    shapes = tuple(shapes)
    key = ("mixed", sig, prm.k, prm.precision, prm.max_iter, shapes, tuple(ctas))
    if key in _cache:
        return dataclasses.replace(prm, **_cache[key][0]), _cache[key][1]
    table = []
    for w, c, mem in shapes:
        for n in ctas:
            p2 = dataclasses.replace(prm, warps=w, cosets=c, messages=mem, ctas_per_sm=n)
            try:
                t = _time(lambda: decode_mixed(packed, offsets, d_of, p2))
            except BbpError:
                continue
            table.append(({"warps": w, "cosets": c, "messages": mem, "ctas_per_sm": n}, t))
    best = min(table, key=lambda x: x[1])
    _cache[key] = (best[0], table)
    return dataclasses.replace(prm, **best[0]), table
