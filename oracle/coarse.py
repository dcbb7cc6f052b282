"""The paper's scheme for blocks of 6 x 6 nodes (Sec. IV, decoder
parameters), step by step in float64.  Test infrastructure only.

For its largest blocks the paper first fuses the network's nodes in groups of
3 x 3 into single tensors, whose legs bundle three bonds of dimension 2 into
one of dimension D' = 8, and then runs blockBP on the fused network with
blocks of 2 x 2 fused tensors (6 x 6 nodes) and MPS messages of bond
chi = 16.  A message then has two sites of dimension 8, so its exact bond
(at most 8) never exceeds chi; what chi = 16 truncates is the boundary MPS
inside a block, whose middle bond reaches 64 after the first fused column.

Parity status: pinned.  Fusing keeps the exact contraction (one block over
the whole fused network with a large bond equals the exact value); with chi
large enough that nothing is truncated the scheme equals the dense
fused-block BP of Remark 9 with 6 x 6 blocks (``oracle.naive``); as chi
grows it converges to that value.  With chi = 16 it is an approximation with
no closed form.

Reading: fused tensors are anchored at (0, 0) like the blocks; the last
fused row / column takes the remainder (Remark 1), so with 2 x 2 fused
blocks the block boundaries are those of 6 x 6 node blocks.  A fused leg
lists its bonds top -> bottom (left -> right), the first one most
significant, the site order of the messages.
"""

from __future__ import annotations

import numpy as np

from . import mps as M
from .blockbp import Params, decide, ranges, run_blockbp
from .lattice import Lattice
from .naive import fuse_block
from .tn import coset_network


def coarse_grain(tensors, f: int = 3):
    """Fuse f x f groups of nodes into single tensors, axes (l, r, u, d)."""
    g = ranges(len(tensors), f)
    return [[fuse_block(tensors, rows, cols) for cols in g] for rows in g]


def decode_coarse(s, d: int, p: float, chi: int = 16, f: int = 3, kb: int = 2, max_iter: int = 20,
                  eta: float = 0.1, delta0: float = 1e-4, delta1: float = 1e-2, cutoff: float = 1e-13):
    """Decode one syndrome with the fused-network scheme; per-coset results
    and the decision of Algorithm 1 / Remark 6."""
    lat = Lattice(d)
    stats = M.Stats()
    P = Params(d=d, k=kb, D=chi, p=p, max_iter=max_iter, eta=eta, delta0=delta0, delta1=delta1, cutoff=cutoff)
    res = [run_blockbp(coarse_grain(coset_network(lat, s, L, p), f), P, stats) for L in range(4)]
    logp = np.array([r.logp for r in res])
    delta = np.array([r.delta for r in res])
    iters = np.array([r.iters for r in res], dtype=np.int64)
    flags = np.array([r.flags for r in res], dtype=np.int64)
    return {"logp": logp, "delta": delta, "iters": iters, "flags": flags,
            "decision": decide(logp, delta, flags), "stats": stats}
