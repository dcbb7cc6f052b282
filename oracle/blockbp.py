"""blockBP decoder, Algorithm 1 with Remarks 1-8, step by step in float64.

Parity status: pinned.  Special cases with exact answers fix every step:
one block covering the network with a large bond is the exact contraction
(Sec. III.D, bMPS limit); a partition into vertical strips is a chain, where
BP with Lemma 1 is exact (Sec. III.C); with k = 3, D = 4 nothing is ever
truncated and the result equals the dense fused-block BP of Remark 9
(``oracle.naive``); the decision rule is checked branch by branch.  Beyond
those cases blockBP is an approximation with no closed form; its distance to
the exact coset probabilities is reported, not gated.

Readings where the paper is silent (each one also listed in the design notes):

* Partition (Algorithm 1, Remark 1): blocks of k x k network nodes anchored
  at (0, 0); the last block row / column takes the remainder W - k(n_b-1).
* Messages (Sec. III.D): the message from block v to block u is an MPS over
  the edges crossing their shared side, sites ordered top -> bottom on a
  vertical side and left -> right on a horizontal side.
* Block update (Eq. BP-update on blocks, Fig. 3): boundary MPS from the
  incoming message on the side opposite the outgoing one, absorbing one
  network column (or row) at a time; the two side messages are absorbed
  site by site at the chain ends, their open bonds riding along as end
  bonds of the running MPS; after every absorbed column the running MPS is
  compressed to bond D (``mps.compress``).
* Normalisation (Remark 3): left-canonical, unit L2 norm.
* Damping (Remark 7): the damped message is compress((1-eta) m_new + eta
  m_old) renormalised, applied at every update including the first.
* Schedule (Remark 8): black blocks (I+J even) send first, then white; one
  iteration is both half-rounds.
* Delta (Remark 4): Frobenius norm, 1/M outside the square root; for unit
  vectors ||aa^T - bb^T||_F^2 = 2 - 2<a|b>^2.
* Read-out (Lemma 1): Z_v contracts block v with all four incoming messages
  by sweeping its columns left to right and closing with the message from
  the right, without compressing after the last column; o_e = <m_uv|m_vu>;
  log P = sum_v log Z_v - sum_e log o_e.  Z_v <= 0 or o_e <= 0 is flagged.
* Decision (Algorithm 1, Remark 6): among cosets with Delta < delta1 and no
  flag take the largest log P; if there is none take the smallest Delta;
  ties go to the lowest index in the order I, X, Y, Z.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import mps as M
from .lattice import Lattice
from .tn import coset_network

FLAG_UNTRUSTED = 1      # Delta >= delta1 (Remark 6)
FLAG_OVERLAP = 2        # some o_e <= 0
FLAG_BLOCK = 4          # some Z_v <= 0
FLAG_NONFINITE = 8      # a norm or log went non-finite

DIRS = ("R", "L", "D", "U")
STEP = {"R": (0, 1), "L": (0, -1), "D": (1, 0), "U": (-1, 0)}
OPPOSITE = {"R": "L", "L": "R", "D": "U", "U": "D"}


@dataclass
class Params:
    d: int
    k: int
    D: int
    p: float
    max_iter: int = 20
    eta: float = 0.1
    delta0: float = 1e-4
    delta1: float = 1e-2
    cutoff: float = 1e-13
    k_cols: int | None = None     # rectangular blocks (tests only)


@dataclass
class CosetResult:
    logp: float
    delta: float
    iters: int
    flags: int
    messages: dict = field(default_factory=dict, repr=False)


def ranges(W: int, k: int):
    """Block index ranges along one axis (Algorithm 1 'partition'; Remark 1)."""
    return [(a, min(a + k, W)) for a in range(0, W, k)]


class BlockNetwork:
    """One coset network partitioned into blocks (Sec. III.D, Fig. 3)."""

    def __init__(self, tensors, k_rows: int, k_cols: int):
        self.T = tensors
        self.W = len(tensors)
        self.rows = ranges(self.W, k_rows)
        self.cols = ranges(self.W, k_cols)
        self.nbr = len(self.rows)
        self.nbc = len(self.cols)

    def has(self, I, J, dr):
        di, dj = STEP[dr]
        return 0 <= I + di < self.nbr and 0 <= J + dj < self.nbc

    def directed_edges(self):
        return [(I, J, dr) for I in range(self.nbr) for J in range(self.nbc)
                for dr in DIRS if self.has(I, J, dr)]

    def side_len(self, I, J, dr):
        r0, r1 = self.rows[I]
        c0, c1 = self.cols[J]
        return (r1 - r0) if dr in ("R", "L") else (c1 - c0)

    def side_dims(self, I, J, dr):
        """Dimensions of the legs crossing side ``dr`` of block (I, J), in
        message site order (2 each in the coset network; a fused network has
        larger legs)."""
        r0, r1 = self.rows[I]
        c0, c1 = self.cols[J]
        T = self.T
        if dr == "R":
            return [T[i][c1 - 1].shape[1] for i in range(r0, r1)]
        if dr == "L":
            return [T[i][c0].shape[0] for i in range(r0, r1)]
        if dr == "D":
            return [T[r1 - 1][j].shape[3] for j in range(c0, c1)]
        return [T[r0][j].shape[2] for j in range(c0, c1)]

    def incoming(self, msgs, I, J, side):
        """Message arriving at (I, J) across ``side``; trivial at the border."""
        if self.has(I, J, side):
            di, dj = STEP[side]
            return msgs[(I + di, J + dj, OPPOSITE[side])]
        return [np.ones((1, 1, 1)) for _ in range(self.side_len(I, J, side))]

    def frame(self, msgs, I, J, dr):
        """Rotate block (I, J) so that ``dr`` points right.

        Returns (columns, in_msg, sideA, sideB): columns in consumption order,
        each a chain of tensors with axes (in, out, chain-prev, chain-next);
        in_msg the MPS on the opposite side; sideA / sideB the side messages'
        sites in consumption order, axes (bond-in, phys, bond-out)."""
        r0, r1 = self.rows[I]
        c0, c1 = self.cols[J]
        T = self.T
        left = self.incoming(msgs, I, J, "L")
        right = self.incoming(msgs, I, J, "R")
        top = self.incoming(msgs, I, J, "U")
        bot = self.incoming(msgs, I, J, "D")
        if dr == "R":
            cols = [[T[i][j] for i in range(r0, r1)] for j in range(c0, c1)]
            return cols, left, top, bot
        if dr == "L":
            cols = [[np.transpose(T[i][j], (1, 0, 2, 3)) for i in range(r0, r1)]
                    for j in range(c1 - 1, c0 - 1, -1)]
            return cols, right, M.reverse(top), M.reverse(bot)
        if dr == "D":
            cols = [[np.transpose(T[i][j], (2, 3, 0, 1)) for j in range(c0, c1)]
                    for i in range(r0, r1)]
            return cols, top, left, right
        cols = [[np.transpose(T[i][j], (3, 2, 0, 1)) for j in range(c0, c1)]
                for i in range(r1 - 1, r0 - 1, -1)]
        return cols, bot, M.reverse(left), M.reverse(right)


def absorb(psi, col, SA, SB, stats):
    """Apply one network column (an MPO) and its two side-message sites.

    Running-MPS bonds are (old bond, MPO bond) pairs; the side messages'
    bonds are the end bonds of the chain."""
    h = len(psi)
    if h == 1:
        A = np.einsum("aib,iocn,acx,bny->xoy", psi[0], col[0], SA, SB)
        stats.contract(*psi[0].shape, *col[0].shape[1:], SA.shape[2], SB.shape[2])
        return [A]
    out = []
    a, i, b = psi[0].shape
    _, o, c, n = col[0].shape
    A = np.einsum("aib,iocn,acx->xobn", psi[0], col[0], SA)
    stats.contract(a, i, b, o, c, n)
    stats.contract(a, c, SA.shape[2], b, o, n)
    out.append(A.reshape(A.shape[0], o, b * n))
    for s in range(1, h - 1):
        p_, i, b = psi[s].shape
        _, o, c, n = col[s].shape
        A = np.einsum("pib,iocn->pcobn", psi[s], col[s])
        stats.contract(p_, i, b, o, c, n)
        out.append(A.reshape(p_ * c, o, b * n))
    p_, i, b = psi[h - 1].shape
    _, o, c, n = col[h - 1].shape
    A = np.einsum("pib,iocn,bny->pcoy", psi[h - 1], col[h - 1], SB)
    stats.contract(p_, i, b, o, c, n)
    stats.contract(p_, c, o, b, n, SB.shape[2])
    out.append(A.reshape(p_ * c, o, A.shape[3]))
    return out


def sweep(cols, in_msg, SA, SB, P: Params, stats, compress_last=True):
    """Boundary-MPS contraction of one block (Sec. III.A inside Sec. III.D).

    Returns (psi, log_scale): the unit-norm running MPS after the last
    column and the log of the norm taken out of it."""
    psi = [A.copy() for A in in_msg]
    log_scale = 0.0
    last = len(cols) - 1
    for t, col in enumerate(cols):
        psi = absorb(psi, col, SA[t], SB[t], stats)
        if t < last or compress_last:
            psi, ln = M.compress(psi, P.D, P.cutoff, stats)
            log_scale += ln
    return psi, log_scale


def block_update(net: BlockNetwork, msgs, I, J, dr, P: Params, stats):
    """Outgoing message of block (I, J) towards ``dr`` (Eq. BP-update)."""
    cols, in_msg, SA, SB = net.frame(msgs, I, J, dr)
    psi, _ = sweep(cols, in_msg, SA, SB, P, stats)
    return psi


def damp(new, old, P: Params, stats):
    """Remark 7 damping, recompressed to D and renormalised (Remark 3)."""
    summed = M.direct_sum(1.0 - P.eta, new, P.eta, old)
    out, _ = M.compress(summed, P.D, P.cutoff, stats)
    return out


def block_log_z(net: BlockNetwork, msgs, I, J, P: Params, stats):
    """log Z_v of Lemma 1 for block (I, J) and whether Z_v > 0."""
    cols, in_msg, SA, SB = net.frame(msgs, I, J, "R")
    psi, log_scale = sweep(cols, in_msg, SA, SB, P, stats, compress_last=False)
    right = net.incoming(msgs, I, J, "R")
    z = M.overlap(psi, right, stats)
    if z == 0.0 or not np.isfinite(z):
        return -np.inf, False
    return log_scale + math.log(abs(z)), z > 0


def run_blockbp(tensors, P: Params, stats=None) -> CosetResult:
    """Algorithm 1 for one coset network: BP loop, Delta, Lemma 1 read-out.

    The arithmetic runs in the tensors' dtype (float64 for the oracle's
    values; float32 only to measure what the method gives in single
    precision); logs and sums of the read-out are Python floats."""
    stats = stats if stats is not None else M.Stats()
    kc = P.k_cols if P.k_cols is not None else P.k
    net = BlockNetwork(tensors, P.k, kc)
    edges = net.directed_edges()
    dt = tensors[0][0].dtype
    msgs = {e: [A.astype(dt) for A in M.uniform_dims(net.side_dims(*e))] for e in edges}   # Remark 2
    Mtot = len(edges)
    delta = 0.0
    iters = 0
    flags = 0
    if Mtot > 0:
        for it in range(1, P.max_iter + 1):
            prev = dict(msgs)
            for color in (0, 1):                                 # Remark 8
                upd = {}
                for (I, J, dr) in edges:
                    if (I + J) % 2 != color:
                        continue
                    new = block_update(net, msgs, I, J, dr, P, stats)
                    upd[(I, J, dr)] = damp(new, msgs[(I, J, dr)], P, stats)
                msgs.update(upd)
            acc = 0.0
            for e in edges:                                      # Remark 4
                o = M.overlap(msgs[e], prev[e], stats)
                acc += 2.0 - 2.0 * o * o
            delta = math.sqrt(max(acc, 0.0)) / Mtot
            iters = it
            if delta < P.delta0:
                break
    # Lemma 1 read-out.
    logp = 0.0
    for I in range(net.nbr):
        for J in range(net.nbc):
            lz, pos = block_log_z(net, msgs, I, J, P, stats)
            logp += lz
            if not pos:
                flags |= FLAG_BLOCK
    for (I, J, dr) in edges:
        if dr not in ("R", "D"):
            continue
        di, dj = STEP[dr]
        o = M.overlap(msgs[(I, J, dr)], msgs[(I + di, J + dj, OPPOSITE[dr])], stats)
        if o == 0.0 or not np.isfinite(o):
            logp = -np.inf
            flags |= FLAG_OVERLAP
            continue
        if o < 0:
            flags |= FLAG_OVERLAP
        logp -= math.log(abs(o))
    if not np.isfinite(logp):
        flags |= FLAG_NONFINITE
    if delta >= P.delta1:
        flags |= FLAG_UNTRUSTED
    return CosetResult(logp=logp, delta=delta, iters=iters, flags=flags, messages=msgs)


def decide(logp, delta, flags) -> int:
    """Decision of Algorithm 1 / Remark 6 over the four cosets."""
    elig = [L for L in range(4) if flags[L] == 0]
    if elig:
        best = elig[0]
        for L in elig[1:]:
            if logp[L] > logp[best]:
                best = L
        return best
    best = 0
    for L in range(1, 4):
        if delta[L] < delta[best]:
            best = L
    return best


def decode(s, P: Params, keep_messages=False, dtype=np.float64):
    """Decode one syndrome: returns a dict of per-coset results and the decision.

    ``dtype`` other than float64 runs the same steps in that precision (the
    network's tensors and every message), to measure the method's own
    rounding error; the oracle's values are float64."""
    lat = Lattice(P.d)
    stats = M.Stats()
    res = []
    for L in range(4):
        T = coset_network(lat, s, L, P.p)
        if dtype is not np.float64:
            T = [[t.astype(dtype) for t in row] for row in T]
        r = run_blockbp(T, P, stats)
        if not keep_messages:
            r.messages = {}
        res.append(r)
    logp = np.array([r.logp for r in res])
    delta = np.array([r.delta for r in res])
    iters = np.array([r.iters for r in res], dtype=np.int64)
    flags = np.array([r.flags for r in res], dtype=np.int64)
    return {
        "logp": logp, "delta": delta, "iters": iters, "flags": flags,
        "decision": decide(logp, delta, flags), "stats": stats, "cosets": res,
    }


def bmps_log_contract(tensors, D: int, cutoff: float = 1e-13, stats=None) -> float:
    """One block covering the whole network: the bMPS contraction (Sec. III.A)."""
    W = len(tensors)
    P = Params(d=(W + 1) // 2, k=W, D=D, p=0.0, max_iter=0, cutoff=cutoff)
    return run_blockbp(tensors, P, stats).logp
