"""Fused-block ("naive") blockBP of Remark 9 with dense vector messages.

Every k x k block is contracted into one tensor F with four legs, one per
side, of dimension 2^(side length) (1 on the network border); plain BP then
runs between these mega-vertices with the same schedule, normalisation,
damping, Delta and Lemma 1 read-out as ``oracle.blockbp``.  It carries no
MPS machinery and no truncation, so wherever ``oracle.blockbp`` truncates
nothing (k = 3, D = 4, for instance) the two must agree to rounding; this
second implementation exists only to pin ``oracle.blockbp``.

Side legs are flattened in C order with the first site most significant:
top -> bottom on vertical sides, left -> right on horizontal sides, the same
site order as the MPS messages.
"""

from __future__ import annotations

import math

import numpy as np

from .blockbp import DIRS, OPPOSITE, STEP, ranges


def fuse_block(T, rows, cols):
    """Contract the nodes of one block; returns F[left, right, top, bottom]."""
    r0, r1 = rows
    c0, c1 = cols
    label = {}
    nxt = [0]

    def lab(key):
        if key not in label:
            label[key] = nxt[0]
            nxt[0] += 1
        return label[key]

    ops = []
    for i in range(r0, r1):
        for j in range(c0, c1):
            l = lab(("h", i, j - 1))       # edge between (i, j-1) and (i, j)
            r = lab(("h", i, j))
            u = lab(("v", i - 1, j))       # edge between (i-1, j) and (i, j)
            dn = lab(("v", i, j))
            ops += [T[i][j], [l, r, u, dn]]
    out_left = [label[("h", i, c0 - 1)] for i in range(r0, r1)]
    out_right = [label[("h", i, c1 - 1)] for i in range(r0, r1)]
    out_top = [label[("v", r0 - 1, j)] for j in range(c0, c1)]
    out_bot = [label[("v", r1 - 1, j)] for j in range(c0, c1)]
    out = out_left + out_right + out_top + out_bot
    F = np.einsum(*ops, out, optimize="greedy")
    dl = int(np.prod(F.shape[:len(out_left)]))
    o = len(out_left)
    dr = int(np.prod(F.shape[o:o + len(out_right)]))
    o += len(out_right)
    dt = int(np.prod(F.shape[o:o + len(out_top)]))
    db = int(np.prod(F.shape[o + len(out_top):]))
    return F.reshape(dl, dr, dt, db)


def run_naive(tensors, k, max_iter, eta, delta0, k_cols=None, init=None):
    """Dense fused-block BP; returns (logp, delta, iters, messages).

    ``init`` optionally maps (I, J, dir) to an initial message (normalised
    here); the default is the uniform start of Remark 2."""
    W = len(tensors)
    kc = k_cols if k_cols is not None else k
    rows, cols = ranges(W, k), ranges(W, kc)
    nbr, nbc = len(rows), len(cols)
    F = {(I, J): fuse_block(tensors, rows[I], cols[J]) for I in range(nbr) for J in range(nbc)}

    def has(I, J, dr):
        di, dj = STEP[dr]
        return 0 <= I + di < nbr and 0 <= J + dj < nbc

    axis = {"L": 0, "R": 1, "U": 2, "D": 3}
    edges = [(I, J, dr) for I in range(nbr) for J in range(nbc) for dr in DIRS if has(I, J, dr)]
    msgs = {}
    for (I, J, dr) in edges:
        dim = F[(I, J)].shape[axis[dr]]
        if init is not None:
            v = np.asarray(init[(I, J, dr)], dtype=np.float64)[:dim]
            msgs[(I, J, dr)] = v / np.linalg.norm(v)
        else:
            msgs[(I, J, dr)] = np.full(dim, 1.0 / math.sqrt(dim))

    def incoming(I, J, side):
        if has(I, J, side):
            di, dj = STEP[side]
            return msgs[(I + di, J + dj, OPPOSITE[side])]
        return np.ones(1)

    def contract_except(I, J, dr):
        f = F[(I, J)]
        vl, vr, vt, vb = (incoming(I, J, s) for s in ("L", "R", "U", "D"))
        full = {"L": vl, "R": vr, "U": vt, "D": vb}
        subs = "lrtb"
        operands = [f]
        spec = [subs]
        for s, c in zip(("L", "R", "U", "D"), subs):
            if s != dr:
                operands.append(full[s])
                spec.append(c)
        out = subs[axis[dr]]
        return np.einsum(",".join(spec) + "->" + out, *operands)

    Mtot = len(edges)
    delta, iters = 0.0, 0
    for it in range(1, max_iter + 1):
        prev = dict(msgs)
        for color in (0, 1):
            upd = {}
            for (I, J, dr) in edges:
                if (I + J) % 2 != color:
                    continue
                new = contract_except(I, J, dr)
                new = new / np.linalg.norm(new)
                dm = (1.0 - eta) * new + eta * msgs[(I, J, dr)]
                upd[(I, J, dr)] = dm / np.linalg.norm(dm)
            msgs.update(upd)
        acc = sum(2.0 - 2.0 * float(msgs[e] @ prev[e]) ** 2 for e in edges)
        delta = math.sqrt(max(acc, 0.0)) / Mtot if Mtot else 0.0
        iters = it
        if delta < delta0:
            break
    logp = 0.0
    for I in range(nbr):
        for J in range(nbc):
            z = np.einsum("lrtb,l,r,t,b->", F[(I, J)], incoming(I, J, "L"), incoming(I, J, "R"),
                          incoming(I, J, "U"), incoming(I, J, "D"))
            logp += math.log(abs(z))
    for (I, J, dr) in edges:
        if dr in ("R", "D"):
            di, dj = STEP[dr]
            logp -= math.log(abs(float(msgs[(I, J, dr)] @ msgs[(I + di, J + dj, OPPOSITE[dr])])))
    return logp, delta, iters, msgs
