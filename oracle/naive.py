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
    """Contract the nodes of one block; returns F[left, right, top, bottom].

    Contracted one row at a time (each row's chain first, then the row onto
    the block through its vertical legs), so that no single contraction
    names more labels than numpy's einsum allows (k = 6 blocks have 84
    internal bonds)."""
    r0, r1 = rows
    c0, c1 = cols
    w = c1 - c0
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    blk = None
    nL = 0                                  # left / right legs collected so far
    for i in range(r0, r1):
        # The row as one tensor: axes l, r, u_0 .. u_{w-1}, d_0 .. d_{w-1}.
        row = T[i][c0]
        for j in range(1, w):
            u_prev = letters[2:2 + j]
            d_prev = letters[2 + j:2 + 2 * j]
            lhs = "a" + "Y" + u_prev + d_prev            # Y: the bond between nodes j-1 and j
            rhs = "Yb" + "X" + "Z"                          # node (l=Y, r=b, u=X, d=Z)
            out = "ab" + u_prev + "X" + d_prev + "Z"
            row = np.einsum(f"{lhs},{rhs}->{out}", row, T[i][c0 + j])
        if blk is None:
            blk = row
            nL = 1
            continue
        # blk axes: L_0..L_{nL-1}, R_0..R_{nL-1}, top_0..top_{w-1}, bot_0..bot_{w-1}
        L = letters[0:nL]
        R = letters[nL:2 * nL]
        top = letters[2 * nL:2 * nL + w]
        bot = letters[2 * nL + w:2 * nL + 2 * w]          # contracted with the row's u legs
        l2, r2 = letters[2 * nL + 2 * w], letters[2 * nL + 2 * w + 1]
        d2 = letters[2 * nL + 2 * w + 2:2 * nL + 3 * w + 2]
        blk = np.einsum(f"{L}{R}{top}{bot},{l2}{r2}{bot}{d2}->{L}{l2}{R}{r2}{top}{d2}", blk, row)
        nL += 1
    sh = blk.shape
    dl = int(np.prod(sh[:nL]))
    dr = int(np.prod(sh[nL:2 * nL]))
    dt = int(np.prod(sh[2 * nL:2 * nL + w]))
    db = int(np.prod(sh[2 * nL + w:]))
    return blk.reshape(dl, dr, dt, db)


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
