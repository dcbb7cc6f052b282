"""Exact references for the coset probabilities (Eq. noise-cosets).

* ``brute_force_coset_logprobs`` sums pi(f_s L g) over all 2^m elements g of
  the stabilizer group -- the definition in Eq. noise-cosets written out.
  Feasible for d <= 3 (m <= 12).
* ``exact_contract_log`` contracts the W x W coset network exactly, node by
  node in row-major order (the quantity Sec. III.A says equals the coset
  probability).  Feasible for W <= 21 (state of 2^(W+1) doubles).

The two are independent routes to the same number and pin each other at
d = 2, 3 (tests/test_oracle_exact.py).
"""

from __future__ import annotations

import itertools

import numpy as np

from .lattice import Lattice
from .tn import coset_network


def _log_pauli_probs(fx, fz, p):
    """log pi(f) for a batch of Paulis [N, n] (product channel, Eq. noise)."""
    err = (fx | fz).astype(bool)
    k = err.sum(axis=1)
    n = fx.shape[1]
    return k * np.log(p / 3.0) + (n - k) * np.log(1.0 - p)


def brute_force_coset_logprobs(lat: Lattice, s, p: float) -> np.ndarray:
    """log pi(f_s L G) for the 4 cosets by summing over all of G."""
    if lat.m > 20:
        raise ValueError("brute force only for tiny codes")
    gx, gz = lat.generator_bits()
    beta = np.array(list(itertools.product((0, 1), repeat=lat.m)), dtype=np.uint8)
    sx = (beta.astype(np.int64) @ gx.astype(np.int64)) % 2
    sz = (beta.astype(np.int64) @ gz.astype(np.int64)) % 2
    out = np.zeros(4)
    for L in range(4):
        fx, fz = lat.coset_frame(s, L)
        lp = _log_pauli_probs((sx ^ fx).astype(np.uint8), (sz ^ fz).astype(np.uint8), p)
        mx = lp.max()
        out[L] = mx + np.log(np.exp(lp - mx).sum())
    return out


def exact_contract_log(tensors) -> float:
    """log of the exact contraction of a square network of (l,r,u,d) tensors.

    The frontier holds the W downward legs of the row being built plus one
    horizontal leg; each node contracts its left leg with the horizontal leg
    and its up leg with the down leg above it.  The frontier is renormalised
    after every row and the scale kept as a log."""
    W = len(tensors)
    shape = [tensors[0][j].shape[2] for j in range(W)] + [1]   # up legs of row 0 (dim 1)
    state = np.ones(shape, dtype=np.float64)
    logscale = 0.0
    for i in range(W):
        for j in range(W):
            T = tensors[i][j]                  # (l, r, u, d)
            # contract state axis j (down leg above) with u, last axis with l
            st = np.moveaxis(state, [j, W], [W - 1, W])      # (..others.., a_j, h)
            others = st.shape[:W - 1]
            st = st.reshape(int(np.prod(others)) if others else 1, st.shape[W - 1], st.shape[W])
            new = np.einsum("xuh,hrun->xnr", st, T)          # (others, d, r)
            new = new.reshape(tuple(others) + (T.shape[3], T.shape[1]))
            state = np.moveaxis(new, [W - 1, W], [j, W])
        nrm = np.abs(state).max()
        if nrm == 0.0:
            return -np.inf
        state = state / nrm
        logscale += np.log(nrm)
    val = float(state.reshape(-1)[0]) if state.size == 1 else float(state.sum())
    if val <= 0:
        return -np.inf
    return logscale + np.log(val)


def exact_coset_logprobs(lat: Lattice, s, p: float) -> np.ndarray:
    """log pi(f_s L G) of the 4 cosets by exact network contraction."""
    return np.array([exact_contract_log(coset_network(lat, s, L, p)) for L in range(4)])
