"""Coset tensor network T_s(L) (Sec. III.A; Fig. 1 caption; Eq. noise-cosets).

The paper defers the construction to Bravyi-Suchara-Vargo; this oracle
rebuilds it from Eq. noise-cosets.  Give every check g a bit beta_g.  Since
the m generators are independent,

    pi(f G) = sum_beta  prod_e  pi_e( f_e * prod_g g^{beta_g} |_e ).

On the (2d-1) x (2d-1) grid every tensor has the legs (l, r, u, d) towards
its four grid neighbours, bond dimension 2, and dimension 1 on the grid
border:

* check node: copy tensor, 1 iff all its legs carry the same beta;
* horizontal-edge qubit: left/right neighbours are sites (Z checks),
  up/down neighbours are plaquettes (X checks), so
  T(l, r, u, d) = pi( f_e (+) (x = u^d, z = l^r) );
* vertical-edge qubit: left/right neighbours are plaquettes, up/down are
  sites, so T(l, r, u, d) = pi( f_e (+) (x = l^r, z = u^d) ).

Depolarizing channel (Sec. IV): pi(I) = 1-p, pi(X) = pi(Y) = pi(Z) = p/3.

Pin: the exact contraction of this network equals the brute-force sum over
the stabilizer group (tests/test_oracle_exact.py, d = 2, 3).
"""

from __future__ import annotations

import numpy as np

from .lattice import Lattice


def pauli_prob(x: int, z: int, p: float) -> float:
    """Single-qubit depolarizing probability (Sec. IV)."""
    return (1.0 - p) if (x == 0 and z == 0) else p / 3.0


def node_tensor(lat: Lattice, i: int, j: int, fx, fz, p: float) -> np.ndarray:
    """Tensor at grid (i, j) with axes (l, r, u, d); border legs have dim 1."""
    W = lat.W
    dims = (1 if j == 0 else 2, 1 if j == W - 1 else 2,
            1 if i == 0 else 2, 1 if i == W - 1 else 2)
    T = np.zeros(dims, dtype=np.float64)
    kind = lat.kind(i, j)
    if kind in ("A", "B"):
        # Copy tensor over the existing legs.
        for l in range(dims[0]):
            for r in range(dims[1]):
                for u in range(dims[2]):
                    for dn in range(dims[3]):
                        vals = []
                        if dims[0] == 2:
                            vals.append(l)
                        if dims[1] == 2:
                            vals.append(r)
                        if dims[2] == 2:
                            vals.append(u)
                        if dims[3] == 2:
                            vals.append(dn)
                        if len(set(vals)) <= 1:
                            T[l, r, u, dn] = 1.0
        return T
    q = lat.qidx[i, j]
    f_x, f_z = int(fx[q]), int(fz[q])
    for l in range(dims[0]):
        for r in range(dims[1]):
            for u in range(dims[2]):
                for dn in range(dims[3]):
                    if kind == "QH":
                        x, z = u ^ dn, l ^ r
                    else:
                        x, z = l ^ r, u ^ dn
                    T[l, r, u, dn] = pauli_prob(f_x ^ x, f_z ^ z, p)
    return T


def coset_network(lat: Lattice, s, coset: int, p: float):
    """All node tensors of T_s(L), as a W x W nested list (Algorithm 1)."""
    fx, fz = lat.coset_frame(s, coset)
    return [[node_tensor(lat, i, j, fx, fz, p) for j in range(lat.W)]
            for i in range(lat.W)]
