"""Planar surface code: qubits, checks, logicals, syndromes (Sec. II.A-B).

Grid picture (Fig. 1 caption; Sec. III.A): the d x d code maps to a
(2d-1) x (2d-1) grid.  Position (i, j) holds

* a horizontal-edge qubit when i and j are both even   (d^2 of them),
* a vertical-edge qubit when i and j are both odd      ((d-1)^2 of them),
* a site check A_u = prod Z when i is even and j odd   (d(d-1) of them),
* a plaquette check B_p = prod X when i is odd, j even (d(d-1) of them),

and every check acts on its grid neighbours (Eq. def:AB).  Qubits are
numbered row-major over the positions with i + j even; syndrome bits are all
A_(r,c) row-major, then all B_(r,j) row-major.

The logicals (Sec. II.B, last paragraph): X-bar is X on the horizontal edges
of row 0 (grid (0, even j)); Z-bar is Z on the horizontal edges of column 0
(grid (even i, 0)).  Cosets are indexed 0..3 = I, X, Y, Z with
L = Xbar^bx Zbar^bz, (bx, bz) = (0,0), (1,0), (1,1), (0,1).

The pure error f_s (Algorithm 1, first step) is not specified by the paper.
This oracle reads it as: for a flagged A_(r,c), X on the horizontal edges
h(r, c+1 .. d-1) (a string to the right rough boundary); for a flagged
B_(r,j), Z on the horizontal edges h(r+1 .. d-1, j) (a string to the bottom
boundary); the product of all of these.

Pins (tests/test_oracle_lattice.py): commutation of every check pair, the
logicals commute with every check and anticommute with each other,
s(f_s) = s, counts n = d^2+(d-1)^2 and m = 2d(d-1), and the syndrome map
agrees with the workload sampler's own (independent) one.
"""

from __future__ import annotations

import numpy as np

COSETS = ("I", "X", "Y", "Z")
COSET_BITS = ((0, 0), (1, 0), (1, 1), (0, 1))   # (bx, bz) of each coset


class Lattice:
    """Index tables of the distance-d planar code (Sec. II.B)."""

    def __init__(self, d: int):
        if d < 2:
            raise ValueError("d must be >= 2")
        self.d = d
        self.W = W = 2 * d - 1
        self.qidx = -np.ones((W, W), dtype=np.int64)
        pos = []
        for i in range(W):
            for j in range(W):
                if (i + j) % 2 == 0:
                    self.qidx[i, j] = len(pos)
                    pos.append((i, j))
        self.qpos = pos
        self.n = len(pos)
        # Checks in syndrome order: A_(r,c) at (2r, 2c+1), then B_(r,j) at (2r+1, 2j).
        self.checks = []          # list of (kind, (i, j), [qubit indices])
        for r in range(d):
            for c in range(d - 1):
                self.checks.append(("A", (2 * r, 2 * c + 1)))
        for r in range(d - 1):
            for j in range(d):
                self.checks.append(("B", (2 * r + 1, 2 * j)))
        self.cidx = -np.ones((W, W), dtype=np.int64)
        supp = []
        for ci, (kind, (i, j)) in enumerate(self.checks):
            self.cidx[i, j] = ci
            q = []
            for (a, b) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if 0 <= a < W and 0 <= b < W:
                    q.append(int(self.qidx[a, b]))
            supp.append(q)
        self.support = supp
        self.m = len(self.checks)

    # -- node classification on the grid ---------------------------------
    def kind(self, i: int, j: int) -> str:
        if i % 2 == 0 and j % 2 == 0:
            return "QH"          # horizontal-edge qubit
        if i % 2 == 1 and j % 2 == 1:
            return "QV"          # vertical-edge qubit
        if i % 2 == 0:
            return "A"           # site check, Z type
        return "B"               # plaquette check, X type

    # -- stabilizer generators as (x, z) bit planes (Eq. def:AB) ---------
    def generator_bits(self):
        gx = np.zeros((self.m, self.n), dtype=np.uint8)
        gz = np.zeros((self.m, self.n), dtype=np.uint8)
        for ci, (kind, _) in enumerate(self.checks):
            for q in self.support[ci]:
                if kind == "A":
                    gz[ci, q] = 1
                else:
                    gx[ci, q] = 1
        return gx, gz

    # -- logical operators (Sec. II.B) -----------------------------------
    def logical_bits(self):
        """(Xbar_x, Zbar_z): X on row-0 horizontal edges, Z on column-0 ones."""
        xb = np.zeros(self.n, dtype=np.uint8)
        zb = np.zeros(self.n, dtype=np.uint8)
        for j in range(0, self.W, 2):
            xb[self.qidx[0, j]] = 1
        for i in range(0, self.W, 2):
            zb[self.qidx[i, 0]] = 1
        return xb, zb

    # -- syndrome map s(f): s_i = 1 iff f anticommutes with g_i -----------
    def syndrome(self, fx, fz) -> np.ndarray:
        fx = np.asarray(fx, dtype=np.uint8)
        fz = np.asarray(fz, dtype=np.uint8)
        s = np.zeros(self.m, dtype=np.uint8)
        for ci, (kind, _) in enumerate(self.checks):
            bits = fx if kind == "A" else fz     # Z check sees x, X check sees z
            v = 0
            for q in self.support[ci]:
                v ^= int(bits[q])
            s[ci] = v
        return s

    # -- pure error f_s (Algorithm 1, first step; construction is a reading)
    def pure_error(self, s):
        s = np.asarray(s, dtype=np.uint8)
        d = self.d
        fx = np.zeros(self.n, dtype=np.uint8)
        fz = np.zeros(self.n, dtype=np.uint8)
        for r in range(d):
            for c in range(d - 1):
                if s[r * (d - 1) + c]:
                    for cc in range(c + 1, d):
                        fx[self.qidx[2 * r, 2 * cc]] ^= 1
        base = d * (d - 1)
        for r in range(d - 1):
            for j in range(d):
                if s[base + r * d + j]:
                    for rr in range(r + 1, d):
                        fz[self.qidx[2 * rr, 2 * j]] ^= 1
        return fx, fz

    def coset_frame(self, s, coset: int):
        """Pauli f_s * L (phases dropped) as (x, z) planes (Algorithm 1, loop)."""
        fx, fz = self.pure_error(s)
        xb, zb = self.logical_bits()
        bx, bz = COSET_BITS[coset]
        if bx:
            fx = fx ^ xb
        if bz:
            fz = fz ^ zb
        return fx, fz

    def true_class(self, ex, ez, s) -> int:
        """Index L* of the coset f_s L* G holding the error e (Sec. II.A).

        e f_s lies in the centraliser; its X-bar component is detected by
        anticommutation with Z-bar and its Z-bar component by X-bar."""
        fx, fz = self.pure_error(s)
        cx = np.asarray(ex, dtype=np.uint8) ^ fx
        cz = np.asarray(ez, dtype=np.uint8) ^ fz
        xb, zb = self.logical_bits()
        bx = int(np.sum(cx & zb) % 2)       # anticommutes with Zbar -> has Xbar
        bz = int(np.sum(cz & xb) % 2)       # anticommutes with Xbar -> has Zbar
        return COSET_BITS.index((bx, bz))


def symplectic(ax, az, bx, bz) -> int:
    """1 iff the Paulis (ax, az) and (bx, bz) anticommute."""
    return int((np.sum(np.asarray(ax) & np.asarray(bz)) + np.sum(np.asarray(az) & np.asarray(bx))) % 2)
