"""Pins of oracle.lattice: stabilizer algebra of the planar code (Sec. II)."""

import itertools

import numpy as np
import pytest

from oracle.lattice import COSET_BITS, Lattice, symplectic

rng = np.random.default_rng(1234)


@pytest.mark.parametrize("d", [2, 3, 4, 5, 7])
def test_counts_and_supports(d):
    lat = Lattice(d)
    assert lat.n == d * d + (d - 1) ** 2          # Sec. II.B
    assert lat.m == 2 * d * (d - 1)               # m = 2d(d-1), k = n - m = 1
    assert lat.n - lat.m == 1
    for ci, (kind, (i, j)) in enumerate(lat.checks):
        assert 2 <= len(lat.support[ci]) <= 4


@pytest.mark.parametrize("d", [2, 3, 5])
def test_generators_commute(d):
    lat = Lattice(d)
    gx, gz = lat.generator_bits()
    for a in range(lat.m):
        for b in range(lat.m):
            assert symplectic(gx[a], gz[a], gx[b], gz[b]) == 0


@pytest.mark.parametrize("d", [2, 3, 5, 7])
def test_logicals(d):
    lat = Lattice(d)
    gx, gz = lat.generator_bits()
    xb, zb = lat.logical_bits()
    zero = np.zeros(lat.n, dtype=np.uint8)
    for a in range(lat.m):
        assert symplectic(xb, zero, gx[a], gz[a]) == 0
        assert symplectic(zero, zb, gx[a], gz[a]) == 0
    assert symplectic(xb, zero, zero, zb) == 1
    assert xb.sum() == d and zb.sum() == d        # weight-d logicals


def test_generators_independent():
    # Rank of the 2n-bit generator matrix over GF(2) must be m (Sec. II.A).
    for d in (2, 3, 4):
        lat = Lattice(d)
        gx, gz = lat.generator_bits()
        A = np.concatenate([gx, gz], axis=1).astype(np.uint8) % 2
        r = 0
        A = A.copy()
        for c in range(A.shape[1]):
            piv = [i for i in range(r, A.shape[0]) if A[i, c]]
            if not piv:
                continue
            A[[r, piv[0]]] = A[[piv[0], r]]
            for i in range(A.shape[0]):
                if i != r and A[i, c]:
                    A[i] ^= A[r]
            r += 1
        assert r == lat.m


@pytest.mark.parametrize("d", [2, 3, 5, 7, 11])
def test_pure_error_reproduces_syndrome(d):
    lat = Lattice(d)
    for _ in range(20):
        s = rng.integers(0, 2, lat.m).astype(np.uint8)
        fx, fz = lat.pure_error(s)
        assert np.array_equal(lat.syndrome(fx, fz), s)
        for L in range(4):
            cx, cz = lat.coset_frame(s, L)
            assert np.array_equal(lat.syndrome(cx, cz), s)


@pytest.mark.parametrize("d", [3, 5])
def test_true_class_of_constructed_errors(d):
    lat = Lattice(d)
    gx, gz = lat.generator_bits()
    xb, zb = lat.logical_bits()
    for _ in range(30):
        s = rng.integers(0, 2, lat.m).astype(np.uint8)
        L = int(rng.integers(0, 4))
        beta = rng.integers(0, 2, lat.m)
        ex, ez = lat.pure_error(s)
        ex = ex ^ (beta @ gx % 2).astype(np.uint8)
        ez = ez ^ (beta @ gz % 2).astype(np.uint8)
        bx, bz = COSET_BITS[L]
        if bx:
            ex = ex ^ xb
        if bz:
            ez = ez ^ zb
        assert lat.true_class(ex, ez, s) == L


def test_d2_pauli_group_partition():
    # d = 2: all 4^5 Paulis; every syndrome class holds |C(G)| = 4 * 2^m
    # operators, and splits into 4 cosets of G of 2^m each (Sec. II.A).
    lat = Lattice(2)
    count = {}
    for bits in itertools.product((0, 1), repeat=2 * lat.n):
        fx = np.array(bits[:lat.n], dtype=np.uint8)
        fz = np.array(bits[lat.n:], dtype=np.uint8)
        s = tuple(lat.syndrome(fx, fz))
        c = lat.true_class(fx, fz, np.array(s, dtype=np.uint8))
        count[(s, c)] = count.get((s, c), 0) + 1
    assert len(count) == 2 ** lat.m * 4
    assert set(count.values()) == {2 ** lat.m}


def test_d3_all_4_13_paulis_split_evenly_into_cosets():
    # All 4^13 Paulis of d = 3: every (syndrome, coset) class, the coset
    # taken relative to the pure error (f_s vanishes on both logicals'
    # supports, so the class is read off the Pauli itself), holds exactly
    # |G| = 2^12 Paulis.  The checks are of one type each (A sees x, B sees
    # z) and so are the class bits (X-bar part from x, Z-bar part from z),
    # so the count over (x, z) is the outer product of two exact counts over
    # the 2^13 x-parts and the 2^13 z-parts.
    lat = Lattice(3)
    n, d = lat.n, lat.d
    nA = d * (d - 1)
    xb, zb = lat.logical_bits()
    bits = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)   # [2^n, n]
    supA = np.zeros((nA, n), dtype=np.int64)
    supB = np.zeros((lat.m - nA, n), dtype=np.int64)
    for ci, (kind, _) in enumerate(lat.checks):
        for q in lat.support[ci]:
            if kind == "A":
                supA[ci, q] = 1
            else:
                supB[ci - nA, q] = 1
    sA = (bits @ supA.T) & 1                        # syndrome bits seen by x parts
    sB = (bits @ supB.T) & 1                        # ... by z parts
    cx = (bits @ zb.astype(np.int64)) & 1           # X-bar component: anticommutes with Z-bar
    cz = (bits @ xb.astype(np.int64)) & 1           # Z-bar component: anticommutes with X-bar
    kx = (sA * (1 << np.arange(nA))).sum(1) * 2 + cx
    kz = (sB * (1 << np.arange(lat.m - nA))).sum(1) * 2 + cz
    hx = np.bincount(kx, minlength=1 << (nA + 1))
    hz = np.bincount(kz, minlength=1 << (lat.m - nA + 1))
    joint = np.outer(hx, hz)                        # [(sA, cx), (sB, cz)] over all 4^13 Paulis
    assert joint.sum() == 4 ** n
    assert np.all(joint == 1 << lat.m)
    # The same classes from the library's own maps on a sample of Paulis.
    rng = np.random.default_rng(3)
    for _ in range(200):
        fx, fz = rng.integers(0, 2, n).astype(np.uint8), rng.integers(0, 2, n).astype(np.uint8)
        s = lat.syndrome(fx, fz)
        ix = int((fx.astype(np.int64) * (1 << np.arange(n))).sum())
        iz = int((fz.astype(np.int64) * (1 << np.arange(n))).sum())
        assert np.array_equal(s, np.concatenate([sA[ix], sB[iz]]).astype(np.uint8))
        c = lat.true_class(fx, fz, s)
        assert c == ((2 if cz[iz] else 1) if cx[ix] else (3 if cz[iz] else 0))
