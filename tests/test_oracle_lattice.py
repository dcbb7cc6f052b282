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
