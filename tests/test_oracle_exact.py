"""Pins of the coset network and the exact references (Eq. noise-cosets)."""

import itertools
import math

import numpy as np
import pytest

import synth
from oracle import blockbp as bb
from oracle.exact import brute_force_coset_logprobs, exact_coset_logprobs
from oracle.lattice import Lattice
from oracle.tn import coset_network

P = 0.1


def _logsumexp(v):
    m = np.max(v)
    return m + math.log(np.sum(np.exp(np.asarray(v) - m)))


@pytest.mark.parametrize("d", [2, 3])
def test_network_contraction_equals_stabilizer_sum(d):
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(5, 0, 8, d, 0.15)
    for s in S:
        bf = brute_force_coset_logprobs(lat, s, 0.15)
        ex = exact_coset_logprobs(lat, s, 0.15)
        np.testing.assert_allclose(ex, bf, rtol=0, atol=1e-12)


def test_d2_cosets_sum_to_one_over_all_syndromes():
    # sum_s sum_L pi(f_s L G) = sum over the whole Pauli group = 1.
    lat = Lattice(2)
    tot = []
    for bits in itertools.product((0, 1), repeat=lat.m):
        s = np.array(bits, dtype=np.uint8)
        tot.extend(exact_coset_logprobs(lat, s, P))
    assert abs(math.exp(_logsumexp(tot)) - 1.0) < 1e-13


def test_d2_cosets_sum_to_syndrome_probability():
    # sum_L pi(f_s L G) = P(s), P(s) summed directly over all 4^n Paulis.
    lat = Lattice(2)
    ps = {}
    for bits in itertools.product((0, 1), repeat=2 * lat.n):
        fx = np.array(bits[:lat.n], dtype=np.uint8)
        fz = np.array(bits[lat.n:], dtype=np.uint8)
        w = int(np.sum(fx | fz))
        s = tuple(lat.syndrome(fx, fz))
        ps[s] = ps.get(s, 0.0) + (P / 3) ** w * (1 - P) ** (lat.n - w)
    for s, prob in ps.items():
        ex = exact_coset_logprobs(lat, np.array(s, dtype=np.uint8), P)
        assert abs(math.exp(_logsumexp(ex)) / prob - 1.0) < 1e-12


def test_zero_syndrome_identity_coset_is_most_likely_at_low_noise():
    lat = Lattice(3)
    s = np.zeros(lat.m, dtype=np.uint8)
    lp = brute_force_coset_logprobs(lat, s, 0.01)
    assert np.argmax(lp) == 0
    # Leading order: pi(G) ~ (1-p)^n for p -> 0.
    assert abs(lp[0] - lat.n * math.log(1 - 0.01)) < 1e-3


def test_one_block_bmps_is_exact_d3():
    # One block covering the network is the bMPS contraction (Sec. III.D);
    # with D >= 2^floor(W/2) = 4 at d = 3 nothing is truncated.
    lat = Lattice(3)
    _, _, S = synth.sample_syndromes(9, 0, 6, 3, P)
    for s in S:
        bf = brute_force_coset_logprobs(lat, s, P)
        bm = [bb.bmps_log_contract(coset_network(lat, s, L, P), D=4, cutoff=1e-15) for L in range(4)]
        np.testing.assert_allclose(bm, bf, rtol=0, atol=1e-11)


def test_one_block_bmps_is_exact_d5():
    lat = Lattice(5)
    _, _, S = synth.sample_syndromes(9, 0, 2, 5, P)
    for s in S:
        ex = exact_coset_logprobs(lat, s, P)
        bm = [bb.bmps_log_contract(coset_network(lat, s, L, P), D=16, cutoff=1e-15) for L in range(4)]
        np.testing.assert_allclose(bm, ex, rtol=0, atol=1e-9)


def test_bmps_converges_as_D_grows():
    # Truncation error of the one-block contraction shrinks to zero as D grows.
    lat = Lattice(5)
    _, _, S = synth.sample_syndromes(21, 0, 1, 5, 0.13)
    s = S[0]
    ex = exact_coset_logprobs(lat, s, 0.13)
    errs = []
    for D in (1, 2, 4, 8, 16):
        bm = np.array([bb.bmps_log_contract(coset_network(lat, s, L, 0.13), D=D, cutoff=1e-15)
                       for L in range(4)])
        errs.append(np.max(np.abs(bm - ex)))
    assert errs[-1] < 1e-9
    assert errs[0] > 1e-3
    for a, b in zip(errs, errs[1:]):
        assert b <= a * 1.5 + 1e-12
