"""Pins of oracle.blockbp (Algorithm 1, Lemma 1, Remarks 1-9)."""

import math

import numpy as np
import pytest

import synth
from oracle import blockbp as bb
from oracle import mps as M
from oracle.exact import exact_coset_logprobs
from oracle.lattice import Lattice
from oracle.naive import run_naive
from oracle.tn import coset_network


def test_partition_remainder_at_the_far_edge():
    # Remark 1: k = 4 on W = 21 gives five blocks of 4 and one of 1.
    assert bb.ranges(21, 4) == [(0, 4), (4, 8), (8, 12), (12, 16), (16, 20), (20, 21)]
    assert bb.ranges(9, 3) == [(0, 3), (3, 6), (6, 9)]


@pytest.mark.parametrize("d,kc,D", [(3, 1, 4), (3, 2, 4), (5, 3, 16)])
def test_strips_are_a_chain_and_blockbp_is_exact(d, kc, D):
    # Vertical strips form a chain (a tree): BP with the Lemma 1 read-out is
    # exact there (Sec. III.C), given an untruncated in-block contraction.
    lat = Lattice(d)
    W = 2 * d - 1
    _, _, S = synth.sample_syndromes(31, 0, 2, d, 0.1)
    for s in S:
        ex = exact_coset_logprobs(lat, s, 0.1)
        P = bb.Params(d=d, k=W, k_cols=kc, D=D, p=0.1, max_iter=60, delta0=1e-15, cutoff=1e-15)
        got = [bb.run_blockbp(coset_network(lat, s, L, 0.1), P).logp for L in range(4)]
        np.testing.assert_allclose(got, ex, rtol=0, atol=1e-9)


def _random_positive_grid(W, seed):
    """A W x W grid of random positive (l, r, u, d) tensors, border legs of dimension 1."""
    rng = np.random.default_rng(seed)
    T = []
    for i in range(W):
        row = []
        for j in range(W):
            dims = (1 if j == 0 else 2, 1 if j == W - 1 else 2, 1 if i == 0 else 2, 1 if i == W - 1 else 2)
            row.append(rng.uniform(0.2, 1.8, size=dims))
        T.append(row)
    return T


@pytest.mark.parametrize("W,k,kc,seed", [(5, 5, 1, 1), (5, 1, 5, 2), (7, 7, 2, 3), (6, 2, 6, 4)])
def test_lemma1_on_random_positive_tree_networks(W, k, kc, seed):
    # Lemma 1 beyond the coset networks: on random positive tensors, strips
    # (k x kc blocks spanning the grid one way) form a chain of blocks, where
    # converged BP with the Bethe read-out gives the exact contraction; the
    # MPS form with an untruncating bond agrees with the dense form.
    from oracle.exact import exact_contract_log
    T = _random_positive_grid(W, seed)
    ref = exact_contract_log(T)
    lp, dl, it, _ = run_naive(T, k, 200, 0.1, 1e-15, k_cols=kc)
    assert dl < 1e-12 and abs(lp - ref) < 1e-9 * max(1.0, abs(ref))
    P = bb.Params(d=(W + 1) // 2, k=k, k_cols=kc, D=1 << W, p=0.1, max_iter=200, delta0=1e-15, cutoff=1e-15)
    r = bb.run_blockbp(T, P)
    assert abs(r.logp - ref) < 1e-9 * max(1.0, abs(ref))


def test_bethe_readout_is_not_exact_on_a_loop():
    # Sanity of the pin above: with 2 x 2 blocks of a 4 x 4 random grid the
    # block graph has a loop and the Bethe value differs from the exact one.
    from oracle.exact import exact_contract_log
    T = _random_positive_grid(4, 9)
    ref = exact_contract_log(T)
    lp, dl, it, _ = run_naive(T, 2, 200, 0.1, 1e-15)
    assert abs(lp - ref) > 1e-6


def test_mps_blockbp_equals_dense_naive_blockbp_when_nothing_truncates():
    # d = 5, k = 3, D = 4: messages have bond <= 2 and the in-block cuts <= 4,
    # so MPS blockBP equals the fused-block dense BP of Remark 9.
    d, p = 5, 0.1
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(synth.workload_seed(1, 0), 0, 3, d, p)
    P = bb.Params(d=d, k=3, D=4, p=p, max_iter=10, delta0=0.0)
    for s in S:
        for L in range(4):
            T = coset_network(lat, s, L, p)
            r = bb.run_blockbp(T, P)
            lp, dl, it, msgs = run_naive(T, 3, 10, 0.1, 0.0)
            assert abs(r.logp - lp) < 1e-10
            # Delta = sqrt(sum 2 - 2<a|b>^2)/M cancels near convergence, so
            # rounding alone moves it by ~sqrt(M * 1e-16) / M.
            assert abs(r.delta - dl) < 1e-7
            for key, m in r.messages.items():
                np.testing.assert_allclose(M.to_dense(m), msgs[key], atol=1e-10)


def test_blockbp_close_to_exact_and_picks_true_coset():
    # Not an identity: reported closeness on a benign case (p = 0.05, d = 5).
    d, p = 5, 0.05
    lat = Lattice(d)
    ex_, ez_, S = synth.sample_syndromes(77, 0, 4, d, p)
    P = bb.Params(d=d, k=3, D=4, p=p, max_iter=20)
    for b, s in enumerate(S):
        r = bb.decode(s, P)
        ex = exact_coset_logprobs(lat, s, p)
        best = int(np.argmax(ex))
        assert abs(r["logp"][best] - ex[best]) < 0.05
        assert r["decision"] == best


def test_decision_rule_branches():
    # Among trusted cosets (no flags) the largest log P wins.
    assert bb.decide([-5, -3, -4, -9], [1e-3] * 4, [0, 0, 0, 0]) == 1
    # Untrusted cosets are skipped even with a larger log P.
    assert bb.decide([-5, -3, -4, -9], [1e-3, 0.5, 1e-3, 1e-3], [0, 1, 0, 0]) == 2
    # None trusted: the smallest Delta wins (Remark 6).
    assert bb.decide([-5, -3, -4, -9], [0.2, 0.5, 0.1, 0.3], [1, 1, 1, 1]) == 2
    # Ties go to the lowest index in the order I, X, Y, Z.
    assert bb.decide([-3, -3, -4, -9], [0, 0, 0, 0], [0, 0, 0, 0]) == 0
    assert bb.decide([-3, -3, -4, -9], [0.1, 0.1, 0.2, 0.3], [1, 1, 1, 1]) == 0


def test_flags_and_delta_threshold():
    d, p = 5, 0.1
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(3, 0, 1, d, p)
    P = bb.Params(d=d, k=3, D=4, p=p, max_iter=1, delta0=0.0, delta1=1e-9)
    r = bb.run_blockbp(coset_network(lat, S[0], 0, p), P)
    assert r.flags & bb.FLAG_UNTRUSTED
    assert r.iters == 1 and r.delta > 0


def test_early_exit_on_delta0():
    d, p = 5, 0.05
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(4, 0, 1, d, p)
    P = bb.Params(d=d, k=3, D=4, p=p, max_iter=50, delta0=1e-4)
    r = bb.run_blockbp(coset_network(lat, S[0], 0, p), P)
    assert r.iters < 50 and r.delta < 1e-4


def test_uniform_noise_free_network_logp():
    # p -> 0 with s = 0: only the identity error survives in coset I, so
    # log P -> n log(1-p); blockBP must reproduce it to O(p) accuracy.
    d = 5
    lat = Lattice(d)
    s = np.zeros(lat.m, dtype=np.uint8)
    p = 1e-6
    r = bb.run_blockbp(coset_network(lat, s, 0, p), bb.Params(d=d, k=3, D=4, p=p, max_iter=5, delta0=0.0))
    assert abs(r.logp - lat.n * math.log(1 - p)) < 1e-4


def test_dense_and_mps_oracles_agree_at_d11_k4_D8():
    # At d = 11, k = 4, D = 8 the MPS form truncates nothing on this shot, so
    # the two independent implementations must give the same log P.
    d, p = 11, 0.10
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(synth.workload_seed(2, 2), 5, 1, d, p)
    stats = M.Stats()
    T = coset_network(lat, S[0], 1, p)
    r = bb.run_blockbp(T, bb.Params(d=d, k=4, D=8, p=p, max_iter=4, delta0=0.0), stats)
    lp, dl, it, _ = run_naive(T, 4, 4, 0.1, 0.0)
    assert stats.truncations == 0
    assert abs(r.logp - lp) < 1e-9


def test_k6_single_block_is_the_exact_contraction():
    # d = 3 (W = 5) with k = 6: one block covers the network, so the fused
    # block tensor's value is the exact coset probability (no BP at all).
    d, p = 3, 0.12
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(31, 0, 3, d, p)
    for s in S:
        ex = exact_coset_logprobs(lat, s, p)
        for L in range(4):
            lp, _, _, _ = run_naive(coset_network(lat, s, L, p), 6, 3, 0.1, 0.0)
            assert abs(lp - ex[L]) < 1e-10


@pytest.mark.parametrize("d,shots", [(4, 2), (7, 1)])
def test_k6_dense_equals_untruncated_mps(d, shots):
    # 6 x 6 blocks: the dense fused-block BP (row-by-row block tensors) and
    # the MPS blockBP with D = 64 (no truncation at k = 6) are independent
    # implementations of the same rule.
    p = 0.08
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(515, 0, shots, d, p)
    P = bb.Params(d=d, k=6, D=64, p=p, max_iter=4, delta0=0.0)
    for s in S:
        for L in range(4):
            T = coset_network(lat, s, L, p)
            r = bb.run_blockbp(T, P)
            lp, dl, _, _ = run_naive(T, 6, 4, 0.1, 0.0)
            assert abs(r.logp - lp) < 1e-9
            assert abs(r.delta - dl) < 1e-7
