"""Pins of the paper's 6 x 6 scheme in the oracle (Sec. IV, decoder
parameters): nodes fused 3 x 3 into tensors with legs of dimension 8, then
blockBP with 2 x 2 fused blocks and chi = 16 (oracle/coarse.py)."""

import numpy as np
import pytest

import synth
from oracle import blockbp as bb
from oracle import mps as M
from oracle.coarse import coarse_grain, decode_coarse
from oracle.exact import exact_contract_log
from oracle.lattice import Lattice
from oracle.naive import run_naive
from oracle.tn import coset_network


@pytest.mark.parametrize("d", [3, 4])
def test_fusing_keeps_the_exact_contraction(d):
    # Fusing nodes only regroups the sum: the exact value of the fused
    # network equals that of the network itself, for every coset.
    p = 0.1
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(808, 0, 2, d, p)
    for s in S:
        for L in range(4):
            T = coset_network(lat, s, L, p)
            assert abs(exact_contract_log(coarse_grain(T)) - exact_contract_log(T)) < 1e-11


def test_fused_leg_dimensions():
    # d = 7: W = 13 = 3 + 3 + 3 + 3 + 1.  Interior legs bundle three bonds
    # (dimension 8), the last row / column one bond (2), the border none (1).
    d = 7
    T = coset_network(Lattice(d), np.zeros(2 * d * (d - 1), dtype=np.uint8), 0, 0.1)
    C = coarse_grain(T)
    assert len(C) == 5 and all(len(row) == 5 for row in C)
    assert C[1][1].shape == (8, 8, 8, 8)
    assert C[0][0].shape == (1, 8, 1, 8)
    assert C[4][4].shape == (2, 1, 2, 1)
    assert C[2][4].shape == (8, 1, 2, 2)


def test_single_fused_block_is_the_exact_contraction():
    # d = 3: W = 5 fuses into 2 x 2 tensors, one 2 x 2 block covers them all;
    # with a bond large enough nothing is truncated and the read-out is the
    # exact contraction (bMPS limit of Sec. III.A).
    d, p = 3, 0.12
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(809, 0, 2, d, p)
    for s in S:
        r = decode_coarse(s, d, p, chi=4096, max_iter=3, delta0=0.0)
        for L in range(4):
            ex = exact_contract_log(coset_network(lat, s, L, p))
            assert abs(r["logp"][L] - ex) < 1e-10


@pytest.mark.parametrize("d", [4, 7])
def test_untruncated_scheme_equals_dense_6x6_blocks(d):
    # 2 x 2 fused blocks are 6 x 6 node blocks with the same boundaries, and
    # a message over two fused legs is exact at bond 8: with chi large
    # enough that the in-block MPS is not truncated either, the scheme
    # equals the dense fused-block BP with 6 x 6 blocks (Remark 9).
    p = 0.08
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(810, 0, 1, d, p)
    for s in S:
        r = decode_coarse(s, d, p, chi=4096, max_iter=4, delta0=0.0)
        assert r["stats"].truncations == 0
        for L in range(4):
            lp, dl, _, _ = run_naive(coset_network(lat, s, L, p), 6, 4, 0.1, 0.0)
            assert abs(r["logp"][L] - lp) < 1e-9
            assert abs(r["delta"][L] - dl) < 1e-7


def test_bond_below_eight_truncates_and_converges_to_the_dense_blocks():
    # d = 7, one syndrome, 6 iterations: chi = 1, 2, 4 truncate the boundary
    # MPS inside the blocks, and the error against the dense 6 x 6 blocks
    # shrinks as chi grows; from chi = 8 on nothing is truncated and the
    # scheme equals the dense blocks.
    d, p = 7, 0.1
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(811, 0, 1, d, p)
    s = S[0]
    exact = np.array([run_naive(coset_network(lat, s, L, p), 6, 6, 0.1, 0.0)[0] for L in range(4)])
    errs = []
    for chi in (1, 2, 4, 8):
        r = decode_coarse(s, d, p, chi=chi, max_iter=6, delta0=0.0)
        assert (r["stats"].truncations > 0) == (chi < 8)
        errs.append(float(np.max(np.abs(r["logp"] - exact))))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-9


@pytest.mark.parametrize("d,p,seed", [(7, 0.15, 813), (9, 0.12, 814)])
def test_paper_chi16_scheme_truncates_nothing(d, p, seed):
    # The paper's bond (chi = 16), 10 iterations: the boundary MPS of a
    # 2 x 2 fused block never needs a bond above 8 here, so the scheme
    # truncates nothing and equals the dense fused-block BP with 6 x 6
    # blocks (which the GPU's k = 6 kernels compute).
    lat = Lattice(d)
    _, _, S = synth.sample_syndromes(seed, 0, 1, d, p)
    s = S[0]
    r = decode_coarse(s, d, p, chi=16, max_iter=10, delta0=0.0, cutoff=1e-15)
    assert r["stats"].truncations == 0
    for L in range(4):
        lp, dl, _, _ = run_naive(coset_network(lat, s, L, p), 6, 10, 0.1, 0.0)
        assert abs(r["logp"][L] - lp) < 1e-9


def test_uniform_messages_over_fused_legs_have_unit_norm():
    m = M.uniform_dims([8, 8, 2])
    assert np.isclose(np.linalg.norm(M.to_dense(m)), 1.0)
    assert np.allclose(M.to_dense(m), 1.0 / np.sqrt(128.0))
    np.testing.assert_array_equal(M.to_dense(M.uniform_dims([2, 2, 2])), M.to_dense(M.uniform(3)))
