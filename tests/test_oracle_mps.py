"""Pins of oracle.mps against linear-algebra facts (Eckart-Young, canonical forms)."""

import numpy as np

from oracle import mps as M

rng = np.random.default_rng(99)


def rand_mps(dims, p=2):
    return [rng.standard_normal((dims[i], p, dims[i + 1])) for i in range(len(dims) - 1)]


def test_compress_exact_when_D_large():
    m = rand_mps([1, 2, 4, 8, 4, 2, 1])
    v = M.to_dense(m)
    c, ln = M.compress(m, D=64, cutoff=0.0)
    np.testing.assert_allclose(np.exp(ln) * M.to_dense(c), v, rtol=0, atol=1e-12 * np.linalg.norm(v))


def test_compress_left_canonical_unit_norm():
    m = rand_mps([1, 2, 4, 8, 4, 2, 1])
    c, _ = M.compress(m, D=3, cutoff=1e-13)
    for A in c[:-1]:
        a, p, b = A.shape
        G = A.reshape(a * p, b).T @ A.reshape(a * p, b)
        np.testing.assert_allclose(G, np.eye(b), atol=1e-13)
    assert abs(np.linalg.norm(M.to_dense(c)) - 1.0) < 1e-13
    assert max(A.shape[2] for A in c) <= 3


def test_two_site_truncation_is_eckart_young():
    # A 2-site MPS is a matrix; truncating its one cut to D is the best rank-D
    # approximation, with error sqrt(sum of discarded sigma^2).
    A = rng.standard_normal((8, 8))
    U, s, Vt = np.linalg.svd(A)
    m = [U.reshape(1, 8, 8) * 1.0, (np.diag(s) @ Vt).reshape(8, 8, 1)]
    for D in (1, 3, 5):
        c, ln = M.compress(m, D=D, cutoff=0.0)
        approx = np.exp(ln) * M.to_dense(c)
        err = np.linalg.norm(approx - A.reshape(-1))
        assert abs(err - np.sqrt(np.sum(s[D:] ** 2))) < 1e-10


def test_cutoff_drops_numerical_zeros():
    # A product state written with a redundant bond of 4 compresses to bond 1.
    a = rng.standard_normal(2)
    b = rng.standard_normal(2)
    A = np.zeros((1, 2, 4))
    A[0, :, 0] = a
    B = np.zeros((4, 2, 1))
    B[0, :, 0] = b
    B[1:, :, 0] = 0.0
    c, _ = M.compress([A, B], D=4, cutoff=1e-13)
    assert c[0].shape[2] == 1


def test_overlap_direct_sum_reverse_match_dense():
    m1 = rand_mps([1, 2, 3, 2, 1])
    m2 = rand_mps([1, 2, 4, 2, 1])
    assert abs(M.overlap(m1, m2) - M.to_dense(m1) @ M.to_dense(m2)) < 1e-12
    s = M.direct_sum(0.3, m1, 0.7, m2)
    np.testing.assert_allclose(M.to_dense(s), 0.3 * M.to_dense(m1) + 0.7 * M.to_dense(m2), atol=1e-12)
    r = M.reverse(m1)
    v = M.to_dense(m1).reshape(2, 2, 2, 2)
    np.testing.assert_allclose(M.to_dense(r), v.transpose(3, 2, 1, 0).reshape(-1), atol=1e-12)


def test_uniform_message_is_unit_and_flat():
    u = M.to_dense(M.uniform(4))
    np.testing.assert_allclose(u, np.full(16, 0.25))


def test_delta_rank_one_identity():
    # Remark 4 uses ||aa^T - bb^T||_F^2; for unit vectors it is 2 - 2<a|b>^2.
    for _ in range(10):
        a = rng.standard_normal(16)
        b = rng.standard_normal(16)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        lhs = np.linalg.norm(np.outer(a, a) - np.outer(b, b)) ** 2
        assert abs(lhs - (2 - 2 * (a @ b) ** 2)) < 1e-13
