"""MPS machinery of the boundary-MPS method (Sec. III.A) in plain numpy.

An MPS is a list of site tensors A[s] with axes (left bond, physical, right
bond).  Compression follows the textbook scheme the paper cites
(Schollwoeck 2011): a right-to-left QR sweep makes sites 1..n-1
right-canonical, then a left-to-right SVD sweep keeps at each cut the
largest singular values, at most ``D`` of them (the truncation bond chi of
Sec. III.A) and only those above ``cutoff * sigma_1``, leaving sites
0..n-2 left-canonical.  The last site is then divided by its Frobenius norm,
which makes the whole MPS left-canonical with unit L2 norm (Remark 3); the
log of the removed norm is returned.

Readings (the paper is silent on these):
* the relative cutoff discards numerically zero Schmidt values, so that the
  bond spaces -- and therefore every later truncation -- are unique;
* end bonds (dimension != 1 at the chain ends) belong to the left system at
  the first cut and to the right system at the last cut; they are never
  truncated.

Library primitives used as steps: numpy.linalg.qr and numpy.linalg.svd
(LAPACK).  Pins: tests/test_oracle_mps.py (Eckart-Young error, canonical
forms, D -> infinity is exact).
"""

from __future__ import annotations

import numpy as np


class Stats:
    """Diagnostics and the algorithmic flop counter of one decode."""

    def __init__(self):
        self.flops = 0.0
        self.min_gap = np.inf     # min relative gap (s_D - s_{D+1}) / s_1 at a real truncation
        self.truncations = 0      # cuts where a Schmidt value above the cutoff was discarded
        self.max_discarded = 0.0  # largest discarded relative Schmidt weight

    # Flop models (Golub & Van Loan, Matrix Computations, 4th ed.):
    #   Householder QR with thin Q of an a x b matrix (a >= b): 4ab^2 - 4b^3/3
    #   R-SVD with thin U, Sigma, V of an a x b matrix (a >= b): 6ab^2 + 11b^3
    def qr(self, a, b):
        a, b = max(a, b), min(a, b)
        self.flops += 4.0 * a * b * b - 4.0 * b ** 3 / 3.0

    def svd(self, a, b):
        a, b = max(a, b), min(a, b)
        self.flops += 6.0 * a * b * b + 11.0 * b ** 3

    def contract(self, *dims):
        """Multiply-add count of an elementwise-product sum over ``dims``."""
        self.flops += 2.0 * float(np.prod(dims))


def truncated_svd(M: np.ndarray, D: int, cutoff: float, stats: Stats | None = None):
    """Thin SVD of M keeping at most D values, all above cutoff * s_1."""
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    if stats is not None:
        stats.svd(*M.shape)
    if s.size == 0 or s[0] == 0.0:
        r = 1
    else:
        r = int(np.count_nonzero(s > cutoff * s[0]))
        r = max(1, min(r, D))
        if stats is not None and r < s.size and s[r] > cutoff * s[0]:
            stats.truncations += 1
            stats.min_gap = min(stats.min_gap, (s[r - 1] - s[r]) / s[0])
            stats.max_discarded = max(stats.max_discarded,
                                      float(np.sum(s[r:] ** 2) / np.sum(s ** 2)))
    return U[:, :r], s[:r], Vt[:r, :]


def right_canonicalize(mps, stats: Stats | None = None):
    """Right-to-left QR sweep: sites 1..n-1 right-canonical (no truncation)."""
    mps = [A.copy() for A in mps]
    for i in range(len(mps) - 1, 0, -1):
        a, p, b = mps[i].shape
        M = mps[i].reshape(a, p * b)
        Q, R = np.linalg.qr(M.T)              # M = R^T Q^T
        if stats is not None:
            stats.qr(p * b, a)
        r = Q.shape[1]
        mps[i] = Q.T.reshape(r, p, b)
        la, lp, lb = mps[i - 1].shape
        mps[i - 1] = np.einsum("xpb,br->xpr", mps[i - 1], R.T)
        if stats is not None:
            stats.contract(la, lp, lb, r)
    return mps


def compress(mps, D: int, cutoff: float, stats: Stats | None = None):
    """QR sweep right-to-left, truncated SVD sweep left-to-right, normalise.

    Returns (new_mps, log_norm) where the new MPS is left-canonical with
    unit norm and ``exp(log_norm) * new_mps`` approximates the input."""
    mps = right_canonicalize(mps, stats)
    n = len(mps)
    for i in range(n - 1):
        a, p, b = mps[i].shape
        U, s, Vt = truncated_svd(mps[i].reshape(a * p, b), D, cutoff, stats)
        r = s.size
        mps[i] = U.reshape(a, p, r)
        SV = s[:, None] * Vt
        na, np_, nb = mps[i + 1].shape
        mps[i + 1] = np.einsum("rb,bpc->rpc", SV, mps[i + 1])
        if stats is not None:
            stats.contract(r, b, np_, nb)
    nrm = float(np.linalg.norm(mps[-1]))
    if nrm == 0.0 or not np.isfinite(nrm):
        return mps, -np.inf
    mps[-1] = mps[-1] / nrm
    return mps, float(np.log(nrm))


def overlap(m1, m2, stats: Stats | None = None) -> float:
    """<m1|m2> of two real MPS with matching physical legs and end bonds 1."""
    E = np.ones((1, 1))
    for A, B in zip(m1, m2):
        E = np.einsum("ab,apc,bpd->cd", E, A, B)
        if stats is not None:
            stats.contract(A.shape[0], B.shape[0], A.shape[1], A.shape[2], B.shape[2])
    return float(E.reshape(-1)[0]) if E.size == 1 else float(np.trace(E))


def direct_sum(a: float, m1, b: float, m2):
    """MPS of the vector a*m1 + b*m2 (bond dims add)."""
    n = len(m1)
    if n == 1:
        return [a * m1[0] + b * m2[0]]
    out = []
    for i, (A, B) in enumerate(zip(m1, m2)):
        la, p, ra = A.shape
        lb, _, rb = B.shape
        if i == 0:
            C = np.concatenate([a * A, b * B], axis=2)
        elif i == n - 1:
            C = np.concatenate([A, B], axis=0)
        else:
            C = np.zeros((la + lb, p, ra + rb))
            C[:la, :, :ra] = A
            C[la:, :, ra:] = B
        out.append(C)
    return out


def to_dense(mps) -> np.ndarray:
    """The vector an MPS with end bonds 1 represents (site 0 most significant)."""
    v = mps[0]
    for A in mps[1:]:
        v = np.einsum("xpb,bqc->xpqc", v, A).reshape(v.shape[0], -1, A.shape[2])
    return v.reshape(-1)


def uniform(w: int):
    """Unit-norm uniform product message (Remark 2)."""
    return [np.full((1, 2, 1), 1.0 / np.sqrt(2.0)) for _ in range(w)]


def uniform_dims(dims):
    """Unit-norm uniform product message over legs of the given dimensions."""
    return [np.full((1, n, 1), 1.0 / np.sqrt(float(n))) for n in dims]


def reverse(mps):
    """The same vector read with the site order reversed."""
    return [np.transpose(A, (2, 1, 0)) for A in mps[::-1]]
