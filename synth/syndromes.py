"""Counter-based depolarizing-noise sampler for the planar surface code.

Workload recipe (Sec. IV, code-capacity model): every qubit independently
suffers I with probability 1-p and X, Y or Z with probability p/3 each; the
syndrome is measured perfectly.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator keyed by (seed, shot, qubit):

    r = mix(mix(mix(seed) ^ shot) ^ qubit),   mix(x) = splitmix64 output of x

The draw for one qubit is decided in integers only, so every implementation
of this recipe (this module, the CUDA sampler) gives the same bits:

    u53 = r >> 11;  identity iff u53 < floor((1 - p) * 2^53)
    otherwise kind = ((mix(r) >> 32) * 3) >> 32  in {0, 1, 2} -> X, Y, Z

Lattice conventions (Sec. II.B, Fig. 1): the (2d-1) x (2d-1) grid holds a
horizontal-edge qubit at (even, even), a vertical-edge qubit at (odd, odd), a
site check A_u at (even, odd) and a plaquette check B_p at (odd, even); a
check acts on its grid neighbours.  Qubits are numbered row-major over the
grid positions with i + j even.  Syndrome bits are all A_(r,c) row-major
(r < d, c < d-1) followed by all B_(r,j) row-major (r < d-1, j < d).
A Pauli is a pair of bit planes (x, z); A_u (Z type) detects x, B_p (X type)
detects z.
"""

from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """One SplitMix64 step applied to the state value(s) ``x`` (uint64)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def counter_u64(seed, shot, qubit):
    """64 random bits for (seed, shot, qubit); broadcasting over arrays."""
    s = splitmix64(np.uint64(seed))
    a = splitmix64(s ^ np.asarray(shot, dtype=np.uint64))
    return splitmix64(a ^ np.asarray(qubit, dtype=np.uint64))


def grid_side(d: int) -> int:
    return 2 * d - 1


def n_qubits(d: int) -> int:
    return d * d + (d - 1) * (d - 1)


def n_checks(d: int) -> int:
    return 2 * d * (d - 1)


def qubit_positions(d: int) -> np.ndarray:
    """Grid positions (i, j) of the qubits, in qubit-index order, shape [n, 2]."""
    W = grid_side(d)
    pos = [(i, j) for i in range(W) for j in range(W) if (i + j) % 2 == 0]
    return np.asarray(pos, dtype=np.int64)


def identity_threshold(p: float) -> int:
    return int((1.0 - float(p)) * 9007199254740992.0)


def sample_errors(seed: int, first_shot: int, B: int, d: int, p: float):
    """Depolarizing errors for shots first_shot .. first_shot+B-1.

    Returns (ex, ez), uint8 arrays of shape [B, n]."""
    n = n_qubits(d)
    shots = np.arange(first_shot, first_shot + B, dtype=np.uint64)[:, None]
    q = np.arange(n, dtype=np.uint64)[None, :]
    r = counter_u64(seed, shots, q)
    u53 = r >> np.uint64(11)
    err = u53 >= np.uint64(identity_threshold(p))
    kind = ((splitmix64(r) >> np.uint64(32)) * np.uint64(3)) >> np.uint64(32)
    ex = (err & ((kind == 0) | (kind == 1))).astype(np.uint8)
    ez = (err & ((kind == 1) | (kind == 2))).astype(np.uint8)
    return ex, ez


def _place(bits: np.ndarray, d: int) -> np.ndarray:
    """Scatter per-qubit bits [B, n] onto a zero-padded grid [B, W+2, W+2]."""
    W = grid_side(d)
    pos = qubit_positions(d)
    g = np.zeros((bits.shape[0], W + 2, W + 2), dtype=np.uint8)
    g[:, pos[:, 0] + 1, pos[:, 1] + 1] = bits
    return g


def syndromes_of(ex: np.ndarray, ez: np.ndarray, d: int) -> np.ndarray:
    """Syndrome bits [B, m] of the Paulis (ex, ez) [B, n]."""
    W = grid_side(d)
    gx = _place(np.asarray(ex, dtype=np.uint8), d)
    gz = _place(np.asarray(ez, dtype=np.uint8), d)

    def nbr_xor(g):
        # XOR of the four grid neighbours of every interior position.
        return (g[:, :-2, 1:-1] ^ g[:, 2:, 1:-1] ^ g[:, 1:-1, :-2] ^ g[:, 1:-1, 2:])

    sx = nbr_xor(gx)  # [B, W, W]
    sz = nbr_xor(gz)
    a = sx[:, 0:W:2, 1:W:2].reshape(ex.shape[0], -1)   # sites (even, odd)
    b = sz[:, 1:W:2, 0:W:2].reshape(ex.shape[0], -1)   # plaquettes (odd, even)
    return np.concatenate([a, b], axis=1).astype(np.uint8)


def sample_syndromes(seed: int, first_shot: int, B: int, d: int, p: float):
    """(ex, ez, syndromes) for B seeded shots."""
    ex, ez = sample_errors(seed, first_shot, B, d, p)
    return ex, ez, syndromes_of(ex, ez, d)


def workload_seed(config: int, p_index: int) -> int:
    """Seed of workload ``config`` at noise level number ``p_index``."""
    return 1000 * int(config) + int(p_index)
