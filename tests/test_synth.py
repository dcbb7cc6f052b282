"""The seeded workload module: generator, sampler statistics, syndrome map."""

import numpy as np

import synth
from oracle.lattice import Lattice


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; the reference C code
    # by Vigna prints these three values first).
    g = np.uint64(0x9E3779B97F4A7C15)
    state = np.uint64(0)
    got = []
    for _ in range(3):
        got.append(int(synth.splitmix64(state)))
        with np.errstate(over="ignore"):
            state = state + g
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counts():
    for d in (2, 3, 5, 11):
        assert synth.n_qubits(d) == d * d + (d - 1) ** 2
        assert synth.n_checks(d) == 2 * d * (d - 1)
        assert len(synth.qubit_positions(d)) == synth.n_qubits(d)


def test_depolarizing_frequencies():
    p = 0.1
    ex, ez = synth.sample_errors(7, 0, 4000, 5, p)
    N = ex.size
    kinds = {
        "I": np.mean((ex == 0) & (ez == 0)), "X": np.mean((ex == 1) & (ez == 0)),
        "Y": np.mean((ex == 1) & (ez == 1)), "Z": np.mean((ex == 0) & (ez == 1)),
    }
    want = {"I": 1 - p, "X": p / 3, "Y": p / 3, "Z": p / 3}
    for k, f in kinds.items():
        sd = np.sqrt(want[k] * (1 - want[k]) / N)
        assert abs(f - want[k]) < 6 * sd, (k, f)


def test_counter_based_shots_are_independent_of_batching():
    a = synth.sample_errors(3, 0, 10, 5, 0.15)
    b = synth.sample_errors(3, 4, 3, 5, 0.15)
    assert np.array_equal(a[0][4:7], b[0]) and np.array_equal(a[1][4:7], b[1])


def test_syndrome_map_matches_oracle_lattice():
    # Two independent implementations of s(f): vectorised grid XOR here,
    # per-check loops over supports in the oracle.
    for d in (2, 3, 5, 7):
        lat = Lattice(d)
        ex, ez, s = synth.sample_syndromes(11, 0, 20, d, 0.2)
        for b in range(20):
            assert np.array_equal(s[b], lat.syndrome(ex[b], ez[b]))
