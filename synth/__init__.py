"""Seeded synthetic workload for the blockBP decoder.

This package is shared by the CPU oracle, the tests, the CUDA path's tests
and the benchmark.  It holds the workload recipe only: a counter-based
random-number generator, the i.i.d. depolarizing error sampler and the
syndrome map of the planar surface code (Sec. II.B).  None of the decoder's
arithmetic (tensor network, message passing, read-out) lives here.
"""

from .syndromes import (  # noqa: F401
    splitmix64,
    counter_u64,
    grid_side,
    n_qubits,
    n_checks,
    qubit_positions,
    sample_errors,
    syndromes_of,
    sample_syndromes,
    workload_seed,
)
