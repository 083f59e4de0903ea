"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package describes circuits and observables only as structure (gate names,
wires, parameter indices) plus seeded random numbers.  It holds none of the
simulation arithmetic: no gate matrices, no index arithmetic, no reductions.
The dense unitaries of :class:`MatrixOp` are random input data.
"""

from .circuits import (  # noqa: F401
    Op,
    MatrixOp,
    Circuit,
    Term,
    GATE_ARITY,
    GATE_NPARAMS,
    layered_circuit,
    strongly_entangling,
    qaoa_maxcut,
    qaoa_param_sets,
    qaoa_mixed_instances,
    regular_graph,
    vqe_givens,
    ry_cz_brick,
    dense_block_wires,
    random_unitary,
    random_circuit,
    random_hamiltonian,
    random_state,
    config_seed,
)
