"""Host arithmetic of the benchmark: the algorithmic flop count behind the
FP64 roofline, checked against closed forms of the workloads."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from workloads import Circuit, Op, strongly_entangling  # noqa: E402


def test_sel24_sweep_flops_closed_form():
    # 8 layers x 24 Rot = 192 Rot, each swept as RZ, RY, RZ: per rotation and
    # amplitude 6 flops on phi and on each of the 24 lambdas, plus 4 per lambda
    # for Im<lambda|G phi>; the CNOT ring is a permutation (0 flops)
    c, _ = strongly_entangling(24, 8)
    m = 24
    want = 192 * 3 * (6 * (1 + m) + 4 * m) * 2.0 ** 24
    assert bench.adjoint_flops(c, m) == pytest.approx(want, rel=1e-15)
    assert want == pytest.approx(2.377e12, rel=1e-3)


def test_controls_halve_the_flops_and_constant_gates_add_no_inner_product():
    n, m = 6, 3
    one = bench.adjoint_flops(Circuit(n, [Op("RX", (0,), (0,))], 1, []), m)
    ctrl = bench.adjoint_flops(Circuit(n, [Op("RX", (1,), (0,), controls=(0,))], 1, []), m)
    had = bench.adjoint_flops(Circuit(n, [Op("Hadamard", (2,))], 0, []), m)
    assert one == (6 * (1 + m) + 4 * m) * 2 ** n
    assert ctrl == one / 2
    assert had == 4 * (1 + m) * 2 ** n


def test_fp64_peak_is_the_pipe_arithmetic():
    # 152 SMs x 2 FP64 FMA per clock x 2 flops x 2070 MHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25856, rel=1e-5)


def test_oracle_layered12_timing_restores_the_thread_count():
    import oracle
    before = oracle.num_threads()
    r = bench.oracle_layered12(reps=1)
    assert oracle.num_threads() == before
    assert r["threads"] == before and r["ms_all_threads"] > 0 and r["ms_one_thread"] > 0


def test_both_arms_print_the_same_config():
    # the reference arm hard-codes the workload's sizes; our arm derives them from the workload
    c, _ = strongly_entangling(bench.N_QUBITS, bench.LAYERS)
    ours = bench.bench_config(bench.N_QUBITS, bench.LAYERS, "c128", 1, c.n_params, len(c.observables))
    ref = bench.bench_config(bench.N_QUBITS, bench.LAYERS, "c128", 1, 576, 24)
    assert ours == ref and ours["workload"] == bench.WORKLOAD
