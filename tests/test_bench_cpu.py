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


def test_json_lines_carry_the_contract_keys(monkeypatch, capsys):
    import argparse
    import json

    cfg = bench.bench_config(bench.N_QUBITS, bench.LAYERS, "c128", 1, 576, 24)
    roofline = {"bound": "alu", "achieved": 1.0, "peak": bench.FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": 1.0 / bench.FP64_PEAK_TFLOPS, "traffic": 1.0}
    cpu = {"value": 1.4e5, "unit": "ms", "cores": 16, "kind": "oracle", "sample": "s"}
    e2e = {"value": 2401.0, "unit": "ms", "h2d_bytes_per_step": 9216, "d2h_bytes_per_step": 110784}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    ours = bench.bench_line(2400.0, 1, 20, 5, "c128", cfg, {"forward_passes": 41}, roofline, cpu, e2e, 2400,
                            clocks, {})
    need = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"}
    assert need <= set(ours)
    assert ours["value"] == 2400.0 and ours["higher_is_better"] is False and ours["dtype"] == "f64"
    assert bench.bench_line(2400.0, 4, 20, 5, "c128", cfg, {}, roofline, cpu, e2e, 1, clocks, {})["value"] == 600.0
    # the reference arm (the oracle), with a stand-in for its timed sample
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(bench, "oracle_sample", lambda rows=1: (1.4e5, 1.5e4, "one row", 16, None))
    bench.run_reference(argparse.Namespace(gpus=1, steps=2, warmup=1))
    ref = json.loads(capsys.readouterr().out)
    assert ref["impl"] == "reference" and need - {"roofline", "gpu_launches", "clocks"} <= set(ref)
    for k in ("metric", "unit", "higher_is_better", "config", "dtype", "scaling"):
        assert ref[k] == ours[k], k
    assert ref["steps"] == 2 and ref["warmup"] == 1 and ref["ms_per_step"] == 1.5e4 and ref["value"] == 1.4e5
    assert ref["e2e"] == {"value": 1.4e5, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert ref["cpu_baseline"]["kind"] == "oracle" and ref["cpu_baseline"]["cores"] == 16


def test_oracle_qaoa_throughput_is_reported():
    r = bench.oracle_qaoa20(count=2, n=10)
    assert r["circuits_per_s"] > 0 and r["threads"] >= 1
