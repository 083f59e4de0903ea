#!/usr/bin/env python
"""Benchmark of the state-vector hot path on one GB300 (or N replicas).

Step = forward pass + expectation values + full adjoint Jacobian of the
24-qubit strongly-entangling-layers workload (8 layers of Rot per wire plus a
CNOT ring of range r = l mod 23 + 1; 576 parameters; 24 single-Z observables)
in complex128, all kernels of the library on the GPU.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the baseline arm) on the host cores.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "adjoint-Jacobian ms & gate HBM GB/s (% peak) at 24-30 qubits; batched circuits/s"
WORKLOAD = ("sel24: 24-qubit StronglyEntanglingLayers, 8 layers of Rot(phi,theta,omega) per wire + CNOT ring "
            "range l mod 23 + 1, 576 parameters, 24 single-Z observables; step = forward + expvals + full "
            "adjoint Jacobian (24 x 576)")
N_QUBITS, LAYERS = 24, 8
FALLBACK_HBM_GBS = 6800.0


def bench_config(n_qubits: int, layers: int, dtype: str, world: int, n_params: int, n_obs: int) -> dict:
    """The `config` of the JSON line, the same dict in both arms for the same
    workload (the plan's pass counts are reported beside it, not in it)."""
    full = (n_qubits, layers) == (N_QUBITS, LAYERS)
    return {"workload": WORKLOAD if full else f"sel{n_qubits} ({layers} layers; reduced size for profiling)",
            "precision": dtype, "n_qubits": n_qubits, "layers": layers, "n_params": n_params,
            "n_observables": n_obs, "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (129 MB): c128 state 268 MB and 24 lambda vectors 6.4 GB per step"
            if full else "reduced size"}


DTYPE_NAMES = {"c128": "f64", "c64": "f32", "c128df": "df64 (f32 pairs; complex128 storage)"}


def bench_line(ms, world, steps, warmup, dtype, config, plan, roofline, cpu, e2e, launches, clocks, extras) -> dict:
    """The GPU arm's JSON line: ms is the slowest replica's time per step."""
    return {"metric": METRIC, "value": replica_value(ms, world), "unit": "ms", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES[dtype], "data": "synthetic",
            "config": config, "plan": plan, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "extras": extras}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--dtype", choices=["c128", "c64", "c128df"], default="c128",
                    help="c128: FP64 arithmetic; c128df: complex128 storage, double-float arithmetic")
    ap.add_argument("--qubits", type=int, default=N_QUBITS, help="smaller sizes are for profiling captures only")
    ap.add_argument("--layers", type=int, default=LAYERS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the complex64 and per-gate side measurements")
    ap.add_argument("--quick-extras", action="store_true", help="only the other precisions of the same step")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="profiling aid: time --steps runs of one batch of N 20-qubit QAOA p=4 parameter sets "
                         "(complex64, default launch shape, no autotuning) and print one JSON line")
    ap.add_argument("--profile-dense", default=None, metavar="K[:cuda]",
                    help="profiling aid: time --steps applications of a random K-qubit unitary on the lowest K "
                         "wires' bits of a --qubits complex64 state (tensor cores for K = 5 unless ':cuda')")
    ap.add_argument("--profile-vqe", action="store_true",
                    help="profiling aid: --steps energy + adjoint-gradient steps of the 24-qubit VQE workload "
                         "(2000-term Hamiltonian) in --dtype; prints one JSON line")
    ap.add_argument("--profile-expval", action="store_true",
                    help="profiling aid: time --steps expectation values of the 24 single-Z observables on the "
                         "--qubits strongly-entangling output state in --dtype; prints one JSON line")
    ap.add_argument("--profile-rycz30", action="store_true",
                    help="profiling aid: --steps forward + adjoint-Jacobian steps of the 30-qubit RY + CZ-brick "
                         "workload (four 5-qubit dense blocks) in --dtype; prints one JSON line")
    ap.add_argument("--profile-gate", default=None, metavar="GATE:WIRE",
                    help="profiling aid: time --steps passes of one gate (RX, Hadamard or CNOT, control "
                         "wire+1) on a --qubits state of --dtype and print one JSON line (not the bench line)")
    return ap.parse_args()


# DRAM bytes (read + write) per adjoint launch from one ncu capture of the
# current kernel on sel22 (22 observables), scaled to sel24 by the state size
# (x4) and the vector count (25 / 23).  Must be re-taken when the kernel changes:
# a precision whose kernel changed after its capture has no entry (traffic null).
# The complex64 kernel's arithmetic changed to packed FP32 after its capture.
PROFILED_TRAFFIC = {
    "c128": (3.028316e9 * 4 * 25 / 23, "ncu dram bytes of one sel22 adjoint launch, scaled x4 x25/23"),
}

# FP64 pipe of a GB300: 152 SMs x 2 FMA lanes/clk x 2 flops x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# Algorithmic flops per amplitude of one gate application (the unfused method,
# each gate a pass): complex multiply 6, real 2x2 rotation 6, RX 6, general
# 2x2 14, Hadamard 4; permutations and sign flips 0.  PhaseShift touches half
# the amplitudes.  A trainable gate adds Im<lambda|G phi>: 4 flops per
# amplitude per lambda (G a Pauli word: a permutation with signs).
_GATE_FLOPS = {"RZ": 6.0, "RY": 6.0, "RX": 6.0, "PhaseShift": 3.0, "Hadamard": 4.0, "Rot": 14.0,
               "IsingZZ": 6.0, "IsingXX": 6.0, "IsingYY": 6.0, "SingleExcitation": 3.0,
               "DoubleExcitation": 6.0 / 8.0}


def adjoint_flops(circ, m):
    """Algorithmic flops of one adjoint sweep with m lambdas (Rot expanded to
    RZ, RY, RZ as the sweep differentiates it)."""
    amps = float(1 << circ.n)
    total = 0.0
    for op in circ.ops:
        parts = ["RZ", "RY", "RZ"] if op.name == "Rot" else [op.name]
        for name in parts:
            f = _GATE_FLOPS.get(name, 0.0)
            ctrl = 0.5 ** len(op.controls)
            total += amps * ctrl * f * (1 + m)
            if op.params:
                total += amps * ctrl * 4.0 * m
    return total


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ---------------------------------------------------------------------------
# oracle (CPU baseline / reference arm) on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(rows: int = 1):
    """Time the FP64 oracle on the sel24 workload, whole parts only.

    Sample: the oracle's own adjoint-Jacobian call for Jacobian rows
    0..rows-1: a complete forward pass (all 384 ops), lambda_j = Z_j psi for
    those rows, and the complete adjoint sweep (all 768 steps of the expanded
    tape) with phi, mu and those lambdas.  The oracle clocks the work done once
    (forward pass; phi's un-apply and mu = G phi) apart from the work done once
    per observable (lambda_j and E_j; the inner products and lambda_j's
    un-apply).  Every observable is a single Z word, so each row repeats the
    same operations on a vector of the same size, and the full step (24 rows)
    is forward + phi part + 24 / rows x (lambda part + rows part).

    Returns (full-step estimate in ms, the sample's own wall ms, description,
    threads, the sample's Jacobian rows)."""
    import oracle
    from workloads import strongly_entangling

    c, p = strongly_entangling(N_QUBITS, LAYERS)
    m = len(c.observables)
    clock = {}
    t0 = time.perf_counter()
    _, J = oracle.adjoint_jacobian(c, p, observables=c.observables[:rows], clock=clock)
    wall_ms = 1e3 * (time.perf_counter() - t0)
    est_ms = 1e3 * (clock["forward"] + clock["phi"] + m / rows * (clock["lambda"] + clock["rows"]))
    sample = (f"oracle FP64 adjoint Jacobian of sel24 at full size for {rows} of its {m} rows: complete forward "
              f"pass (384 ops) and complete adjoint sweep (768 steps), timed; the full step is forward + phi part "
              f"+ {m}/{rows} x per-row part (forward {clock['forward']:.2f} s, phi {clock['phi']:.2f} s, "
              f"per-row {clock['lambda'] + clock['rows']:.2f} s)")
    return est_ms, wall_ms, sample, oracle.num_threads(), J


def oracle_layered12(reps: int = 3):
    """The oracle on the 12-qubit layered workload (10 layers of RX, RY, RZ on
    every wire plus a CNOT ladder, O = sum_i Z_i, 360 parameters): forward pass
    plus full adjoint Jacobian, median ms over `reps` calls with all host
    threads and with one thread (the thread count is restored afterwards)."""
    import oracle
    from workloads import layered_circuit

    c, p = layered_circuit(12, 10)
    threads = oracle.num_threads()

    def med():
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.adjoint_jacobian(c, p)
            ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts)

    try:
        all_ms = med()
        oracle.set_num_threads(1)
        one_ms = med()
    finally:
        oracle.set_num_threads(threads)
    return {"workload": "layered12: forward + 360-parameter adjoint Jacobian of sum_i Z_i, oracle FP64",
            "ms_all_threads": all_ms, "threads": threads, "ms_one_thread": one_ms, "reps": reps}


def oracle_qaoa20(count: int = 4, n: int = 20):
    """The oracle on the batched QAOA workload: energies of the first `count`
    of the 512 parameter sets of the 20-node p = 4 MaxCut circuit (forward
    pass plus <H_C>, all host threads), as circuits per second."""
    import oracle
    from workloads import qaoa_maxcut, qaoa_param_sets

    c = qaoa_maxcut(n, 4)
    sets = qaoa_param_sets(512, 4)[:count]
    t0 = time.perf_counter()
    for p in sets:
        oracle.expval(oracle.forward(c, p), c.observables[0])
    dt = time.perf_counter() - t0
    return {"workload": f"QAOA MaxCut, {n} nodes, p = 4: energy of {count} parameter sets, oracle FP64",
            "circuits_per_s": count / dt, "threads": oracle.num_threads()}


def max_over_ranks(value: float, world: int, device) -> float:
    """The job's time: the slowest replica's (all-reduce MAX over the process
    group; the replicas themselves exchange nothing)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_max: float, world: int) -> float:
    """Whole-job time per step: `world` replicas each finish one step in ms_max."""
    return ms_max / world if world > 1 else ms_max


def run_reference(args):
    """The oracle arm: each step is one oracle_sample (one complete Jacobian
    row, about 10 s on 16 cores); `value` is the full sel24 step it gives,
    `ms_per_step` the sample's own wall time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    est, wall = [], []
    sample = cores = None
    for i in range(args.warmup + args.steps):
        e, w, sample, cores, _ = oracle_sample(rows=1)
        if i >= args.warmup:
            est.append(e)
            wall.append(w)
    value = statistics.mean(est)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(wall),
            "value_is": "the full sel24 step (forward + 24 x 576 Jacobian) from each timed sample; ms_per_step is "
                        "the sample's own wall time (one complete Jacobian row)",
            "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(N_QUBITS, LAYERS, "c128", int(os.environ.get("WORLD_SIZE", "1")), 576, 24),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample,
                             "samples": len(est), "spread_ms": [min(est), max(est)]},
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# side measurements of the other workload shapes (rank 0, untimed by the contract)
# ---------------------------------------------------------------------------
def _timed(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def extra_gates(hbm_peak, wires_step=1):
    """Per-gate pass at 30 qubits for every target wire (the per-index study):
    RX, Hadamard, CNOT (control wire t+1 mod n).  Reported per wire as GB/s of
    algorithmic bytes (2V, or V for a one-control gate: half the pairs) and as
    a fraction of the measured HBM peak."""
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import Op
    out = {}
    for dtype in ("c128", "c128df", "c64"):
        n = 30
        sv = StateVector(n, dtype, renormalize=False)  # time the gate pass alone
        V = (8 if dtype == "c64" else 16) << n
        res = {}
        for name in ("RX", "Hadamard", "CNOT"):
            fr, ms_l = [], []
            for t in range(0, n, wires_step):
                if name == "CNOT":
                    op = Op("PauliX", (t,), (), ((t + 1) % n,))
                else:
                    op = Op(name, (t,), (0,) if name == "RX" else ())
                prog = Program(sv, [op], 1 if name == "RX" else 0)
                prog.set_params([0.3] if name == "RX" else [])
                ms = _timed(lambda: prog.forward(reset=False), 5, torch.cuda.current_stream())
                alg = (V if name == "CNOT" else 2.0 * V)
                fr.append(round(alg / ms / 1e6 / hbm_peak, 4))
                ms_l.append(round(ms, 3))
                prog.close()
            res[name] = {"wires": list(range(0, n, wires_step)), "ms": ms_l, "frac_of_hbm": fr,
                         "frac_min": min(fr), "frac_median": float(np.median(fr)), "frac_max": max(fr)}
        out[dtype] = res
        sv.close()
        torch.cuda.empty_cache()
    # dense 5-qubit block, complex64, 28 qubits: tensor cores vs CUDA cores.  Algorithmic: 2V bytes;
    # 32 complex multiply-adds per amplitude = 256 real flops per amplitude.
    n = 28
    V = 8 << n
    dense = {}
    for tc in (True, False):
        ms = _dense_block_ms(n, 5, tc, 5, 2)
        dense["tensor_cores" if tc else "cuda_cores"] = {"ms": ms, "frac_of_hbm": 2.0 * V / ms / 1e6 / hbm_peak,
                                                         "tflops": (1 << n) * 256.0 / ms / 1e9}
    out["dense5_n28_c64"] = dense
    return out


def extra_qaoa():
    """Batched QAOA MaxCut: 512 parameter sets of one 20-node circuit and 256
    mixed 14-22-qubit instances, complex64 with FP64 reductions, one persistent
    graph-captured launch each; beside it the plain per-circuit complex128 form."""
    import torch
    from paper_2403_02512_gb300 import _lib as L
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import qaoa_maxcut, qaoa_mixed_instances, qaoa_param_sets
    res = {}
    c = qaoa_maxcut(20, 4)
    sets = qaoa_param_sets(512, 4)
    b = L.Batch([c] * len(sets), L.SV_C64)
    b.set_params(sets.ravel())
    b.autotune()
    b.run()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        e64 = b.run()
    dt = (time.perf_counter() - t0) / reps
    res["qaoa20_x512_c64_batch"] = {"circuits_per_s": len(sets) / dt, "ms_per_batch": dt * 1e3, **b.info()}
    b.close()
    # plain per-circuit complex128 form on a sample of the same parameter sets
    sv = StateVector(20, "c128")
    prog = Program.from_circuit(sv, c)
    k = 32
    e128 = np.zeros(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(k):
        prog.forward(sets[i])
        e128[i] = float(prog.expval()[0])
    dt128 = (time.perf_counter() - t0) / k
    res["qaoa20_per_circuit_c128"] = {"circuits_per_s": 1.0 / dt128, "sample": k,
                                      "max_abs_diff_c64_batch_vs_c128": float(np.abs(e64[:k] - e128).max())}
    # energy + adjoint gradient (8 parameters) of one parameter set, per precision
    for dtype in ("c128", "c64"):
        g_sv = StateVector(20, dtype)
        g_prog = Program.from_circuit(g_sv, c)
        g_prog.set_params(sets[0])

        def grad_step():
            g_prog.forward()
            return g_prog.jacobian()

        ms = _timed(grad_step, 5, torch.cuda.current_stream())
        res[f"qaoa20_energy_and_gradient_{dtype}"] = {"ms": ms, "adjoint_passes": g_prog.stats()[1]}
        g_prog.close()
        g_sv.close()
    prog.close()
    sv.close()
    inst = qaoa_mixed_instances(256, 14, 22, 4)
    b = L.Batch([ci for ci, _ in inst], L.SV_C64)
    b.set_params(np.concatenate([pi for _, pi in inst]))
    b.autotune()
    b.run()
    t0 = time.perf_counter()
    for _ in range(reps):
        b.run()
    dt = (time.perf_counter() - t0) / reps
    res["qaoa_mixed14to22_x256_c64_batch"] = {"circuits_per_s": 256 / dt, "ms_per_batch": dt * 1e3, **b.info()}
    b.close()
    torch.cuda.empty_cache()
    return res


def extra_vqe():
    """24-qubit Givens ansatz, 2000-term Hamiltonian: forward + energy + adjoint gradient (one lambda),
    as one Jacobian call (the energy from lambda = H psi) and as separate energy and VJP calls."""
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import vqe_givens
    c, p = vqe_givens(24, 12, 40, 120, 2000)
    out = {}
    grads = {}
    for dtype in ("c128", "c64"):
        sv = StateVector(24, dtype, basis_state=c.basis_state)
        prog = Program.from_circuit(sv, c)

        def step():
            prog.forward(p)
            prog.expval()
            return prog.vjp(np.ones(1))

        def step_jac():
            prog.forward(p)
            return prog.jacobian()

        ms = _timed(step, 2, torch.cuda.current_stream())
        ms_jac = _timed(step_jac, 2, torch.cuda.current_stream())
        grads[dtype] = step().cpu().numpy()
        out[dtype] = {"ms_energy_and_gradient": ms_jac, "ms_energy_then_vjp": ms,
                      "forward_passes": prog.stats()[0], "adjoint_passes": prog.stats()[1]}
        prog.close()
        sv.close()
        torch.cuda.empty_cache()
    out["c64_max_abs_gradient_diff_vs_c128"] = float(np.abs(grads["c64"] - grads["c128"]).max())
    return out


def extra_measurements(hbm_peak):
    """Measurement processes on the sel24 output state: a forward-mode
    Jacobian-vector product (one tangent pass plus the 24 dots), expectation
    values and variances of the 24 single-Z observables, marginal probabilities
    of all 24 wires, 10^4 samples.  Algorithmic bytes: JVP 2 x 2V per forward
    pass (psi and d psi) + 2 m V; expval V; variance V + 2 m V (lambda passes
    write m vectors, the norms read them); probabilities V; samples V plus the
    2^24-entry CDF."""
    import torch
    from paper_2403_02512_gb300 import _lib as L
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import strongly_entangling
    c, p = strongly_entangling(N_QUBITS, LAYERS)
    m = len(c.observables)
    out = {}
    u = np.random.default_rng(7).random(10000)
    wires = list(range(N_QUBITS))
    for dtype in ("c128", "c64"):
        sv = StateVector(N_QUBITS, dtype)
        prog = Program.from_circuit(sv, c)
        prog.forward(p)
        V = (8 if dtype == "c64" else 16) << N_QUBITS
        res = {}
        tangent = np.random.default_rng(8).normal(size=c.n_params)
        prog.set_params(p)
        for name, fn, alg in (("jvp_forward_mode", lambda: prog.jvp(tangent), 2 * 2 * V * prog.stats()[0] + 2 * m * V),
                              ("expval", lambda: sv.expval(c.observables), V),
                              ("variance", lambda: sv.var(c.observables), V + 2 * m * V),
                              ("probs_all_wires_to_host", lambda: sv.probs(wires), V + 8 * (1 << N_QUBITS)),
                              ("sample_1e4_all_wires", lambda: sv.sample(wires, u), V + 3 * 8 * (1 << N_QUBITS))):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()  # the JVP leaves its output on the device
            ms = (time.perf_counter() - t0) / reps * 1e3
            res[name] = {"ms": ms, "frac_of_hbm": alg / ms / 1e6 / hbm_peak}
        # sparse observable: 8 stored entries per row (the diagonal plus 7 seeded columns)
        rows = 1 << N_QUBITS
        rng = np.random.default_rng(9)
        cols = np.concatenate([np.arange(rows)[:, None], rng.integers(0, rows, (rows, 7))], axis=1)
        cols.sort(axis=1)
        vals = rng.normal(size=cols.shape) + 1j * rng.normal(size=cols.shape)
        sp = L.Sparse(N_QUBITS, np.arange(0, 8 * rows + 1, 8), cols.ravel(), vals.ravel())
        alg_sp = 8 * (rows + 1) + 24 * 8 * rows + V + 8 * V  # CSR arrays, psi rows, gathered columns
        L.sv_sparse_expval(sv.handle, sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            L.sv_sparse_expval(sv.handle, sp)
        ms = (time.perf_counter() - t0) / 3 * 1e3
        res["sparse_expval_8_per_row"] = {"ms": ms, "frac_of_hbm": alg_sp / ms / 1e6 / hbm_peak}
        sp.close()
        del cols, vals
        out[dtype] = res
        prog.close()
        sv.close()
        torch.cuda.empty_cache()
    return out


def extra_layered12():
    """12-qubit layered RX/RY/RZ + CNOT ladder, O = sum_i Z_i, complex128:
    forward + expval + full adjoint Jacobian (360 parameters).  The state is
    64 KiB, so the step is bound by launch and pass latency, not HBM: reported
    in microseconds per step (its parity with the oracle is a test case)."""
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import layered_circuit
    c, p = layered_circuit(12, 10)
    sv = StateVector(12, "c128")
    prog = Program.from_circuit(sv, c)

    def step():
        prog.forward(p)
        return prog.jacobian()

    for _ in range(3):
        step()
    ms = _timed(step, 50, torch.cuda.current_stream())
    out = {"us_forward_and_jacobian": ms * 1e3, "forward_passes": prog.stats()[0], "adjoint_passes": prog.stats()[1]}
    prog.close()
    sv.close()
    return out


def extra_dense_fusion_layer30(hbm_peak):
    """Dense-block fusion measured per layer of the 30-qubit RY + CZ-brick
    workload (complex64): (a) one layer as the planner runs it, RY on all 30
    wires plus the layer's CZ brick in tile passes; (b) the same layer fused
    into 5-wire windows, i.e. six 5-qubit dense blocks on the tensor cores
    (wires 5w .. 5w + 4) plus the CZ gates that cross a window boundary.  The
    kernels' time does not depend on the matrices' entries, so (b) uses seeded
    unitaries."""
    import torch
    from paper_2403_02512_gb300 import _lib as L
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import Op
    n = 30
    out = {}
    sv = StateVector(n, "c64", renormalize=False)
    for parity in (0, 1):
        layer = [Op("RY", (w,), (w,)) for w in range(n)]
        layer += [Op("PauliZ", (a + 1,), controls=(a,)) for a in range(parity, n - 1, 2)]
        prog = Program(sv, layer, n)
        prog.set_params(np.linspace(0.1, 3.0, n))
        ms_tiles = _timed(lambda: prog.forward(reset=False), 5, torch.cuda.current_stream())
        passes = prog.stats()[0]
        prog.close()
        cross = [Op("PauliZ", (a + 1,), controls=(a,)) for a in range(parity, n - 1, 2) if (a + 1) % 5 == 0]
        pc = Program(sv, cross, 0)
        pc.set_params([])
        rng = np.random.default_rng(parity)
        mats = [np.linalg.qr(rng.normal(size=(32, 32)) + 1j * rng.normal(size=(32, 32)))[0] for _ in range(6)]

        def fused():
            for w in range(6):
                sv.apply_matrix(list(range(5 * w, 5 * w + 5)), mats[w])
            if cross:
                pc.forward(reset=False)

        ms_fused = _timed(fused, 3, torch.cuda.current_stream())
        pc.close()
        out["even_layer" if parity == 0 else "odd_layer"] = {
            "tile_passes_ms": ms_tiles, "tile_passes": passes, "fused_dense_ms": ms_fused,
            "fused_blocks": 6, "boundary_cz": len(cross)}
    sv.close()
    torch.cuda.empty_cache()
    return out


def _kernel_split(kt):
    total = sum(v[0] for v in kt.values()) or 1.0
    return {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / total, 4)}
            for k, v in kt.items() if v[1] > 0}


def extra_rycz30(hbm_peak, reps=3):
    """30-qubit RY layers + CZ brick + a 5-qubit dense block after every fifth
    layer, <Z0 Z29>: forward + full adjoint Jacobian (600 params), `reps`
    timed repetitions (no kernel events), then one repetition with per-kernel
    CUDA events for the kernel split and the rooflines of the adjoint tile
    kernel (2V(1 + m) bytes per launch, m = 1; FP64 flops of the unfused
    method) and of the dense-block kernels (2V bytes and 256 flops per
    amplitude per application).  The dense blocks run on the tensor cores in
    complex64 and on the CUDA cores in complex128."""
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import ry_cz_brick
    from paper_2403_02512_gb300 import _lib as L
    c, p = ry_cz_brick(30, 20)
    n_dense = sum(op.name == "QubitUnitary" for op in c.ops)
    out = {}
    # the last run applies the complex64 dense blocks on the CUDA cores instead
    for key, dtype, tc in (("c128", "c128", True), ("c64", "c64", True), ("c64_dense_on_cuda_cores", "c64", False)):
        L.sv_set_dense_tensor_cores(tc)
        sv = StateVector(30, dtype)
        prog = Program.from_circuit(sv, c)

        def step():
            prog.forward(p)
            return prog.jacobian()

        try:
            step()
            torch.cuda.synchronize()
            times = [_timed(step, 1, torch.cuda.current_stream()) for _ in range(reps if tc else 1)]
            L.sv_kernel_timing_reset()
            L.sv_kernel_timing_enable(True)
            E, J = step()
            torch.cuda.synchronize()
            L.sv_kernel_timing_enable(False)
            kt = L.sv_kernel_timing_read()
        finally:
            L.sv_set_dense_tensor_cores(True)
        V = (8 if dtype == "c64" else 16) << 30
        res = {"ms_forward_and_jacobian": float(np.median(times)), "ms_reps": times, "expval": float(E[0]),
               "forward_passes": prog.stats()[0], "adjoint_passes": prog.stats()[1], "J_sum": float(J.sum()),
               "kernels": _kernel_split(kt)}
        adj_ms, adj_n = kt["tile_adjoint"]
        if adj_n:
            fl = adjoint_flops(c, 1) / adj_n  # one sweep per repetition
            res["roofline_tile_adjoint"] = {
                "launches": adj_n, "avg_launch_ms": adj_ms / adj_n,
                "hbm_frac": 2.0 * V * 2 / (adj_ms / adj_n * 1e-3) / 1e9 / hbm_peak,
                "fp64_tflops_algorithmic": fl / (adj_ms / adj_n * 1e-3) / 1e12,
                "fp64_frac": (fl / (adj_ms / adj_n * 1e-3) / 1e12 / FP64_PEAK_TFLOPS) if dtype == "c128" else None}
        dk_ms, dk_n = kt["dense_k"]
        if dk_n:
            res["roofline_dense_blocks"] = {
                "launches": dk_n, "applications": 3 * n_dense, "avg_launch_ms": dk_ms / dk_n,
                "hbm_frac": 2.0 * V * 3 * n_dense / (dk_ms * 1e-3) / 1e9 / hbm_peak,
                "tflops_algorithmic": 256.0 * (1 << 30) * 3 * n_dense / (dk_ms * 1e-3) / 1e12}
        out[key] = res
        prog.close()
        sv.close()
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2403_02512_gb300 import _lib as L
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import strongly_entangling

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    hbm_peak, peak_kind = peaks()
    NQ = args.qubits
    c, p = strongly_entangling(NQ, args.layers)
    m, P = len(c.observables), c.n_params

    def measure(dtype, steps, warmup, timing):
        sv = StateVector(NQ, dtype)
        prog = Program.from_circuit(sv, c)
        params = torch.tensor(p, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()

        def step():
            prog.set_params(params)
            prog.forward()
            return prog.jacobian()

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        if timing:
            clocks.start()
        # the headline region: kernel-timing events off
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launches = 0
        for _ in range(steps):
            prog.set_params(params)
            launches += prog.stats()[2]
            prog.forward()
            launches += prog.stats()[2]
            E, J = prog.jacobian()
            launches += prog.stats()[2]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if timing else None
        ms = e0.elapsed_time(e1) / steps
        kt = None
        if timing:
            # the roofline region: the same steps again with a CUDA event pair
            # around every library kernel launch (on the library's stream)
            L.sv_kernel_timing_reset()
            L.sv_kernel_timing_enable(True)
            for _ in range(min(steps, 5)):
                step()
            torch.cuda.synchronize()
            L.sv_kernel_timing_enable(False)
            kt = L.sv_kernel_timing_read()
        fp, ap, _ = prog.stats()
        out = {"ms": ms, "launches": launches, "kt": kt, "clocks": clk, "fwd_passes": fp, "adj_passes": ap,
               "J": J, "E": E, "vec_bytes": (8 if dtype == "c64" else 16) << NQ}
        prog.close()
        sv.close()
        del params
        torch.cuda.empty_cache()
        return out

    main = measure(args.dtype, args.steps, args.warmup, timing=True)
    ms = max_over_ranks(main["ms"], world, "cuda")

    # roofline of the dominant kernel (tile_adjoint).  HBM: algorithmic bytes
    # 2V(1 + m) per launch.  Arithmetic: the sweep's algorithmic flops
    # (adjoint_flops) over all launches.  Native complex128 is bound by the FP64
    # pipe and reports "alu"; complex64 and double-float report HBM.
    kt = main["kt"]
    V = main["vec_bytes"]
    adj_ms, adj_n = kt["tile_adjoint"]
    bytes_per_launch = 2.0 * V * (1 + m)
    hbm_achieved = bytes_per_launch * adj_n / (adj_ms * 1e-3) / 1e9 if adj_ms > 0 else None
    flops_per_launch = adjoint_flops(c, m) / max(1, main["adj_passes"])  # one sweep = adj_passes launches
    flops_achieved = flops_per_launch * adj_n / (adj_ms * 1e-3) / 1e12 if adj_ms > 0 else None
    total_kernel_ms = sum(v[0] for v in kt.values())
    shares = {k: round(v[0] / total_kernel_ms, 4) for k, v in kt.items() if v[1] > 0}
    common = {"kernel": "k_tile_adjoint", "avg_launch_ms": adj_ms / max(1, adj_n), "launches": adj_n,
              "timed_in": "a second region of min(steps, 5) steps with per-launch CUDA events",
              "algorithmic_bytes_per_launch": bytes_per_launch,
              "algorithmic_flops_per_launch": flops_per_launch,
              "hbm_achieved_gbs": hbm_achieved, "hbm_frac": (hbm_achieved / hbm_peak) if hbm_achieved else None,
              "kernel_time_shares": shares, "traffic": None}
    if (NQ, args.layers) == (N_QUBITS, LAYERS) and args.dtype in PROFILED_TRAFFIC:
        common["traffic"], common["traffic_source"] = PROFILED_TRAFFIC[args.dtype]
    if args.dtype == "c128":
        roofline = {"bound": "alu", "achieved": flops_achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": flops_achieved / FP64_PEAK_TFLOPS if flops_achieved else None,
                    "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2070 MHz (FP64 pipe)", **common}
    else:
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": (hbm_achieved / hbm_peak) if hbm_achieved else None, "peak_kind": peak_kind,
                    "fp_tflops_algorithmic": flops_achieved, **common}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        dt = L.SV_C64 if args.dtype == "c64" else L.SV_C128
        h = L.sv_create(NQ, dt)
        if args.dtype == "c128df":
            L.sv_set_compute(h, L.SV_COMPUTE_DOUBLE_FLOAT)
        L.sv_set_stream(h, torch.cuda.current_stream().cuda_stream)
        tape, obs = L.Tape(c.ops, P), L.PauliSums(c.observables)
        pin = torch.tensor(p, dtype=torch.float64).pin_memory()
        p_host = pin.numpy()
        for _ in range(1):
            L.sv_reset(h, 0)
            L.sv_forward(h, tape, p_host)
            L.sv_adjoint_jacobian(h, tape, p_host, obs)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            L.sv_reset(h, 0)
            L.sv_forward(h, tape, p_host)
            E_h, J_h = L.sv_adjoint_jacobian(h, tape, p_host, obs)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        barrier()
        L.sv_destroy(h)
        err = float(np.abs(J_h - main["J"].cpu().numpy()).max())
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 2 * P * 8,
               "d2h_bytes_per_step": (m + m * P) * 8, "api": "sv_reset + sv_forward + sv_adjoint_jacobian",
               "max_abs_diff_vs_device_path": err}

    extras = {}
    if not args.no_extras and rank == 0:
        for other in [d for d in ("c128", "c128df", "c64") if d != args.dtype]:
            o = measure(other, max(2, args.steps // 2), 2, timing=False)
            dJ = float(np.abs(o["J"].cpu().numpy() - main["J"].cpu().numpy()).max())
            extras[other] = {"ms_per_step": o["ms"], "max_abs_jacobian_diff_vs_" + args.dtype: dJ}
            del o
            torch.cuda.empty_cache()
        if NQ == N_QUBITS and not args.quick_extras:
            extras["gate_pass_n30"] = extra_gates(hbm_peak)
            extras["qaoa_batched"] = extra_qaoa()
            extras["vqe24_2000_terms"] = extra_vqe()
            extras["rycz30"] = extra_rycz30(hbm_peak)
            extras["dense_fusion_layer30_c64"] = extra_dense_fusion_layer30(hbm_peak)
            try:
                extras["layered12"] = extra_layered12()
            except Exception as exc:  # an extra never takes the bench line down
                extras["layered12"] = {"error": repr(exc)}
            extras["measurements_sel24"] = extra_measurements(hbm_peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        runs = [oracle_sample(rows=1) for _ in range(2)]
        est = statistics.mean(r[0] for r in runs)
        Jo = runs[0][4]
        cpu = {"value": est, "unit": "ms", "cores": runs[0][3], "kind": "oracle", "sample": runs[0][2],
               "samples": len(runs), "spread_ms": [min(r[0] for r in runs), max(r[0] for r in runs)],
               "sample_wall_s": sum(r[1] for r in runs) / 1e3}
        if (NQ, args.layers) == (N_QUBITS, LAYERS):
            cpu["max_abs_diff_row0_vs_gpu"] = float(np.abs(main["J"].cpu().numpy()[0] - Jo[0]).max())
        for key, fn in (("layered12", oracle_layered12), ("qaoa20", oracle_qaoa20)):
            try:  # a side figure never takes the bench line down
                cpu[key] = fn()
            except Exception as exc:
                cpu[key] = {"error": repr(exc)}

    if rank == 0:
        line = bench_line(ms, world, args.steps, args.warmup, args.dtype,
                          bench_config(NQ, args.layers, args.dtype, world, P, m),
                          {"forward_passes": main["fwd_passes"], "adjoint_passes": main["adj_passes"]},
                          roofline, cpu, e2e, main["launches"], main["clocks"], extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _dense_block_ms(n, k, tensor_cores, reps, warmup):
    import torch
    from paper_2403_02512_gb300 import _lib as L
    from paper_2403_02512_gb300.torch_api import StateVector
    rng = np.random.default_rng(k)
    U, _ = np.linalg.qr(rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k)))
    wires = list(range(n - k, n))  # the lowest index bits: each group is contiguous
    L.sv_set_dense_tensor_cores(tensor_cores)
    try:
        sv = StateVector(n, "c64", renormalize=False)
        for _ in range(warmup):
            sv.apply_matrix(wires, U)
        ms = _timed(lambda: sv.apply_matrix(wires, U), reps, torch.cuda.current_stream())
        sv.close()
    finally:
        L.sv_set_dense_tensor_cores(True)
    return ms


def run_profile_dense(args):
    k, _, mode = args.profile_dense.partition(":")
    ms = _dense_block_ms(args.qubits, int(k), mode != "cuda", args.steps, args.warmup)
    V = 8 << args.qubits
    print(json.dumps({"profile_dense": args.profile_dense, "n": args.qubits, "ms": ms,
                      "gbs_algorithmic": 2.0 * V / ms / 1e6}))


def run_profile_vqe(args):
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import vqe_givens
    c, p = vqe_givens(24, 12, 40, 120, 2000)
    sv = StateVector(24, args.dtype, basis_state=c.basis_state)
    prog = Program.from_circuit(sv, c)

    def step():
        prog.forward(p)
        return prog.jacobian()

    for _ in range(args.warmup):
        step()
    ms = _timed(step, args.steps, torch.cuda.current_stream())
    print(json.dumps({"profile_vqe": args.dtype, "ms_energy_and_gradient": ms}))


def run_profile_expval(args):
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import strongly_entangling
    c, p = strongly_entangling(args.qubits, args.layers)
    sv = StateVector(args.qubits, args.dtype)
    prog = Program.from_circuit(sv, c)
    prog.forward(p)
    for _ in range(args.warmup):
        sv.expval(c.observables)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sv.expval(c.observables)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / args.steps * 1e3
    V = (8 if args.dtype == "c64" else 16) << args.qubits
    print(json.dumps({"profile_expval": args.dtype, "n": args.qubits, "words": len(c.observables), "ms": ms,
                      "gbs_algorithmic": V / ms / 1e6}))


def run_profile_rycz30(args):
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import ry_cz_brick
    c, p = ry_cz_brick(30, 20)
    sv = StateVector(30, args.dtype)
    prog = Program.from_circuit(sv, c)

    def step():
        prog.forward(p)
        return prog.jacobian()

    for _ in range(args.warmup):
        step()
    ms = _timed(step, args.steps, torch.cuda.current_stream())
    print(json.dumps({"profile_rycz30": args.dtype, "ms_forward_and_jacobian": ms,
                      "adjoint_passes": prog.stats()[1]}))


def run_profile_gate(args):
    import torch
    from paper_2403_02512_gb300.torch_api import Program, StateVector
    from workloads import Op
    name, wire = args.profile_gate.split(":")
    t, n = int(wire), args.qubits
    sv = StateVector(n, args.dtype, renormalize=False)  # time the gate pass alone
    if name == "CNOT":
        op = Op("PauliX", (t,), (), ((t + 1) % n,))
    else:
        op = Op(name, (t,), (0,) if name == "RX" else ())
    prog = Program(sv, [op], 1 if name == "RX" else 0)
    prog.set_params([0.3] if name == "RX" else [])
    for _ in range(args.warmup):
        prog.forward(reset=False)
    ms = _timed(lambda: prog.forward(reset=False), args.steps, torch.cuda.current_stream())
    V = (8 if args.dtype == "c64" else 16) << n
    alg = V if name == "CNOT" else 2.0 * V
    print(json.dumps({"profile_gate": args.profile_gate, "dtype": args.dtype, "n": n, "ms": ms,
                      "gbs_algorithmic": alg / ms / 1e6}))


def run_profile_batch(args):
    import torch
    from paper_2403_02512_gb300 import _lib as L
    from workloads import qaoa_maxcut, qaoa_param_sets
    c = qaoa_maxcut(20, 4)
    sets = qaoa_param_sets(args.profile_batch, 4)
    b = L.Batch([c] * len(sets), L.SV_C64)
    b.set_params(sets.ravel())
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.run()
    dt = (time.perf_counter() - t0) / args.steps
    print(json.dumps({"profile_batch": len(sets), "ms_per_batch": dt * 1e3, "circuits_per_s": len(sets) / dt,
                      **b.info()}))
    b.close()


def main():
    args = parse()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.profile_vqe:
        run_profile_vqe(args)
    elif args.profile_dense:
        run_profile_dense(args)
    elif args.profile_gate:
        run_profile_gate(args)
    elif args.profile_expval:
        run_profile_expval(args)
    elif args.profile_rycz30:
        run_profile_rycz30(args)
    elif args.profile_batch:
        run_profile_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
