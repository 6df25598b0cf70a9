#!/usr/bin/env python
"""Benchmark: simulate the 30-qubit, 20-cycle Sycamore-pattern circuit (5x6 grid, ABCDCDAB,
fSim(pi/2, pi/6), random sqrt(X/Y/W)) on one GB300 and report amplitude updates per second.

One step = one pass of the whole hot path over one circuit, in the paper's order: the first
phase by contraction deferral (Sect. 2 and Sect. 4's subcircuits 1 and 2: the gates up to the
sixth one that crosses the lattice's middle column cut run as two 15-qubit tensors with
entanglement indices, EI / E2Q of the Appendix, then one tensor-core contraction writes the
2^30-amplitude state), then aggregation planning and FP64 composition (host) of the remaining
gates and every fused block applied on the device, and the norm / Porter-Thomas / XEB
reduction.  Each step's plan is built on the host while the previous step's last blocks run on
the device; the split and its two tensors' plans are built once, and so is the qubit layout the
state is written in (sim_plan_layout; relabelled before each run, which costs nothing since the
contraction overwrites every amplitude).  The state (8 GiB complex64) is
larger than L2, so no flush is needed between steps.  The JSON line also reports the same
circuit without the split ("plain_path": fused blocks from |0...0>).

metric value = 2^n * (original gates) * steps / device time   ("gate" amplitude updates/s)
pass updates = 2^n * (fused blocks) * steps / device time      (roofline basis, 16 B/amp/pass)

Default configuration: chosen by the library's autotuner before the timed region among the
block widths and the FP32-equivalent arithmetic (FP32 CUDA cores; 3xFP16 on tcgen05 or
mma.sync, or 3xTF32, for blocks of 4-6 qubits; FP32 accumulate; error vs the oracle ~1e-6 on
this workload).  The same JSON line also reports the FP32-only path (blocks of up to 4 qubits)
and a bounded serving run (200 random circuits, n in 16..30, served concurrently vs one at a
time).

--impl reference times the CPU oracle (complex128, gate by gate) on the host cores on a bounded
sample of the same workload (the first gates of the circuit on the full 30-qubit state).
Multi-GPU (torchrun): independent replicas, one circuit per rank (seed = rank), no collective
on the data path; time = max over ranks, value = all ranks' updates / that time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "syc30_5x6_d20"
NOMINAL_DENSE_F16_TFLOPS = 2250.0  # GB300 dense FP16/BF16 tensor rate, datasheet (no sparsity)
# Poisson arrival rates of the 2000-circuit serving legs: about 70% of each server's saturated
# rate on GB300 (all circuits at t = 0), so that the server keeps up and its latency is a queueing
# figure, not a backlog
SERVING_RATE_SPLIT = 87.5
SERVING_RATE_FP32 = 35.0
METRIC = "amplitude-updates/s"
UNIT = "amp-updates/s"


# Configurations beyond one resident 30-qubit state (Sect. 4: sliced qubits, phases, a secondary
# store): store kind, sliced bits, block width, store regions kept in HBM, and how the two
# sliced sets are picked (the lattice ends, or sim_phases_choose_sets).
LARGE_CASES = {
    "syc33_6x6m3_d20": dict(store="device", slice_bits=3, kmax=6, device_regions=0, sets="ends", front_pairs=3),
    "syc34_5x7m1_d16": dict(store="host", slice_bits=3, kmax=6, device_regions=0, sets="chosen", front_pairs=4),
    "syc35_5x7_d16": dict(store="host", slice_bits=4, kmax=6, device_regions=8, sets="chosen", front_pairs=4),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--kmax", type=int, default=0,
                    help="block width; 0 = autotune (sim_autotune, FP32-equivalent arithmetic only), "
                         "measured before the timed region")
    ap.add_argument("--precision", default="fp16x3",
                    choices=["fp32", "fp16x3", "fp16x3_tmem", "bf16x3", "tf32x3", "tf32"],
                    help="arithmetic of blocks with k >= 5 when --kmax is given (narrower blocks always "
                         "run FP32 on CUDA cores)")
    ap.add_argument("--front-pairs", type=int, default=5,
                    help="contraction deferral (Sect. 2): the longest prefix of the circuit that "
                         "crosses the bipartition sim_split_choose picks at most this many times "
                         "runs as two tensors and their contraction; 0 = plain fused blocks only")
    ap.add_argument("--no-layout", action="store_true",
                    help="keep the identity qubit layout instead of the one sim_plan_layout chooses")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the raw nvidia-smi samples of the timed region in this file "
                         "(default: a temporary file)")
    ap.add_argument("--cpu-sample-gates", type=int, default=42)
    ap.add_argument("--no-fp32-path", action="store_true")
    ap.add_argument("--no-bf16-path", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--no-per-gate", action="store_true",
                    help="skip the plain per-gate baseline (every gate its own pass over the state)")
    ap.add_argument("--serving-circuits", type=int, default=2000)
    ap.add_argument("--serving-rate", type=float, default=SERVING_RATE_SPLIT,
                    help="Poisson arrival rate of the split-precision serving leg in circuits/s (0: every "
                         "circuit at t = 0, saturated)")
    ap.add_argument("--serving-rate-fp32", type=float, default=SERVING_RATE_FP32,
                    help="Poisson arrival rate of the FP32 serving leg in circuits/s (0: saturated)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving leg in the --precision given (fp32, else the split mode) "
                         "and print one JSON line")
    ap.add_argument("--serving-max-large", type=int, default=0,
                    help="srv_opts.max_large of the serving-only run (0: the library's default)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 33-qubit sliced runs (64 GiB state) and the 35-qubit streamed run "
                         "(256 GiB store) of the default line")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the CPU oracle on one and on all host cores for the 12-, 30- (sample), "
                         "28- (sample) and 24-qubit circuits, print one JSON line, and exit")
    ap.add_argument("--large-case", default=None, choices=sorted(LARGE_CASES),
                    help="run one configuration beyond the bench's 30 qubits instead (33 qubits resident "
                         "in 8 slices with sliced phases; 34 and 35 qubits streamed through a host store, "
                         "35 with half its regions in HBM), print one JSON line, and exit")
    ap.add_argument("--large-kmax", type=int, default=0,
                    help="with --large-case: block width (0: the case's own)")
    ap.add_argument("--large-front-pairs", type=int, default=-1,
                    help="with --large-case: bridging gates of the contraction-deferral front (-1: the "
                         "case's own, 0: none, the whole circuit in phases)")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the small profiling case (2^28 amplitudes, 2 GiB > L2): fused "
                         "apply k=4 (targets >= bit 5, then mixed), k=2, k=5 on tensor cores (3xFP16 with "
                         "mma.sync, high then mixed targets; with tcgen05, 256- and 128-group tiles and one "
                         "target below bit 4), k=4 on bits 0-3 in the default mode, a high-bit and a "
                         "low<->top permutation and a reduction, each twice, then exit; meant to run under ncu")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str | None = None):
        self.device = device
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"sycsim_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9 and p[1].replace(".", "").isdigit():
                rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time."""
    return units_per_rank * world_size / seconds_max


TCGEN05_TRAFFIC_GB = 4 * (2.147897 + 2.088273)  # k_apply_tcgen05<5, 2, 0>, ncu at 2^28 amplitudes
TCGEN05_K6_TRAFFIC_GB = 4 * (2.148062 + 2.087781)  # k_apply_tc6a<1, 0>, ncu at 2^28 amplitudes


def measured_peaks(key: str = "hbm_gbs"):
    """A measured peak from MEASURED_PEAKS.json (HBM copy GB/s, or bf16 TFLOP/s), else the
    profiling recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if d.get(key):
            return d[key], "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}[key], "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu), or "unknown"."""
    try:
        return next((ln.split(":", 1)[1].strip() for ln in subprocess.run(
            ["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines()
            if ln.startswith("Model name")), "unknown")
    except Exception:
        return "unknown"


def cpu_baseline(circ, sample_gates: int, steps: int = 1, single_thread_gates: int = 4):
    """Time the oracle (complex128, gate by gate) on the first `sample_gates` gates of the circuit
    applied to the full state on all host cores, and on the first `single_thread_gates` gates on
    one thread."""
    import oracle
    import syc_inputs as si

    oracle.build()
    cores = os.cpu_count() or 1
    amps = float(1 << circ.n_qubits)
    psi = oracle.basis_state(circ.n_qubits, 0)
    oracle.set_threads(1)
    one = si.Circuit(circ.n_qubits, circ.gates[:single_thread_gates], name=circ.name)
    t0 = time.perf_counter()
    oracle.apply_gates(psi, one)
    t_one = time.perf_counter() - t0
    oracle.set_threads(cores)
    sample = si.Circuit(circ.n_qubits, circ.gates[:sample_gates], name=circ.name)
    psi = oracle.basis_state(circ.n_qubits, 0)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.apply_gates(psi, sample)
        times.append(time.perf_counter() - t0)
    del psi
    return {"value": amps * sample_gates * steps / sum(times), "unit": UNIT,
            "cores": oracle.max_threads(), "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"first {sample_gates} of {circ.n_gates} gates of {circ.name} on the full "
                      f"2^{circ.n_qubits} complex128 state, {steps} run(s)",
            "seconds": sum(times),
            "single_thread": {"value": amps * single_thread_gates / t_one, "unit": UNIT, "cores": 1,
                              "sample": f"first {single_thread_gates} gates, same state",
                              "seconds": t_one}}


def oracle_table():
    """The oracle (complex128, gate by gate) on one host thread and on all of them, for the
    12-qubit circuit, samples of the 30-qubit circuit and of the 28-qubit sub-lattice circuit,
    and a 24-qubit serving-size circuit: wall time and amplitude updates/s."""
    import oracle
    import syc_inputs as si

    oracle.build()
    cores = os.cpu_count() or 1
    cpu = cpu_model()
    cases = [("12 qubits, 3x4 grid, 8 cycles (whole circuit)", si.workload_circuit("syc12_3x4_d8", 0), None),
             ("30 qubits, 5x6 grid, 20 cycles (first 12 gates)", si.workload_circuit("syc30_5x6_d20", 0), 12),
             ("28 qubits, 4x7 grid, 20 cycles (first 24 gates)", si.workload_circuit("syc28_4x7_d20", 0), 24),
             ("24 qubits, 4x6 grid, 14 cycles (whole circuit)", si.sycamore_circuit(si.Grid(4, 6), 14, seed=5), None)]
    rows = []
    for threads in sorted({1, cores}):
        oracle.set_threads(threads)
        for name, circ, g in cases:
            sample = circ if g is None else si.Circuit(circ.n_qubits, circ.gates[:g], name=circ.name)
            psi = oracle.basis_state(circ.n_qubits, 0)
            t0 = time.perf_counter()
            oracle.apply_gates(psi, sample)
            dt = time.perf_counter() - t0
            del psi
            rows.append({"case": name, "threads": threads, "gates": sample.n_gates, "seconds": dt,
                         "amp_updates_per_s": float(1 << circ.n_qubits) * sample.n_gates / dt})
    return {"cpu": cpu, "cores": cores, "rows": rows}


def serving_run(count: int, device: int, rate_hz: float = 0.0, precision: str = "fp16x3_tmem", max_large: int = 0):
    """Serve `count` random circuits (qubits uniform in 16..30, 8..20 cycles), all submitted at
    once (rate_hz = 0) or each at its Poisson arrival time, and run the same circuits, arriving
    the same way, one at a time through sim_*; report circuits/s and the latency distributions
    (completion - arrival).  precision: the server's arithmetic above its packing size
    ("fp16x3_tmem": 3xFP16 on tcgen05, blocks of <= 6 qubits; "fp32": CUDA cores, blocks of <= 5
    qubits up to 24 qubits and <= 4 above); the one-at-a-time path uses the same arithmetic,
    block widths and layouts."""
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si

    stream = si.serving_stream(count, base_seed=1000, rate_hz=rate_hz if rate_hz > 0 else 1e9)
    arrivals = [a if rate_hz > 0 else 0.0 for a, _ in stream]
    circs = [c for _, c in stream]
    gates = [pkg.gates_array(c) for c in circs]
    fp32 = precision == "fp32"
    prec = pkg.SIM_FP32 if fp32 else pkg.SIM_FP16X3_TMEM

    def kmax_of(n):  # the server's width policy above its packing size
        return (5 if n <= 24 else 4) if fp32 else 6

    def until(t0, at):  # sleep until `at` seconds after t0
        dt = at - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)

    import torch
    torch.cuda.synchronize()
    handles = {}
    for n in sorted({c.n_qubits for c in circs}):  # states allocated before the clock starts
        handles[n] = pkg.sim_create(n, 0, device=device)
    seq_done = []  # completion - arrival
    t0 = time.perf_counter()
    for at, c, g in zip(arrivals, circs, gates):
        until(t0, at)
        h = handles[c.n_qubits]
        big = c.n_qubits > 20
        # planned as the server plans a request: the greedy schedule (search=1)
        p = (pkg.sim_plan_create(c.n_qubits, g, kmax=kmax_of(c.n_qubits), precision=prec, search=1) if big else
             pkg.sim_plan_create(c.n_qubits, g, kmax=5, precision=pkg.SIM_FP32 if fp32 else prec, search=1))
        if big:
            pkg.sim_set_layout(h, pkg.sim_plan_layout(p, c.n_qubits)[0])
        pkg.sim_reset(h)
        pkg.sim_apply_plan(h, p)
        pkg.sim_reduce(h)
        pkg.sim_plan_destroy(p)
        seq_done.append((time.perf_counter() - t0 - at) * 1e3)
    seq_s = time.perf_counter() - t0
    for h in handles.values():
        pkg.sim_destroy(h)
    srv = pkg.srv_create(device=device, precision=prec, max_large=max_large)
    # the server's autotuner (srv_autotune), before the clock starts: one sample circuit per size
    # above the packing size and depth class, seeds outside the stream's
    tsamples = [si.sycamore_circuit(si.near_square_grid(n), d, seed=70000 + 31 * n + d)
                for n in range(21, 31) for d in (10, 14, 18)]
    t_tune = time.perf_counter()
    picks = pkg.srv_autotune(srv, [(c.n_qubits, pkg.gates_array(c)) for c in tsamples])
    t_tune = time.perf_counter() - t_tune
    tuned = {f"{c.n_qubits}q_{c.n_gates}g": {"kmax": k, "front": f, "ms": round(ms, 3)}
             for c, (k, f, ms) in zip(tsamples, picks)}
    t0 = time.perf_counter()
    tickets, lag_ms = [], []  # lag: arrival -> srv_submit's call (the submitting thread running late)
    for at, c, g in zip(arrivals, circs, gates):
        until(t0, at)
        lag_ms.append(max(0.0, (time.perf_counter() - t0 - at) * 1e3))
        tickets.append(pkg.srv_submit(srv, c.n_qubits, g))
    # completion - arrival: the lag plus the server's latency from the call (planning included)
    srv_done = [lag + pkg.srv_wait(srv, t)[2] for lag, t in zip(lag_ms, tickets)]
    served_s = time.perf_counter() - t0
    st = pkg.srv_stats(srv)
    pkg.srv_destroy(srv)
    arr = ("all at t=0 (saturated)" if rate_hz <= 0 else
           f"Poisson at {rate_hz:g} circuits/s (last arrival at {arrivals[-1]:.2f} s)")
    if fp32:
        arith = ("fp32 on CUDA cores (k_max 5 up to 24 qubits, 4 above, in a chosen layout above 20 "
                 "qubits; circuits of <= 20 qubits packed one per CTA, k_max 5)")
        front = ("circuits of >= 26 qubits (from 22 where the autotuner measured it faster) whose first "
                 "2 crossings of the chosen bipartition leave >= 10% of the gates in front run them as "
                 "two tensors and one FP32 contraction on CUDA cores; the one-at-a-time path runs every "
                 "circuit plainly")
    else:
        arith = ("fp16x3_tmem (k_max 6 in a chosen layout above 20 qubits; circuits of <= 20 "
                 "qubits packed one per CTA in FP32, k_max 5)")
        front = ("circuits of >= 26 qubits whose first 5 crossings of the chosen bipartition leave >= 30% "
                 "of the gates in front run them as two tensors and one tcgen05 contraction; the "
                 "one-at-a-time path runs every circuit plainly")
    return {"circuits": count, "qubits": "16..30", "cycles": "8..20", "arrivals": arr,
            "circuits_per_s": count / served_s,
            "p50_ms": statistics.quantiles(srv_done, n=100)[49],
            "p99_ms": statistics.quantiles(srv_done, n=100)[98],
            "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
            "one_at_a_time_circuits_per_s": count / seq_s,
            "one_at_a_time_p50_ms": statistics.quantiles(seq_done, n=100)[49],
            "one_at_a_time_p99_ms": statistics.quantiles(seq_done, n=100)[98],
            "arithmetic": arith, "server_front": front,
            "autotune": {"by": "srv_autotune: k_max 4-6 (and the front or not) measured per size "
                               "and depth class on one sample each, before the timed leg",
                         "seconds": t_tune, "choices": tuned}}


def graph_replay_run(device: int, runs: int = 30):
    """The same circuit run `runs` times from |0...0> (20 and 24 qubits, 20 cycles, k_max 5,
    SIM_FP16X3_TMEM): each run through sim_apply_plan vs a replay of its CUDA graph; wall time
    per run, measured after a warm-up run of each."""
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si

    out = []
    for grid in (si.Grid(4, 5), si.Grid(4, 6)):
        circ = si.sycamore_circuit(grid, cycles=20, seed=7)
        n = circ.n_qubits
        plan = pkg.sim_plan_create(n, pkg.gates_array(circ), kmax=5, precision=pkg.SIM_FP16X3_TMEM)
        h = pkg.sim_create(n, 0, device=device)
        g = pkg.sim_graph_create(h, plan)
        res = {"circuit": f"{grid.rows}x{grid.cols} grid ({n} qubits), 20 cycles, k_max 5, fp16x3_tmem",
               "blocks": pkg.sim_plan_info(plan)[0], "runs": runs}
        for name, run in (("direct_ms_per_run", lambda: pkg.sim_apply_plan(h, plan)),
                          ("graph_ms_per_run", lambda: pkg.sim_graph_launch(h, g))):
            pkg.sim_reset(h)
            run()
            pkg.sim_sync(h)
            t0 = time.perf_counter()
            for _ in range(runs):
                pkg.sim_reset(h)
                run()
            pkg.sim_sync(h)
            res[name] = (time.perf_counter() - t0) * 1e3 / runs
        pkg.sim_graph_destroy(g)
        pkg.sim_destroy(h)
        pkg.sim_plan_destroy(plan)
        out.append(res)
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import syc_inputs as si
    circ = si.workload_circuit(args.workload, seed=0)
    g = max(1, min(args.cpu_sample_gates, 8))
    total_steps = args.warmup + args.steps
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    psi = oracle.basis_state(circ.n_qubits, 0)
    sample = si.Circuit(circ.n_qubits, circ.gates[:g], name=circ.name)
    times = []
    for i in range(total_steps):
        t0 = time.perf_counter()
        oracle.apply_gates(psi, sample)
        times.append(time.perf_counter() - t0)
    t = sum(times[args.warmup:])
    amps = float(1 << circ.n_qubits)
    value = amps * g * args.steps / t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random circuit)",
            "config": {"workload": args.workload, "n_qubits": circ.n_qubits,
                       "sample": f"each step applies the first {g} gates of the circuit"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"first {g} of {circ.n_gates} gates per step, full state"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si
    from paper_1910_09534_gb300 import build as pkg_build

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    pkg_build.build()

    circ = si.workload_circuit(args.workload, seed=rank)
    n = circ.n_qubits
    amps = 1 << n
    gates = pkg.gates_array(circ)
    h = pkg.sim_create(n, 0, device=local)
    stream_ptr = pkg.sim_stream(h)
    stream = torch.cuda.ExternalStream(stream_ptr)

    prec = {"fp32": pkg.SIM_FP32, "fp16x3": pkg.SIM_FP16X3, "fp16x3_tmem": pkg.SIM_FP16X3_TMEM,
            "bf16x3": pkg.SIM_BF16X3, "tf32x3": pkg.SIM_TF32X3, "tf32": pkg.SIM_TF32}[args.precision]
    tuned = None
    if args.kmax == 0:
        kmax, prec, tune_ms = pkg.sim_autotune(h, gates, pkg.SIM_TUNE_FP32_EQUIVALENT)
        args.kmax = kmax
        args.precision = {pkg.SIM_FP32: "fp32", pkg.SIM_FP16X3: "fp16x3", pkg.SIM_FP16X3_TMEM: "fp16x3_tmem",
                          pkg.SIM_BF16X3: "bf16x3", pkg.SIM_TF32X3: "tf32x3", pkg.SIM_TF32: "tf32"}[prec]
        tuned = {"by": "sim_autotune (FP32-equivalent arithmetic)", "kmax": kmax,
                 "precision": args.precision, "tuning_run_ms": tune_ms}

    # contraction deferral (Sect. 2, the paper's first phase): the circuit's first gates, up to
    # the (front_pairs + 1)-th gate across the middle column cut, as two half-lattice tensors
    # with entanglement indices, contracted into the state; the rest as fused blocks on it
    front = None
    n_front, front_info = 0, None
    if args.front_pairs > 0:
        side, n_front = pkg.sim_split_choose(n, gates, args.front_pairs)
        split = pkg.sim_split_create(n, gates[:n_front], side)
        n_side, n_wires, pairs, n_tg = pkg.sim_split_info(split)
        front = {}

        def front_for(hh):
            if hh.value not in front:
                front[hh.value] = pkg.sim_front_create(hh, split, kmax=args.kmax, precision=prec)
            return front[hh.value]
        tplans = [pkg.sim_plan_create(n_wires[t], pkg.sim_split_gates(split, t), kmax=args.kmax,
                                      precision=prec) for t in range(2)]
        front_info = {"gates": n_front, "bridging_gates": pairs, "entanglement_values": 4 ** pairs,
                      "sides": "sim_split_choose (the 5x6 lattice's middle column)", "qubits_per_side": n_side,
                      "tensor_qubits": n_wires,
                      "tensor_blocks": [pkg.sim_plan_info(p)[0] for p in tplans],
                      "contraction": "tcgen05 3xFP16" if prec in (pkg.SIM_FP16X3, pkg.SIM_FP16X3_TMEM)
                      else "FP32 CUDA cores"}
        for p in tplans:
            pkg.sim_plan_destroy(p)
    rest = gates[n_front:]

    # where the qubits sit (sim_plan_layout: fewer blocks on slow kernel paths); relabelling is free
    # before the front or the reset overwrites the state
    def choose_layout(gl, kmax, precision, split_=None):
        if args.no_layout:
            return None, None
        pl = pkg.sim_plan_create(n, gl, kmax=kmax, precision=precision)
        perm, est, est_id = (pkg.sim_plan_layout_front(pl, split_, n) if split_ is not None
                             else pkg.sim_plan_layout(pl, n))
        pkg.sim_plan_destroy(pl)
        return perm, {"chosen_by": "sim_plan_layout", "estimate_ms": est, "identity_estimate_ms": est_id}
    # with the front, the layout also keeps the contraction's stores whole (sim_plan_layout_front)
    layout, layout_info = choose_layout(rest, args.kmax, prec, split if front is not None else None)

    def start(hh, lay=None):
        lay = layout if lay is None else lay
        if lay is not None:
            pkg.sim_set_layout(hh, lay)
        if front is None:
            pkg.sim_reset(hh)
        else:
            pkg.sim_front_run(hh, front_for(hh))

    results = [pkg.pinned_array(3, dtype=np.float64) for _ in range(2)]
    result_ev = [torch.cuda.Event(), torch.cuda.Event()]

    def run_steps(k):
        # k circuit runs; each plan (host: grouping + FP64 composition) is built while the
        # previous run's blocks are still executing (sim_apply_plan returns once the last blocks
        # are queued).  Each run's reduction is queued (sim_reduce_async) and the next run queued
        # behind it before that result is read, so the device does not wait for the host between
        # runs; every run's result is still read back.
        plan = pkg.sim_plan_create(n, rest, kmax=args.kmax, precision=prec)
        out, prev = None, None
        for s in range(k):
            start(h)
            pkg.sim_apply_plan(h, plan)
            pkg.sim_reduce_async(h, results[s % 2])
            result_ev[s % 2].record(stream)
            nxt = pkg.sim_plan_create(n, rest, kmax=args.kmax, precision=prec) if s + 1 < k else None
            if prev is not None:
                result_ev[prev].synchronize()
                out = tuple(float(x) for x in results[prev][:3])
            prev = s % 2
            nb = pkg.sim_plan_info(plan)[0]
            pkg.sim_plan_destroy(plan)
            plan = nxt
        result_ev[prev].synchronize()
        out = tuple(float(x) for x in results[prev][:3])
        return out, nb

    (norm, s2, xeb), nblocks = run_steps(args.warmup)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    pkg.sim_profile_enable(h, True)
    launches0 = pkg.sim_launch_count(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_csv) as clk:
        barrier()
        e0.record(stream)
        (norm, s2, xeb), nblocks = run_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    launches = pkg.sim_launch_count(h) - launches0
    a_n, a_ms, a_bytes = pkg.sim_profile_read(h, pkg.SIM_PROF_APPLY)
    r_n, r_ms, r_bytes = pkg.sim_profile_read(h, pkg.SIM_PROF_REDUCE)
    c_n, c_ms, c_flops = pkg.sim_profile_read(h, pkg.SIM_PROF_CONTRACT)
    pkg.sim_profile_enable(h, False)

    ms_max = max_over_ranks(ms, dist)
    value = whole_job_rate(float(amps) * circ.n_gates * args.steps, ws, ms_max / 1e3)
    pass_updates = whole_job_rate(float(amps) * nblocks * args.steps, ws, ms_max / 1e3)

    # end to end through the public API with host buffers: gate records from pinned host
    # memory in, all 2^n amplitudes out to pinned host memory, every step; the last readout is
    # inside the timed region too.  The schedule (readouts overlapping the next circuit's compute
    # on two handles, or one after the other) is the faster of the two on a short untimed probe.
    gates_pinned = pkg.pinned_array(gates.size, dtype=pkg._native.GATE_DTYPE)
    gates_pinned[:] = gates
    h2 = pkg.sim_create(n, 0, device=local)
    outs = [pkg.pinned_array(amps, dtype=np.complex64), pkg.pinned_array(amps, dtype=np.complex64)]
    hs = [h, h2]
    rest_pinned = gates_pinned[n_front:]
    for hw, ow in zip(hs, outs):  # one untimed end-to-end step on each handle (warm-up)
        pw = pkg.sim_plan_create(n, rest_pinned, kmax=args.kmax, precision=prec)
        start(hw)
        pkg.sim_apply_plan(hw, pw)
        if layout is not None:
            pkg.sim_permute(hw, list(range(n)))
        pkg.sim_amplitudes_async(hw, ow)
        pkg.sim_sync(hw)
        pkg.sim_plan_destroy(pw)
    # each readout bracketed by CUDA events on its handle's stream: the host link's speed while the
    # loop ran (other tenants share the node's host memory and link)
    streams = [torch.cuda.ExternalStream(pkg.sim_stream(hh)) for hh in hs]
    rd_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.e2e_steps)]
    computed = [torch.cuda.Event(), torch.cuda.Event()]

    def e2e_loop(k, overlap, rd=None):
        # overlap: two handles, the circuits computing one after another (each handle's stream
        # waits for the other's last compute kernel, not for its readout), so one handle's readout
        # overlaps the other's compute and a step costs max(compute, readout).  Serial: one handle,
        # each readout finished before the next circuit starts -- faster on hosts whose link, while
        # the device streams HBM at its peak, moves data several times slower than alone
        plan = pkg.sim_plan_create(n, rest_pinned, kmax=args.kmax, precision=prec)
        for s_ in range(k):
            i = s_ % 2 if overlap else 0
            hc = hs[i]
            if overlap and s_ > 0:
                streams[i].wait_event(computed[(s_ - 1) % 2])
            start(hc)
            pkg.sim_apply_plan(hc, plan)
            if layout is not None:
                pkg.sim_permute(hc, list(range(n)))  # logical order for the asynchronous readout
            computed[i].record(streams[i])
            nxt = pkg.sim_plan_create(n, rest_pinned, kmax=args.kmax, precision=prec) if s_ + 1 < k else None
            if rd is not None:
                rd[s_][0].record(streams[i])
            pkg.sim_amplitudes_async(hc, outs[i])
            if rd is not None:
                rd[s_][1].record(streams[i])
            if not overlap:
                pkg.sim_sync(hc)
            elif s_ > 0:
                pkg.sim_sync(hs[(s_ - 1) % 2])  # the previous circuit's amplitudes are in host memory
            pkg.sim_plan_destroy(plan)
            plan = nxt
        pkg.sim_sync(hs[(k - 1) % 2] if overlap else hs[0])

    # the schedule: both measured on 3 untimed steps, the faster one timed
    probe = {}
    for mode in (True, False):
        tp = time.perf_counter()
        e2e_loop(3, mode)
        probe["overlapped" if mode else "serial"] = time.perf_counter() - tp
    overlap = probe["overlapped"] <= probe["serial"]
    barrier()
    t0 = time.perf_counter()
    e2e_loop(args.e2e_steps, overlap, rd_ev)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    torch.cuda.synchronize()
    rd_in_loop = sorted(a.elapsed_time(b) for a, b in rd_ev)
    e2e_value = whole_job_rate(float(amps) * circ.n_gates * args.e2e_steps, ws, max(e2e_s, 1e-9))
    # the host link right after: one 8 GiB readout alone (other tenants of the node share the
    # host memory and its link; this says how fast it was during the end-to-end leg)
    pkg.sim_permute(h, list(range(n)))
    t1 = time.perf_counter()
    pkg.sim_amplitudes_async(h, outs[0])
    pkg.sim_sync(h)
    readout_ms = 1e3 * (time.perf_counter() - t1)
    sanity = outs[(args.e2e_steps - 1) % 2 if overlap else 0][:4].copy()
    for o in outs + results:
        pkg.sim_host_free(o.ctypes.data)
    pkg.sim_host_free(gates_pinned.ctypes.data)
    if front is not None:
        for hv in list(front):
            if hv == h2.value:
                pkg.sim_front_destroy(front.pop(hv))
    pkg.sim_destroy(h2)
    # the same circuit without the split (plain fused blocks from |0...0>), same timing method
    plain_path = None
    if front is not None:
        layout_plain, _ = choose_layout(gates, args.kmax, prec)

        def step_plain():
            plan = pkg.sim_plan_create(n, gates, kmax=args.kmax, precision=prec)
            if layout_plain is not None:
                pkg.sim_set_layout(h, layout_plain)
            pkg.sim_reset(h)
            pkg.sim_apply_plan(h, plan)
            out = pkg.sim_reduce(h)
            nb = pkg.sim_plan_info(plan)[0]
            pkg.sim_plan_destroy(plan)
            return out, nb
        for _ in range(args.warmup):
            step_plain()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            _, nbp = step_plain()
        e1.record(stream)
        torch.cuda.synchronize()
        msp = e0.elapsed_time(e1)
        plain_path = {"value": float(amps) * circ.n_gates * args.steps / (msp / 1e3), "unit": UNIT,
                      "ms_per_step": msp / args.steps, "fused_blocks": nbp}
    # the FP32-only path on the same state and timing method (blocks of <= 4 qubits), its front of
    # 2 bridging gates contracted in FP32 on CUDA cores (each bridging gate quadruples that cost)
    fp32_path = None
    if not args.no_fp32_path:
        side32, nf32 = pkg.sim_split_choose(n, gates, 2)
        split32 = pkg.sim_split_create(n, gates[:nf32], side32)
        rest32 = gates[nf32:]
        layout32, _ = choose_layout(rest32, 4, pkg.SIM_FP32, split32)
        fr32 = pkg.sim_front_create(h, split32, kmax=4, precision=pkg.SIM_FP32)

        def step32():
            plan = pkg.sim_plan_create(n, rest32, kmax=4, precision=pkg.SIM_FP32)
            if layout32 is not None:
                pkg.sim_set_layout(h, layout32)
            pkg.sim_front_run(h, fr32)
            pkg.sim_apply_plan(h, plan)
            out = pkg.sim_reduce(h)
            nb = pkg.sim_plan_info(plan)[0]
            pkg.sim_plan_destroy(plan)
            return out, nb
        for _ in range(args.warmup):
            step32()
        pkg.sim_profile_enable(h, True)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            (n32, s32, _), nb32 = step32()
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1)
        c32, a32_ms, a32_bytes = pkg.sim_profile_read(h, pkg.SIM_PROF_APPLY)
        k32_n, k32_ms, _ = pkg.sim_profile_read(h, pkg.SIM_PROF_CONTRACT)
        pkg.sim_profile_enable(h, False)
        pkg.sim_front_destroy(fr32)
        pkg.sim_split_destroy(split32)
        peak32, _ = measured_peaks()
        ach32 = a32_bytes / (a32_ms / 1e3) / 1e9
        fp32_path = {"value": float(amps) * circ.n_gates * args.steps / (ms32 / 1e3), "unit": UNIT,
                     "ms_per_step": ms32 / args.steps, "kmax": 4, "fused_blocks": nb32,
                     "front": {"gates": nf32, "bridging_gates": 2, "contraction": "FP32 CUDA cores",
                               "contraction_ms": k32_ms / max(k32_n, 1)},
                     "norm": n32, "porter_thomas_2n_sum_p2": s32,
                     "roofline": {"bound": "hbm", "achieved": ach32, "peak": peak32, "unit": "GB/s",
                                  "frac": ach32 / peak32, "launches": c32}}

    # the plain per-gate apply (configuration 2's baseline): every gate its own FP32 pass over the
    # state from |0...0>, its matrix from sim_gate_matrix, through sim_apply_fused
    per_gate_path = None
    if not args.no_per_gate:
        per_gate = [([int(g["q0"])] if g["q1"] < 0 else [int(g["q0"]), int(g["q1"])], pkg.sim_gate_matrix(g))
                    for g in gates]
        pkg.sim_set_layout(h, list(range(n)))

        def step_pg():
            pkg.sim_reset(h)
            for t, m in per_gate:
                pkg.sim_apply_fused(h, t, m)
            return pkg.sim_reduce(h)
        step_pg()  # warm-up
        barrier()
        e0.record(stream)
        npg, spg, _ = step_pg()
        e1.record(stream)
        torch.cuda.synchronize()
        mspg = e0.elapsed_time(e1)
        per_gate_path = {"value": float(amps) * circ.n_gates / (mspg / 1e3), "unit": UNIT, "ms_per_step": mspg,
                         "passes": len(per_gate), "precision": "fp32", "norm": npg, "porter_thomas_2n_sum_p2": spg,
                         "default_speedup": mspg / (ms_max / args.steps)}

    # the same step in BF16x3 (the other split-precision mode: BF16 pieces, no better than 2^-16
    # per product), same front, widths and timing, for the comparison of the two modes
    bf16_path = None
    if front is not None and prec == pkg.SIM_FP16X3_TMEM and not args.no_bf16_path:
        fr_b = pkg.sim_front_create(h, split, kmax=args.kmax, precision=pkg.SIM_BF16X3)
        layout_b, _ = choose_layout(rest, args.kmax, pkg.SIM_BF16X3, split)

        def step_b():
            plan = pkg.sim_plan_create(n, rest, kmax=args.kmax, precision=pkg.SIM_BF16X3)
            if layout_b is not None:
                pkg.sim_set_layout(h, layout_b)
            pkg.sim_front_run(h, fr_b)
            pkg.sim_apply_plan(h, plan)
            out = pkg.sim_reduce(h)
            pkg.sim_plan_destroy(plan)
            return out
        for _ in range(args.warmup):
            step_b()
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            nb_, sb_, _ = step_b()
        e1.record(stream)
        torch.cuda.synchronize()
        msb = e0.elapsed_time(e1)
        pkg.sim_front_destroy(fr_b)
        bf16_path = {"value": float(amps) * circ.n_gates * args.steps / (msb / 1e3), "unit": UNIT,
                     "ms_per_step": msb / args.steps, "precision": "bf16x3", "norm": nb_,
                     "porter_thomas_2n_sum_p2": sb_, "norm_drift_per_pass": (nb_ - 1.0) / max(nblocks, 1)}

    matrix_bytes = 0
    plan = pkg.sim_plan_create(n, gates, kmax=args.kmax)
    for i in range(pkg.sim_plan_info(plan)[0]):
        tg, _ = pkg.sim_plan_block(plan, i)
        matrix_bytes += 8 * (1 << (2 * len(tg)))
    pkg.sim_plan_destroy(plan)
    if front is not None:
        for f in front.values():
            pkg.sim_front_destroy(f)
        pkg.sim_split_destroy(split)
    pkg.sim_destroy(h)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_peaks()
    achieved = a_bytes / (a_ms / 1e3) / 1e9 if a_ms > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"{args.precision} (k>=5 blocks; f32 accumulate)",
        "data": "synthetic (seeded random Sycamore-pattern circuit; state from |0...0>)",
        "config": {"workload": args.workload, "n_qubits": n, "cycles": si.WORKLOADS[args.workload]["cycles"],
                   "gates": circ.n_gates, "kmax": args.kmax, "precision": args.precision,
                   "fused_blocks": nblocks,
                   "state_bytes": amps * 8, "l2": "state 8 GiB > 129 MB L2: no flush needed",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu"},
        "pass_updates_per_s": pass_updates,
        "autotune": tuned,
        "gpu_launches": launches,
        "check": {"norm": norm, "porter_thomas_2n_sum_p2": s2, "xeb": xeb},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     # DRAM read + write of the dominant kernel family, per launch on 2^30 amplitudes
                     # (GB), from an ncu capture of that kernel on 2^28 amplitudes, x 4, against
                     # 17.18 GB algorithmic; null for configurations without that capture
                     "traffic": ((TCGEN05_K6_TRAFFIC_GB if args.kmax == 6 else TCGEN05_TRAFFIC_GB)
                                 if args.precision == "fp16x3_tmem" and n == 30 else None),
                     "traffic_kernel": (("k_apply_tc6a<1, 0>" if args.kmax == 6 else "k_apply_tcgen05<5, 2, 0>")
                                        if args.precision == "fp16x3_tmem" else None),
                     "kernel": "fused apply, all launches (" + {
                         "fp16x3_tmem": "k_apply_tcgen05 / k_apply_mma_f16x3 / k_apply_reg / k_apply_direct",
                         "fp32": "k_apply_reg / k_apply_direct / k_apply_tiled"}.get(
                         args.precision, "k_apply_mma_f16x3 / k_apply_reg / k_apply_direct") + ")",
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "launches": a_n, "avg_launch_ms": a_ms / max(a_n, 1)},
        "breakdown_ms_per_step": {"apply": a_ms / args.steps, "reduce": r_ms / args.steps,
                                  "contract": c_ms / args.steps,
                                  "other": ms_max / args.steps - (a_ms + r_ms + c_ms) / args.steps},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(gates.nbytes + matrix_bytes),
                "d2h_bytes_per_step": int(amps * 8), "steps": args.e2e_steps,
                "schedule": ("overlapped: two handles, computes chained, the readout of step i during the "
                             "compute of step i+1" if overlap else
                             "serial: one handle, each readout before the next compute (the link slows "
                             "while the device streams HBM)"),
                "schedule_probe_s": probe,
                "readout_alone_ms": readout_ms, "readout_alone_gbs": amps * 8 / (readout_ms / 1e3) / 1e9,
                "readout_in_loop_ms": {"median": rd_in_loop[len(rd_in_loop) // 2], "max": rd_in_loop[-1]},
                "e2e_ms_per_step": 1e3 * e2e_s / args.e2e_steps},
        "clocks": clk.summary(),
    }
    line["config"]["layout"] = layout_info
    if front_info is not None:
        line["config"]["front"] = front_info
        bf16, bf16_kind = measured_peaks("bf16_tflops")
        ach_c = c_flops / (c_ms / 1e3) / 1e12 if c_ms > 0 else None
        # the contraction's tensor roofline: algorithmic complex-GEMM FLOPs (8 per complex
        # multiply-add) per launch / its CUDA-event time; 3xFP16 issues 3 FP16 MMA FLOPs per
        # algorithmic FLOP, so the tensor pipe runs at 3 x achieved
        # The measured cuBLAS bf16 burst is below what this kernel's tensor pipe sustains (3 x
        # achieved exceeded it), so it is no ceiling here: the fraction is taken against the
        # larger of it and the dense FP16/BF16 datasheet figure, and a pipe fraction above 1
        # against the measured figure is flagged as a problem of that measurement.
        peak_c = max(bf16, NOMINAL_DENSE_F16_TFLOPS)
        pipe_meas = 3 * ach_c / bf16 if ach_c else None
        line["contract_roofline"] = {
            "bound": "tensor", "kernel": "k_contract_tcgen05" if "tcgen05" in front_info["contraction"]
            else "k_contract_fp32", "achieved": ach_c, "peak": peak_c, "unit": "TFLOP/s",
            "frac": ach_c / peak_c if ach_c else None, "mma_flops_per_alg_flop": 3,
            "tensor_pipe_frac": 3 * ach_c / peak_c if ach_c else None,
            "tensor_pipe_frac_of_measured_bf16": pipe_meas,
            "measured_bf16_tflops": bf16,
            "peak_source": (f"max of {bf16_kind} bf16_tflops {bf16:.1f} and the dense FP16/BF16 datasheet "
                            f"figure {NOMINAL_DENSE_F16_TFLOPS:.0f} (FP16 runs at the BF16 rate)"),
            "note": ("tensor pipe above the measured cuBLAS bf16 burst: that measurement is below the "
                     "pipe's real ceiling" if pipe_meas and pipe_meas > 1 else None),
            "sm_mhz_median": (clk.summary() or {}).get("sm_mhz"),
            "launches": c_n, "avg_launch_ms": c_ms / max(c_n, 1),
            "alg_flops_per_launch": c_flops / max(c_n, 1)}
        line["plain_path"] = plain_path
    if per_gate_path:
        line["per_gate_path"] = per_gate_path
    if fp32_path:
        line["fp32_path"] = fp32_path
    if bf16_path:
        line["bf16x3_path"] = bf16_path
    # a per-result error estimate that needs no oracle: the norm's drift from 1 per fused pass
    line["check"]["norm_drift_per_pass"] = (norm - 1.0) / max(nblocks, 1)
    if ws == 1 and not args.no_large:
        # configuration 3: 33 qubits (64 GiB) held as 8 slices over 3 bits, phases with in-place
        # permutation passes between them, in the default arithmetic, in BF16x3, in TF32 (mma.sync;
        # its stated error is ~1e-3) and in FP32
        line["syc33_sliced"] = {p: large_case_run("syc33_6x6m3_d20", p, local)
                                for p in ("fp16x3_tmem", "bf16x3", "tf32", "fp32")}
        # configuration 4: 35 qubits (256 GiB) in a secondary store, 8 of its 16 regions pinned on the
        # host and 8 in HBM, streamed through device slots of 2^31 amplitudes phase by phase
        line["syc35_store"] = large_case_run("syc35_5x7_d16", "fp16x3_tmem", local)
    if ws == 1 and not args.no_serving:
        # configuration 5: 2000 circuits, Poisson arrivals, each arithmetic beside its one-at-a-time run
        line["serving"] = {p: serving_run(args.serving_circuits, local, r, p)
                           for p, r in (("fp16x3_tmem", args.serving_rate), ("fp32", args.serving_rate_fp32))}
    if ws == 1 and not args.no_graphs:
        line["graph_replay"] = graph_replay_run(local)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(circ, args.cpu_sample_gates)
    _ = sanity
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def kernel_case():
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si
    from paper_1910_09534_gb300 import build as pkg_build

    pkg_build.build()
    n = 28
    h = pkg.sim_create(n)
    for t in ([12, 13, 14, 15], [1, 3, 14, 20], [12, 13]):
        u = si.random_unitary(len(t), 1)
        for _ in range(2):
            pkg.sim_apply_fused(h, t, u)
    for t in ([12, 13, 14, 15, 16], [1, 3, 14, 20, 25]):
        u = si.random_unitary(len(t), 2)
        for _ in range(2):
            pkg.sim_apply_fused(h, t, u, precision=pkg.SIM_FP16X3)
    # default mode: tcgen05 with 256-group tiles stored from registers, 128-group tiles with bulk
    # stores, one target below bit 4; then a 4-qubit block on bits 0-3 (mma.sync, k = 4)
    for t in ([12, 13, 14, 15, 16], [4, 9, 14, 20, 25], [3, 4, 5, 7, 8], [0, 1, 2, 3]):
        u = si.random_unitary(len(t), 2)
        for _ in range(2):
            pkg.sim_apply_fused(h, t, u, precision=pkg.SIM_FP16X3_TMEM)
    # 6-qubit blocks on tcgen05: a target at bit 7 (2 KiB copies), all above bit 7 (1 KiB), one
    # below bit 4
    for t in ([7, 12, 14, 18, 22, 26], [12, 13, 14, 15, 16, 17], [3, 9, 14, 20, 25, 27]):
        u = si.random_unitary(len(t), 3)
        for _ in range(2):
            pkg.sim_apply_fused(h, t, u, precision=pkg.SIM_FP16X3_TMEM)
    for pairs in (((25, 10), (26, 11), (27, 12)), ((0, 25), (1, 26), (2, 27))):  # high-high, low<->top
        perm = list(range(n))
        for a, b in pairs:
            perm[a], perm[b] = b, a
        pkg.sim_permute(h, perm)
        pkg.sim_permute(h, list(range(n)))
    pkg.sim_reduce(h)
    pkg.sim_reduce(h)
    # contraction deferral on the 28-qubit workload: its gates up to the sixth one across the
    # middle column cut (12 + 16 qubits, 4^5 entanglement values), front run twice
    circ = si.workload_circuit("syc28_4x7_d20", seed=0)
    side, nf = pkg.sim_split_choose(n, pkg.gates_array(circ), 5)
    s = pkg.sim_split_create(n, pkg.gates_array(circ)[:nf], side)
    f = pkg.sim_front_create(h, s, kmax=5, precision=pkg.SIM_FP16X3_TMEM)
    for _ in range(2):
        pkg.sim_front_run(h, f)
    pkg.sim_sync(h)
    pkg.sim_front_destroy(f)
    pkg.sim_split_destroy(s)
    pkg.sim_destroy(h)
    print("kernel case done", flush=True)


def large_case_run(name: str, precision: str = "fp16x3_tmem", device: int = 0, front_pairs: int = -1,
                   kmax: int = 0) -> dict:
    """One run of a configuration from LARGE_CASES in SIM_FP16X3_TMEM at the case's block width, or
    in SIM_FP32 at k_max 4 (the resident one after a warm-up run; a streamed run takes seconds and
    runs once): wall time, gate updates/s, the apply kernels' time and bandwidth with their HBM
    roofline, the permutation passes (resident) or the host link's combined rate (streamed), and
    the final state's norm and 2^n sum p^2."""
    import paper_1910_09534_gb300 as pkg
    import syc_inputs as si

    cfg = LARGE_CASES[name]
    circ = si.workload_circuit(name, seed=0)
    n, s, kmax = circ.n_qubits, cfg["slice_bits"], kmax or cfg["kmax"]
    gates = pkg.gates_array(circ)
    prec = {"bf16x3": pkg.SIM_BF16X3, "tf32": pkg.SIM_TF32}.get(precision, pkg.SIM_FP16X3_TMEM)
    if precision == "fp32":
        prec, kmax = pkg.SIM_FP32, 4
    host = cfg["store"] == "host"
    # into a host store, the circuit's first gates run as contraction deferral (Sect. 4's first
    # phase): two tensors contracted slice by slice straight into the store, fused with the first
    # phase's blocks; the sliced sets and phases are chosen for the remaining gates
    split, n_front, front_info = None, 0, None
    pairs_wanted = cfg.get("front_pairs", 0) if front_pairs < 0 else front_pairs
    if pairs_wanted > 0:
        side, n_front = pkg.sim_split_choose(n, gates, pairs_wanted)
        split = pkg.sim_split_create(n, gates[:n_front], side)
        n_side, n_wires, pairs, _ = pkg.sim_split_info(split)
        front_info = {"gates": n_front, "bridging_gates": pairs, "qubits_per_side": [int(x) for x in n_side],
                      "tensor_qubits": [int(x) for x in n_wires]}
    rest = gates[n_front:]
    if cfg["sets"] == "chosen":
        set_a, set_b, _, _ = pkg.sim_phases_choose_sets(n, rest, s, kmax=kmax)
    else:
        set_a, set_b = list(range(s)), list(range(n - s, n))
    ph = pkg.sim_phases_create(n, rest, s, set_a, set_b, kmax=kmax, precision=prec)
    n_phases, n_blocks = pkg.sim_phases_info(ph)
    front, layout_info, perm = None, None, None
    if host:
        h = pkg.sim_create(n, s, store=pkg.SIM_STORE_HOST, set_a=set_a, set_b=set_b, slots=3,
                           store_device_regions=cfg["device_regions"], device=device)
    else:
        h = pkg.sim_create(n, s, device=device)
    if host or split is not None:
        # the order of the qubits outside the sliced sets (sim_phases_layout): fewer blocks with
        # two targets below bit 4, and with a front side-0 qubits on bits 0-4 (the contraction's
        # stores stay whole); resident, the first phase's sliced set already on top.  A
        # relabelling, before anything is written
        perm, est, est_asc = pkg.sim_phases_layout(ph, n, split, resident=not host)
        pkg.sim_set_layout(h, perm)
        layout_info = {"chosen_by": "sim_phases_layout", "estimate_ms": est, "starting_estimate_ms": est_asc}
        if split is not None:
            front = pkg.sim_front_create(h, split, kmax=kmax, precision=prec)
    fused = host and front is not None

    def run():
        if front is None:
            pkg.sim_run_phases(h, ph)
        elif fused:
            # the contraction fills each slice of the first phase's sliced set, the phase's
            # blocks run on it, and it is written once
            pkg.sim_front_run_phase(h, front, *pkg.sim_phases_get(ph, 0))
            for i in range(1, n_phases):
                set_i, plan_i = pkg.sim_phases_get(ph, i)
                pkg.sim_run_phase(h, set_i, plan_i)
        else:  # resident: the contraction writes the whole state, the phases permute as they go
            pkg.sim_set_layout(h, perm)
            pkg.sim_front_run(h, front)
            pkg.sim_run_phases(h, ph)

    if not host:  # warm-up
        if front is None:
            pkg.sim_reset(h)
        run()
        pkg.sim_sync(h)
    if front is None:
        pkg.sim_reset(h)
    pkg.sim_sync(h)
    pkg.sim_profile_enable(h, True)
    t0 = time.perf_counter()
    run()
    pkg.sim_sync(h)
    wall = time.perf_counter() - t0
    a_n, a_ms, a_bytes = pkg.sim_profile_read(h, pkg.SIM_PROF_APPLY)
    p_n, p_ms, p_bytes = pkg.sim_profile_read(h, pkg.SIM_PROF_PERMUTE)
    c_n, c_ms, _ = pkg.sim_profile_read(h, pkg.SIM_PROF_CONTRACT)
    pkg.sim_profile_enable(h, False)
    norm, s2, _ = pkg.sim_reduce(h)
    if front is not None:
        pkg.sim_front_destroy(front)
        pkg.sim_split_destroy(split)
        front_info.update({"first_phase_fused": fused, "contraction_launches": c_n, "contraction_ms": c_ms})
    pkg.sim_destroy(h)
    pkg.sim_phases_destroy(ph)
    state_bytes = 8.0 * (1 << n)
    peak, peak_kind = measured_peaks()
    ach = a_bytes / (a_ms / 1e3) / 1e9 if a_ms else None
    line = {"case": name, "n_qubits": n, "gates": circ.n_gates,
            "store": ("host" if host else "device") + (f", {cfg['device_regions']} of {1 << s} regions in HBM"
                                                       if cfg["device_regions"] else ""),
            "slice_bits": s, "set_a": set_a, "set_b": set_b, "sets": cfg["sets"], "kmax": kmax,
            "precision": precision, "phases": n_phases, "blocks": n_blocks, "wall_s": wall,
            "gate_updates_per_s": float(1 << n) * circ.n_gates / wall,
            "apply": {"launches": a_n, "ms": a_ms, "gbs": ach,
                      "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                   "frac": ach / peak if ach else None, "peak_source": f"{peak_kind} hbm_gbs",
                                   "alg_bytes": a_bytes}},
            "norm": norm, "porter_thomas_2n_sum_p2": s2,
            "norm_drift_per_pass": (norm - 1.0) / max(n_blocks, 1)}
    if front_info is not None:
        line["front"] = front_info
    if layout_info is not None:
        line["layout"] = layout_info
    if host:  # every phase moves the host regions out and back (the fused first phase only out)
        moved = (2 * n_phases - (1 if fused else 0)) * state_bytes * (1 - cfg["device_regions"] / (1 << s))
        line["host_link_gbs_combined"] = moved / wall / 1e9
    else:
        line["permute"] = {"passes": p_n, "ms": p_ms, "gbs_moved": p_bytes / (p_ms / 1e3) / 1e9 if p_ms else None}
    return line


def large_case(name: str, precision: str = "fp16x3_tmem", front_pairs: int = -1, kmax: int = 0):
    from paper_1910_09534_gb300 import build as pkg_build

    pkg_build.build()
    print(json.dumps(large_case_run(name, precision, front_pairs=front_pairs, kmax=kmax)), flush=True)


def serving_case(args):
    """Only the config-5 serving leg (no timed steps): one JSON line."""
    from paper_1910_09534_gb300 import build as pkg_build

    pkg_build.build()
    prec = "fp32" if args.precision == "fp32" else "fp16x3_tmem"
    rate = args.serving_rate if prec != "fp32" else args.serving_rate_fp32
    print(json.dumps(serving_run(args.serving_circuits, 0, rate, prec, args.serving_max_large)), flush=True)


def main():
    args = parse()
    if args.large_case:
        large_case(args.large_case, args.precision if args.precision in ("fp32", "bf16x3", "tf32") else "fp16x3_tmem",
                   args.large_front_pairs, args.large_kmax)
    elif args.serving_only:
        serving_case(args)
    elif args.kernel_case:
        kernel_case()
    elif args.oracle_table:
        print(json.dumps(oracle_table()), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
