"""Benchmark of the simulator's hot path on the 28-qubit brickwork workload.

One step = the whole path over one circuit: |0...0> start (qc_state_init_basis),
the 540-gate brickwork of Haar-random two-qubit unitaries on 28 qubits (depth 40,
seed 2), the probability vector (qc_probs), 1e6 shots by inverse CDF on seeded
uniforms (qc_sample) and <sum_i Z_i Z_{i+1}> (qc_expect_pauli).  The headline runs the
circuit in complex64 through the fusion planner (QC_RUN_FUSED); the plain complex128
per-gate path ("plain FP64") is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (under torchrun) every rank runs an
independent replica of the workload (the workload does not shard); the value is the
total number of circuits per second over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "circuit time & HBM GB/s (frac of peak) at 28–32 qubits: fused/FP32 vs plain FP64"
N_QUBITS, DEPTH, SEED, SHOTS, SHOT_SEED = 28, 40, 2, 1_000_000, 102


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1922.7)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------

def oracle_rate(gates_per_step: int, steps: int, warmup: int, ops):
    """Circuits/s of the oracle extrapolated from `gates_per_step` gates of the
    28-qubit brickwork per step (plus nothing else: gates dominate)."""
    import oracle
    psi = oracle.basis_state(N_QUBITS, 0)
    times = []
    it = 0
    for s in range(warmup + steps):
        t0 = time.perf_counter()
        for _ in range(gates_per_step):
            oracle.apply_op(psi, ops[it % len(ops)])
            it += 1
        dt = time.perf_counter() - t0
        if s >= warmup:
            times.append(dt)
    t = sum(times)
    return (gates_per_step * steps / len(ops)) / t, t / steps, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ops = W.brickwork(N_QUBITS, DEPTH, SEED)
    rate, sec_per_step, cores = oracle_rate(args.ref_gates, args.steps, args.warmup, ops)
    sample = "%d of the %d brickwork gates per step on 28 qubits (complex128), extrapolated" % (
        args.ref_gates, len(ops))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "circuits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "brickwork n=28 depth=40 Haar 2q (540 gates), 1e6 shots", "n_qubits": N_QUBITS},
            "cpu_baseline": {"value": rate, "unit": "circuits/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": "circuits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

class StreamTimer:
    def __init__(self, stream):
        import torch
        self.stream = stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def start(self):
        self.e0.record(self.stream)

    def stop(self) -> float:
        self.e1.record(self.stream)
        self.e1.synchronize()
        return self.e0.elapsed_time(self.e1)


def run_ours(args):
    import torch

    import paper_2503_03016_gb300 as P

    rank, world, local = dist_setup(args.gpus)
    hbm_gbs, bf16_tflops, peak_src = peaks()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ops = W.brickwork(N_QUBITS, DEPTH, SEED)
    circ = P.Circuit(N_QUBITS, ops)
    u_host = torch.tensor(W.uniforms(SHOTS, SHOT_SEED), dtype=torch.float64).pin_memory()
    u_dev = u_host.to("cuda", non_blocking=True)
    out_dev = torch.empty(SHOTS, dtype=torch.int64, device="cuda")
    out_host = torch.empty(SHOTS, dtype=torch.int64).pin_memory()
    zz = W.zz_terms(N_QUBITS, ring=False)
    mode = P.QC_RUN_FUSED if args.mode == "fused" else P.QC_RUN_PER_GATE
    prec = P.QC_PREC_TF32X3 if args.prec == "tf32x3" else P.QC_PREC_NATIVE
    st = P.State(N_QUBITS, "c64", stream)
    probs = torch.empty(1 << N_QUBITS, dtype=torch.float64, device="cuda")

    def step(e2e: bool):
        if e2e:
            u_dev.copy_(u_host, non_blocking=True)
        P.qc_state_init_basis(st.handle, 0)
        P.qc_run_circuit(st.handle, circ, None, mode, prec)
        P.qc_probs(st.handle, probs)
        P.qc_sample(st.handle, u_dev, SHOTS, out_dev)
        ev = P.qc_expect_pauli(st.handle, zz)  # synchronising: returns host values
        if e2e:
            out_host.copy_(out_dev, non_blocking=True)
        return ev

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = P.qc_launch_count()
    timer = StreamTimer(stream)
    torch.cuda.synchronize()
    timer.start()
    for _ in range(args.steps):
        step(False)
    ms = timer.stop()
    launches = P.qc_launch_count() - launches0
    torch.cuda.synchronize()
    barrier(world)
    ms_max = max_over_ranks(ms, world)

    # end to end through the public API: host uniforms in, host samples out
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(True)
    stream.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world)

    # dominant kernel: time the circuit alone with events
    torch.cuda.synchronize()
    timer.start()
    for _ in range(args.steps):
        P.qc_run_circuit(st.handle, circ, None, mode, prec)
    circ_ms = timer.stop() / args.steps
    clk = clocks.stop()

    # plain FP64: complex128 per-gate sweeps
    plain = None
    if args.plain_steps > 0:
        st128 = P.State(N_QUBITS, "c128", stream)
        P.qc_state_init_basis(st128.handle, 0)
        P.qc_run_circuit(st128.handle, circ, None, P.QC_RUN_PER_GATE, P.QC_PREC_NATIVE)
        torch.cuda.synchronize()
        timer.start()
        for _ in range(args.plain_steps):
            P.qc_state_init_basis(st128.handle, 0)
            P.qc_run_circuit(st128.handle, circ, None, P.QC_RUN_PER_GATE, P.QC_PREC_NATIVE)
        p_ms = timer.stop() / args.plain_steps
        sbytes128 = (1 << N_QUBITS) * 16
        plain = {"ms_per_circuit": p_ms, "dtype": "f64", "algorithmic_gb": len(ops) * 2 * sbytes128 / 1e9,
                 "effective_gbs": len(ops) * 2 * sbytes128 / (p_ms * 1e-3) / 1e9}
        st128.free()

    sbytes = (1 << N_QUBITS) * 8
    passes = P.qc_last_pass_count() if args.mode == "fused" else len(ops)
    algo_bytes = (passes or len(ops)) * 2 * sbytes
    achieved = algo_bytes / (circ_ms * 1e-3) / 1e9
    # cpu baseline (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and args.cpu_gates > 0:
        rate, _, cores = oracle_rate(args.cpu_gates, 1, 0, ops)
        cpu = {"value": rate, "unit": "circuits/s", "cores": cores, "kind": "oracle",
               "sample": "%d of %d brickwork gates on 28 qubits (complex128), extrapolated" % (args.cpu_gates, len(ops))}
    if rank == 0:
        steps_total = args.steps * world
        line = {
            "metric": METRIC, "value": steps_total / (ms_max * 1e-3), "unit": "circuits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic",
            "config": {"workload": "brickwork n=28 depth=40 Haar 2q (540 gates, seed 2) + probs + 1e6 shots + <ZZ>",
                       "mode": args.mode, "prec": args.prec, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (2 GiB state)"},
            "circuit_ms": circ_ms,
            "plain_fp64": plain,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s",
                         "frac": achieved / hbm_gbs, "traffic": None, "peak_source": peak_src,
                         "kernel": "circuit (%s)" % args.mode, "passes": passes},
            "cpu_baseline": cpu,
            "e2e": {"value": steps_total / (e2e_ms * 1e-3), "unit": "circuits/s",
                    "h2d_bytes_per_step": SHOTS * 8, "d2h_bytes_per_step": SHOTS * 8 + 8 * len(zz)},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    st.free()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch_bench(args):
    """Opt-in secondary measurement: the 4096-circuit batched ansatz workload (n uniform
    in 12..20, 8 layers, seed 4), one persistent launch per step, replayed from a CUDA
    graph; prints its own JSON line."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    layers = 8
    ns, params = W.batch_workload(4096, layers, 12, 20, 4)
    offs = np.cumsum([0] + [p.size for p in params[:-1]]).astype(np.int64)
    flat = np.concatenate(params).astype(np.float32)
    dparams = torch.tensor(flat, device="cuda")
    out = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    nsi = np.asarray(ns, dtype=np.int32)
    for _ in range(max(args.warmup, 1)):
        P.qc_run_batch(nsi, layers, offs, dparams, flat.size, out)
    torch.cuda.synchronize()
    timer = StreamTimer(stream)
    timer.start()
    for _ in range(args.steps):
        P.qc_run_batch(nsi, layers, offs, dparams, flat.size, out)
    ms = timer.stop() / args.steps
    flops = sum(8.0 * layers * 2 * int(n) * (1 << int(n)) for n in ns)
    print(json.dumps({"metric": "batched ansatz circuits/s", "value": len(ns) / (ms * 1e-3), "unit": "circuits/s",
                      "ms_per_step": ms, "steps": args.steps, "fusion_width": P.qc_batch_fusion_width(),
                      "approx_fp32_tflops": flops / (ms * 1e-3) / 1e12,
                      "config": {"workload": "4096 ansatz circuits, n in 12..20, 8 layers RY.RZ + CZ chain, <ZZ>"}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["fused", "per_gate"])
    ap.add_argument("--prec", default="native", choices=["native", "tf32x3"])
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-gates", type=int, default=24)
    ap.add_argument("--ref-gates", type=int, default=8)
    ap.add_argument("--qubits", type=int, default=28, help="smaller cases for profiling only")
    ap.add_argument("--workload", default="brickwork", choices=["brickwork", "batch"],
                    help="batch: opt-in secondary measurement of the batched launch")
    args = ap.parse_args()
    global N_QUBITS
    N_QUBITS = args.qubits
    if args.workload == "batch" and args.impl == "ours":
        run_batch_bench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
