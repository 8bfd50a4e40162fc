"""Benchmark of the simulator's hot path on the 28-qubit brickwork workload.

One step = the whole path over one circuit: |0...0> start (qc_state_init_basis),
the 540-gate brickwork of Haar-random two-qubit unitaries on 28 qubits (depth 40,
seed 2), the probability vector (qc_probs), 1e6 shots by inverse CDF on seeded
uniforms (qc_sample) and <sum_i Z_i Z_{i+1}> (qc_expect_pauli).  The headline runs the
circuit in complex64 through the fusion planner (QC_RUN_FUSED); the plain complex128
per-gate path (the metric's "plain FP64": binary64 storage, its sweeps computed in
double-float arithmetic) is timed beside it.

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
WORKLOAD = "brickwork n=28 depth=40 Haar 2q (540 gates, seed 2) + probs + 1e6 shots + <ZZ>"
# FP32 peak from unit counts at the maximum SM clock
ALU_PEAK_TF = 152 * 128 * 2 * 2070e6 / 1e12
ALU_PEAK_SRC = "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1922.7)), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


_TF32_PEAK = None


def tf32_peak():
    """Dense TF32 tensor throughput measured on this GPU: torch FP32 matmul of 8192^3
    with TF32 allowed (2 N^3 flops), best of 10, CUDA events.  The library never calls
    this; it is the roofline denominator of the TF32 tensor-core kernels."""
    global _TF32_PEAK
    if _TF32_PEAK is None:
        import torch
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = True
        try:
            N = 8192
            a = torch.randn(N, N, device="cuda")
            b = torch.randn(N, N, device="cuda")
            c = torch.empty(N, N, device="cuda")
            for _ in range(3):
                torch.matmul(a, b, out=c)
            best = None
            for _ in range(10):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            _TF32_PEAK = 2.0 * N ** 3 / (best * 1e-3) / 1e12
            del a, b, c
            torch.cuda.empty_cache()
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
    return _TF32_PEAK


TF32_PEAK_SRC = "measured: torch FP32 matmul 8192^3 with TF32 allowed, best of 10"


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
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ms_local: float, steps: int, world: int):
    """(value, ms_max): every rank ran `steps` independent circuits; the whole job's
    throughput is all ranks' circuits over the slowest rank's time."""
    ms_max = max_over_ranks(ms_local, world)
    return steps * world / (ms_max * 1e-3), ms_max


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


def oracle_step_baseline(ops, gates: int, single_gates: int):
    """The oracle timed on one step of the workload: `gates` of the brickwork's gates
    (extrapolated to all of them) plus the whole readout on the resulting 28-qubit
    state -- FP64 probabilities, the double-double CDF, 1e6 shots by bisection and
    <sum Z_i Z_i+1> -- on all host threads; and `single_gates` gates on one thread."""
    import oracle
    threads = oracle.num_threads()
    psi = oracle.basis_state(N_QUBITS, 0)
    t0 = time.perf_counter()
    for i in range(gates):
        oracle.apply_op(psi, ops[i])
    t_gate = (time.perf_counter() - t0) / gates
    u = W.uniforms(SHOTS, SHOT_SEED)
    # Z_i Z_i+1: z mask on index bits n-1-i and n-2-i
    zz = [(0, 3 << (N_QUBITS - 2 - i), 1.0) for i in range(N_QUBITS - 1)]
    t0 = time.perf_counter()
    p = oracle.probs(psi)
    c = oracle.cdf(p)
    oracle.sample(c, u)
    del p, c
    oracle.expect_masks(psi, zz)
    t_read = time.perf_counter() - t0
    t1 = None
    if single_gates > 0:
        oracle.set_threads(1)
        try:
            t0 = time.perf_counter()
            for i in range(single_gates):
                oracle.apply_op(psi, ops[gates + i])
            t1 = (time.perf_counter() - t0) / single_gates
        finally:
            oracle.set_threads(threads)
    step_s = t_gate * len(ops) + t_read
    out = {"value": 1.0 / step_s, "unit": "circuits/s", "cores": threads, "kind": "oracle",
           "sample": ("%d of %d brickwork gates on 28 qubits (complex128) extrapolated to the circuit, plus the "
                      "whole readout (FP64 probabilities, CDF, 1e6 shots, <sum ZZ>) timed once" % (gates, len(ops))),
           "readout_s": t_read, "readout_share": t_read / step_s, "gate_s": t_gate}
    if t1 is not None:
        out["one_thread"] = {"value": 1.0 / (t1 * len(ops) + t_read * threads), "unit": "circuits/s",
                             "gate_s": t1, "sample": "%d gates on one thread; readout scaled by the thread count"
                                                     % single_gates}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ops = W.brickwork(N_QUBITS, DEPTH, SEED)
    rate, sec_per_step, cores = oracle_rate(args.ref_gates, args.steps, args.warmup, ops)
    sample = ("%d of the %d brickwork gates per step on 28 qubits (complex128), extrapolated to the circuit; "
              "gates only (the probabilities, shots and <ZZ> would add to the oracle's time)" % (
                  args.ref_gates, len(ops)))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "circuits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": "oracle (plain per-gate loops, complex128)",
                       "parallelism": "host cores", "n_qubits": N_QUBITS},
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
    prec = {"tf32x3": P.QC_PREC_TF32X3, "native": P.QC_PREC_NATIVE, "auto": P.QC_PREC_AUTO}[args.prec]
    st = P.State(N_QUBITS, "c64", stream)
    probs = torch.empty(1 << N_QUBITS, dtype=torch.float64, device="cuda")

    def step(e2e: bool):
        if e2e:
            u_dev.copy_(u_host, non_blocking=True)
        P.qc_state_init_basis(st.handle, 0)
        P.qc_run_circuit(st.handle, circ, None, mode, prec)
        P.qc_probs(st.handle, probs)
        # shots drawn from the FP64 probabilities just computed (the same values the
        # sampler would form from the amplitudes, so the same outcomes)
        P.qc_sample_probs(st.handle, probs, N_QUBITS, u_dev, SHOTS, out_dev)
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
    value, ms_max = whole_job_rate(ms, args.steps, world)

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

    # the plain arm: complex128 per-gate sweeps (double-float arithmetic on the FP32
    # pipe at this size; FP64 storage)
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
        plain = {"ms_per_circuit": p_ms, "dtype": "c128",
                 "arith": "double-float (FP32 pairs, 48-bit significands; no FP64 instructions)",
                 "algorithmic_gb": len(ops) * 2 * sbytes128 / 1e9,
                 "effective_gbs": len(ops) * 2 * sbytes128 / (p_ms * 1e-3) / 1e9,
                 "frac_hbm": len(ops) * 2 * sbytes128 / (p_ms * 1e-3) / 1e9 / hbm_gbs}
        st128.free()

    sbytes = (1 << N_QUBITS) * 8
    passes = P.qc_last_pass_count() if args.mode == "fused" else len(ops)
    tc_path = args.mode == "fused" and P.qc_last_fused_path() == 2
    if tc_path:
        # dominant kernel: the tile pass with tensor-core stages.  Each stage is a
        # 128 x 64 x 64 real GEMM per 4096-amplitude tile, three TF32 products:
        # 2 * 64 * 64 * 128 * 3 / 4096 = 768 flops per amplitude per stage.
        stages = P.qc_last_stage_count()
        flops = stages * 768.0 * (1 << N_QUBITS)
        tf32_pk = tf32_peak()
        achieved = flops / (circ_ms * 1e-3) / 1e12
        # DRAM bytes of one tensor-core tile pass (box copies) in an ncu capture at 26
        # qubits (537.35 MB read + 480.32 MB written), scaled by the larger state
        roof = {"bound": "tensor", "achieved": achieved, "peak": tf32_pk, "unit": "TFLOP/s",
                "frac": achieved / tf32_pk, "traffic": 1013.80352e6 * (1 << (N_QUBITS - 26)),
                "traffic_note": "per pass, ncu at 26 qubits scaled by 2^(n-26)",
                "peak_source": TF32_PEAK_SRC,
                "kernel": "k_tile_pass_tc", "passes": passes, "stages": stages,
                "gate_tflops_fp32_equivalent": len(ops) * 32.0 * (1 << N_QUBITS) / (circ_ms * 1e-3) / 1e12}
    elif args.mode == "fused":
        # dominant kernel: the tile pass, bound by FP32 FMA for Haar gates.  Algorithmic
        # work: every two-qubit gate is 4 complex multiply-adds (32 flops) per amplitude.
        # Peak from unit counts: SMs x 128 FP32 lanes x 2 flops x SM clock under load.
        flops = len(ops) * 32.0 * (1 << N_QUBITS)
        sm_mhz = (clk.get("sm_mhz") or 2070.0) if isinstance(clk, dict) else 2070.0
        peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
        achieved = flops / (circ_ms * 1e-3) / 1e12
        # DRAM bytes of one tile pass in an ncu capture at 26 qubits (537.43 + 476.53 MB),
        # scaled by the larger state (a pass moves the state once each way)
        traffic = 1013.959168e6 * (1 << (N_QUBITS - 26))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_note": "per pass, ncu at 26 qubits scaled by 2^(n-26)",
                "algorithmic_bytes_per_pass": 2 * sbytes, "hbm_gbs_over_passes": passes * 2 * sbytes / (circ_ms * 1e-3) / 1e9,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x %.0f MHz" % sm_mhz,
                "kernel": "k_tile_pass<float,512,4>", "passes": passes}
    else:
        algo_bytes = len(ops) * 2 * sbytes
        achieved = algo_bytes / (circ_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
                "traffic": None, "peak_source": peak_src, "kernel": "k_2q_dense<float,1>", "launches": len(ops)}
    # cpu baseline (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and args.cpu_gates > 0:
        cpu = oracle_step_baseline(ops, args.cpu_gates, args.cpu_single_gates)
    if rank == 0:
        steps_total = args.steps * world
        line = {
            "metric": METRIC, "value": value, "unit": "circuits/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "tf32x3" if tc_path else "c64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": args.mode, "prec": args.prec,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (2 GiB state)"},
            "circuit_ms": circ_ms,
            "plain_c128": plain,
            "roofline": roof,
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
    subset = ""
    if args.batch_range:
        # profiling only: the circuits of the workload whose qubit counts lie in LO..HI
        lo, hi = (int(x) for x in args.batch_range.split("-"))
        keep = [i for i, n in enumerate(ns) if lo <= n <= hi][:args.batch_count or None]
        ns, params = [ns[i] for i in keep], [params[i] for i in keep]
        subset = " (subset: %d circuits with %d..%d qubits)" % (len(ns), lo, hi)
    offs = np.cumsum([0] + [p.size for p in params[:-1]]).astype(np.int64)
    flat = np.concatenate(params).astype(np.float32)
    dparams = torch.tensor(flat, device="cuda")
    out = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    nsi = np.asarray(ns, dtype=np.int32)
    for _ in range(max(args.warmup, 1)):
        P.qc_run_ansatz_batch(nsi, layers, offs, dparams, flat.size, out)
    torch.cuda.synchronize()
    timer = StreamTimer(stream)
    timer.start()
    for _ in range(args.steps):
        P.qc_run_ansatz_batch(nsi, layers, offs, dparams, flat.size, out)
    ms = timer.stop() / args.steps
    # a fused RZ.RY layer gate costs 2 complex multiply-adds = 16 real flops per amplitude
    flops = sum(16.0 * layers * int(n) * (1 << int(n)) for n in ns)
    tf = flops / (ms * 1e-3) / 1e12
    print(json.dumps({"metric": "batched ansatz circuits/s", "value": len(ns) / (ms * 1e-3), "unit": "circuits/s",
                      "ms_per_step": ms, "steps": args.steps, "fusion_width": P.qc_batch_fusion_width(),
                      "approx_fp32_tflops": tf,
                      "roofline": {"bound": "alu", "achieved": tf, "peak": ALU_PEAK_TF, "unit": "TFLOP/s",
                                   "frac": tf / ALU_PEAK_TF, "peak_source": ALU_PEAK_SRC},
                      "config": {"workload": "4096 ansatz circuits, n in 12..20, 8 layers RY.RZ + CZ chain, <ZZ>" +
                                 subset}}))


def run_batch_general_bench(args):
    """Opt-in secondary measurement: the general batch entry point on a mixed family of
    1024 circuits (QFTs, depth-8 Haar brickworks, 4-layer RY.RZ ansatz with a CZ ring;
    n uniform in 10..16, seed 9), each with its own sum_i Z_i Z_i+1 + sum_i X_i
    observable, in one launch per step (complex64)."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    rng = np.random.default_rng(9)
    circs, hams, offs, flat = [], [], [], []
    nps = 0
    for i in range(1024):
        n = int(rng.integers(10, 17))
        kind = i % 3
        if kind == 0:
            ops, p = W.qft(n), None
        elif kind == 1:
            ops, p = W.brickwork(n, 8, 1000 + i), None
        else:
            ops, p = W.ansatz(n, 4, ring=True), W.ansatz_params(n, 4, 2000 + i)
        circs.append(P.Circuit(n, ops))
        hams.append(P.Hamiltonian.from_strings(W.zz_terms(n, True) + W.x_terms(n)))
        offs.append(nps)
        if p is not None:
            flat.append(p)
            nps += p.size
    dparams = torch.tensor(np.concatenate(flat), dtype=torch.float64, device="cuda")
    out = torch.empty(len(circs), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 1)):
        P.qc_run_batch(circs, hams, dparams, offs, None, out)
    torch.cuda.synchronize()
    t = StreamTimer(stream)
    t.start()
    for _ in range(args.steps):
        P.qc_run_batch(circs, hams, dparams, offs, None, out)
    ms = t.stop() / args.steps
    print(json.dumps({"metric": "general batch circuits/s", "value": len(circs) / (ms * 1e-3), "unit": "circuits/s",
                      "ms_per_step": ms, "steps": args.steps, "path": P.qc_last_batch_path(),
                      "config": {"workload": "1024 circuits (QFT, brickwork depth 8, ansatz 4 layers), n in 10..16, "
                                             "observable ring ZZ + sum X, one launch (tables uploaded per call)"}}))


def run_block_bench(args):
    """Opt-in secondary measurement: a dense 5-qubit block (Haar 32x32) on spread qubits
    and on index bits 10..14, and a dense 6-qubit block (Haar 64x64), on a 28-qubit
    complex64 state, CUDA-core FMA (k_kq_native) vs tensor cores (TF32x3: the one-stage
    tile pass with box copies where the block's tile has a box plan, else k_block_tc;
    k_block_tc6)."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    n = args.qubits or 28
    hbm, bf16, _ = peaks()
    tf32_pk = tf32_peak()
    st = P.State(n, "c64").init_gaussian(7)
    stream = torch.cuda.current_stream()
    res = {}
    # spread qubits (index bits 24, 18, 13, 7, 1 at 28 qubits) and a block on index bits
    # 10..14
    cases = (("k5", 5, [3, 9, 14, 20, n - 2]), ("k5_mid", 5, [n - 15 + j for j in range(5)]),
             ("k6", 6, [3, 9, 14, 20, 23, n - 2]))
    for label, k, qs in cases:
        U = W.haar_unitaries(1, 1 << k, 11)[0]
        for name, prec in (("native", P.QC_PREC_NATIVE), ("tf32x3", P.QC_PREC_TF32X3)):
            for _ in range(max(args.warmup, 1)):
                P.qc_apply_fused_k(st.handle, qs, U, prec)
            torch.cuda.synchronize()
            t = StreamTimer(stream)
            t.start()
            for _ in range(args.steps):
                P.qc_apply_fused_k(st.handle, qs, U, prec)
            ms = t.stop() / args.steps
            # 2^k complex multiply-adds per amplitude, 8 flops each (x3 for the split)
            flops = 8.0 * (1 << k) * (1 << n) * (3 if prec == P.QC_PREC_TF32X3 else 1)
            gbs = 2 * 8 * (1 << n) / (ms * 1e-3) / 1e9
            tf = flops / (ms * 1e-3) / 1e12
            r = {"ms": ms, "gbs": gbs, "frac_hbm": gbs / hbm, "tflops": tf}
            if prec == P.QC_PREC_TF32X3:
                r["frac_tf32"] = tf / tf32_pk
            else:
                r["frac_alu"] = tf / ALU_PEAK_TF
            res["%s_%s" % (label, name)] = r
    print(json.dumps({"metric": "fused 5- and 6-qubit blocks on %d qubits" % n, "results": res,
                      "peaks": {"hbm_gbs": hbm, "tf32_tflops": tf32_pk, "alu_tflops": ALU_PEAK_TF,
                                "tf32_source": TF32_PEAK_SRC}}))


def run_qft_bench(args):
    """Opt-in secondary measurement: the 32-qubit QFT (544 gates) on the seeded Gaussian
    state, per-gate vs fused tile passes, complex64 (32 GiB) and complex128 (64 GiB)."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    n = args.qubits or 32
    hbm, _, _ = peaks()
    ops = W.qft(n)
    # per-gate sweeps: H moves the whole state, a controlled phase the quarter with both
    # bits set, a swap the half where the bits differ
    per_gate_sweeps = n + (n * (n - 1) / 2) / 4 + (n // 2) / 2
    circ = P.Circuit(n, ops)
    stream = torch.cuda.current_stream()
    res = {}
    for dt in ("c64", "c128"):
        st = P.State(n, dt).init_gaussian(3)
        sbytes = (1 << n) * (8 if dt == "c64" else 16)
        runs = [("fused", P.QC_RUN_FUSED, P.QC_PREC_NATIVE)]
        if dt == "c64":  # tensor-core stage passes (TF32x3)
            runs.append(("fused_tf32x3", P.QC_RUN_FUSED, P.QC_PREC_TF32X3))
        runs.append(("per_gate", P.QC_RUN_PER_GATE, P.QC_PREC_NATIVE))
        for mode_name, mode, prec in runs:
            if dt == "c128" and mode_name == "per_gate" and args.steps > 1:
                reps = 1
            else:
                reps = args.steps
            P.qc_run_circuit(st.handle, circ, None, mode, prec)  # warm-up
            torch.cuda.synchronize()
            t = StreamTimer(stream)
            t.start()
            for _ in range(reps):
                P.qc_run_circuit(st.handle, circ, None, mode, prec)
            ms = t.stop() / reps
            passes = P.qc_last_pass_count() if mode == P.QC_RUN_FUSED else None
            alg = 2 * sbytes * (passes if passes else per_gate_sweeps)
            gbs = alg / (ms * 1e-3) / 1e9
            res["%s_%s" % (dt, mode_name)] = {"ms": ms, "passes": passes, "algorithmic_gb": alg / 1e9,
                                              "gbs": gbs, "frac_hbm": gbs / hbm}
            if mode == P.QC_RUN_FUSED:
                res["%s_%s" % (dt, mode_name)]["path"] = P.qc_last_fused_path()
                res["%s_%s" % (dt, mode_name)]["stages"] = P.qc_last_stage_count()
        st.free()
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "QFT on %d qubits (%d gates)" % (n, len(ops)), "results": res,
                      "peaks": {"hbm_gbs": hbm}}))


def run_window_bench(args):
    """Opt-in secondary measurement: where the tensor-core stages pay.  540 Haar gates in
    brickwork order on a window of the lowest 5 or 10 qubits of a 28-qubit complex64
    state (deep stages: many gates per 5-bit block), on the CUDA-core tile passes and on
    the passes with tensor-core stages."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    n = args.qubits or 28
    _, bf16, src = peaks()
    sm_peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * 2070e6 / 1e12
    tf32_pk = tf32_peak()
    stream = torch.cuda.current_stream()
    st = P.State(n, "c64").init_gaussian(3)
    res = {}
    for width in (5, 10):
        ops = W.window_chain(n, n - width, width, 540, 7)
        circ = P.Circuit(n, ops)
        for name, prec in (("fp32", P.QC_PREC_NATIVE), ("tf32x3", P.QC_PREC_TF32X3)):
            P.qc_run_circuit(st.handle, circ, None, P.QC_RUN_FUSED, prec)  # warm-up
            torch.cuda.synchronize()
            t = StreamTimer(stream)
            t.start()
            for _ in range(args.steps):
                P.qc_run_circuit(st.handle, circ, None, P.QC_RUN_FUSED, prec)
            ms = t.stop() / args.steps
            gate_tf = len(ops) * 32.0 * (1 << n) / (ms * 1e-3) / 1e12
            r = {"ms": ms, "path": P.qc_last_fused_path(), "passes": P.qc_last_pass_count(),
                 "stages": P.qc_last_stage_count(), "gate_tflops_fp32_equivalent": gate_tf}
            if r["path"] == 2:
                tf = r["stages"] * 768.0 * (1 << n) / (ms * 1e-3) / 1e12
                r.update({"tf32_tflops": tf, "frac_tf32_peak": tf / tf32_pk})
            else:
                r.update({"frac_fp32_peak": gate_tf / sm_peak})
            res["w%d_%s" % (width, name)] = r
    st.free()
    print(json.dumps({"metric": "540 Haar gates on the lowest 5 / 10 of %d qubits (complex64)" % n,
                      "results": res, "peaks": {"fp32_tflops": sm_peak, "tf32_tflops": tf32_pk,
                                                "tf32_source": TF32_PEAK_SRC}}))


def run_adjoint_bench(args):
    """Opt-in secondary measurement: energy + full gradient of the 24-qubit, 10-layer
    ansatz (480 parameters, H = ring ZZ + sum X) by the adjoint sweep."""
    import paper_2503_03016_gb300 as P
    import torch
    torch.cuda.set_device(0)
    n, layers = 24, 10
    ops, params, terms, coeffs = W.adjoint_workload(n, layers, 5)
    circ = P.Circuit(n, ops)
    hbm, _, _ = peaks()
    # reverse sweep bytes: both dtypes run it as tile passes over psi and lambda together
    # (each pass reads and writes both states: 4 S per pass)
    res = {}
    for dt, code in (("c64", P.QC_C64), ("c128", P.QC_C128)):
        sbytes = (1 << n) * (8 if dt == "c64" else 16)
        P.qc_adjoint_grad(circ, params, terms, coeffs, code)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e, g = P.qc_adjoint_grad(circ, params, terms, coeffs, code)
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        passes = P.qc_last_pass_count()
        alg, form = 4 * sbytes * passes, "fused: %d tile passes over both states" % passes
        gbs = alg / (ms * 1e-3) / 1e9
        res[dt] = {"ms_energy_and_gradient": ms, "energy": e, "grad_norm": float(np.linalg.norm(g)),
                   "reverse_sweep": form, "reverse_sweep_algorithmic_gb": alg / 1e9, "gbs": gbs,
                   "frac_hbm": gbs / hbm}
    print(json.dumps({"metric": "adjoint gradient, %d qubits, %d gates, %d parameters" % (n, len(ops), len(params)),
                      "results": res, "peaks": {"hbm_gbs": hbm},
                      "note": "wall clock per synchronising call (forward pass, H psi and energy included); "
                              "bytes count the reverse sweep only"}))


def run_sweeps_bench(args):
    """Opt-in secondary measurement: each single-kernel step of the path on its own
    (28 qubits, complex64 and complex128, seeded Gaussian state) against the measured
    HBM bandwidth.  Algorithmic bytes: what the step must read and write at least."""
    import torch

    import paper_2503_03016_gb300 as P
    torch.cuda.set_device(0)
    n = args.qubits or 28
    hbm, _, _ = peaks()
    stream = torch.cuda.current_stream()
    U1 = W.haar_unitaries(1, 2, 21)[0]
    U2 = W.haar_unitaries(1, 4, 22)[0]
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    shots = 1_000_000
    u = torch.tensor(W.uniforms(shots, 102), device="cuda")
    idx = torch.empty(shots, dtype=torch.int64, device="cuda")  # 8-byte outcome indices
    zz = W.zz_terms(n, ring=False)
    N = 1 << n
    res = {}
    for dt in ("c64", "c128"):
        st = P.State(n, dt).init_gaussian(3)
        S = N * (8 if dt == "c64" else 16)
        probs = torch.empty(N, dtype=torch.float64, device="cuda")
        h = st.handle
        cases = [
            ("init_basis", lambda: P.qc_state_init_basis(h, 0), S),
            ("init_gaussian", lambda: P.qc_state_init_gaussian(h, 3), S),
            ("1q_dense_q5", lambda: P.qc_apply_1q(h, 5, U1), 2 * S),
            ("1q_dense_q0", lambda: P.qc_apply_1q(h, 0, U1), 2 * S),
            ("1q_dense_bit0", lambda: P.qc_apply_1q(h, n - 1, U1), 2 * S),
            ("2q_dense", lambda: P.qc_apply_2q(h, 3, 17, U2), 2 * S),
            ("2q_dense_bit0", lambda: P.qc_apply_2q(h, 9, n - 1, U2), 2 * S),
            ("cnot", lambda: P.qc_apply_ctrl(h, [2], None, 9, X), S),  # the half with the control set
            ("cz", lambda: P.qc_apply_ctrl(h, [2], None, 9, Z), S / 2),  # the quarter with both bits set
            ("outcome_prob", lambda: P.qc_outcome_prob(h, 7, 0), S),
            ("probs", lambda: P.qc_probs(h, probs), S + 8 * N),
            ("sample_1e6", lambda: P.qc_sample(h, u, shots, idx), S),
            ("expect_zz_chain", lambda: P.qc_expect_pauli(h, zz), S),
            # P(outcome) (read S), then keep half (read S/2) and write the whole state
            ("collapse", lambda: P.qc_collapse(h, 7, 0), 2.5 * S),
        ]
        out = {}
        for name, fn, alg in cases:
            fn()
            torch.cuda.synchronize()
            t = StreamTimer(stream)
            t.start()
            for _ in range(args.steps):
                fn()
            ms = t.stop() / args.steps
            gbs = alg / (ms * 1e-3) / 1e9
            out[name] = {"ms": ms, "algorithmic_gb": alg / 1e9, "gbs": gbs, "frac_hbm": gbs / hbm}
        res[dt] = out
        st.free()
        del probs
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "single-kernel steps on %d qubits" % n, "results": res, "peaks": {"hbm_gbs": hbm},
                      "l2": "state (2 GiB / 4 GiB) larger than L2"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="fused", choices=["fused", "per_gate"])
    ap.add_argument("--prec", default="auto", choices=["auto", "native", "tf32x3"],
                    help="fused passes: auto (the faster of the two for the circuit, timed once), CUDA-core "
                         "(native) or tensor-core stages (tf32x3)")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-gates", type=int, default=16)
    ap.add_argument("--cpu-single-gates", type=int, default=2)
    ap.add_argument("--ref-gates", type=int, default=8)
    ap.add_argument("--batch-range", default=None, help="batch workload: profile only circuits with LO-HI qubits")
    ap.add_argument("--batch-count", type=int, default=0, help="batch workload: at most this many of them")
    ap.add_argument("--qubits", type=int, default=None,
                    help="register size (default: 28 brickwork and block, 32 QFT); smaller for profiling")
    ap.add_argument("--workload", default="brickwork",
                    choices=["brickwork", "batch", "batch_general", "block", "qft", "adjoint", "sweeps", "window"],
                    help="batch: opt-in secondary measurement of the batched launch")
    args = ap.parse_args()
    global N_QUBITS
    N_QUBITS = args.qubits or 28
    if args.workload == "batch" and args.impl == "ours":
        run_batch_bench(args)
    elif args.workload == "batch_general" and args.impl == "ours":
        run_batch_general_bench(args)
    elif args.workload == "block" and args.impl == "ours":
        run_block_bench(args)
    elif args.workload == "qft" and args.impl == "ours":
        run_qft_bench(args)
    elif args.workload == "adjoint" and args.impl == "ours":
        run_adjoint_bench(args)
    elif args.workload == "sweeps" and args.impl == "ours":
        run_sweeps_bench(args)
    elif args.workload == "window" and args.impl == "ours":
        run_window_bench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
