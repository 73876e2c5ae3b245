"""Benchmark: batched gradients of the paper's circuit workloads on one GB300.

Default workload (one step = one full gradient): the 28-qubit multi-contracted
VQE -- 8 layers of Ry on every qubit + CNOT ladder (224 parameters), the Eq. 2
exciton Hamiltonian over nearest and next-nearest pairs (268 Pauli terms,
synthetic coefficients), 8 reference states of 2^28 complex64 amplitudes
(2 GiB each) in device memory -- by the adjoint sweep of tile passes.
Inputs are seeded and synthetic.

Printed (one JSON line on rank 0): gradients/s (value), the HBM roofline of
the dominant kernel (the reverse tile passes) and of gate application (the
identity-layout forward passes), the CPU oracle timed on the host cores
(extrapolated from a bounded sample), an end-to-end number through the C ABI
with host buffers, and under ``forms`` the 8-qubit MC-VQE (585 shifted
circuits in one batched launch; adjoint; complex128; the plain
one-circuit-per-launch complex128 form) and the 20-qubit circuit-learning
gate application.

``--workload`` selects another configuration (mcvqe8, qcl20, qcl-uneven,
ddcl).  ``--impl reference`` times the CPU oracle (the reference arm: there
is no runnable reference implementation, only the paper) on the same
workload.  Multi-GPU: ``--gpus N`` without a torchrun environment starts N
ranks itself under ``torch.distributed.run``; every rank runs its own replica
of the workload and the value is the gradients of all ranks over the slowest
rank's time.  ``--workload mcvqe8 --split vqpu`` instead splits one
parameter-shift batch into one contiguous segment per rank with one
allgather of the energies (the paper's virtual-QPU split, Sec. 4.1).
"""
from __future__ import annotations

import argparse
import json
import os
import socket
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "gradients/sec & shifted circuits/sec, batched/adjoint vs plain; % HBM roofline"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the
# 28-qubit gradient's reverse sweep, the 16 k_tile_rev launches of one
# adjoint at tile shape (10, 4) with stored states every second pass, summed
# from one ncu capture of `bench.py --tile-shape 10,4 --steps 1 --warmup 1
# --no-extras`.  It is reported only while the library sources hash to the
# digest they had when it was taken (a changed kernel gives null).
REVERSE_TRAFFIC = {"workload": "mcvqe28", "tile_bits": 10, "reg_bits": 4, "checkpoint_every": 2,
                   "csrc_sha256": "3be433daaaea0c271931339ce6c6b2d4bd0f76597376013fa58373f7f09f626b",
                   "bytes": 961372915968}


def csrc_digest() -> str:
    """SHA-256 over the library's C++/CUDA sources, in name order."""
    import hashlib
    d = os.path.join(ROOT, "paper_2406_03466_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh", ".cpp", ".h")):
            h.update(name.encode())
            with open(os.path.join(d, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()


def reverse_traffic(w, tile_bits, reg_bits, every):
    """The captured reverse-sweep traffic when it applies to this run, else None."""
    t = REVERSE_TRAFFIC
    if t["bytes"] is None or w.name != t["workload"] or (tile_bits, reg_bits) != (
            t["tile_bits"], t["reg_bits"]) or every != t["checkpoint_every"]:
        return None
    return t["bytes"] if csrc_digest() == t["csrc_sha256"] else None
WORKLOAD_MCVQE8 = ("mcvqe8: multi-contracted VQE gradient, 8 qubits, 4 layers Ry + CNOT ladder "
            "(32 params), 128-term Eq. 2 Hamiltonian, 9 references, 585 shifted circuits")
L2_FLUSH_BYTES = 256 << 20   # larger than the 126.5 MiB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--workload", default="mcvqe28",
                    choices=["mcvqe8", "qcl20", "mcvqe28", "qcl-uneven", "ddcl"],
                    help="mcvqe28 (default): adjoint gradient of the 28-qubit MC-VQE (8 states "
                         "of 2 GiB in device memory); qcl20: the same for the 20-qubit circuit "
                         "learning; mcvqe8: batched parameter-shift gradient of the 8-qubit "
                         "MC-VQE (on chip); "
                         "qcl-uneven: adjoint gradients of 8 circuit-learning circuits of "
                         "20-24 qubits and depth 4-12 in one graph launch; ddcl: data-driven "
                         "circuit learning (Sec. 4.2) at 26 qubits (--qubits for 20-24)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--split", default="replicas", choices=["replicas", "vqpu"],
                    help="multi-GPU mode: replicas (default; every rank its own gradients) or "
                         "vqpu (mcvqe8 only: one parameter-shift batch split into one segment "
                         "per rank, one allgather of energies, Sec. 4.1)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true", help="skip adjoint/plain/c128 side runs")
    ap.add_argument("--energy-shape", default="",
                    help="mcvqe8 only: 'R,T' pins the energy kernel to R register bits and T "
                         "threads per block instead of autotuning (for profiler captures)")
    ap.add_argument("--tile-shape", default="",
                    help="qcl20 / mcvqe28 only: 't,R' pins the tile passes to 2^t amplitudes and "
                         "R register bits instead of autotuning (for profiler captures)")
    ap.add_argument("--tensor-blocks", action="store_true",
                    help="qcl20 / mcvqe28 with --tile-shape t,4 (t = 11 or 12): forward passes as "
                         "dense 16x16 blocks on the tensor cores (for profiler captures)")
    ap.add_argument("--qubits", type=int, default=0,
                    help="qcl20 / mcvqe28 only: the same workload family at this qubit count "
                         "(a smaller case for profiler captures; not a bench line)")
    return ap.parse_args()


def job_throughput(t_dev, units_per_rank, dist, device):
    """Whole-job rate of a replicas run: every rank did `units_per_rank` units
    in its own t_dev seconds; the job took the slowest rank's time."""
    import torch
    world = 1
    if dist:
        t = torch.tensor([t_dev], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
        world = dist.get_world_size()
    return world * units_per_rank / t_dev, t_dev


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------- CPU oracle

def cpu_baseline(seconds: float):
    """The oracle's parameter-shift gradient of the same workload, as it stands,
    repeated for about `seconds` on the host cores."""
    import oracle
    w = wl.config(1)
    threads = oracle.max_threads()
    oracle.grad_param_shift(w)  # load + warm
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.grad_param_shift(w)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "gradients/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} full gradients of the benchmark workload (585 circuits each, "
                      f"complex128, OpenMP over circuits) in {dt:.1f} s"}


# -------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="svclocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- timing

def timed_loop(fn, steps, flush, stream):
    """Device time of `steps` calls of fn, L2 flushed (untimed) before each."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3  # seconds


def algorithmic_flops(w, n_slots):
    """FLOPs of one launch of the batched energy kernel, counted from the
    unfused circuit: 6 per amplitude per rotation (a real 2x2-structured
    rotation on a complex amplitude), 0 per CNOT, and per Pauli term 8 per
    amplitude (the complex product conj(psi_{j^x}) psi_j and its signed sum)."""
    dim = 1 << w.n_qubits
    rot = sum(1 for g in w.gates if g.op in ("RX", "RY", "RZ", "ENC_RY_ASIN", "ENC_RZ_ACOS_SQ"))
    per_circuit = 6 * rot * dim + 8 * w.n_terms * dim
    return per_circuit * n_slots


def fp32_peak_tflops():
    """FP32 FMA peak from unit counts and the maximum SM clock: 152 SMs x 128
    lanes x 2 FLOP x 2.07 GHz."""
    return 152 * 128 * 2 * 2.07e9 / 1e12


def measured_hbm_gbs():
    """The measured copy bandwidth of the GB300s, else the
    recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def forward_passes_roofline(sv, w, dev, flush, stream, reps=5, opts=None):
    """Times the forward simulation of workload `w` (all instances, states in
    device memory) and reports it against the HBM roofline: each tile pass
    reads and writes every state once, the |ref> initialisation writes them."""
    import torch
    d = 0 if w.inputs is None else 1
    circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, d)
    # the states come back in qubit order: identity-layout passes
    o = sv.plan_opts() if opts is None else opts
    ident = sv.plan_opts(o.reg_bits, o.threads_per_block, bool(o.no_fusion), o.epilogue,
                         o.tile_bits, o.coalesce_bits, no_relabel=True,
                         tensor_blocks=bool(o.tensor_blocks))
    info = sv.sv_plan_info(circ, "c64", ident)
    n, I = w.n_qubits, w.n_instances
    st = sv.sv_alloc(n, I, "c64", device=dev)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev).reshape(1, -1)
    xin = None if w.inputs is None else torch.as_tensor(w.inputs, device=dev)
    slots = sv.make_slots([(0, 0, -1, i if d else -1, int(w.refs[i]), 0.0) for i in range(I)])
    fn = lambda: sv.sv_apply_circuit_batch(st, [circ], slots, theta, xin, opts)  # noqa: E731
    fn()
    t = timed_loop(fn, reps, flush, stream) / reps
    nbytes = (2 * info["n_passes"] + 1) * I * (8 << n)
    peak, src = measured_hbm_gbs()
    achieved = nbytes / t / 1e9
    st.free()
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": f"{'k_tile_fwd_tc' if o.tensor_blocks else 'k_tile_fwd'} x "
                      f"{info['n_passes']} identity-layout tile passes of "
                      f"2^{info['tile_bits']} amplitudes ({w.name}: {I} states of {n} qubits)",
            "forward_ms": t * 1e3, "bytes_per_forward": nbytes, "peak_source": src}


def adjoint_phases(sv, w, prob, theta, out, info, flush, stream, reps, step=None, reg_bits=None):
    """Per-phase CUDA-event times of the device-memory adjoint (the library's
    phase timer records events on the call's stream), each step after an L2
    flush; the reverse tile passes are the dominant kernel: per pass they
    read psi (or its stored state) and lambda of every state and write
    lambda, and psi unless the next pass restarts from a stored state (the
    library reports the bytes of the passes it launched)."""
    import torch
    sv.sv_phase_timing(True)
    ph = {"forward_ms": 0.0, "h_ms": 0.0, "reverse_ms": 0.0}
    for _ in range(reps):
        flush.fill_(1.0)
        if step is None:
            sv.sv_grad_adjoint(prob, theta, None, *out)
        else:
            step()
        got = sv.sv_last_phase_ms()
        for k in ph:
            ph[k] += got[k] / reps
    sv.sv_phase_timing(False)
    torch.cuda.synchronize()
    n, I = w.n_qubits, w.n_instances
    state = I * (8 << n)
    last = sv.sv_last_adjoint_info()
    nbytes = last["reverse_bytes"]
    peak, src = measured_hbm_gbs()
    achieved = nbytes / (ph["reverse_ms"] * 1e-3) / 1e9
    # the gradient's own forward passes (the same relabeling plan), 16 B per
    # amplitude per pass; the phase also holds |ref>, the group matrices and
    # the stored checkpoint copies
    fwd_bytes = 2 * info["n_passes"] * state
    traffic = reverse_traffic(w, info["tile_bits"], reg_bits, last["checkpoint_every"])
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": f"k_tile_rev x {info['n_passes']} reverse tile passes of "
                      f"2^{info['tile_bits']} amplitudes ({w.name}: {I} states of {n} qubits; "
                      "psi and lambda read and lambda written per pass, psi written "
                      "unless the next pass restarts from a stored state)",
            "reverse_ms": ph["reverse_ms"], "bytes_per_reverse": nbytes,
            "checkpoint_every": last["checkpoint_every"], "peak_source": src,
            "phases_ms": ph,
            "forward_phase_frac": fwd_bytes / (ph["forward_ms"] * 1e-3) / 1e9 / peak}


def cpu_baseline_device_memory(w, seconds):
    """The oracle on a bounded sample of a large workload: whole circuits
    (each with its full <H>) for about `seconds`, scaled to parameter-shift
    gradients (2P + 1 circuits per instance)."""
    import oracle
    threads = oracle.max_threads()
    # Above 22 qubits one oracle circuit per core already runs for minutes:
    # time the same family at 20 qubits and scale by the state size and the
    # gate + term count.
    ws, scale = w, 1.0
    if w.n_qubits > 22:
        ws = wl.mcvqe(20, w.meta.get("layers", 8), w.meta.get("pairs", "nn+nnn"),
                      n_refs=w.n_instances)
        cost = lambda x: (1 << x.n_qubits) * (len(x.gates) + 3 * x.n_terms)  # noqa: E731
        scale = cost(w) / cost(ws)
    t0 = time.perf_counter()
    n_done = 0
    while True:
        k = max(1, threads)
        oracle.energies(ws, None, np.arange(k) % ws.n_instances)
        n_done += k
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    per_circuit = dt / n_done * scale
    circuits = w.n_slots_param_shift
    how = (f"{n_done} full circuits of {ws.name} in {dt:.1f} s" +
           (f", scaled x{scale:.0f} to {w.name} by 2^n x (gates + 3 terms)" if ws is not w else "") +
           f"; scaled to {circuits} circuits per parameter-shift gradient (extrapolated)")
    return {"value": 1.0 / (per_circuit * circuits), "unit": "gradients/s", "cores": threads,
            "kind": "oracle", "sample": how}


def device_workload(args):
    """Config 4 (qcl20) or 5 (mcvqe28), or the same family at --qubits."""
    w = wl.config(3 if args.workload == "qcl20" else 4)
    if args.qubits:
        w = (wl.qcl(args.qubits, w.meta.get("layers", 10), w.n_instances) if args.workload == "qcl20"
             else wl.mcvqe(args.qubits, w.meta.get("layers", 8), w.meta.get("pairs", "nn+nnn"),
                           n_refs=w.n_instances))
    return w


def device_workload_name(w):
    return (f"{w.name}: adjoint gradient, {w.n_instances} states of {w.n_qubits} qubits in "
            f"device memory, {w.n_params} params")


def run_device_memory(args, sv, dev, stream, dist, world, rank):
    """Adjoint gradient of a workload whose states live in device memory."""
    import torch
    w = device_workload(args)
    pinned = None
    if args.tile_shape:
        tile_bits, R = (int(x) for x in args.tile_shape.split(","))
        pinned = sv.plan_opts(reg_bits=R, tile_bits=tile_bits, tensor_blocks=args.tensor_blocks)
    prob = sv.Problem.from_spec(w, "c64", device=dev, opts=pinned)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev)
    out = sv._outputs(prob, dev, None, None, None)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tc = bool(args.tensor_blocks)
    if pinned is None:
        # tile shape (tile bits, register bits, tensor-core forward passes)
        # picked by timing
        sv.sv_autotune(prob, theta, 2)
        tile_bits, R, tc, _ = sv.sv_tuned_tile(prob, 2)
    opts = sv.plan_opts(reg_bits=R, tile_bits=tile_bits, tensor_blocks=tc)

    def step():
        sv.sv_grad_adjoint(prob, theta, None, *out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    t_dev = timed_loop(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    gps, t_dev = job_throughput(t_dev, args.steps, dist, dev)
    d = 0 if w.inputs is None else 1
    info = sv.sv_plan_info(sv.Circuit(w.n_qubits, w.gates, w.n_params, d), "c64", opts)
    hinfo = sv.sv_h_plan_info(sv.PauliSum(w.n_qubits, w.pauli_letters, w.pauli_coeffs), "c64")
    result = {"metric": METRIC, "value": gps, "unit": "gradients/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
              "config": {"workload": device_workload_name(w), "tile_passes": info["n_passes"],
                         "tuned_tile": {"tile_bits": tile_bits, "reg_bits": R,
                                        "tensor_blocks": tc},
                         "h_passes": hinfo["n_passes"],
                         "l2": "states larger than L2; 256 MiB flush before each step",
                         "parallelism": f"replicas x{world}"},
              # per adjoint: group matrices, |ref>, forward and reverse passes, the
              # passes of lambda = H psi, per-slot gradients, combination
              "gpu_launches": args.steps * (2 * info["n_passes"] + hinfo["n_passes"] + 4),
              "clocks": clk, "wall_s_timed_region": t_wall}
    if rank == 0:
        result["roofline"] = adjoint_phases(sv, w, prob, theta, out, info, flush, stream,
                                            reps=2 if w.n_qubits > 24 else 5, reg_bits=R)
        result["roofline_forward"] = forward_passes_roofline(sv, w, dev, flush, stream,
                                                             reps=3 if w.n_qubits > 24 else 5,
                                                             opts=opts)
        # end to end through the C ABI with host buffers: theta from host
        # memory in, loss + gradient + instance energies back to host memory
        # (sv_grad_adjoint_host returns once they are there)
        th_host = torch.as_tensor(w.theta, dtype=torch.float64)
        g_host = torch.empty(w.n_params, dtype=torch.float64)
        l_host = torch.empty(1, dtype=torch.float64)
        e_host = torch.empty(w.n_instances, dtype=torch.float64)
        sv.sv_grad_adjoint_host(prob, th_host, e_host, l_host, g_host, stream=stream)
        reps = max(2, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(reps):
            sv.sv_grad_adjoint_host(prob, th_host, e_host, l_host, g_host, stream=stream)
        result["e2e"] = {"value": reps / (time.perf_counter() - t0), "unit": "gradients/s",
                         "h2d_bytes_per_step": 8 * w.n_params,
                         "d2h_bytes_per_step": 8 * (w.n_params + 1 + w.n_instances),
                         "timing": "host wall clock per step; sv_grad_adjoint_host returns once "
                                   "the results are in host memory"}
        result["cpu_baseline"] = cpu_baseline_device_memory(w, min(args.cpu_seconds, 10.0))
        if not args.no_extras and not args.qubits:
            forms = {}
            if args.workload == "mcvqe28":
                # gate application with complex Rx.Rz.Rx groups: the 20-qubit
                # circuit-learning batch (64 states, 512 MiB), register
                # stages and the same stages as tensor-core blocks
                q20 = wl.config(3)
                forms["qcl20_gate_application"] = forward_passes_roofline(
                    sv, q20, dev, flush, stream, opts=sv.plan_opts(reg_bits=4, tile_bits=11))
                forms["qcl20_gate_application_tensor_blocks"] = forward_passes_roofline(
                    sv, q20, dev, flush, stream,
                    opts=sv.plan_opts(reg_bits=4, tile_bits=12, tensor_blocks=True))
            _, _, _, side = mcvqe8_side(sv, dev, stream, flush, 2000)
            side["cpu_baseline"] = cpu_baseline(min(args.cpu_seconds, 3.0))
            forms["mcvqe8"] = side
            result["forms"] = forms
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# Table 3 of the paper (DDCL gradient, 10 layers, one V100 per virtual QPU,
# Aer + cuStateVec): runtime at one GPU from the printed fits, 10^intercept s.
PAPER_DDCL_1GPU_S = {20: 418.8, 22: 532.1, 24: 907.8, 26: 2500.0}


def cpu_baseline_ddcl(w, seconds):
    """The oracle on whole DDCL circuits at 20 qubits for about `seconds`,
    scaled by 2^n x gates to the workload and to the 2P + 1 circuits of one
    parameter-shift gradient (extrapolated)."""
    import oracle
    ws = wl.ddcl(min(20, w.n_qubits), w.meta.get("layers", 10))
    t0 = time.perf_counter()
    n_done = 0
    while True:
        oracle.output_distribution(ws)
        n_done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    scale = ((1 << w.n_qubits) * len(w.gates)) / ((1 << ws.n_qubits) * len(ws.gates))
    per_grad = dt / n_done * scale * (2 * w.n_params + 1)
    return {"value": 1.0 / per_grad, "unit": "gradients/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"{n_done} whole circuits of {ws.name} in {dt:.1f} s (one circuit at a "
                      f"time), scaled x{scale:.0f} by 2^n x gates to {w.name} and to "
                      f"{2 * w.n_params + 1} circuits per parameter-shift gradient (extrapolated)"}


def run_ddcl(args, sv, dev, stream, dist, world, rank):
    """Adjoint gradient of the JS divergence of data-driven circuit learning."""
    import torch
    n = args.qubits or 26
    w = wl.ddcl(n, 10)
    prob = sv.Problem.from_spec(w, "c64", device=dev)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev)
    target = torch.as_tensor(w.target_dist, dtype=torch.float64, device=dev)
    js = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(w.n_params, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        sv.sv_grad_ddcl(prob, theta, target, js, grad)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    t_dev = timed_loop(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    gps, t_dev = job_throughput(t_dev, args.steps, dist, dev)
    opts = sv.plan_opts(reg_bits=4, tile_bits=11)
    info = sv.sv_plan_info(sv.Circuit(n, w.gates, w.n_params, 0), "c64", opts)
    paper_s = PAPER_DDCL_1GPU_S.get(n)
    result = {"metric": METRIC, "value": gps, "unit": "gradients/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
              "config": {"workload": ddcl_workload_name(w), "tile_passes": info["n_passes"],
                         "l2": f"one {8 << n >> 20} MiB state; 256 MiB flush before each step",
                         "parallelism": f"replicas x{world}"},
              "gpu_launches": args.steps * (2 * info["n_passes"] + 5),
              "clocks": clk, "wall_s_timed_region": t_wall,
              "paper_context": None if paper_s is None else {
                  "gradients_per_s": 1.0 / paper_s,
                  "source": "Table 3 fit intercept at one GPU: NVIDIA V100, Aer + cuStateVec, "
                            f"parameter shift over {2 * w.n_params} circuits, {n} qubits, "
                            "10 layers (another machine, another layer layout and target)"}}
    if rank == 0:
        result["roofline"] = adjoint_phases(sv, w, prob, theta, None, info, flush, stream,
                                            reps=3, step=step)
        th_host = torch.as_tensor(w.theta, dtype=torch.float64).pin_memory()
        g_host = torch.empty(w.n_params, dtype=torch.float64).pin_memory()
        th_dev = torch.empty_like(theta)
        t0 = time.perf_counter()
        reps = max(1, args.steps // 2)
        for _ in range(reps):
            th_dev.copy_(th_host, non_blocking=True)
            sv.sv_grad_ddcl(prob, th_dev, target, js, grad)
            g_host.copy_(grad, non_blocking=True)
            stream.synchronize()
        result["e2e"] = {"value": reps / (time.perf_counter() - t0), "unit": "gradients/s",
                         "h2d_bytes_per_step": 8 * w.n_params, "d2h_bytes_per_step": 8 * w.n_params}
        result["cpu_baseline"] = cpu_baseline_ddcl(w, min(args.cpu_seconds, 10.0))
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def ddcl_workload_name(w):
    return (f"{w.name}: data-driven circuit learning gradient (JS divergence, Eq. 3), "
            f"{w.n_qubits} qubits, {w.meta['layers']} layers, {w.n_params} params, adjoint")


def uneven_workload_name(ws):
    return (f"qcl-uneven: adjoint gradients of {len(ws)} circuit-learning circuits (n, layers) = "
            + ", ".join(f"({w.n_qubits},{w.meta['layers']})" for w in ws)
            + f", {ws[0].n_instances} inputs each, one CUDA graph launch (persistent sweeps)")


def uneven_cost_model(w):
    return (1 << w.n_qubits) * (len(w.gates) + 3 * w.n_terms)


def cpu_baseline_uneven(ws, seconds):
    """The oracle on whole circuits of the batch's smallest circuit for about
    `seconds`, scaled by 2^n x (gates + 3 terms) to every circuit of the
    batch and to one parameter-shift gradient per circuit (extrapolated)."""
    import oracle
    threads = oracle.max_threads()
    ws0 = min(ws, key=uneven_cost_model)
    t0 = time.perf_counter()
    n_done = 0
    while True:
        k = max(1, threads)
        oracle.energies(ws0, None, np.arange(k) % ws0.n_instances)
        n_done += k
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    per = dt / n_done / uneven_cost_model(ws0)
    total = sum(w.n_slots_param_shift * uneven_cost_model(w) * per for w in ws)
    return {"value": len(ws) / total, "unit": "gradients/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_done} full circuits of {ws0.name} in {dt:.1f} s; scaled by 2^n x "
                      f"(gates + 3 terms) to the {len(ws)} circuits' parameter-shift gradients "
                      "(extrapolated)"}


def run_uneven(args, sv, dev, stream, dist, world, rank):
    """Adjoint gradients of the uneven circuit-learning batch in one graph launch."""
    import torch
    ws = wl.qcl_uneven()
    probs = [sv.Problem.from_spec(w, "c64", device=dev) for w in ws]
    thetas = [torch.as_tensor(w.theta, dtype=torch.float64, device=dev) for w in ws]
    outs = sv.sv_grad_adjoint_multi(probs, thetas)  # plans, runs, captures
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        sv.sv_grad_adjoint_multi(probs, thetas, outputs=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    t_dev = timed_loop(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    gps, t_dev = job_throughput(t_dev, args.steps * len(ws), dist, dev)
    # algorithmic HBM bytes of one step: |ref> writes, forward passes (read +
    # write), lambda = H psi passes, reverse passes (psi and lambda, read + write)
    nbytes, launches, max_pass = 0, 0, 0
    for w in ws:
        circ = sv.Circuit(w.n_qubits, w.gates, w.n_params, 1)
        npass = sv.sv_plan_info(circ, "c64")["n_passes"]
        nh = sv.sv_h_plan_info(sv.PauliSum(w.n_qubits, w.pauli_letters, w.pauli_coeffs))["n_passes"]
        state = w.n_instances * (8 << w.n_qubits)
        nbytes += state * (1 + 2 * npass + 2 + 3 * (nh - 1) + 4 * npass)
        launches += 4 + nh
        max_pass = max(max_pass, npass)
    launches += 2  # the two persistent sweeps (forward, reverse) of all circuits
    peak, src = measured_hbm_gbs()
    achieved = nbytes * args.steps / t_dev / 1e9 / world
    result = {"metric": METRIC, "value": gps, "unit": "gradients/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
              "config": {"workload": uneven_workload_name(ws),
                         "l2": "states larger than L2; 256 MiB flush before each step",
                         "parallelism": f"replicas x{world}"},
              "gpu_launches": args.steps * launches,
              "clocks": clk, "wall_s_timed_region": t_wall,
              "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "traffic": None,
                           "kernel": "whole step: persistent forward sweep (k_tile_sweep) + k_tile_h "
                                     "+ persistent reverse sweep of all circuits, one graph",
                           "bytes_per_step": nbytes, "peak_source": src}}
    if rank == 0:
        th_host = [torch.as_tensor(w.theta, dtype=torch.float64).pin_memory() for w in ws]
        g_host = [torch.empty(w.n_params, dtype=torch.float64).pin_memory() for w in ws]
        t0 = time.perf_counter()
        reps = max(1, args.steps // 2)
        for _ in range(reps):
            for th_d, th_h in zip(thetas, th_host):
                th_d.copy_(th_h, non_blocking=True)
            step()
            for o, gh, w in zip(outs, g_host, ws):
                gh.copy_(o[2][: w.n_params], non_blocking=True)
            stream.synchronize()
        result["e2e"] = {"value": reps * len(ws) / (time.perf_counter() - t0), "unit": "gradients/s",
                         "h2d_bytes_per_step": sum(8 * w.n_params for w in ws),
                         "d2h_bytes_per_step": sum(8 * w.n_params for w in ws)}
        result["cpu_baseline"] = cpu_baseline_uneven(ws, min(args.cpu_seconds, 10.0))
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def mcvqe8_side(sv, dev, stream, flush, steps, extras=True):
    """The 8-qubit MC-VQE batched parameter-shift gradient (585 circuits in one
    energy launch + the dependent assembly) and its side forms: the energy
    kernel alone against the FP32 ALU roof, the host-buffer entry point, the
    adjoint, both complex128 forms and the plain one-circuit-per-launch
    complex128 form.  Returns (problem, outputs, dict)."""
    import torch
    w = wl.config(1)
    B = w.n_slots_param_shift
    prob = sv.Problem.from_spec(w, "c64", device=dev)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev)
    out = sv._outputs(prob, dev, None, None, None)
    e_buf = torch.empty(B, dtype=torch.float64, device=dev)
    sv.sv_autotune(prob, theta)
    tuned = {"energy": sv.sv_tuned_shape(prob, 1)[:2], "adjoint": sv.sv_tuned_shape(prob, 2)[:2]}
    fn = lambda: sv.sv_grad_param_shift(prob, theta, *out)  # noqa: E731
    for _ in range(20):
        fn()
    res = {"workload": WORKLOAD_MCVQE8, "circuits_per_gradient": B,
           "tuned_shape_c64": {k: {"reg_bits": v[0], "threads_per_block": v[1]}
                               for k, v in tuned.items()}}
    t = timed_loop(fn, steps, flush, stream)
    res["gradients_per_s"] = steps / t
    res["shifted_circuits_per_s"] = steps / t * B
    # dominant kernel alone: the batched energies of all 585 circuits
    k_steps = max(200, steps // 4)
    fn = lambda: sv.sv_param_shift_energies(prob, theta, e_buf)  # noqa: E731
    for _ in range(20):
        fn()
    t_k = timed_loop(fn, k_steps, flush, stream) / k_steps
    flops = algorithmic_flops(w, B)
    peak = fp32_peak_tflops()
    achieved = flops / t_k / 1e12
    res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak, "traffic": None,
                       "kernel": f"k_energy<float,{tuned['energy'][0]}> (batched shifted-circuit "
                                 "energies; the gradient assembly follows as a dependent launch)",
                       "kernel_us": t_k * 1e6,
                       "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    # end to end through the C ABI: theta from host memory in, loss +
    # gradient + energies back to host memory, every step
    th_host = torch.as_tensor(w.theta, dtype=torch.float64).pin_memory()
    g_host = torch.empty(w.n_params, dtype=torch.float64).pin_memory()
    l_host = torch.empty(1, dtype=torch.float64).pin_memory()
    e_host = torch.empty(w.n_instances, dtype=torch.float64).pin_memory()
    e2e_steps = max(200, steps // 4)
    # the C-ABI call itself, arguments marshalled once (the binding's per-call
    # argument checks are Python work, not the library's)
    import ctypes
    c_fn = sv.library().sv_grad_param_shift_host
    c_args = (ctypes.byref(prob.struct), ctypes.c_void_p(th_host.data_ptr()),
              ctypes.c_void_p(e_host.data_ptr()), ctypes.c_void_p(l_host.data_ptr()),
              ctypes.c_void_p(g_host.data_ptr()), ctypes.c_void_p(stream.cuda_stream))

    def e2e_step():
        if c_fn(*c_args) != sv.SV_OK:
            raise RuntimeError(sv.sv_last_error())

    for _ in range(10):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    t_e2e = time.perf_counter() - t0
    res["e2e"] = {"value": e2e_steps / t_e2e, "unit": "gradients/s",
                  "h2d_bytes_per_step": 8 * w.n_params,
                  "d2h_bytes_per_step": 8 * (w.n_params + 1 + w.n_instances),
                  "timing": "host wall clock per step of the C-ABI call "
                            "sv_grad_param_shift_host (returns once the results are in host "
                            "memory), arguments marshalled once"}
    if extras:
        n = max(200, steps // 4)
        fn = lambda: sv.sv_grad_adjoint(prob, theta, None, *out)  # noqa: E731
        for _ in range(20):
            fn()
        res["adjoint_c64_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
        prob128 = sv.Problem.from_spec(w, "c128", device=dev)
        out128 = sv._outputs(prob128, dev, None, None, None)
        sv.sv_autotune(prob128, theta)
        fn = lambda: sv.sv_grad_param_shift(prob128, theta, *out128)  # noqa: E731
        for _ in range(20):
            fn()
        res["batched_c128_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
        fn = lambda: sv.sv_grad_adjoint(prob128, theta, None, *out128)  # noqa: E731
        for _ in range(20):
            fn()
        res["adjoint_c128_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
        # the plain form is host-driven (one launch per gate and term): wall clock
        sv.sv_grad_param_shift_plain(prob128, theta, *out128)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 2
        for _ in range(reps):
            sv.sv_grad_param_shift_plain(prob128, theta, *out128)
        torch.cuda.synchronize()
        res["plain_c128_gradients_per_s"] = reps / (time.perf_counter() - t0)
        res["plain_c128_launches_per_gradient"] = B * (1 + len(w.gates) + w.n_terms) + 1
    return prob, theta, out, res


def run_mcvqe8(args, sv, dev, stream, dist, world, rank):
    """The 8-qubit batched parameter-shift gradient as the bench line
    (replicas, or --split vqpu: one batch split over the ranks)."""
    import torch
    w = wl.config(1)
    B = w.n_slots_param_shift
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    shape_opts = None
    if args.energy_shape:
        R_, T_ = (int(x) for x in args.energy_shape.split(","))
        shape_opts = sv.plan_opts(reg_bits=R_, threads_per_block=T_)
    prob = sv.Problem.from_spec(w, "c64", device=dev, opts=shape_opts)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev)
    out = sv._outputs(prob, dev, None, None, None)
    if shape_opts is None:
        sv.sv_autotune(prob, theta)
    vqpu_split = args.split == "vqpu" and dist is not None
    if vqpu_split:
        from paper_2406_03466_gb300 import vqpu

        def step():
            vqpu.param_shift_gradient(prob, theta, dist, stream=stream)
    else:
        def step():
            sv.sv_grad_param_shift(prob, theta, *out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    t_dev = timed_loop(step, args.steps, flush, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if vqpu_split:
        # one gradient per step for the whole job: strong scaling
        t = torch.tensor([t_dev], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
        grads_per_s = args.steps / t_dev
    else:
        grads_per_s, t_dev = job_throughput(t_dev, args.steps, dist, dev)
    lo, hi = (0, B)
    if vqpu_split:
        from paper_2406_03466_gb300 import vqpu
        lo, hi = vqpu.segment(B, world, rank)
    result = {"metric": METRIC, "value": grads_per_s, "unit": "gradients/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
              "scaling": "strong" if vqpu_split else "weak", "vs_baseline": None, "dtype": "c64",
              "data": "synthetic",
              "config": {"workload": WORKLOAD_MCVQE8, "circuits_per_gradient": B,
                         "l2": "flushed before every timed step (256 MiB write, untimed)",
                         "parallelism": (f"vqpu x{world}: one segment of the batch per rank "
                                         f"(rank 0: slots [{lo}, {hi})) + NCCL allgather of "
                                         "energies" if vqpu_split else f"replicas x{world}")},
              "shifted_circuits_per_s": grads_per_s * B,
              # k_energy + k_ps_combine_dep, or per rank its segment's k_energy + the combine
              "gpu_launches": 2 * args.steps,
              "clocks": clk, "wall_s_timed_region": t_wall}
    if rank == 0:
        _, _, _, side = mcvqe8_side(sv, dev, stream, flush, max(200, args.steps // 4),
                                    extras=not args.no_extras)
        result["config"]["tuned_shape_c64"] = side.pop("tuned_shape_c64")
        result["roofline"] = side.pop("roofline")
        result["e2e"] = side.pop("e2e")
        for k in ("workload", "circuits_per_gradient", "gradients_per_s", "shifted_circuits_per_s"):
            side.pop(k, None)
        if not args.no_extras:
            # the metric's "% HBM roofline": gate application on the 20-qubit
            # circuit-learning batch (64 states, 512 MiB)
            result["hbm_gate_passes"] = forward_passes_roofline(sv, wl.config(3), dev, flush, stream)
            result["forms"] = side
        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def relaunch_cmd(argv, gpus, port):
    """The torch.distributed.run command that starts `gpus` ranks of this
    script with the same arguments (one node, rendezvous on 127.0.0.1)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
            f"--nproc-per-node={gpus}", "--master-addr", "127.0.0.1", "--master-port", str(port),
            os.path.abspath(__file__)] + list(argv)


def main():
    args = parse()
    rank, world, local = rank_info()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # --gpus N outside torchrun: start the N ranks here
        sys.exit(subprocess.call(relaunch_cmd(sys.argv[1:], args.gpus, _free_port())))
    if args.steps is None:
        args.steps = {"mcvqe8": 4000, "qcl20": 20, "mcvqe28": 5, "qcl-uneven": 5, "ddcl": 5}[args.workload]
    if args.warmup is None:
        args.warmup = {"mcvqe8": 50, "qcl20": 3, "mcvqe28": 3, "qcl-uneven": 3, "ddcl": 3}[args.workload]

    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload == "mcvqe8":
            cb, workload = cpu_baseline(args.cpu_seconds), WORKLOAD_MCVQE8
        elif args.workload == "ddcl":
            w = wl.ddcl(args.qubits or 26, 10)
            cb, workload = cpu_baseline_ddcl(w, min(args.cpu_seconds, 10.0)), ddcl_workload_name(w)
        elif args.workload == "qcl-uneven":
            ws = wl.qcl_uneven()
            cb = cpu_baseline_uneven(ws, min(args.cpu_seconds, 10.0))
            workload = uneven_workload_name(ws)
        else:
            w = device_workload(args)
            cb = cpu_baseline_device_memory(w, min(args.cpu_seconds, 10.0))
            workload = device_workload_name(w)
        v = cb["value"]
        line = {"metric": METRIC, "value": v, "unit": "gradients/s", "impl": "reference",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": {"workload": workload}, "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "gradients/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2406_03466_gb300 as sv

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    if args.workload == "qcl-uneven":
        return run_uneven(args, sv, dev, stream, dist, world, rank)
    if args.workload == "ddcl":
        return run_ddcl(args, sv, dev, stream, dist, world, rank)
    if args.workload == "mcvqe8":
        return run_mcvqe8(args, sv, dev, stream, dist, world, rank)
    return run_device_memory(args, sv, dev, stream, dist, world, rank)


if __name__ == "__main__":
    main()
