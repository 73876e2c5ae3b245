"""Benchmark: batched parameter-shift gradients of a multi-contracted VQE.

Workload (one step = one full gradient): 8 qubits (monomers), 4 layers of Ry
on every qubit + CNOT ladder (32 parameters), the Eq. 2 exciton Hamiltonian
with all 28 pairs (128 Pauli terms, synthetic coefficients), 9 reference
states; the parameter-shift batch is 2 x 32 x 9 + 9 = 585 circuits, each with
its full <H>, run by one batched kernel launch whose last block assembles
the gradient.
Inputs are seeded and synthetic.

Printed (one JSON line on rank 0): gradients/s of the batched complex64
path (value), shifted circuits/s, the adjoint gradient, the plain
one-circuit-per-launch complex128 form and the batched complex128 form, the
roofline of the dominant kernel, the CPU oracle timed on the host cores, and
an end-to-end number through the C ABI with host buffers.

``--impl reference`` times the CPU oracle (the reference arm: there is no
runnable reference implementation, only the paper) on the same workload.
Multi-GPU (torchrun): every rank runs its own replica of the workload; the
value is the gradients of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "gradients/sec & shifted circuits/sec, batched/adjoint vs plain; % HBM roofline"
WORKLOAD = ("mcvqe8: multi-contracted VQE gradient, 8 qubits, 4 layers Ry + CNOT ladder "
            "(32 params), 128-term Eq. 2 Hamiltonian, 9 references, 585 shifted circuits")
L2_FLUSH_BYTES = 256 << 20   # larger than the 126.5 MiB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true", help="skip adjoint/plain/c128 side runs")
    return ap.parse_args()


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
        self.path = os.path.join("/tmp", f"svclocks_{os.getpid()}.csv")

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


def main():
    args = parse()
    rank, world, local = rank_info()

    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(args.cpu_seconds)
        v = cb["value"]
        line = {"metric": METRIC, "value": v, "unit": "gradients/s", "impl": "reference",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c128", "data": "synthetic",
                "config": {"workload": WORKLOAD}, "cpu_baseline": cb,
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

    w = wl.config(1)
    B = w.n_slots_param_shift
    prob = sv.Problem.from_spec(w, "c64", device=dev)
    theta = torch.as_tensor(w.theta, dtype=torch.float64, device=dev)
    out = sv._outputs(prob, dev, None, None, None)
    e_buf = torch.empty(B, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # launch shapes (register bits, threads per block) picked by timing
    sv.sv_autotune(prob, theta)
    tuned = {"energy": sv.sv_tuned_shape(prob, 1)[:2], "adjoint": sv.sv_tuned_shape(prob, 2)[:2]}

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
    if dist:
        t = torch.tensor([t_dev], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_dev = float(t.item())
    grads_per_s = world * args.steps / t_dev

    result = {"metric": METRIC, "value": grads_per_s, "unit": "gradients/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
              "config": {"workload": WORKLOAD, "circuits_per_gradient": B,
                         "l2": "flushed before every timed step (256 MiB write, untimed)",
                         "tuned_shape_c64": {k: {"reg_bits": v[0], "threads_per_block": v[1]}
                                             for k, v in tuned.items()},
                         "parallelism": f"replicas x{world}"},
              "shifted_circuits_per_s": grads_per_s * B,
              "gpu_launches": args.steps,
              "clocks": clk, "wall_s_timed_region": t_wall}

    if rank == 0:
        # dominant kernel alone: the batched energies of all 585 circuits
        k_steps = max(200, args.steps // 4)
        fn = lambda: sv.sv_param_shift_energies(prob, theta, e_buf)  # noqa: E731
        for _ in range(20):
            fn()
        t_k = timed_loop(fn, k_steps, flush, stream) / k_steps
        flops = algorithmic_flops(w, B)
        peak = fp32_peak_tflops()
        achieved = flops / t_k / 1e12
        result["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak,
                              "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                              "kernel": f"k_energy<float,{tuned['energy'][0]}> (batched "
                                        "shifted-circuit energies + fused gradient assembly)",
                              "kernel_us": t_k * 1e6,
                              "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

        # end to end through the C ABI: theta from pinned host memory in,
        # loss + gradient back to pinned host memory, every step.
        th_host = torch.as_tensor(w.theta, dtype=torch.float64).pin_memory()
        g_host = torch.empty(w.n_params, dtype=torch.float64).pin_memory()
        l_host = torch.empty(1, dtype=torch.float64).pin_memory()
        th_dev = torch.empty_like(theta)
        e2e_steps = max(200, args.steps // 4)

        def e2e_step():
            th_dev.copy_(th_host, non_blocking=True)
            l_, e_, g_ = sv.sv_grad_param_shift(prob, th_dev, *out)
            g_host.copy_(g_[: w.n_params], non_blocking=True)
            l_host.copy_(l_, non_blocking=True)
            stream.synchronize()

        for _ in range(10):
            e2e_step()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        t_e2e = time.perf_counter() - t0
        result["e2e"] = {"value": e2e_steps / t_e2e, "unit": "gradients/s",
                         "h2d_bytes_per_step": 8 * w.n_params,
                         "d2h_bytes_per_step": 8 * (w.n_params + 1),
                         "timing": "host wall clock incl. stream synchronize per step"}

        if not args.no_extras:
            extras = {}
            fn = lambda: sv.sv_grad_adjoint(prob, theta, None, *out)  # noqa: E731
            for _ in range(20):
                fn()
            n = max(200, args.steps // 4)
            extras["adjoint_c64_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
            prob128 = sv.Problem.from_spec(w, "c128", device=dev)
            out128 = sv._outputs(prob128, dev, None, None, None)
            sv.sv_autotune(prob128, theta)
            fn = lambda: sv.sv_grad_param_shift(prob128, theta, *out128)  # noqa: E731
            for _ in range(20):
                fn()
            extras["batched_c128_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
            fn = lambda: sv.sv_grad_adjoint(prob128, theta, None, *out128)  # noqa: E731
            for _ in range(20):
                fn()
            extras["adjoint_c128_gradients_per_s"] = n / timed_loop(fn, n, flush, stream)
            # the plain form is host-driven (one launch per gate and term): wall clock
            sv.sv_grad_param_shift_plain(prob128, theta, *out128)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 2
            for _ in range(reps):
                sv.sv_grad_param_shift_plain(prob128, theta, *out128)
            torch.cuda.synchronize()
            extras["plain_c128_gradients_per_s"] = reps / (time.perf_counter() - t0)
            extras["plain_c128_launches_per_gradient"] = B * (1 + len(w.gates) + w.n_terms) + 1
            result["forms"] = extras

        result["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
