#!/usr/bin/env python
"""Benchmark of the parallel-in-time Newton solver (arXiv 2409.20027) on GB300.

Workload (one "step" = one complete constrained solve): force-limited cart-pole,
primal log-barrier IP (mu 1e-1 -> 1e-6), T = 16384 steps over a fixed 2.56 s horizon
(RK4, dt = 2.56/T), |u| <= 10, |p| <= 2, solved to KKT residual <= 1e-6, FP32 LQR
arithmetic with FP64 solves.  Initial states are seeded (seed = step index mod 10).

Prints one JSON line.  --impl reference times the serial FP64 CPU oracle instead.
Multi-GPU (torchrun): independent replicas, one instance per rank.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-solve (ms) vs horizon T at KKT residual ≤1e-6; batched solves/sec; grads/sec"
HORIZON_S = 2.56
L2_FLUSH_BYTES = 256 << 20


def algorithmic_flops(n, m, T, info):
    """Per-solve algorithmic FLOPs (unit counts per time step, per Newton iteration):
    value scan 2 x 16.7 n^3, co-state and state scans 2 x 2 x (2 n^3 + 2 n^2), element
    init and feedback 10 n^2 m + 2 m^3; every multiple-shooting rollout iteration one
    affine scan 2 (2 n^3 + 2 n^2)."""
    per_it = 2 * 16.7 * n ** 3 + 4 * (2 * n ** 3 + 2 * n ** 2) + 10 * n * n * m + 2 * m ** 3
    per_roll = 2 * (2 * n ** 3 + 2 * n ** 2)
    return T * (info["newton_iters"] * per_it + info["roll_iters"] * per_roll)


def alu_peak_tflops():
    # FP32 FMA pipes: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (maximum SM clock)
    return 152 * 128 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        for r in rows:
            for name, v in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


def cartpole_instance(T):
    from paper_2409_20027_gb300 import workloads as W
    return W.cartpole(T=T, horizon=HORIZON_S)


def oracle_solve_ms(T, seed):
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    p = cartpole_instance(T)
    t0 = time.perf_counter()
    r = O.solve_ip(p, W.cartpole_x0(seed), T)
    return (time.perf_counter() - t0) * 1e3, r["info"]


def run_reference(args, T):
    """The serial FP64 CPU oracle on a bounded sample of the workload: a T_s = 1024
    solve of the same problem family, scaled by T / T_s (the oracle's cost per Newton
    iteration is linear in T and its iteration count does not grow with T)."""
    Ts = min(T, 1024)
    for k in range(args.warmup):
        oracle_solve_ms(Ts, k % 10)
    times = []
    for k in range(args.steps):
        ms, info = oracle_solve_ms(Ts, k % 10)
        times.append(ms * T / Ts)
    v = sum(times) / len(times)
    sample = f"oracle IP solve at T={Ts} (same 2.56 s horizon), time scaled x{T / Ts:g} to T={T}"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(T), "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                                                   "sample": sample},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(T):
    return {"workload": f"cart-pole swing-stabilisation, primal log-barrier IP, T={T}, fixed {HORIZON_S} s "
                        f"horizon (RK4, dt={HORIZON_S / T:.4g}), |u|<=10, |p|<=2, KKT<=1e-6",
            "T": T, "method": "ip", "precision": "fp32 LQR with fp64 solves",
            "l2": "flushed between timed solves (256 MiB write)", "seeds": "step index mod 10"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--T", type=int, default=16384)
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    T = args.T

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, T)
        return

    import torch
    from paper_2409_20027_gb300 import ptn, workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    p = cartpole_instance(T)
    solver = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE)
    x0s = [torch.tensor(W.cartpole_x0((k + 100 * rank) % 10 + 0), dtype=torch.float64, device=dev)
           for k in range(10)]
    xo = torch.empty((T + 1, 4), dtype=torch.float64, device=dev)
    uo = torch.empty((T, 1), dtype=torch.float64, device=dev)
    lo = torch.empty((T + 1, 4), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    infos = []
    for k in range(args.warmup):
        _, _, _, info = solver.solve_ip(x0s[k % 10], T, x_out=xo, u_out=uo, lam_out=lo)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            _, _, _, info = solver.solve_ip(x0s[k % 10], T, x_out=xo, u_out=uo, lam_out=lo)
            ev[k][1].record(stream)
            infos.append(info)
        torch.cuda.synchronize()
    barrier()
    clocks = clk.summary()
    per = [a.elapsed_time(b) for a, b in ev]
    ms = sum(per) / len(per)
    if dist is not None:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ok = all(i["status"] == 0 and i["r_kkt"] <= 1e-6 * (1 + 1e-9) for i in infos)

    # end to end through the public API with host buffers (pinned), copies in the region
    x0h = torch.tensor(W.cartpole_x0(0), dtype=torch.float64).pin_memory()
    xh = torch.empty((T + 1, 4), dtype=torch.float64).pin_memory()
    uh = torch.empty((T, 1), dtype=torch.float64).pin_memory()
    x0d = torch.empty(4, dtype=torch.float64, device=dev)
    e2e = []
    for k in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x0d.copy_(x0h, non_blocking=True)
        solver.solve_ip(x0d, T, x_out=xo, u_out=uo, lam_out=lo)
        xh.copy_(xo, non_blocking=True)
        uh.copy_(uo, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = sum(e2e) / len(e2e)

    sweep = {}
    if not args.no_sweep:
        for Ts in [256, 1024, 4096]:
            ps = cartpole_instance(Ts)
            sv = ptn.Solver(ps, max_T=Ts, precision=ptn.PTN_FP32_FP64SOLVE)
            x0 = x0s[0]
            sv.solve_ip(x0, Ts)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            _, _, _, inf = sv.solve_ip(x0, Ts)
            b.record(stream)
            torch.cuda.synchronize()
            sweep[str(Ts)] = {"ms": a.elapsed_time(b), "newton_iters": inf["newton_iters"], "status": inf["status"],
                              "r_kkt": inf["r_kkt"]}
            sv.close()
        sweep[str(T)] = {"ms": ms, "newton_iters": infos[-1]["newton_iters"], "status": infos[-1]["status"],
                         "r_kkt": infos[-1]["r_kkt"]}

    if rank != 0:
        return
    last = infos[-1]
    flops = algorithmic_flops(4, 1, T, last)
    achieved = flops / (per[-1] * 1e-3) / 1e12
    peak = alu_peak_tflops()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_solve_grid<CartPole,float>",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        Ts = 1024
        t_ms, _ = oracle_solve_ms(Ts, 0)
        cpu = {"value": t_ms * T / Ts, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"one oracle IP solve at T={Ts} (same horizon), time scaled x{T // Ts} to T={T}"}
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config(T),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 4 * 8,
                    "d2h_bytes_per_step": ((T + 1) * 4 + T) * 8},
            "gpu_launches": args.steps, "clocks": clocks, "kkt_ok": ok,
            "newton_iters": last["newton_iters"], "sweep": sweep}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
