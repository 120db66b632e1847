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
TUNED_TABLE = os.path.join(ROOT, "paper_2409_20027_gb300", "tuned_gb300.json")
BATCH_HORIZON_S = 1.28  # keeps dt_b <= 0.02 for every batch horizon (T_b >= 64)
SWEEP_T = [256, 1024, 4096, 16384, 32768, 65536]


def algorithmic_flops(n, m, T, info):
    """Per-solve algorithmic FLOPs (unit counts per time step, per Newton iteration):
    value scan 2 x 16.7 n^3, co-state and state scans 2 x 2 x (2 n^3 + 2 n^2), element
    init and feedback 10 n^2 m + 2 m^3; every multiple-shooting rollout iteration one
    affine scan 2 (2 n^3 + 2 n^2)."""
    per_it = 2 * 16.7 * n ** 3 + 4 * (2 * n ** 3 + 2 * n ** 2) + 10 * n * n * m + 2 * m ** 3
    per_roll = 2 * (2 * n ** 3 + 2 * n ** 2)
    return T * (info["newton_iters"] * per_it + info["roll_iters"] * per_roll)


# DRAM bytes (read + write) of one k_solve_grid launch of this workload (seed 0), from the
# ncu launch list summarised in profiles/k_solve_grid_cartpole_T16384.md (mean of the
# three launches after the first)
TRAFFIC_BYTES = ((3.645440 + 2.659584) + (3.320576 + 2.477824) + (3.235584 + 2.478336)) / 3 * 1e6


def flop_split(n, m, T, info):
    """(FP32, FP64) algorithmic FLOPs of one solve.  The FP64 share is the inverse of
    I + C1 J2 (about 2 n^3 per combination, two combinations per element) in the value
    scan; everything else runs in FP32."""
    total = algorithmic_flops(n, m, T, info)
    f64 = T * info["newton_iters"] * 2 * 2 * n ** 3
    return total - f64, f64


def measured_fma_peaks():
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), measured by the probe kernel of
    include/ptn_peaks.h (full occupancy, 8 independent chains per thread, CUDA-event timed),
    with the SM count of the device; None where the probe is unavailable."""
    import ctypes as C
    from paper_2409_20027_gb300 import build as B
    try:
        lib = C.CDLL(B.build_peaks())
        lib.ptn_peak_fma.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        out = {}
        for name, fp64, iters in [("fp32", 0, 200000), ("fp64", 1, 2000)]:
            best = 0.0
            for _ in range(3):
                tf, ms = C.c_double(), C.c_double()
                rc = lib.ptn_peak_fma(fp64, 8, iters, C.byref(tf), C.byref(ms))
                if rc != 0:
                    return None
                best = max(best, tf.value)
            out[name] = best
        return out
    except (OSError, RuntimeError):
        return None


def blended_peak_tflops(f32, f64, p32, p64):
    """Peak rate of a kernel doing f32 FP32 and f64 FP64 flops with each pipe at its own
    peak: (f32 + f64) / (f32 / P32 + f64 / P64)."""
    return (f32 + f64) / (f32 / p32 + f64 / p64)


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


def _oracle_ref(job):
    """One oracle solve of a benchmark workload (also run in spawn-pool workers): the
    solution arrays, the oracle's report and the solve's wall time in ms.  Jobs:
    ("cartpole", T, seed) the single-solve workload at horizon T; ("pendulum", seed) the
    pendulum at T = 64; ("batch", k) instance k of the batch workload; ("quad", b, T)
    instance b of the quadrotor workload."""
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    kind = job[0]
    if kind == "cartpole":
        _, T, seed = job
        args = (W.cartpole(T=T, horizon=HORIZON_S), W.cartpole_x0(seed), T)
        kw = {}
    elif kind == "pendulum":
        args = (W.pendulum(), W.pendulum_x0(job[1]), 64)
        kw = {}
    elif kind == "batch":
        k = job[1]
        T = int(W.batch_horizons(1024, seed=0)[k])
        args = (W.cartpole(T=T, horizon=BATCH_HORIZON_S), W.cartpole_batch_x0(1024, seed=0)[k], T)
        kw = {}
    elif kind == "synth":
        _, T, k = job
        args = (W.synth(0), W.synth_x0(k), T)
        kw = {"opts": O.Options(costate_mode=1)}
    elif kind == "quad":
        _, b, T = job
        args = (W.quadrotor(W.quadrotor_waypoints(b + 1, seed=0)[b]), np.zeros(12), T)
        kw = {"u_init": np.full((T, 4), W.quadrotor_hover_u())}
    elif kind == "admm_pend":
        # ADMM on the paper's pendulum with the bench's settings (rho, the 1e-2 rule)
        T = job[1]
        t0 = time.perf_counter()
        r = O.solve_admm(W.pendulum_paper(dt=3.2 / T), W.pendulum_x0(0), T,
                         opts=O.Options(rho=W.PAPER_ADMM["pendulum_rho"], admm_tol=W.PAPER_ADMM["tol"],
                                        max_outer=2000))
        r["ms"] = (time.perf_counter() - t0) * 1e3
        return r
    else:
        raise ValueError(job)
    t0 = time.perf_counter()
    r = O.solve_ip(*args, **kw)
    r["ms"] = (time.perf_counter() - t0) * 1e3
    return r


def err_vs_oracle(ref, x, u, lam, J):
    """Relative error of a GPU result against the oracle's, max|a - b| / max(1, max|b|) for
    x, u, lam and |J - J_o| / max(1, |J_o|), with the oracle's status and iteration count."""
    def rel(a, b):
        a = np.asarray(a)
        b = np.asarray(b)
        return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))
    return {"x": rel(x, ref["x"]), "u": rel(u, ref["u"]),
            "lam": None if lam is None else rel(lam, ref["lam"]),
            "J": abs(J - ref["info"]["J"]) / max(1.0, abs(ref["info"]["J"])),
            "oracle_status": ref["info"]["status"], "oracle_newton_iters": ref["info"]["newton_iters"]}


def oracle_pool(jobs, timeout=900):
    """Oracle solves of `jobs` in a spawn pool over the host cores (safe after CUDA is
    initialised), one job per process; returns (results in job order, processes used)."""
    import multiprocessing as mp
    procs = max(1, min(os.cpu_count() or 1, len(jobs)))
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=procs) as pool:  # leaving the block terminates it
        return pool.map_async(_oracle_ref, jobs, chunksize=1).get(timeout=timeout), procs


BATCH_SAMPLE = 16


def batch_sample_indices():
    rng = np.random.default_rng(7)
    return sorted(int(k) for k in rng.choice(1024, size=BATCH_SAMPLE, replace=False))


def cpu_batch_baseline():
    """The oracle on a sample of the batch workload, one instance per worker process over
    the host cores: solves/s of the sample (which scales to the batch as its mean horizon
    does) and the sample's solutions.  Never raises: a failure is reported instead."""
    from paper_2409_20027_gb300 import workloads as W
    try:
        ks = batch_sample_indices()
        Tb = W.batch_horizons(1024, seed=0)
        oracle_pool([("batch", ks[0])])  # start-up (imports, library build) outside the timing
        t0 = time.perf_counter()
        res, procs = oracle_pool([("batch", k) for k in ks])
        wall = time.perf_counter() - t0
        steps = sum(int(Tb[k]) for k in ks)
        return {"solves_per_s": len(ks) / wall, "unit": "solves/s", "cores": procs, "kind": "oracle",
                "sample": f"{len(ks)} instances of the batch workload (seed 7 draw), {steps} steps; the whole "
                          f"batch has {int(Tb.sum())} steps, one instance per process",
                "converged": sum(1 for r in res if r["info"]["status"] == 0)}, dict(zip(ks, res))
    except Exception as e:  # the GPU numbers must not depend on the host baseline
        return {"error": f"{type(e).__name__}: {e}"}, {}


def host_cpu():
    """Model name of the host CPU (Linux /proc/cpuinfo, lscpu-style keys), or the machine."""
    import platform
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def run_reference(args, T):
    """The serial FP64 CPU oracle on the benchmark's workload itself: every timed step is
    one complete oracle solve of the T = 16384 cart-pole (seed = step index mod 10), single
    thread.  The warm-up steps are T = 1024 solves of the same problem family (the oracle
    has no compilation step; warm-up only pages in its code and data)."""
    for k in range(args.warmup):
        _oracle_ref(("cartpole", min(T, 1024), k % 10))
    times, iters = [], []
    for k in range(args.steps):
        r = _oracle_ref(("cartpole", T, k % 10))
        times.append(r["ms"])
        iters.append(r["info"]["newton_iters"])
    v = sum(times) / len(times)
    sample = (f"one complete oracle IP solve of the workload per step (T={T}, seed = step mod 10), "
              f"single thread on {host_cpu()}; warm-up steps are T=1024 solves; mean Newton iterations "
              f"{sum(iters) / len(iters):.1f}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(T), "cpu_baseline": {"value": v, "unit": "ms", "cores": 1, "kind": "oracle",
                                                   "sample": sample},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (every rank gets it): a step takes as long as its
    slowest replica."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_pendulum(ptn, W, dev, flush, stream, tuned):
    """The pendulum swing-up (n = 2, m = 1, Euler dt = 0.05, T = 64, |u| <= 5, mu 1e-1 ->
    1e-6), FP64 throughout, seeds 0-9 (x0 = N(0, 0.05^2) per component), tuned launch shape;
    each seed's solve timed with CUDA events after warm-up, L2 flushed before each."""
    import torch
    from paper_2409_20027_gb300 import autotune
    T = 64
    sv = ptn.Solver(W.pendulum(), max_T=T, precision=ptn.PTN_FP64)
    launch = autotune.apply(sv, tuned, T)
    x0s = [torch.tensor(W.pendulum_x0(sd), dtype=torch.float64, device=dev) for sd in range(10)]
    for x in x0s[:3]:
        sv.solve_ip(x, T)
    torch.cuda.synchronize()
    ms, its, st, infos, outs = [], [], [], [], {}
    for sd, x in enumerate(x0s):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xs, us, ls, inf = sv.solve_ip(x, T)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        its.append(inf["newton_iters"])
        st.append(inf["status"])
        infos.append(inf)
        outs[("pendulum", sd)] = (xs.cpu().numpy(), us.cpu().numpy(), ls.cpu().numpy(), inf["J"])
    sv.close()
    return {"workload": "pendulum swing-up, IP, T=64 (Euler dt=0.05), |u|<=5, FP64, seeds 0-9, KKT<=1e-6",
            "ms_median": float(np.median(ms)), "ms_mean": float(np.mean(ms)), "ms": ms,
            "newton_iters_mean": float(np.mean(its)),
            "us_per_newton_iter": float(1e3 * np.sum(ms) / max(np.sum(its), 1)),
            "status_counts": {str(k): st.count(k) for k in set(st)}, "launch": launch or "defaults",
            "phase_share": phase_share(infos)}, outs


def run_batch(args, ptn, W, dev, flush, stream):
    """Batched workload: B cart-pole instances (RK4), horizons T_b log-uniform in [64, 4096]
    from seed 0, each covering the same 1.28 s at dt_b = 1.28 / T_b; one launch for the
    whole batch (one CTA per instance).  Also the same instances solved one by one with
    the single-instance path (cluster or grid tier)."""
    import torch
    B = args.batch
    Tb = W.batch_horizons(B, seed=0)
    dtb = BATCH_HORIZON_S / Tb  # every instance covers the same 1.28 s at its own sampling rate
    x0 = torch.tensor(W.cartpole_batch_x0(B, seed=0), dtype=torch.float64, device=dev)
    p = W.cartpole()
    sv = ptn.Solver(p, max_T=int(Tb.max()), max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE)
    S = int(Tb.sum())
    xo = torch.empty((S + B, 4), dtype=torch.float64, device=dev)
    uo = torch.empty((S, 1), dtype=torch.float64, device=dev)
    lo = torch.empty((S + B, 4), dtype=torch.float64, device=dev)
    sv.solve_batch(x0, Tb, x_out=xo, u_out=uo, lam_out=lo, dt_b=dtb)
    torch.cuda.synchronize()
    times, infos = [], None
    for k in range(2):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, _, infos = sv.solve_batch(x0, Tb, x_out=xo, u_out=uo, lam_out=lo, dt_b=dtb)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ms = min(times)
    st = [i["status"] for i in infos]
    # the solutions of the instances the CPU leg also solves (for the error against it)
    xoff = np.concatenate([[0], np.cumsum(Tb + 1)])
    uoff = np.concatenate([[0], np.cumsum(Tb)])
    xs, us, ls = xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy()
    outs = {k: (xs[xoff[k]:xoff[k + 1]], us[uoff[k]:uoff[k + 1]], ls[xoff[k]:xoff[k + 1]], infos[k]["J"])
            for k in batch_sample_indices() if k < B}
    # the same instances one at a time (a sample of 32, scaled to B)
    one = ptn.Solver(p, max_T=int(Tb.max()), precision=ptn.PTN_FP32_FP64SOLVE)
    ns = min(B, 32)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(ns):
        one.solve_batch(x0[i:i + 1], Tb[i:i + 1], dt_b=dtb[i:i + 1])
    b.record(stream)
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b) * B / ns
    sv.close()
    one.close()
    return {"workload": f"{B} cart-pole instances, IP, RK4, 1.28 s horizon at dt_b=1.28/T_b, T_b log-uniform [64, 4096] "
                        f"(seed 0, {S} steps), one launch", "solves_per_s": B / (ms * 1e-3), "ms": ms,
            "converged": int(sum(1 for x in st if x == 0)), "status_counts": {str(k): st.count(k) for k in set(st)},
            "one_by_one_solves_per_s": B / (seq_ms * 1e-3),
            "one_by_one_sample": f"first {ns} instances as single solves (cluster or grid tier), time scaled to {B}"}, outs


def run_multiplier(args, ptn, W, dev, flush, stream, tuned, x0):
    """The multiplier form of the co-states (option costate_mode; a variant of the method:
    dynamics multipliers moved to the LQR duals instead of the co-state scan), pure (1) and
    restarted from the scan's co-states at every barrier level (2), beside the co-state
    form (0) on the same single solves (same x0, same tuned launch shapes), and modes 1, 2
    on the batch workload.  All forms end at the same KKT point."""
    import torch
    from paper_2409_20027_gb300 import autotune
    out = {"single": {}}
    sols = {}
    for Ts in [1024, 4096, args.T]:
        ps = cartpole_instance(Ts)
        row = {}
        for mode in [0, 1, 2]:
            sv = ptn.Solver(ps, max_T=Ts, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=mode)
            autotune.apply(sv, tuned, Ts)
            sv.solve_ip(x0, Ts)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            xs_, us_, ls_, inf = sv.solve_ip(x0, Ts)
            b.record(stream)
            torch.cuda.synchronize()
            row[f"mode{mode}"] = {"ms": a.elapsed_time(b), "newton_iters": inf["newton_iters"],
                                  "status": inf["status"], "r_kkt": inf["r_kkt"]}
            if mode > 0:
                sols[("mult", Ts, mode)] = (xs_.cpu().numpy(), us_.cpu().numpy(), ls_.cpu().numpy(), inf["J"])
            sv.close()
        out["single"][str(Ts)] = row
    B = args.batch
    Tb = W.batch_horizons(B, seed=0)
    dtb = BATCH_HORIZON_S / Tb
    xb = torch.tensor(W.cartpole_batch_x0(B, seed=0), dtype=torch.float64, device=dev)
    out["batch"] = {}
    for mode in [1, 2]:
        sv = ptn.Solver(W.cartpole(), max_T=int(Tb.max()), max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE,
                        costate_mode=mode)
        sv.solve_batch(xb, Tb, dt_b=dtb)
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, _, infos = sv.solve_batch(xb, Tb, dt_b=dtb)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        st = [i["status"] for i in infos]
        out["batch"][f"mode{mode}"] = {"solves_per_s": B / (ms * 1e-3), "ms": ms,
                                       "status_counts": {str(k): st.count(k) for k in set(st)},
                                       "newton_iters_mean": float(np.mean([i["newton_iters"] for i in infos]))}
        sv.close()
    out["workload"] = ("cart-pole IP as the sweep (2.56 s horizon, tuned launch, x0 seed 0) in co-state forms "
                       "0 (scan), 1 (multiplier), 2 (multiplier restarted per barrier level); the batch "
                       "workload in forms 1 and 2 (form 0: the batch section)")
    return out, sols


def _admm_solve(ptn, prob, T, x0, stream, flush, tuned, **opt):
    import torch
    from paper_2409_20027_gb300 import autotune
    sv = ptn.Solver(prob, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, **opt)
    autotune.apply(sv, tuned, T)
    sv.solve_admm(x0, T)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    a.record(stream)
    xs, us, ls, inf = sv.solve_admm(x0, T)
    b.record(stream)
    torch.cuda.synchronize()
    sv.close()
    row = {"ms": a.elapsed_time(b), "status": inf["status"], "outer_iters": inf["outer_iters"],
           "newton_iters": inf["newton_iters"], "r_p": inf["r_p"], "r_d": inf["r_d"], "r_stat": inf["r_stat"]}
    return row, (xs.cpu().numpy(), us.cpu().numpy(), None, inf["J"])


def run_admm(args, ptn, W, dev, flush, stream, tuned, x0):
    """ADMM (Sec. II-C) with the paper's stopping rule max|w - z| <= 1e-2 and max|z - z_prev|
    <= 1e-2, at most 2000 outer iterations (the oracle's own cap), each sub-problem solved by
    Newton to 1e-6, FP32 LQR with FP64 solves:
      - the paper's pendulum (g, l, m, b = 1e-3, Euler, |tau| <= 5; rho = 1 as the paper sets
        it) on a fixed 3.2 s horizon, T = 256 ... 16384: time-to-solve at the rule;
      - the configuration's cart-pole (rho = 1, 2.56 s horizon) at T = 256, 1024, which does not
        meet the rule within 2000 outer iterations, on the GPU or in the oracle."""
    import torch
    out = {"pendulum_paper": {}, "cartpole": {}}
    xp = torch.tensor(W.pendulum_x0(0), dtype=torch.float64, device=dev)
    sols = {}
    for Ts in [256, 1024, 4096, 16384]:
        row, sol = _admm_solve(ptn, W.pendulum_paper(dt=3.2 / Ts), Ts, xp, stream, flush, tuned,
                               rho=W.PAPER_ADMM["pendulum_rho"], admm_tol=W.PAPER_ADMM["tol"], max_outer=2000)
        out["pendulum_paper"][str(Ts)] = row
        if Ts == 256:
            sols[("admm_pend", Ts)] = sol
    for Ts in [256, 1024]:
        out["cartpole"][str(Ts)], _ = _admm_solve(ptn, cartpole_instance(Ts), Ts, x0, stream, flush, tuned, rho=1.0,
                                                  admm_tol=1e-2, max_outer=2000)
    out["workload"] = ("ADMM, stop at max|w-z|, max|z-z_prev| <= 1e-2 or 2000 outer iterations; the paper's pendulum "
                       "(rho 1) on 3.2 s at dt = 3.2/T, x0 seed 0; the cart-pole of the sweep (rho 1, 2.56 s, x0 seed "
                       "0); Newton sub-problems to 1e-6, FP32 LQR with FP64 solves")
    return out, sols


PHASES = ["costate", "second_order", "value", "state", "line_search", "initial_rollout", "other"]


def phase_share(infos):
    """Share of SM cycles per phase of the Newton step, summed over instances (the
    solver's own clock64 counters, first thread of each group)."""
    tot = np.zeros(7)
    for i in infos:
        tot += np.asarray(i["cycles"], dtype=np.float64)
    return {k: round(float(v / max(tot.sum(), 1.0)), 4) for k, v in zip(PHASES, tot)}


QUAD_ORACLE_SAMPLE = 2


def run_quadrotor(args, ptn, W, dev, flush, stream):
    """Quadrotor workload: B instances (n = 12, m = 4, Euler dt = 0.01, T = 1024), hover
    start at the origin, waypoints uniform in the 2 m cube (seed 0), hover thrust as the
    strictly feasible initial control; one batched IP solve (wide tier), then the adjoint
    of J* plus a trajectory loss with respect to x0, diag Q, diag R, diag Qf and the model
    constants (mass, inertia, arm, yaw coefficient, g).  grads/s counts one gradient of
    every instance per forward + adjoint."""
    import torch
    B, T = args.quad_batch, args.quad_T
    wps = W.quadrotor_waypoints(B, seed=0)
    xrefs = torch.tensor(np.stack([W.quadrotor(w).xref for w in wps]), dtype=torch.float64, device=dev)
    Tb = np.full(B, T, dtype=np.int32)
    sv = ptn.Solver(W.quadrotor(), max_T=T, max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE)
    x0 = torch.zeros((B, 12), dtype=torch.float64, device=dev)
    u0 = torch.full((B * T, 4), W.quadrotor_hover_u(), dtype=torch.float64, device=dev)
    xo = torch.empty((B * (T + 1), 12), dtype=torch.float64, device=dev)
    uo = torch.empty((B * T, 4), dtype=torch.float64, device=dev)
    gx = torch.zeros_like(xo)
    gx[T::T + 1, :3] = 1.0  # d loss / d final position
    fw, ad = [], []
    for k in range(2):
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        _, _, lq, infos = sv.solve_batch(x0, Tb, xref=xrefs, u_init=u0, x_out=xo, u_out=uo)
        b.record(stream)
        sv.adjoint(Tb, x0, xo, uo, infos[0]["mu"], 1.0, gx, None, xref=xrefs)
        c.record(stream)
        torch.cuda.synchronize()
        fw.append(a.elapsed_time(b))
        ad.append(b.elapsed_time(c))
    st = [i["status"] for i in infos]
    xs, us, ls = xo.cpu().numpy(), uo.cpu().numpy(), lq.cpu().numpy()
    outs = {b: (xs[b * (T + 1):(b + 1) * (T + 1)], us[b * T:(b + 1) * T], ls[b * (T + 1):(b + 1) * (T + 1)],
                infos[b]["J"])
            for b in range(min(B, QUAD_ORACLE_SAMPLE))}
    sv.close()
    f, g = min(fw), min(ad)
    return {"workload": f"{B} quadrotor instances (n=12, m=4), T={T}, Euler dt=0.01, waypoints in a 2 m cube, "
                        "IP fp32 LQR with fp64 solves (wide tier); adjoint in fp64",
            "forward_ms": f, "adjoint_ms": g, "solves_per_s": B / (f * 1e-3), "grads_per_s": B / ((f + g) * 1e-3),
            "converged": int(sum(1 for x in st if x == 0)), "status_counts": {str(k): st.count(k) for k in set(st)},
            "newton_iters_mean": float(np.mean([i["newton_iters"] for i in infos])),
            "phase_share": phase_share(infos)}, outs


def _mpc_loop(ptn, W, prob, x0, target, steps):
    """One closed-loop experiment: B loops from the rows of x0, horizon N at the problem's
    rate, `steps` periods, each one batched solve warm-started with the shifted controls;
    synchronous solves, then the same loop replayed period by period from one CUDA graph."""
    import torch
    from paper_2409_20027_gb300 import mpc
    B = x0.shape[0]
    N = W.PAPER_MPC["horizon"]
    sv = ptn.Solver(prob, max_T=N, max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE, block_threads=64)
    mpc.closed_loop(sv, x0, N, 2)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = mpc.closed_loop(sv, x0, N, steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    gl = mpc.GraphLoop(sv, x0, N)
    gl.run(2)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    resg = gl.run(steps)
    torch.cuda.synchronize()
    wall_g = time.perf_counter() - t0
    same = bool(torch.equal(res["x"], resg["x"]) and torch.equal(res["u"], resg["u"]))
    del gl
    sv.close()
    st, its = res["status"], res["iters"]
    err = (res["x"][-1] - torch.tensor(target, device=x0.device)).abs()
    lim = float(prob.uhi[0])
    return {"loops": B, "periods": steps, "horizon": N, "dt": prob.dt,
            "period_ms": 1e3 * wall / steps, "loop_periods_per_s": B * steps / wall,
            "graph_period_ms": 1e3 * wall_g / steps, "graph_loop_periods_per_s": B * steps / wall_g,
            "graph_same_trajectories": same,
            "newton_iters_first": float(its[0].mean()), "newton_iters_warm": float(its[1:].mean()),
            "converged_share": float((st == 0).mean()),
            "final_state_abs_err_max": err.max(dim=0).values.tolist(),
            "final_state_abs_err_median": err.median(dim=0).values.tolist(),
            "max_abs_control": float(res["u"].abs().max().item()), "control_limit": lim}


def run_mpc(ptn, W, dev, stream):
    """Closed-loop MPC as the paper's experiment (Sec. IV-C): 4 s at 100 Hz (400 periods),
    horizon N = 60, Euler, the paper's pendulum (|tau| <= 5) and cart-pole (m_c = 10, m_p = 1,
    |F| <= 60), target upright (and the cart at the origin); 256 loops per system."""
    import torch
    m = W.PAPER_MPC
    steps = int(round(m["duration_s"] * m["rate_hz"]))
    B = 256
    xc = torch.tensor(W.cartpole_batch_x0(B, seed=1), dtype=torch.float64, device=dev)
    xp = torch.tensor(np.stack([W.pendulum_upright_x0(1000 + b) for b in range(B)]), dtype=torch.float64, device=dev)
    return {"workload": f"{B} closed loops per system, {m['duration_s']:g} s at {m['rate_hz']} Hz (Euler), N="
                        f"{m['horizon']}, the paper's pendulum (|tau|<=5) and cart-pole (m_c=10, m_p=1, |F|<=60, "
                        "R=1e-4), both from near upright, shifted warm start, fp32 LQR with fp64 solves, one "
                        "batched solve per period",
            "cartpole": _mpc_loop(ptn, W, W.cartpole_paper(), xc, [0.0, np.pi, 0.0, 0.0], steps),
            "pendulum": _mpc_loop(ptn, W, W.pendulum_paper(), xp, [np.pi, 0.0], steps)}


def run_synth(args, ptn, W, dev, flush, stream):
    """The synthetic scaling workload x+ = A x + B u + 0.1 tanh(W x) (n = 32, m = 8; A 0.98 x
    Haar orthogonal, B ~ N(0, 1/m), W ~ N(0, 1/n), random SPD Q, R = 0.1 I, |u| <= 1, x0 ~
    N(0, I); matrices from seed 0), IP with the multiplier form of the co-states (the co-state
    products of A + 0.1 W grow like 1.0167^T at this seed), FP32 LQR data with FP64 solves,
    wide tier: one instance at T = 65536 on the cooperative grid, and a batch of 64 instances
    with T uniform in [1024, 8192] (seed 0), one CTA each."""
    import torch
    p = W.synth(0)
    out = {"workload": "synthetic x+ = A x + B u + 0.1 tanh(W x), n=32, m=8 (seed 0), |u|<=1, IP, multiplier "
                       "form of the co-states, fp32 LQR with fp64 solves, wide tier",
           "spectral_radius_A_plus_cW": float(np.abs(np.linalg.eigvals(p.A + 0.1 * p.W)).max())}
    T = args.synth_T
    sv = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1)
    x0 = torch.tensor(W.synth_x0(0), dtype=torch.float64, device=dev)
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    xs, us, ls, inf = sv.solve_ip(x0, T)
    b.record(stream)
    torch.cuda.synchronize()
    out["single"] = {"T": T, "ms": a.elapsed_time(b), "status": inf["status"], "newton_iters": inf["newton_iters"],
                     "r_kkt": inf["r_kkt"], "r_stat": inf["r_stat"], "r_dyn": inf["r_dyn"], "J": inf["J"],
                     "us_per_newton_iter": 1e3 * a.elapsed_time(b) / max(inf["newton_iters"], 1),
                     "phase_share": phase_share([inf]), "note": "one solve, cold (the first of this model)"}
    sv.close()
    B = args.synth_batch
    Tb = W.uniform_horizons(B, seed=0, lo=1024, hi=8192)
    S = int(Tb.sum())
    sb = ptn.Solver(p, max_T=(S + B - 1) // B, max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1)
    xb = torch.tensor(np.stack([W.synth_x0(k) for k in range(B)]), dtype=torch.float64, device=dev)
    flush.zero_()
    a.record(stream)
    X, U, _, infos = sb.solve_batch(xb, Tb)
    b.record(stream)
    torch.cuda.synchronize()
    st = [i["status"] for i in infos]
    k = int(np.argmin(Tb))
    xoff = int(np.sum(Tb[:k] + 1))
    uoff = int(np.sum(Tb[:k]))
    sample = (X[xoff:xoff + int(Tb[k]) + 1].cpu().numpy(), U[uoff:uoff + int(Tb[k])].cpu().numpy(), None,
              infos[k]["J"])
    out["batch"] = {"instances": B, "steps": S, "ms": a.elapsed_time(b), "solves_per_s": B / (a.elapsed_time(b) * 1e-3),
                    "status_counts": {str(v): st.count(v) for v in set(st)},
                    "newton_iters_mean": float(np.mean([i["newton_iters"] for i in infos])),
                    "horizons": "uniform in [1024, 8192], seed 0", "x0": "synth_x0(b) for instance b"}
    sb.close()
    return out, {("synth", int(Tb[k]), k): sample}


LITERAL_T = [256, 1024, 4096, 16384]


def run_literal_dt(args, ptn, W, dev, flush, stream, tuned):
    """The cart-pole at the configuration's literal time step dt = 0.01 for every T (the
    horizon grows to 163.84 s): the co-state form (0) and the multiplier form (1), FP32 LQR
    with FP64 solves, tuned launch shape per T; status, Newton iterations and time."""
    import torch
    from paper_2409_20027_gb300 import autotune
    out = {"workload": "cart-pole IP at dt = 0.01 for every T (horizon 0.01 T s), x0 seed 0, FP32 LQR with FP64 "
                       "solves; the open-loop co-state map of the upright cart-pole grows like 1.0476^T"}
    x0 = torch.tensor(W.cartpole_x0(0), dtype=torch.float64, device=dev)
    for T in LITERAL_T:
        row = {}
        for mode in [0, 1]:
            sv = ptn.Solver(W.cartpole(dt=0.01), max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=mode)
            autotune.apply(sv, tuned, T)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, _, inf = sv.solve_ip(x0, T)
            b.record(stream)
            torch.cuda.synchronize()
            row[f"mode{mode}"] = {"ms": a.elapsed_time(b), "status": inf["status"], "newton_iters": inf["newton_iters"],
                                  "r_stat": inf["r_stat"], "J": inf["J"]}
            sv.close()
        out[str(T)] = row
    return out


def oracle_literal(T):
    """The oracle on the literal-dt cart-pole (seed 0): its status, Newton iterations, the
    largest co-state and log10 of the norm of the open-loop Jacobian product along its result."""
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    p = W.cartpole(dt=0.01)
    t0 = time.perf_counter()
    r = O.solve_ip(p, W.cartpole_x0(0), T)
    ms = (time.perf_counter() - t0) * 1e3
    M = np.eye(4)
    lg = 0.0
    for t in range(T):
        F, _ = O.jac(p, r["x"][t], r["u"][t])
        M = F @ M
        nm = np.linalg.norm(M)
        lg += np.log10(nm)
        M /= nm
    return {"status": r["info"]["status"], "newton_iters": r["info"]["newton_iters"], "ms": ms, "J": r["info"]["J"],
            "max_abs_lam": float(np.abs(r["lam"]).max()), "log10_norm_prod_F": lg}


def run_sequential(args, ptn, W, dev, flush, stream):
    """The paper's comparison axis on this GPU: the same single cart-pole solve (2.56 s
    horizon, T = 1024, FP32 LQR with FP64 solves) by the sequential-in-time baseline (one
    thread running the serial recursions) next to the parallel-in-time solve of the sweep.
    (Bounded to one solve: the FP64 sequential baseline runs for minutes on this GPU.)"""
    import torch
    out, sols = {}, {}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for T in [1024]:
        p = cartpole_instance(T)
        sv = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, sequential=1)
        xs = torch.tensor(W.cartpole_x0(0), dtype=torch.float64, device=dev)
        flush.zero_()
        a.record(stream)
        xq, uq, lq, inf = sv.solve_ip(xs, T)
        b.record(stream)
        torch.cuda.synchronize()
        out[str(T)] = {"ms": a.elapsed_time(b), "newton_iters": inf["newton_iters"], "status": inf["status"]}
        sols[("seq", T)] = (xq.cpu().numpy(), uq.cpu().numpy(), lq.cpu().numpy(), inf["J"])
        sv.close()
    return out, sols


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
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--no-quad", action="store_true")
    ap.add_argument("--quad-batch", type=int, default=256)
    ap.add_argument("--quad-T", type=int, default=1024)
    ap.add_argument("--no-mpc", action="store_true")
    ap.add_argument("--no-seq", action="store_true")
    ap.add_argument("--no-mult", action="store_true")
    ap.add_argument("--no-admm", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-pend", action="store_true")
    ap.add_argument("--no-synth", action="store_true")
    ap.add_argument("--no-literal", action="store_true")
    ap.add_argument("--synth-T", type=int, default=65536)
    ap.add_argument("--synth-batch", type=int, default=64)
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

    from paper_2409_20027_gb300 import autotune
    tuned = autotune.load(TUNED_TABLE) if os.path.exists(TUNED_TABLE) else {}
    p = cartpole_instance(T)
    solver = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE)
    launch = autotune.apply(solver, tuned, T)
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
        ms = max_over_ranks(ms, dist, dev)
    ok = all(i["status"] == 0 and i["r_kkt"] <= 1e-6 * (1 + 1e-9) for i in infos)

    # end to end through the public API with host buffers (pinned), copies in the region
    # (same inputs, in the same order, as the device-timed steps)
    x0hs = [x.cpu().pin_memory() for x in x0s]
    xh = torch.empty((T + 1, 4), dtype=torch.float64).pin_memory()
    uh = torch.empty((T, 1), dtype=torch.float64).pin_memory()
    x0d = torch.empty(4, dtype=torch.float64, device=dev)
    e2e = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x0d.copy_(x0hs[k % 10], non_blocking=True)
        solver.solve_ip(x0d, T, x_out=xo, u_out=uo, lam_out=lo)
        xh.copy_(xo, non_blocking=True)
        uh.copy_(uo, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = sum(e2e) / len(e2e)

    # the solution of the seed-0 solve, for the error against the oracle
    _, _, _, info0 = solver.solve_ip(x0s[0], T, x_out=xo, u_out=uo, lam_out=lo)
    gpu_out = {("cartpole", T, 0): (xo.cpu().numpy(), uo.cpu().numpy(), lo.cpu().numpy(), info0["J"])}

    # the sections below are single-GPU measurements: with N replicas only the headline
    # solve above is repeated on every GPU
    single = world == 1
    sweep = {}
    if not args.no_sweep and single:
        for Ts in SWEEP_T:
            if Ts == T:
                continue
            ps = cartpole_instance(Ts)
            sv = ptn.Solver(ps, max_T=Ts, precision=ptn.PTN_FP32_FP64SOLVE)
            autotune.apply(sv, tuned, Ts)
            x0 = x0s[0]
            sv.solve_ip(x0, Ts)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            xs_, us_, ls_, inf = sv.solve_ip(x0, Ts)
            b.record(stream)
            torch.cuda.synchronize()
            sweep[str(Ts)] = {"ms": a.elapsed_time(b), "newton_iters": inf["newton_iters"], "status": inf["status"],
                              "fp64_finish_iters": inf["finish_iters"],
                              "r_kkt": inf["r_kkt"], "us_per_newton_iter": 1e3 * a.elapsed_time(b) /
                              max(inf["newton_iters"], 1)}
            gpu_out[("cartpole", Ts, 0)] = (xs_.cpu().numpy(), us_.cpu().numpy(), ls_.cpu().numpy(), inf["J"])
            sv.close()
        sweep[str(T)] = {"ms": ms, "newton_iters": infos[-1]["newton_iters"], "status": infos[-1]["status"],
                         "fp64_finish_iters": [i["finish_iters"] for i in infos],
                         "r_kkt": infos[-1]["r_kkt"], "us_per_newton_iter": 1e3 * ms / max(infos[-1]["newton_iters"], 1),
                         "note": "the headline solves (mean over the timed steps)"}
        sweep["workload"] = ("cart-pole IP on the fixed 2.56 s horizon (dt = 2.56/T, RK4), x0 seed 0, tuned launch "
                             "shape per T, fp32 LQR with fp64 solves, KKT <= 1e-6")

    pend = None
    if not args.no_pend and single:
        pend, pend_out = run_pendulum(ptn, W, dev, flush, stream, tuned)
        gpu_out.update(pend_out)

    batch = None
    batch_out = {}
    if not args.no_batch and single:
        batch, batch_out = run_batch(args, ptn, W, dev, flush, stream)
    quad = None
    quad_out = {}
    if not args.no_quad and single:
        quad, quad_out = run_quadrotor(args, ptn, W, dev, flush, stream)
    literal = None
    if not args.no_literal and single:
        literal = run_literal_dt(args, ptn, W, dev, flush, stream, tuned)
    synth = None
    synth_out = {}
    if not args.no_synth and single:
        synth, synth_out = run_synth(args, ptn, W, dev, flush, stream)
    mpcl = None
    if not args.no_mpc and single:
        mpcl = run_mpc(ptn, W, dev, stream)
    # solutions compared with an oracle solve of another section's workload: key ->
    # (the oracle job, the GPU solution)
    cross_out = {}
    seq = None
    if not args.no_seq and single:
        seq, so = run_sequential(args, ptn, W, dev, flush, stream)
        cross_out.update({k: (("cartpole", k[1], 0), v) for k, v in so.items()})
    admm = None
    admm_out = {}
    if not args.no_admm and single:
        admm, admm_out = run_admm(args, ptn, W, dev, flush, stream, tuned, x0s[0])
    mult = None
    if not args.no_mult and single:
        mult, mo = run_multiplier(args, ptn, W, dev, flush, stream, tuned, x0s[0])
        cross_out.update({k: (("cartpole", k[1], 0), v) for k, v in mo.items()})
    peaks = measured_fma_peaks() if rank == 0 else None

    if rank != 0:
        return
    last = infos[-1]
    f32, f64 = flop_split(4, 1, T, last)
    achieved = (f32 + f64) / (per[-1] * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if peaks:
        p32, p64 = peaks["fp32"], peaks["fp64"]
        src = "measured"
        how = ("measured on this GPU by the FMA-throughput probe (include/ptn_peaks.h): FP32 %.1f TFLOP/s, FP64 "
               "%.2f TFLOP/s" % (p32, p64))
    else:
        p32 = sms * 128 * 2 * 2.07e9 / 1e12
        p64 = 1.25
        src = "nominal"
        how = "nominal: FP32 %d SMs x 128 lanes x 2 x 2.07 GHz = %.1f TFLOP/s, FP64 1.25 TFLOP/s" % (sms, p32)
    peak = blended_peak_tflops(f32, f64, p32, p64)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC_BYTES if T == 16384 else None, "kernel": "k_solve_grid<CartPole,float,double>",
            "peak_source": "%s; blended by this solve's FP32/FP64 flop split (%.1f%% FP64); %d SMs"
                           % (how, 100 * f64 / (f32 + f64), sms),
            "peak_kind": src, "fp32_peak": p32, "fp64_peak": p64}
    cpu = None
    errs = {}
    if not args.no_cpu_baseline and world == 1:
        # the oracle on the headline workload itself (one full solve, single thread) ...
        r16 = _oracle_ref(("cartpole", T, 0))
        cpu = {"value": r16["ms"], "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"one complete oracle IP solve of the workload (T={T}, seed 0), single thread on "
                         f"{host_cpu()}", "oracle_newton_iters": r16["info"]["newton_iters"]}
        refs = {("cartpole", T, 0): r16}
        # ... and every other result's reference solve, in parallel over the host cores
        jobs = [k for k in gpu_out if k not in refs]
        jobs += [("quad", b, args.quad_T) for b in quad_out]
        jobs += list(synth_out)
        jobs += list(admm_out)
        jobs += [j for j, _ in cross_out.values() if j not in refs and j not in jobs]
        if batch is not None:
            bc, bref = cpu_batch_baseline()
            batch["cpu_baseline"] = bc
            refs.update({("batch", k): r for k, r in bref.items()})
        try:
            res, _ = oracle_pool(jobs)
            refs.update(dict(zip(jobs, res)))
        except Exception as e:  # the GPU numbers must not depend on the host references
            errs["error"] = f"{type(e).__name__}: {e}"
        outs = dict(gpu_out)
        outs.update({("quad", b, args.quad_T): v for b, v in quad_out.items()})
        outs.update({("batch", k): v for k, v in batch_out.items()})
        outs.update(synth_out)
        outs.update(admm_out)
        for key, (x, u, lam, J) in outs.items():
            if key in refs:
                errs["/".join(str(v) for v in key)] = err_vs_oracle(refs[key], x, u, lam, J)
        for key, (job, (x, u, lam, J)) in cross_out.items():
            if job in refs:
                errs["/".join(str(v) for v in key)] = err_vs_oracle(refs[job], x, u, lam, J)
        if pend is not None:
            pend["oracle_ms_median"] = float(np.median([refs[("pendulum", sd)]["ms"] for sd in range(10)
                                                        if ("pendulum", sd) in refs] or [np.nan]))
    head_err = errs.get(f"cartpole/{T}/0")
    if not args.no_sweep and single and errs:
        for Ts in SWEEP_T:
            e = errs.get(f"cartpole/{Ts}/0")
            if e is not None:
                sweep[str(Ts)]["err_vs_oracle"] = e
    if pend is not None and errs:
        pend["err_vs_oracle_max"] = max_err([errs.get(f"pendulum/{sd}") for sd in range(10)])
    if batch is not None and errs:
        batch["err_vs_oracle_max"] = max_err([v for k, v in errs.items() if k.startswith("batch/")])
        batch["err_vs_oracle_sample"] = "the instances of cpu_baseline's sample"
    if quad is not None and errs:
        quad["err_vs_oracle_max"] = max_err([v for k, v in errs.items() if k.startswith("quad/")])
        quad["err_vs_oracle_sample"] = f"instances 0..{QUAD_ORACLE_SAMPLE - 1}"
    if literal is not None and not args.no_cpu_baseline and world == 1:
        for Tl in LITERAL_T[:3]:
            literal[str(Tl)]["oracle_mode0"] = oracle_literal(Tl)
    if synth is not None and errs:
        synth["batch"]["err_vs_oracle"] = max_err([v for k, v in errs.items() if k.startswith("synth/")])
        synth["batch"]["err_vs_oracle_sample"] = "the batch's shortest instance (oracle time grows as n^3 T)"
    if synth is not None:
        # the oracle's own solve of the single T = 65536 instance (stored: it takes minutes)
        gold = os.path.join(ROOT, "tests", "golden", "synth_T65536.json")
        if os.path.exists(gold) and synth["single"]["T"] == 65536:
            with open(gold) as f:
                g = json.load(f)["info"]
            synth["single"]["oracle"] = {"status": g["status"], "newton_iters": g["newton_iters"], "J": g["J"],
                                         "note": "stored oracle solve (tests/golden/synth_reference.py): the FP64 "
                                                 "oracle does not converge on this instance, so no error is stated"}
    if errs:
        if seq is not None:
            for Tq in seq:
                seq[Tq]["err_vs_oracle"] = errs.get(f"seq/{Tq}")
        if mult is not None:
            for Tm, row in mult["single"].items():
                for mode in [1, 2]:
                    e = errs.get(f"mult/{Tm}/{mode}")
                    if e is not None:
                        row[f"mode{mode}"]["err_vs_oracle"] = e
            mult["err_vs_oracle_reference"] = "the oracle's co-state form (mode 0) at the same instance"
        if admm is not None and "admm_pend/256" in errs:
            admm["pendulum_paper"]["256"]["err_vs_oracle"] = errs["admm_pend/256"]
    if literal is not None:
        for Tl, row in literal.items():
            o = row.get("oracle_mode0") if isinstance(row, dict) else None
            if o and o["status"] == 0:
                for mode in ["mode0", "mode1"]:
                    if row[mode]["status"] == 0:
                        row[mode]["J_err_vs_oracle"] = abs(row[mode]["J"] - o["J"]) / max(1.0, abs(o["J"]))
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": config(T),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": 4 * 8,
                    "d2h_bytes_per_step": ((T + 1) * 4 + T) * 8},
            "gpu_launches": sum(1 + (i["finish_iters"] > 0) for i in infos), "clocks": clocks, "kkt_ok": ok,
            "err_vs_oracle": head_err, "newton_iters": [i["newton_iters"] for i in infos],
            "fp64_finish_iters": [i["finish_iters"] for i in infos], "launch": launch or "defaults",
            "phase_share": phase_share(infos), "sweep": sweep, "pendulum": pend,
            "batch": batch, "quadrotor": quad, "synthetic": synth, "literal_dt": literal, "mpc": mpcl,
            "sequential": seq,
            "multiplier_form": mult, "admm": admm}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def max_err(es):
    """Component-wise maximum of err_vs_oracle records (None entries skipped)."""
    es = [e for e in es if e]
    if not es:
        return None
    out = {k: max((e[k] for e in es if e.get(k) is not None), default=None) for k in ("x", "u", "lam", "J")}
    out["instances"] = len(es)
    out["oracle_not_converged"] = sum(1 for e in es if e["oracle_status"] != 0)
    return out


if __name__ == "__main__":
    main()
