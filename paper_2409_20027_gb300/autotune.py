"""Launch-shape autotuner: an offline sweep of the launch options of a solve (threads per
CTA, time steps per thread, whether a single solve may use a thread-block cluster) for
each horizon bucket of a model and precision, and the lookup that applies the fastest
shape to a solver before a solve.

The sweep times real solves through the C ABI (``ptn.Solver``), so it needs the CUDA
library and a GPU; the table it writes is plain JSON and the lookup is host logic.
"""
from __future__ import annotations

import json
import os

# upper bounds of the horizon buckets
BUCKETS = [64, 256, 1024, 4096, 16384, 65536]

# launch shapes swept by default (fields of ptn_options)
CANDIDATES = [
    {"block_threads": 64, "grid_steps_per_thread": 2, "cluster_max_blocks": 16},
    {"block_threads": 128, "grid_steps_per_thread": 2, "cluster_max_blocks": 16},
    {"block_threads": 256, "grid_steps_per_thread": 2, "cluster_max_blocks": 16},
    {"block_threads": 128, "grid_steps_per_thread": 4, "cluster_max_blocks": 16},
    {"block_threads": 128, "grid_steps_per_thread": 2, "cluster_max_blocks": 0},
    {"block_threads": 128, "grid_steps_per_thread": 1, "cluster_max_blocks": 0},
    {"block_threads": 128, "grid_steps_per_thread": 4, "cluster_max_blocks": 0},
    {"block_threads": 32, "grid_steps_per_thread": 2, "cluster_max_blocks": 16},
    {"block_threads": 64, "grid_steps_per_thread": 1, "cluster_max_blocks": 16},
    {"block_threads": 128, "grid_steps_per_thread": 1, "cluster_max_blocks": 16},
]


def bucket_of(T: int) -> int:
    """The smallest bucket bound >= T (the largest bound for longer horizons)."""
    if T < 1:
        raise ValueError("horizon must be >= 1")
    for b in BUCKETS:
        if T <= b:
            return b
    return BUCKETS[-1]


def key(model: int, precision: int) -> str:
    return f"model{int(model)}-prec{int(precision)}"


def tuned_options(table: dict, model: int, precision: int, T: int) -> dict:
    """Launch options for a solve of horizon T, or {} when the table has no entry for the
    model, precision and bucket (the solver's options then stay as they are)."""
    ent = table.get(key(model, precision), {}).get(str(bucket_of(T)))
    return dict(ent["options"]) if ent else {}


def apply(solver, table: dict, T: int) -> dict:
    """Set the solver's launch options for horizon T from the table; returns them."""
    opts = tuned_options(table, solver.prob.model, solver.options.precision, T)
    if opts:
        solver.set_options(**opts)
    return opts


def sweep(prob, x0, Ts, precision: int, candidates=None, reps: int = 2, u_init=None, table=None) -> dict:
    """Time every candidate shape on a solve of each horizon in Ts (one representative per
    bucket) and record the fastest converged one.  x0: a CUDA float64 tensor.  Returns
    the updated table."""
    import torch

    from . import ptn

    table = {} if table is None else table
    cands = CANDIDATES if candidates is None else candidates
    ent = table.setdefault(key(prob.model, precision), {})
    for T in Ts:
        s = ptn.Solver(prob, max_T=T, precision=precision)
        best = None
        for c in cands:
            s.set_options(**c)
            ui = None if u_init is None else u_init(T)
            try:
                s.solve_ip(x0, T, u_init=ui)  # warm-up
            except ptn.PtnError:
                continue  # a shape this device or horizon cannot take
            torch.cuda.synchronize()
            times = []
            ok = True
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                _, _, _, info = s.solve_ip(x0, T, u_init=ui)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
                ok &= info["status"] == 0
            ms = min(times)
            if ok and (best is None or ms < best["ms"]):
                best = {"options": dict(c), "ms": ms, "T": int(T)}
        s.close()
        if best is not None:
            ent[str(bucket_of(T))] = best
    return table


def save(table: dict, path: str) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)


def default_sweep(out_path: str) -> dict:
    """Sweep the cart-pole workload (fixed 2.56 s horizon, FP32 LQR with FP64 solves) at
    T = 256 ... 16384 and the pendulum (FP64) at T = 64; write the table to out_path."""
    import torch

    from . import ptn, workloads as W

    dev = torch.device("cuda:0")
    table = {}
    for T in [256, 1024, 4096, 16384]:
        x0 = torch.tensor(W.cartpole_x0(0), dtype=torch.float64, device=dev)
        sweep(W.cartpole(T=T, horizon=2.56), x0, [T], ptn.PTN_FP32_FP64SOLVE, table=table)
    x0 = torch.tensor(W.pendulum_x0(0), dtype=torch.float64, device=dev)
    sweep(W.pendulum(), x0, [64], ptn.PTN_FP64, table=table)
    save(table, out_path)
    return table


if __name__ == "__main__":
    import sys

    default_sweep(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "tuned_gb300.json"))
