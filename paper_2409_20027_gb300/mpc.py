"""Closed-loop model predictive control with the batched solver: at every control period
solve the horizon-N problem from the current states of all closed loops at once, apply
the first control, advance the plant one step, and warm-start the next solve with the
shifted control sequence (receding horizon; the paper's closed-loop experiment, Sec. IV).

The plant is the same discrete model the controller uses (nominal MPC), so the next
state is the solve's predicted x_1.  Everything between solves is index arithmetic on
device tensors; every solve runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def shift_controls(u, T: int):
    """Warm start for the next period: drop the applied control and repeat the last one.
    u: (B * T, m) concatenated horizons of B loops.  Returns a new tensor."""
    import torch
    m = u.shape[1]
    v = u.reshape(-1, T, m)
    return torch.cat([v[:, 1:, :], v[:, -1:, :]], dim=1).reshape(-1, m).contiguous()


def closed_loop(solver, x0, T: int, steps: int, u_init=None, warm_start: bool = True, xref=None):
    """Run `steps` control periods for the B loops whose initial states are the rows of
    x0 (CUDA float64, B x n) with horizon T.  u_init: (B * T, m) first warm start (None:
    zeros, which must be strictly feasible for the interior-point method).
    Returns dict(x: (steps + 1, B, n) states, u: (steps, B, m) applied controls,
    iters: (steps, B) Newton iterations, status: (steps, B))."""
    import torch
    B, n = x0.shape
    m = solver.nu
    xs = [x0.clone()]
    us, its, sts = [], [], []
    x = x0.contiguous()
    u_ws = u_init
    Tb = np.full(B, T, dtype=np.int32)
    for _ in range(steps):
        X, U, _, infos = solver.solve_batch(x, Tb, xref=xref, u_init=u_ws)
        Xv = X.reshape(B, T + 1, n)
        Uv = U.reshape(B, T, m)
        us.append(Uv[:, 0, :].clone())
        its.append([i["newton_iters"] for i in infos])
        sts.append([i["status"] for i in infos])
        x = Xv[:, 1, :].contiguous()
        xs.append(x.clone())
        u_ws = shift_controls(U, T) if warm_start else u_init
    return {"x": torch.stack(xs), "u": torch.stack(us), "iters": np.asarray(its), "status": np.asarray(sts)}
