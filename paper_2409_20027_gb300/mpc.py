"""Closed-loop model predictive control with the batched solver: at every control period
solve the horizon-N problem from the current states of all closed loops at once, apply
the first control, advance the plant one step, and warm-start the next solve with the
shifted control sequence (receding horizon; the paper's closed-loop experiment, Sec. IV).

The plant is the same discrete model the controller uses (nominal MPC), so the next
state is the solve's predicted x_1.  Everything between solves is index arithmetic on
device tensors; every solve runs in the CUDA library.  closed_loop_graph records one
control period (solve, plant step, warm-start shift) as a CUDA graph and replays it, so
consecutive periods run without a host round trip.
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


class GraphLoop:
    """One control period of closed_loop (batched solve by ptn_solve_batch_async, plant
    step x <- x_1, shifted warm start) captured once as a CUDA graph on fixed device
    buffers; run() replays it period after period from the initial states, copying the
    history out between replays without synchronising.  Arguments as closed_loop
    (u_init None: zeros)."""

    def __init__(self, solver, x0, T: int, u_init=None, xref=None):
        import torch

        from . import ptn

        B, n = x0.shape
        m = solver.nu
        dev = x0.device
        self.B, self.n, self.m, self.dev = B, n, m, dev
        solver.prepare_batch(np.full(B, T, dtype=np.int32))
        self.x_init = x0.clone().contiguous()
        self.w_init = (torch.zeros((B * T, m), dtype=torch.float64, device=dev) if u_init is None
                       else u_init.clone().contiguous())
        x = self.x_init.clone()
        u_ws = self.w_init.clone()
        X = torch.empty((B * (T + 1), n), dtype=torch.float64, device=dev)
        U = torch.empty((B * T, m), dtype=torch.float64, device=dev)
        lam = torch.empty_like(X)
        u_first = torch.empty((B, m), dtype=torch.float64, device=dev)
        info = solver.new_info_buffer(B, dev)
        Uv, Xv, Wv = U.view(B, T, m), X.view(B, T + 1, n), u_ws.view(B, T, m)

        def period():
            solver.solve_batch_async(x, xref=xref, u_init=u_ws, x_out=X, u_out=U, lam_out=lam, info_dev=info)
            u_first.copy_(Uv[:, 0, :])
            x.copy_(Xv[:, 1, :])
            Wv[:, :-1, :].copy_(Uv[:, 1:, :])
            Wv[:, -1, :].copy_(Uv[:, -1, :])

        # one eager period on a side stream loads every kernel before the capture
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            period()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            period()
        self.x, self.u_ws, self.u_first = x, u_ws, u_first
        self.status = ptn.status_view(info, B)
        self._keep = (X, U, lam, info)

    def run(self, steps: int) -> dict:
        import torch

        B, n, m, dev = self.B, self.n, self.m, self.dev
        self.x.copy_(self.x_init)
        self.u_ws.copy_(self.w_init)
        xs = torch.empty((steps + 1, B, n), dtype=torch.float64, device=dev)
        us = torch.empty((steps, B, m), dtype=torch.float64, device=dev)
        st = torch.empty((steps, B, 2), dtype=torch.int32, device=dev)
        xs[0].copy_(self.x)
        for k in range(steps):
            self.graph.replay()
            xs[k + 1].copy_(self.x)
            us[k].copy_(self.u_first)
            st[k].copy_(self.status)
        stc = st.cpu().numpy()
        return {"x": xs, "u": us, "iters": stc[:, :, 1], "status": stc[:, :, 0]}


def closed_loop_graph(solver, x0, T: int, steps: int, u_init=None, xref=None):
    """closed_loop with warm starts, each period replayed from one captured CUDA graph
    (GraphLoop).  Same arguments and result as closed_loop."""
    return GraphLoop(solver, x0, T, u_init=u_init, xref=xref).run(steps)
