"""Pins for time-varying tracking targets in the oracle (stage cost l_t with targets
x*_t, u*_t that vary with t; Sec. II-A's l_t): the problem statement allows a different
stage cost at every step, and a tracking reference trajectory is the common case.

R1  LQ special case: one Newton step from any point is the exact minimiser of the dense
    condensed QP whose targets are the trajectories (not a constant).
R2  constant trajectories reproduce the constant-target solve bit for bit.
R3  the adjoint's weight gradients with time-varying targets match finite differences of
    re-solved problems.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2409_20027_gb300 import workloads as W

INF = np.inf


def test_lq_newton_step_tracks_time_varying_targets():
    rng = np.random.default_rng(3)
    n, m, T = 4, 2, 10
    p = W.synth(0, nx=n, nu=m)
    xr_t = rng.normal(size=(T + 1, n))
    ur_t = rng.normal(size=(T, m))
    p = p.replace(W=np.zeros((n, n)), ulo=np.full(m, -INF), uhi=np.full(m, INF), Qf=2.0 * p.Q,
                  xref_traj=xr_t, uref_traj=ur_t)
    x0 = rng.normal(size=n)
    u = rng.normal(size=(T, m))
    x = O.rollout(p, x0, u)
    nd = O.newton_direction(p, x, u, 0.0, "none")
    assert nd["status"] == 0
    Su = np.zeros(((T + 1) * n, T * m)); sx = np.zeros((T + 1) * n)
    for t in range(T + 1):
        sx[t * n:(t + 1) * n] = np.linalg.matrix_power(p.A, t) @ x0
        for k in range(t):
            Su[t * n:(t + 1) * n, k * m:(k + 1) * m] = np.linalg.matrix_power(p.A, t - 1 - k) @ p.B
    Qb = sla.block_diag(*([p.Q] * T + [p.Qf]))
    Rb = sla.block_diag(*([p.R] * T))
    H = 2 * (Su.T @ Qb @ Su + Rb)
    g = 2 * (Su.T @ Qb @ (sx - xr_t.ravel()) - Rb @ ur_t.ravel())
    ustar = np.linalg.solve(H, -g).reshape(T, m)
    assert np.allclose(u + nd["du"], ustar, rtol=1e-9, atol=1e-9)
    # the cost evaluates the targets step by step
    xs = O.rollout(p, x0, ustar)
    J = sum((xs[t] - xr_t[t]) @ p.Q @ (xs[t] - xr_t[t]) + (ustar[t] - ur_t[t]) @ p.R @ (ustar[t] - ur_t[t])
            for t in range(T)) + (xs[T] - xr_t[T]) @ p.Qf @ (xs[T] - xr_t[T])
    assert O.cost(p, xs, ustar)[1] == pytest.approx(J, rel=1e-12)


def test_constant_trajectories_reproduce_constant_targets():
    p = W.cartpole(T=64, horizon=2.56)
    T = 64
    x0 = W.cartpole_x0(1)
    a = O.solve_ip(p, x0, T)
    q = p.replace(xref_traj=np.tile(p.xref, (T + 1, 1)), uref_traj=np.tile(p.uref, (T, 1)))
    b = O.solve_ip(q, x0, T)
    assert a["info"]["newton_iters"] == b["info"]["newton_iters"]
    for k in ["x", "u", "lam"]:
        assert np.array_equal(a[k], b[k])


def _loss(p, x0, T, mu, u_warm):
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, u_warm)
    assert r["info"]["status"] == 0
    return r["info"]["J_c"]


def test_adjoint_weight_gradients_with_time_varying_targets():
    p, T, mu = W.pendulum(), 15, 1e-2
    t = np.arange(T + 1)
    xr_t = np.stack([np.pi * t / T, 0.3 * np.sin(t)], axis=1)   # swing up along a ramp
    ur_t = 0.5 * np.cos(t[:T])[:, None]
    p = p.replace(xref_traj=xr_t, uref_traj=ur_t)
    x0 = W.pendulum_x0(2)
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, np.zeros((T, 1)))
    assert r["info"]["status"] == 0
    a = O.adjoint(p, mu, r["x"], r["u"], 1.0)
    assert a["status"] == 0
    us = r["u"]

    def fd(mod, h=1e-5):
        def cd(hh):
            return (_loss(mod(+hh), x0, T, mu, us) - _loss(mod(-hh), x0, T, mu, us)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    for i in range(p.nx):
        E = np.zeros((p.nx, p.nx)); E[i, i] = 1
        num = fd(lambda s: p.replace(Q=p.Q + s * E))
        assert a["Qd"][i] == pytest.approx(num, rel=1e-5, abs=1e-6 * max(1.0, abs(num)))
        num = fd(lambda s: p.replace(Qf=p.Qf + s * E))
        assert a["Qfd"][i] == pytest.approx(num, rel=1e-5, abs=1e-6 * max(1.0, abs(num)))
    E = np.ones((1, 1))
    num = fd(lambda s: p.replace(R=p.R + s * E))
    assert a["Rd"][0] == pytest.approx(num, rel=1e-5, abs=1e-6 * max(1.0, abs(num)))
