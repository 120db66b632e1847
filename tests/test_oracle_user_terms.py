"""Pins for user-written terms in the oracle (the general stage cost l_t, terminal cost l_T
and inequality rows g_t(x, u) <= 0 of Sec. II-A, eq. ocp), given as callbacks with their
derivatives over z = (x, u).

U1  callbacks that restate the quadratic tracking cost and the box bounds reproduce the
    built-in terms (same iterates, same solution);
U2  LQ special case with an x-u cross term in the user cost: one Newton step is the exact
    minimiser of the dense condensed QP (pins the cross block of the Hessian);
U3  the control gradient d_t with a non-quadratic user cost and a nonlinear user row
    equals finite differences of the barrier cost along the rollout;
U4  KKT invariants at the interior-point solution with a nonlinear user row.
"""
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2409_20027_gb300 import workloads as W

INF = np.inf


def quad_terms(p, box_rows=None):
    """User callbacks restating l_t = e^T Q e + eu^T R eu and l_T = e^T Qf e (and, with
    box_rows = [(is_x, index, sign, bound)], the box rows sign (z_k - bound) <= 0)."""
    n, m = p.nx, p.nu
    Hs = sla.block_diag(p.Q + p.Q.T, p.R + p.R.T)

    def stage(t, x, u):
        e, eu = x - p.xref, u - p.uref
        return e @ p.Q @ e + eu @ p.R @ eu, Hs @ np.concatenate([e, eu]), Hs

    def terminal(x):
        e = x - p.xref
        return e @ p.Qf @ e, (p.Qf + p.Qf.T) @ e, p.Qf + p.Qf.T

    ut = SimpleNamespace(stage=stage, terminal=terminal, constraints=None, nc=0)
    if box_rows:
        K = n + m

        def constraints(t, x, u):
            z = np.concatenate([x, u])
            g = np.array([sg * (z[(0 if isx else n) + k] - b) for isx, k, sg, b in box_rows])
            J = np.zeros((len(box_rows), K))
            for r, (isx, k, sg, b) in enumerate(box_rows):
                J[r, (0 if isx else n) + k] = sg
            return g, J, np.zeros((len(box_rows), K, K))
        ut.constraints, ut.nc = constraints, len(box_rows)
    return ut


def test_restated_quadratic_cost_and_box_rows_reproduce_builtin():
    p, T = W.pendulum(), 40
    x0 = W.pendulum_x0(3)
    a = O.solve_ip(p, x0, T)
    rows = [(False, 0, 1.0, p.uhi[0]), (False, 0, -1.0, p.ulo[0])]
    q = p.replace(ulo=np.full(1, -INF), uhi=np.full(1, INF), user_terms=quad_terms(p, rows))
    b = O.solve_ip(q, x0, T)
    assert b["info"]["status"] == 0 and a["info"]["newton_iters"] == b["info"]["newton_iters"]
    for k in ["x", "u", "lam"]:
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(1.0, np.abs(a[k]).max())


def test_lq_user_cost_with_cross_term_newton_step_is_exact():
    rng = np.random.default_rng(8)
    n, m, T = 4, 2, 9
    p = W.synth(1, nx=n, nu=m)
    p = p.replace(W=np.zeros((n, n)), ulo=np.full(m, -INF), uhi=np.full(m, INF), Qf=2.0 * p.Q)
    Cxu = 0.2 * rng.normal(size=(n, m))   # l_t = x^T Q x + u^T R u + 2 x^T Cxu u + c^T x
    cx = rng.normal(size=n)
    H = np.block([[p.Q + p.Q.T, 2 * Cxu], [2 * Cxu.T, p.R + p.R.T]])

    def stage(t, x, u):
        z = np.concatenate([x, u])
        g = H @ z + np.concatenate([cx, np.zeros(m)])
        return x @ p.Q @ x + u @ p.R @ u + 2 * x @ Cxu @ u + cx @ x, g, H

    def terminal(x):
        return x @ p.Qf @ x, (p.Qf + p.Qf.T) @ x, p.Qf + p.Qf.T

    q = p.replace(user_terms=SimpleNamespace(stage=stage, terminal=terminal, constraints=None, nc=0))
    x0 = rng.normal(size=n)
    u = rng.normal(size=(T, m))
    x = O.rollout(q, x0, u)
    nd = O.newton_direction(q, x, u, 0.0, "none")
    assert nd["status"] == 0
    # dense condensed QP over u: x = sx + Su u
    Su = np.zeros(((T + 1) * n, T * m)); sx = np.zeros((T + 1) * n)
    for t in range(T + 1):
        sx[t * n:(t + 1) * n] = np.linalg.matrix_power(p.A, t) @ x0
        for k in range(t):
            Su[t * n:(t + 1) * n, k * m:(k + 1) * m] = np.linalg.matrix_power(p.A, t - 1 - k) @ p.B
    Qb = sla.block_diag(*([p.Q + p.Q.T] * T + [p.Qf + p.Qf.T]))
    Rb = sla.block_diag(*([p.R + p.R.T] * T))
    Cb = np.zeros(((T + 1) * n, T * m))
    for t in range(T):
        Cb[t * n:(t + 1) * n, t * m:(t + 1) * m] = 2 * Cxu
    cb = np.concatenate([np.tile(cx, T), np.zeros(n)])
    Hu = Su.T @ Qb @ Su + Rb + Su.T @ Cb + Cb.T @ Su
    gu = Su.T @ Qb @ sx + Cb.T @ sx + Su.T @ cb
    ustar = np.linalg.solve(Hu, -gu).reshape(T, m)
    assert np.allclose(u + nd["du"], ustar, rtol=1e-9, atol=1e-9)


def pendulum_user_problem():
    """The pendulum with a non-quadratic user stage cost (a quartic term on the angle
    error and a 1 - cos term), a user terminal cost, and a time-varying nonlinear row
    on the angular rate: w^2 <= 9 + 0.05 t."""
    p = W.pendulum()
    n, m = 2, 1

    def stage(t, x, u):
        e = x[0] - np.pi
        l = e ** 2 + 0.1 * x[1] ** 2 + 0.01 * u[0] ** 2 + 0.05 * e ** 4 + 0.3 * (1 - np.cos(x[0] - np.pi))
        g = np.array([2 * e + 0.2 * e ** 3 + 0.3 * np.sin(x[0] - np.pi), 0.2 * x[1], 0.02 * u[0]])
        H = np.diag([2 + 0.6 * e ** 2 + 0.3 * np.cos(x[0] - np.pi), 0.2, 0.02])
        return l, g, H

    def terminal(x):
        e = x[0] - np.pi
        return 10 * e ** 2 + x[1] ** 2, np.array([20 * e, 2 * x[1]]), np.diag([20.0, 2.0])

    def constraints(t, x, u):
        g = np.array([x[1] ** 2 - (9.0 + 0.05 * t)])
        J = np.array([[0.0, 2 * x[1], 0.0]])
        Hc = np.zeros((1, 3, 3)); Hc[0, 1, 1] = 2.0
        return g, J, Hc

    return p.replace(user_terms=SimpleNamespace(stage=stage, terminal=terminal, constraints=constraints, nc=1))


def test_user_terms_gradient_matches_finite_differences():
    p, T, mu = pendulum_user_problem(), 12, 0.05
    rng = np.random.default_rng(4)
    x0 = W.pendulum_x0(1)
    u = 0.5 * rng.uniform(-1, 1, size=(T, 1))
    x = O.rollout(p, x0, u)
    d = O.newton_direction(p, x, u, 1e6, "barrier", mu)["d"]
    h = 1e-6
    fd = np.zeros_like(u)
    for t in range(T):
        up = u.copy(); up[t, 0] += h
        um = u.copy(); um[t, 0] -= h
        fd[t, 0] = (O.cost(p, O.rollout(p, x0, up), up, "barrier", mu)[0]
                    - O.cost(p, O.rollout(p, x0, um), um, "barrier", mu)[0]) / (2 * h)
    assert np.abs(d - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_ip_with_user_row_satisfies_kkt_invariants():
    p, T = pendulum_user_problem(), 64
    r = O.solve_ip(p, W.pendulum_x0(0), T)
    i = r["info"]
    assert i["status"] == 0 and i["r_kkt"] <= 1e-6 * (1 + 1e-9) and i["r_feas"] == 0.0
    w = r["x"][:T, 1]
    assert np.all(w ** 2 < 9.0 + 0.05 * np.arange(T))   # strictly inside the user row
    # the row is active somewhere (else the test would not exercise it)
    assert np.max(w ** 2 - (9.0 + 0.05 * np.arange(T))) > -0.5
