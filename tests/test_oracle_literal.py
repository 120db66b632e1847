"""Pins of the oracle's update of Alg. 4 as printed (update_mode 1: x <- x + dx, u <- u + du,
no rollout), against things other than the update loop itself:

- on a linear-quadratic problem (the synthetic map with c = 0, no bounds) the linearised
  dynamics are exact, so the printed update and the rollout update reach the same KKT point
  with no dynamics defect;
- one printed update from a consistent nominal equals (dx, du) of the oracle's one-step
  routine (newton_direction, separate code);
- the dynamics defect it leaves is the model's Taylor remainder
  -(f(x + dx, u + du) - f(x, u) - F dx - G du), and near the solution it matches the
  second-order term -1/2 dz^T f_zz dz from the model's Hessians.
"""
import numpy as np

import oracle as O
from paper_2409_20027_gb300 import workloads as W

LITERAL = O.Options(update_mode=1)
MU = 0.1


def test_printed_update_on_a_linear_quadratic_problem():
    p = W.synth(3, nx=4, nu=2)
    p = p.replace(prm=np.array([0.0]), ulo=np.full(2, -np.inf), uhi=np.full(2, np.inf))
    x0 = W.synth_x0(3, nx=4)
    T = 20
    a = O.solve_ip(p, x0, T, opts=LITERAL)
    b = O.solve_ip(p, x0, T)
    assert a["info"]["status"] == 0 and b["info"]["status"] == 0
    assert np.abs(a["x"] - b["x"]).max() <= 1e-10 and np.abs(a["u"] - b["u"]).max() <= 1e-10
    assert a["info"]["r_dyn"] <= 1e-12 and a["info"]["r_stat"] <= 1e-6


def _one_literal_step(p, x0, u0, T):
    opts = O.Options(update_mode=1, mu0=MU, mu_final=MU, max_newton=1, tol_final=1e-14, tol_inner=1e-14)
    return O.solve_ip(p, x0, T, u_init=u0, opts=opts)


def _near_solution(p, x0, T):
    """A strictly feasible nominal near the solution at barrier weight MU (small, feasible
    steps): its controls shrunk by 0.1 % towards zero, inside the torque box."""
    sol = O.solve_ip(p, x0, T, opts=O.Options(mu0=MU, mu_final=MU))
    return 0.999 * sol["u"]


def test_one_printed_update_is_the_newton_direction():
    p = W.pendulum()
    T = 30
    x0 = W.pendulum_x0(4)
    u0 = _near_solution(p, x0, T)
    xh = O.rollout(p, x0, u0)
    nd = O.newton_direction(p, xh, u0, 1e-6, "barrier", MU)
    r = _one_literal_step(p, x0, u0, T)
    assert r["info"]["newton_iters"] == 1
    assert np.abs(r["x"] - (xh + nd["dx"])).max() <= 1e-12 * max(1.0, np.abs(xh).max())
    assert np.abs(r["u"] - (u0 + nd["du"])).max() <= 1e-12 * max(1.0, np.abs(u0 + nd["du"]).max())


def test_defects_of_the_printed_update_are_the_taylor_remainder():
    p = W.pendulum()
    T = 30
    x0 = W.pendulum_x0(4)
    u0 = _near_solution(p, x0, T)
    xh = O.rollout(p, x0, u0)
    r = _one_literal_step(p, x0, u0, T)
    dx, du = r["x"] - xh, r["u"] - u0
    for t in range(T):
        F, G = O.jac(p, xh[t], u0[t])
        remainder = O.step(p, r["x"][t], r["u"][t]) - O.step(p, xh[t], u0[t]) - F @ dx[t] - G @ du[t]
        defect = r["x"][t + 1] - O.step(p, r["x"][t], r["u"][t])
        assert np.abs(defect + remainder).max() <= 1e-12
        # second order: -1/2 dz^T (e_i^T f)_zz dz per component i
        pred = np.zeros(2)
        for i in range(2):
            Hxx, Hxu, Huu = O.hess(p, xh[t], u0[t], np.eye(2)[i])
            pred[i] = -0.5 * (dx[t] @ Hxx @ dx[t] + 2 * dx[t] @ Hxu @ du[t] + du[t] @ Huu @ du[t])
        scale = max(np.abs(pred).max(), 1e-14)
        assert np.abs(defect - pred).max() <= 0.1 * scale + 1e-13, (t, defect, pred)
