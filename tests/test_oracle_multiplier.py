"""Pins for the oracle's multiplier form of the co-states (a variant of the method: the
co-state recursion of Sec. III-B is replaced by multipliers nu of the dynamics, updated
by the duals of each Newton step's LQR).

M1  Linear dynamics: the model Hessian vanishes and the multiplier terms of the
    Lagrangian telescope along the linearised dynamics, so the Newton direction and the
    model terms G1, G2 equal those of the co-state form for ANY nu; with nu = the
    co-states, the x-gradient q vanishes and d is the co-state form's d.
M2  LQ problem, alpha = 0: one step reaches the optimum, and nu + dnu are the co-states
    there, computed here by the backward recursion written from the problem definition.
M3  Nonlinear IP problems: the multiplier form ends at the co-state form's KKT point
    (x, u and lam = nu), which the pins of test_oracle_newton tie to the paper.
M4  ADMM at a fixed outer count: the same iterate (x, u, z, v).
Mode 2 restarts the multipliers from the recursion's co-states at every Newton
sub-problem (barrier level); it must reach the same KKT point as well, including on a
batch instance where the pure form stalls.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

RNG = np.random.default_rng(23)
INF = np.inf


def _lq_problem(n=4, m=2, seed=0):
    p = W.synth(seed, nx=n, nu=m)
    return p.replace(W=np.zeros((n, n)), ulo=np.full(m, -INF), uhi=np.full(m, INF),
                     xref=RNG.normal(size=n), uref=RNG.normal(size=m), Qf=2.0 * p.Q)


def _lq_costates(p, x):
    """Co-states of the LQ problem at states x: stage cost (x - x*)^T Q (x - x*) + ...
    (no 1/2), so lam_{N+1} = 2 Qf (x_{N+1} - x*), lam_t = 2 Q (x_t - x*) + A^T lam_{t+1}."""
    T = x.shape[0] - 1
    lam = np.zeros_like(x)
    lam[T] = 2.0 * p.Qf @ (x[T] - p.xref)
    for t in range(T - 1, -1, -1):
        lam[t] = 2.0 * p.Q @ (x[t] - p.xref) + p.A.T @ lam[t + 1]
    return lam


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(1.0, np.abs(np.asarray(b)).max()))


@pytest.mark.parametrize("seed", [0, 1])
def test_direction_is_independent_of_multipliers_for_linear_dynamics(seed):
    p = _lq_problem(seed=seed)
    n, m, T = p.nx, p.nu, 12
    x0 = RNG.normal(size=n)
    u = RNG.normal(size=(T, m))
    x = O.rollout(p, x0, u)
    nu = 5.0 * RNG.normal(size=(T + 1, n))
    a = O.newton_direction(p, x, u, 1e-3, "none")
    b = O.newton_direction_mult(p, x, u, nu, 1e-3, "none")
    assert a["status"] == 0 and b["status"] == 0
    assert np.allclose(b["du"], a["du"], rtol=1e-9, atol=1e-9)
    assert np.allclose(b["dx"], a["dx"], rtol=1e-9, atol=1e-9)
    assert b["G1"] == pytest.approx(a["G1"], rel=1e-9, abs=1e-9)
    assert b["G2"] == pytest.approx(a["G2"], rel=1e-9, abs=1e-9)
    # with the co-states as multipliers the Lagrangian's x-gradient vanishes
    c = O.newton_direction_mult(p, x, u, a["lam"], 1e-3, "none")
    assert np.abs(c["q"]).max() <= 1e-9 * max(1.0, np.abs(a["lam"]).max())
    assert np.allclose(c["d"], a["d"], rtol=1e-10, atol=1e-10)


def test_dual_step_lands_on_the_lq_costates():
    p = _lq_problem(n=3, m=2, seed=4)
    n, m, T = p.nx, p.nu, 10
    x0 = RNG.normal(size=n)
    u = RNG.normal(size=(T, m))
    x = O.rollout(p, x0, u)
    nu = 3.0 * RNG.normal(size=(T + 1, n))
    b = O.newton_direction_mult(p, x, u, nu, 0.0, "none")
    assert b["status"] == 0
    x1, u1 = x + b["dx"], u + b["du"]
    assert np.allclose(x1, O.rollout(p, x0, u1), rtol=1e-10, atol=1e-10)
    lam = _lq_costates(p, x1)
    # row 0 of nu is replaced by its local definition before the step
    nu0 = nu.copy()
    nu0[0] = 2.0 * p.Q @ (x[0] - p.xref) + p.A.T @ nu[1]
    assert np.allclose(nu0 + b["dnu"], lam, rtol=1e-8, atol=1e-8)
    # and the step reached the optimum: the co-state form's gradient vanishes there
    a = O.newton_direction(p, x1, u1, 0.0, "none")
    assert np.abs(a["d"]).max() <= 1e-8 * max(1.0, np.abs(lam).max())


CASES = {
    "pendulum-64": (W.pendulum(), W.pendulum_x0(0), 64),
    "cartpole-128": (W.cartpole(), W.cartpole_x0(1), 128),
    "cartpole-256-fixed-horizon": (W.cartpole(T=256, horizon=2.56), W.cartpole_x0(2), 256),
}


def _batch_instance(k, B=1024, horizon=1.28):
    """Instance k of the batch workload: T_b log-uniform [64, 4096] (seed 0), the 1.28 s
    horizon at dt_b = 1.28 / T_b with the stage weights scaled by dt_b / dt."""
    Tb = W.batch_horizons(B, seed=0)
    base = W.cartpole()
    dt = horizon / float(Tb[k])
    sc = dt / base.dt
    return base.replace(dt=dt, Q=base.Q * sc, R=base.R * sc), W.cartpole_batch_x0(B, seed=0)[k], int(Tb[k])


# instance 310 (T = 130): the pure multiplier form stalls there (as on a few other short
# batch instances); the form restarted from the co-states at each barrier level does not
CASES["batch-310"] = _batch_instance(310)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", list(CASES))
def test_multiplier_form_reaches_the_costate_form_kkt_point(case, mode):
    p, x0, T = CASES[case]
    if case == "batch-310" and mode == 1:
        r = O.solve_ip(p, x0, T, opts=O.Options(costate_mode=1))
        assert r["info"]["status"] == -3  # documented limitation of the pure form
        return
    a = O.solve_ip(p, x0, T)
    b = O.solve_ip(p, x0, T, opts=O.Options(costate_mode=mode))
    assert a["info"]["status"] == 0 and b["info"]["status"] == 0
    assert rel(b["x"], a["x"]) <= 1e-9
    assert rel(b["u"], a["u"]) <= 1e-9
    assert rel(b["lam"], a["lam"]) <= 1e-9
    assert b["info"]["J"] == pytest.approx(a["info"]["J"], rel=1e-12)
    assert b["info"]["r_stat"] <= 1e-6 and b["info"]["r_dyn"] <= 1e-9


def test_multiplier_form_admm_fixed_outer_count():
    p = W.cartpole()
    x0, T, K = W.cartpole_x0(3), 120, 10
    a = O.solve_admm(p, x0, T, opts=O.Options(admm_fixed_iters=K, tol_final=1e-9))
    b = O.solve_admm(p, x0, T, opts=O.Options(admm_fixed_iters=K, tol_final=1e-9, costate_mode=1))
    assert a["info"]["status"] == 0 and b["info"]["status"] == 0
    # (lam is not compared: after the last z, v update the co-state form recomputes its
    # co-states under the new penalty terms, while nu stays the multiplier of the last
    # Newton sub-problem)
    for k in ["x", "u", "z", "v"]:
        assert rel(b[k], a[k]) <= 1e-8, k


def test_multiplier_form_solves_where_the_costate_recursion_breaks_down():
    # synthetic x+ = A x + B u + c tanh(W x), n = 6, m = 2, seed 9: the Jacobian at the
    # origin has spectral radius 1.017, so the co-state recursion's products of F_t^T grow
    # like 1.017^T.  At T = 512 both forms reach the same KKT point; at T = 1024 the
    # recursion-based Newton step breaks down while the multiplier form converges, to the
    # same cost (the state has settled by step 512, so the longer horizon adds nothing)
    p = W.synth(9, nx=6, nu=2)
    rho = max(abs(np.linalg.eigvals(p.A + p.prm[0] * p.W)))
    assert rho > 1.01
    x0 = W.synth_x0(9, nx=6)
    a = O.solve_ip(p, x0, 512)
    b = O.solve_ip(p, x0, 512, opts=O.Options(costate_mode=1))
    assert a["info"]["status"] == 0 and b["info"]["status"] == 0
    assert rel(b["u"], a["u"]) <= 1e-9 and b["info"]["J"] == pytest.approx(a["info"]["J"], rel=1e-12)
    c = O.solve_ip(p, x0, 1024)
    assert c["info"]["status"] != 0
    d = O.solve_ip(p, x0, 1024, opts=O.Options(costate_mode=1))
    i = d["info"]
    assert i["status"] == 0 and i["r_stat"] <= 1e-6 and i["r_dyn"] <= 1e-9 and i["r_feas"] == 0.0
    assert np.abs(d["lam"]).max() < 1e3
    assert i["J"] == pytest.approx(a["info"]["J"], rel=1e-6)
