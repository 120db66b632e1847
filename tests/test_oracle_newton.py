"""Pins for the oracle's Newton step, IP and ADMM loops, and adjoint.

P1  LQ special case: one Newton step is the exact optimum (dense KKT) and the
    Riccati S_t tends to the DARE solution.
P4  d_t equals the gradient of the rollout cost (finite differences).
P5  the Newton direction equals -(Hessian + alpha I)^{-1} gradient, Hessian by FD.
P6  local quadratic convergence of Newton (Sec. III-E).
P7  KKT invariants at the IP result.
P8  brute-force minimisation on a tiny horizon finds the same minimiser.
P9  adjoint gradients vs finite differences of re-solved problems.
P10 ADMM at tight tolerance agrees with IP at small mu.
"""
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import minimize

import oracle as O
from paper_2409_20027_gb300 import workloads as W

RNG = np.random.default_rng(11)
INF = np.inf


def _lq_problem(n=4, m=2, seed=0):
    p = W.synth(seed, nx=n, nu=m)
    return p.replace(W=np.zeros((n, n)), ulo=np.full(m, -INF), uhi=np.full(m, INF),
                     xref=RNG.normal(size=n), uref=RNG.normal(size=m), Qf=2.0 * p.Q)


# ---------------------------------------------------------------- P1

def test_lq_one_newton_step_is_exact_optimum():
    p = _lq_problem()
    n, m, T = p.nx, p.nu, 12
    x0 = RNG.normal(size=n)
    u = RNG.normal(size=(T, m))
    x = O.rollout(p, x0, u)
    nd = O.newton_direction(p, x, u, 0.0, "none")
    assert nd["status"] == 0
    u1 = u + nd["du"]
    # dense condensed QP: x_t = A^t x0 + sum_k A^{t-1-k} B u_k
    Su = np.zeros(((T + 1) * n, T * m)); sx = np.zeros((T + 1) * n)
    Ak = np.eye(n)
    for t in range(T + 1):
        sx[t * n:(t + 1) * n] = np.linalg.matrix_power(p.A, t) @ x0
        for k in range(t):
            Su[t * n:(t + 1) * n, k * m:(k + 1) * m] = np.linalg.matrix_power(p.A, t - 1 - k) @ p.B
    Qb = sla.block_diag(*([p.Q] * T + [p.Qf]))
    Rb = sla.block_diag(*([p.R] * T))
    xr = np.tile(p.xref, T + 1); ur = np.tile(p.uref, T)
    H = 2 * (Su.T @ Qb @ Su + Rb)
    g = 2 * (Su.T @ Qb @ (sx - xr) - Rb @ ur)
    ustar = np.linalg.solve(H, -g).reshape(T, m)
    assert np.allclose(u1, ustar, rtol=1e-9, atol=1e-9)
    assert np.allclose(x + nd["dx"], O.rollout(p, x0, ustar), rtol=1e-9, atol=1e-9)


def test_lq_riccati_tends_to_dare():
    p = _lq_problem(n=3, m=1, seed=2)
    T = 400
    x0 = RNG.normal(size=p.nx)
    u = np.zeros((T, p.nu))
    x = O.rollout(p, x0, u)
    nd = O.newton_direction(p, x, u, 0.0, "none")
    # costs carry no 1/2, so the value matrix in the 1/2 x^T S x convention is 2 * DARE
    Pd = sla.solve_discrete_are(p.A, p.B, p.Q, p.R)
    assert np.allclose(nd["S"][0], 2 * Pd, rtol=1e-8, atol=1e-8)
    K = np.linalg.solve(p.R + p.B.T @ Pd @ p.B, p.B.T @ Pd @ p.A)
    assert np.allclose(nd["Gam"][0], -K, rtol=1e-8, atol=1e-8)


# ---------------------------------------------------------------- P4 / P5

CASES = [
    (W.pendulum(), lambda: W.pendulum_x0(1), 12, 0.5),
    (W.cartpole(T=10, horizon=0.2), lambda: W.cartpole_x0(1), 10, 1.0),
    (W.quadrotor(waypoint=[0.4, -0.3, 0.2]), lambda: np.zeros(12), 5, 0.1),
    (W.synth(1, nx=6, nu=2), lambda: W.synth_x0(1, nx=6), 7, 0.2),
]


def _start(p, x0f, T, scale):
    if p.model == W.QUADROTOR:
        return x0f(), W.quadrotor_hover_u() + scale * RNG.uniform(-1, 1, size=(T, 4))
    return x0f(), scale * RNG.uniform(-1, 1, size=(T, p.nu))


def _grad(p, x0, u, mu):
    x = O.rollout(p, x0, u)
    return O.newton_direction(p, x, u, 1e6, "barrier", mu)["d"]


@pytest.mark.parametrize("k", range(4))
def test_costate_gradient_matches_finite_differences(k):
    p, x0f, T, sc = CASES[k]
    x0, u = _start(p, x0f, T, sc)
    mu = 0.05
    d = _grad(p, x0, u, mu)
    h = 1e-6
    fd = np.zeros_like(u)
    for t in range(T):
        for i in range(p.nu):
            up = u.copy(); up[t, i] += h
            um = u.copy(); um[t, i] -= h
            fd[t, i] = (O.cost(p, O.rollout(p, x0, up), up, "barrier", mu)[0]
                        - O.cost(p, O.rollout(p, x0, um), um, "barrier", mu)[0]) / (2 * h)
    assert np.abs(d - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("k", range(4))
def test_newton_direction_matches_dense_newton(k):
    p, x0f, T, sc = CASES[k]
    T = min(T, 6)
    x0, u = _start(p, x0f, T, sc)
    mu, alpha = 0.05, 2.0
    x = O.rollout(p, x0, u)
    nd = O.newton_direction(p, x, u, alpha, "barrier", mu)
    assert nd["status"] == 0
    # Hessian of the reduced cost by central differences of the (pinned) gradient
    h = 1e-5
    nz = T * p.nu
    H = np.zeros((nz, nz))
    for j in range(nz):
        up = u.copy().ravel(); up[j] += h
        um = u.copy().ravel(); um[j] -= h
        H[:, j] = (_grad(p, x0, up.reshape(u.shape), mu) - _grad(p, x0, um.reshape(u.shape), mu)).ravel() / (2 * h)
    H = 0.5 * (H + H.T)
    du = -np.linalg.solve(H + alpha * np.eye(nz), nd["d"].ravel())
    assert np.allclose(nd["du"].ravel(), du, rtol=1e-5, atol=1e-6 * max(1, np.abs(du).max()))
    # dx is the linearised response to du (eq. linearized-ocp)
    dx = np.zeros(p.nx)
    for t in range(T):
        dx = nd["F"][t] @ dx + nd["G"][t] @ nd["du"][t]
    assert np.allclose(nd["dx"][T], dx, atol=1e-10)


# ---------------------------------------------------------------- P6

def test_local_quadratic_convergence():
    p = W.pendulum()
    T, mu = 30, 1e-2
    x0 = W.pendulum_x0(0)
    ref = O.solve_fixed_mu(p, x0, T, mu, 1e-12, np.zeros((T, 1)))
    assert ref["info"]["status"] == 0
    u = ref["u"] + 5e-4 * RNG.normal(size=(T, 1))
    norms = []
    for _ in range(12):
        x = O.rollout(p, x0, u)
        nd = O.newton_direction(p, x, u, 0.0, "barrier", mu)
        norms.append(np.abs(nd["d"]).max())
        if norms[-1] < 1e-11:
            break
        u = u + nd["du"]          # pure Newton on the reduced problem
    assert norms[-1] < 1e-9
    # in the final phase the gradient norm is squared each step (bounded ratio)
    tail = [i for i in range(len(norms) - 1) if norms[i] < 1e-2 and norms[i + 1] > 1e-12]
    assert len(tail) >= 2
    assert max(norms[i + 1] / norms[i] ** 2 for i in tail) < 10.0


# ---------------------------------------------------------------- P7

@pytest.mark.parametrize("seed", [0, 1])
def test_ip_result_satisfies_kkt_invariants(seed):
    p = W.pendulum()
    T = 64
    r = O.solve_ip(p, W.pendulum_x0(seed), T)
    i = r["info"]
    assert i["status"] == 0
    assert i["r_stat"] <= 1e-6 and i["r_dyn"] <= 1e-12 and i["r_feas"] == 0.0
    assert i["r_kkt"] <= 1e-6 * (1 + 1e-9)
    assert i["mu"] == pytest.approx(1e-6)
    w = np.array([O.constraints(p, r["x"][t], r["u"][t]) for t in range(T)])
    assert (w < 0).all()
    # complementarity of the implied duals y = mu / (-w): y >= 0, y (-w) = mu
    y = i["mu"] / (-w)
    assert (y > 0).all() and np.allclose(y * (-w), i["mu"])
    # the barrier objective at the result is below the start's
    u0 = np.zeros((T, 1))
    assert i["J_c"] < O.cost(p, O.rollout(p, W.pendulum_x0(seed), u0), u0, "barrier", 1e-6)[0]


# ---------------------------------------------------------------- P8

def test_bruteforce_tiny_horizon_same_minimiser():
    # pendulum, T = 3: minimise the barrier objective with an independent numpy model
    p = W.pendulum()
    T, mu = 3, 1e-2
    x0 = np.array([0.3, -0.2])
    g, l, m, b = p.prm[:4]

    def J(u):
        if np.any(np.abs(u) >= 5):
            return 1e30
        x = x0.copy(); c = 0.0
        for t in range(T):
            e = x - p.xref
            c += e @ p.Q @ e + p.R[0, 0] * u[t] ** 2 - mu * (np.log(5 - u[t]) + np.log(5 + u[t]))
            x = x + p.dt * np.array([x[1], -(g / l) * np.sin(x[0]) - b / (m * l * l) * x[1] + u[t] / (m * l * l)])
        e = x - p.xref
        return c + e @ p.Qf @ e

    best = None
    for s in range(30):
        u0 = np.random.default_rng(s).uniform(-4.9, 4.9, size=T)
        res = minimize(J, u0, method="Nelder-Mead", options=dict(xatol=1e-11, fatol=1e-13, maxiter=20000))
        if best is None or res.fun < best.fun:
            best = res
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, np.zeros((T, 1)))
    assert r["info"]["status"] == 0
    assert np.allclose(r["u"][:, 0], best.x, atol=1e-5)
    assert r["info"]["J_c"] == pytest.approx(best.fun, rel=1e-10)


# ---------------------------------------------------------------- P9

def _loss(p, x0, T, mu, u_warm, gx, gu):
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, u_warm)
    assert r["info"]["status"] == 0
    return r["info"]["J_c"] + (gx * r["x"]).sum() + (gu * r["u"]).sum()


@pytest.mark.parametrize("which", ["pendulum", "quadrotor"])
def test_adjoint_matches_finite_differences(which):
    if which == "pendulum":
        p, T, mu = W.pendulum(), 15, 1e-2
        x0 = W.pendulum_x0(2)
        uw = np.zeros((T, 1))
        prm_idx = [0, 1, 2, 3]
    else:
        p, T, mu = W.quadrotor(waypoint=[0.3, 0.1, -0.2]), 8, 1e-2
        xr = p.xref.copy(); xr[3:6] = [0.2, -0.3, 0.8]     # excite all three axes
        p = p.replace(xref=xr)
        x0 = np.zeros(12)
        uw = np.full((T, 4), W.quadrotor_hover_u())
        prm_idx = [0, 1, 2, 3]
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, uw)
    assert r["info"]["status"] == 0
    xs, us = r["x"], r["u"]
    gx = RNG.normal(size=xs.shape); gu = RNG.normal(size=us.shape)
    a = O.adjoint(p, mu, xs, us, 1.0, gx, gu)
    assert a["status"] == 0
    def fd(mod, h=1e-5):
        # central differences with one Richardson step (error O(h^4))
        def cd(hh):
            pp, xp = mod(+hh); pm, xm = mod(-hh)
            return (_loss(pp, xp, T, mu, us, gx, gu) - _loss(pm, xm, T, mu, us, gx, gu)) / (2 * hh)
        return (4 * cd(h / 2) - cd(h)) / 3

    def chk(an, num):
        assert an == pytest.approx(num, rel=1e-5, abs=1e-6 * max(1.0, abs(num)))

    for i in range(p.nx):
        e = np.zeros(p.nx); e[i] = 1
        chk(a["x0"][i], fd(lambda s: (p, x0 + s * e)))
    for i in range(p.nx):
        E = np.zeros((p.nx, p.nx)); E[i, i] = 1
        chk(a["Qd"][i], fd(lambda s: (p.replace(Q=p.Q + s * E), x0)))
        chk(a["Qfd"][i], fd(lambda s: (p.replace(Qf=p.Qf + s * E), x0)))
    for i in range(p.nu):
        E = np.zeros((p.nu, p.nu)); E[i, i] = 1
        chk(a["Rd"][i], fd(lambda s: (p.replace(R=p.R + s * E), x0)))
    for k in prm_idx:
        def mod(s, k=k):
            pr = p.prm.copy(); pr[k] += s
            return p.replace(prm=pr), x0
        chk(a["prm"][k], fd(mod, h=2e-3 * abs(p.prm[k])))


def test_adjoint_x0_gradient_is_first_costate():
    # envelope theorem: dJ*/dx0 = lam_1 (gx = gu = 0)
    p, T, mu = W.pendulum(), 20, 1e-2
    x0 = W.pendulum_x0(4)
    r = O.solve_fixed_mu(p, x0, T, mu, 1e-12, np.zeros((T, 1)))
    a = O.adjoint(p, mu, r["x"], r["u"], 1.0)
    assert np.allclose(a["x0"], r["lam"][0], rtol=1e-12)


# ---------------------------------------------------------------- P10

def test_admm_tight_agrees_with_ip_small_mu():
    p = W.pendulum()
    T = 40
    x0 = W.pendulum_x0(5)
    ip = O.solve_ip(p, x0, T)
    ad = O.solve_admm(p, x0, T, opts=O.Options(admm_tol=1e-6, max_outer=3000))
    assert ip["info"]["status"] == 0 and ad["info"]["status"] == 0
    assert ad["info"]["r_p"] <= 1e-6 and ad["info"]["r_d"] <= 1e-6
    assert ad["info"]["J"] == pytest.approx(ip["info"]["J"], rel=1e-4)
    assert np.abs(ad["u"] - ip["u"]).max() < 2e-3
