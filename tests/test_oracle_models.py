"""Pins for the oracle's models and their derivatives.

Each model is tied to physics it must obey (energy balance, equilibria, rotation
kinematics), the integrators to an independent ODE solver, and every derivative
to central finite differences of the oracle's own step function.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O
from paper_2409_20027_gb300 import workloads as W

RNG = np.random.default_rng(1234)


def _problems():
    return [W.pendulum(), W.cartpole(), W.quadrotor(waypoint=[0.3, -0.2, 0.5]), W.synth(0, nx=6, nu=2)]


# ---------------------------------------------------------------- physics pins

def test_pendulum_energy_balance():
    # E = 1/2 m l^2 w^2 - m g l cos(th);  dE/dt = w (u - b w)  (Sec. IV-A model)
    p = W.pendulum()
    g, l, m, b = p.prm[:4]
    for _ in range(20):
        x = RNG.normal(size=2) * 2
        u = RNG.normal(size=1) * 3
        xd = O.rhs(p, x, u)
        dE = m * l * l * x[1] * xd[1] + m * g * l * np.sin(x[0]) * xd[0]
        assert dE == pytest.approx(x[1] * (u[0] - b * x[1]), rel=1e-12, abs=1e-12)


def test_cartpole_energy_balance_pins_theta_dot_squared():
    # Cart-pole energy E = 1/2 (mc+mp) p'^2 + mp l p' th' cos th + 1/2 mp l^2 th'^2 - mp g l cos th
    # obeys dE/dt = F p' (the force is the only power input).  This only holds with the
    # l*th'^2 term in the cart equation (the paper prints l*th').
    p = W.cartpole()
    mc, mp, l, g = p.prm[:4]
    for _ in range(20):
        x = RNG.normal(size=4) * np.array([1, 3, 2, 4])
        F = RNG.normal() * 5
        xd = O.rhs(p, x, [F])
        th, pd, td = x[1], x[2], x[3]
        pdd, tdd = xd[2], xd[3]
        dE = ((mc + mp) * pd * pdd + mp * l * (pdd * td * np.cos(th) + pd * tdd * np.cos(th)
                                              - pd * td * td * np.sin(th))
              + mp * l * l * td * tdd + mp * g * l * np.sin(th) * td)
        assert dE == pytest.approx(F * pd, rel=1e-10, abs=1e-10)
        # kinematic rows
        assert xd[0] == x[2] and xd[1] == x[3]


def _rot(phi, th, psi):
    cx, sx, cy, sy, cz, sz = np.cos(phi), np.sin(phi), np.cos(th), np.sin(th), np.cos(psi), np.sin(psi)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def test_quadrotor_hover_equilibrium():
    p = W.quadrotor()
    xd = O.rhs(p, np.zeros(12), np.full(4, W.quadrotor_hover_u()))
    assert np.abs(xd).max() < 1e-14


def test_quadrotor_rigid_body_kinematics_and_energy():
    # (1) Euler-angle rates: d/dt R(eta) = R [w]x for body rates w.
    # (2) thrust acts along the body z axis R e3: v' = (sum F / m) R e3 - g e3.
    # (3) energy E = 1/2 m |v|^2 + m g z + 1/2 w^T I w, dE/dt = sum F (R e3).v + tau.w,
    #     with tau from the '+' layout (torque = sum r_i x F_i e3, yaw k_m (f1-f2+f3-f4)).
    p = W.quadrotor()
    mass, Ixx, Iyy, Izz, arm, km, g = p.prm[:7]
    I = np.diag([Ixx, Iyy, Izz])
    r = [np.array([arm, 0, 0]), np.array([0, arm, 0]), np.array([-arm, 0, 0]), np.array([0, -arm, 0])]
    for _ in range(10):
        x = RNG.normal(size=12) * 0.5
        u = RNG.uniform(0, 4, size=4)
        xd = O.rhs(p, x, u)
        eta, v, w = x[3:6], x[6:9], x[9:12]
        R = _rot(*eta)
        h = 1e-6
        dR = (_rot(*(eta + h * xd[3:6])) - _rot(*(eta - h * xd[3:6]))) / (2 * h)
        assert np.allclose(dR, R @ _skew(w), atol=1e-8)
        assert np.allclose(xd[6:9], u.sum() / mass * R[:, 2] - np.array([0, 0, g]), atol=1e-12)
        tau = sum(np.cross(ri, np.array([0, 0, fi])) for ri, fi in zip(r, u))
        tau[2] = km * (u[0] - u[1] + u[2] - u[3])
        dE = mass * v @ xd[6:9] + mass * g * xd[2] + w @ I @ xd[9:12]
        assert dE == pytest.approx(u.sum() * R[:, 2] @ v + tau @ w, rel=1e-9, abs=1e-9)
        assert np.allclose(xd[:3], v)


def test_synth_map_special_cases():
    p = W.synth(0, nx=6, nu=2)
    # W x = 0 (x = 0): the map is A x + B u exactly, i.e. B u
    u = RNG.normal(size=2)
    assert np.allclose(O.step(p, np.zeros(6), u), p.B @ u, atol=1e-15)
    # odd symmetry f(-x, -u) = -f(x, u)
    x = RNG.normal(size=6)
    assert np.allclose(O.step(p, -x, -u), -O.step(p, x, u), atol=1e-14)
    # with W = 0 the map is linear: Jacobians are A and B
    p0 = p.replace(W=np.zeros((6, 6)))
    F, G = O.jac(p0, x, u)
    assert np.allclose(F, p.A) and np.allclose(G, p.B)


# ---------------------------------------------------------------- integrators

def test_euler_step_is_one_explicit_euler_step():
    for p in [W.pendulum(), W.quadrotor()]:
        for _ in range(5):
            x = RNG.normal(size=p.nx) * 0.3
            u = RNG.uniform(0.5, 2, size=p.nu)
            assert np.allclose(O.step(p, x, u), x + p.dt * O.rhs(p, x, u), atol=1e-15, rtol=1e-14)


def test_rk4_matches_ode_solution_to_fifth_order():
    # local error of a 4th-order method is O(dt^5): halving dt divides it by ~32
    p = W.cartpole()
    x = np.array([0.2, 2.5, -0.4, 1.1])
    u = np.array([3.0])
    errs = []
    for dt in [0.04, 0.02, 0.01]:
        q = p.replace(dt=dt)
        ref = solve_ivp(lambda t, y: O.rhs(p, y, u), (0, dt), x, rtol=1e-13, atol=1e-13, method="DOP853").y[:, -1]
        errs.append(np.abs(O.step(q, x, u) - ref).max())
    assert errs[-1] < 1e-8
    assert 20 < errs[0] / errs[1] < 45 and 20 < errs[1] / errs[2] < 45


# ---------------------------------------------------------------- derivatives vs FD

@pytest.mark.parametrize("k", range(4))
def test_jacobian_matches_central_differences(k):
    p = _problems()[k]
    n, m = p.nx, p.nu
    x = RNG.normal(size=n) * 0.4
    u = RNG.uniform(0.5, 2.0, size=m)
    F, G = O.jac(p, x, u)
    h = 1e-6
    for j in range(n + m):
        e = np.zeros(n + m); e[j] = h
        fp = O.step(p, x + e[:n], u + e[n:])
        fm = O.step(p, x - e[:n], u - e[n:])
        col = (fp - fm) / (2 * h)
        ref = F[:, j] if j < n else G[:, j - n]
        assert np.allclose(ref, col, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("k", range(4))
def test_hessian_contraction_matches_differences_of_jacobian(k):
    # (lam . f_zz) e_j = d/dz_j [ J(z)^T lam ]
    p = _problems()[k]
    n, m = p.nx, p.nu
    x = RNG.normal(size=n) * 0.4
    u = RNG.uniform(0.5, 2.0, size=m)
    lam = RNG.normal(size=n)
    Hxx, Hxu, Huu = O.hess(p, x, u, lam)
    H = np.block([[Hxx, Hxu], [Hxu.T, Huu]])
    h = 1e-6

    def jt(z):
        F, G = O.jac(p, z[:n], z[n:])
        return np.concatenate([F.T @ lam, G.T @ lam])

    z = np.concatenate([x, u])
    for j in range(n + m):
        e = np.zeros(n + m); e[j] = h
        col = (jt(z + e) - jt(z - e)) / (2 * h)
        assert np.allclose(H[:, j], col, rtol=1e-5, atol=1e-7)
    assert np.allclose(H, H.T)


def test_param_jacobian_matches_differences():
    p = W.quadrotor()
    x = RNG.normal(size=12) * 0.3
    u = RNG.uniform(0.5, 2.0, size=4)
    D = O.param_jac(p, x, u)
    h = 1e-7
    for k in range(7):
        pp = p.prm.copy(); pm = p.prm.copy()
        pp[k] += h * max(1, abs(pp[k])); pm[k] -= h * max(1, abs(pm[k]))
        col = (O.step(p.replace(prm=pp), x, u) - O.step(p.replace(prm=pm), x, u)) / (2 * h * max(1, abs(p.prm[k])))
        assert np.allclose(D[:, k], col, rtol=1e-5, atol=1e-7)
