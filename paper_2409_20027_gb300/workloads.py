"""Seeded synthetic workloads shaped like the paper's examples (Sec. IV) and the
benchmark configurations built on them.

This module only builds problem data (model constants, weights, bounds, initial
states, horizons) from numpy ``default_rng`` seeds.  It contains none of the
method's arithmetic, so both the CUDA path and the CPU oracle consume identical
inputs from it.

Models (``Problem.model``): 0 pendulum (Sec. IV-A), 1 cart-pole (Sec. IV-B),
2 quadrotor (12 states, 4 rotor thrusts), 3 synthetic ``x+ = A x + B u + c tanh(W x)``.
Cost: ``sum_t (x-xref)^T Q (x-xref) + (u-uref)^T R (u-uref) + (x_T-xref)^T Qf (x_T-xref)``
(no 1/2 factor).  Constraints: box bounds on states and controls (``inf`` = none).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PENDULUM, CARTPOLE, QUADROTOR, SYNTH = 0, 1, 2, 3
EULER, RK4 = 0, 1
INF = np.inf


@dataclass
class Problem:
    model: int
    nx: int
    nu: int
    dt: float
    integrator: int
    prm: np.ndarray                  # model constants (<= 8)
    Q: np.ndarray
    R: np.ndarray
    Qf: np.ndarray
    xref: np.ndarray
    uref: np.ndarray
    xlo: np.ndarray
    xhi: np.ndarray
    ulo: np.ndarray
    uhi: np.ndarray
    A: np.ndarray | None = None      # synthetic model only
    B: np.ndarray | None = None
    W: np.ndarray | None = None
    name: str = ""
    xref_traj: np.ndarray | None = None  # time-varying targets, (T+1) x nx (replaces xref)
    uref_traj: np.ndarray | None = None  # T x nu (replaces uref)
    user_terms: object | None = None     # user-written stage / terminal costs and rows (oracle side)

    def replace(self, **kw) -> "Problem":
        d = dict(self.__dict__)
        d.update(kw)
        return Problem(**d)


def _f(a):
    return np.asarray(a, dtype=np.float64)


# ---------------------------------------------------------------- pendulum
def pendulum(dt: float = 0.05, b: float = 0.1) -> Problem:
    """Torque-limited pendulum swing-up: g=9.81, l=1, m=1, damping b, Euler step dt,
    Q=diag(1,0.1), R=0.01, Qf=diag(10,1), target (pi, 0), |u| <= 5."""
    return Problem(model=PENDULUM, nx=2, nu=1, dt=dt, integrator=EULER,
                   prm=_f([9.81, 1.0, 1.0, b]),
                   Q=np.diag([1.0, 0.1]), R=np.array([[0.01]]), Qf=np.diag([10.0, 1.0]),
                   xref=_f([np.pi, 0.0]), uref=_f([0.0]),
                   xlo=_f([-INF, -INF]), xhi=_f([INF, INF]), ulo=_f([-5.0]), uhi=_f([5.0]),
                   name="pendulum")


def pendulum_x0(seed: int) -> np.ndarray:
    """x0 = (0, 0) + N(0, 0.05^2) per component."""
    return np.random.default_rng(seed).normal(0.0, 0.05, size=2)


# ---------------------------------------------------------------- cart-pole
CARTPOLE_DT = 0.01


def cartpole(T: int | None = None, dt: float = CARTPOLE_DT, horizon: float | None = None) -> Problem:
    """Force-limited cart-pole: m_c=1, m_p=0.1, l=0.5, g=9.81, RK4 step.  State
    (p, theta, p', theta'), theta = pi upright.  Q=diag(1,10,0.1,0.1), R=0.01, Qf=100 Q,
    target (0, pi, 0, 0), |u| <= 10, |p| <= 2, all at dt = 0.01.

    With ``horizon`` the step is horizon/T (fixed physical time, varying sampling rate,
    as in Sec. IV) and the stage weights Q, R are scaled by dt/0.01 so that every T
    discretises the same continuous-time cost (T = 256, horizon 2.56 s is the dt = 0.01
    problem exactly)."""
    Q = np.diag([1.0, 10.0, 0.1, 0.1])
    R = np.array([[0.01]])
    Qf = 100.0 * Q
    if horizon is not None:
        dt = horizon / T
        Q = Q * (dt / CARTPOLE_DT)
        R = R * (dt / CARTPOLE_DT)
    return Problem(model=CARTPOLE, nx=4, nu=1, dt=dt, integrator=RK4,
                   prm=_f([1.0, 0.1, 0.5, 9.81]),
                   Q=Q, R=R, Qf=Qf,
                   xref=_f([0.0, np.pi, 0.0, 0.0]), uref=_f([0.0]),
                   xlo=_f([-2.0, -INF, -INF, -INF]), xhi=_f([2.0, INF, INF, INF]),
                   ulo=_f([-10.0]), uhi=_f([10.0]), name="cartpole")


def cartpole_x0(seed: int) -> np.ndarray:
    """p ~ U[-0.5, 0.5], theta ~ U[pi-0.3, pi+0.3], velocities 0."""
    r = np.random.default_rng(seed)
    p = r.uniform(-0.5, 0.5)
    th = r.uniform(np.pi - 0.3, np.pi + 0.3)
    return _f([p, th, 0.0, 0.0])


def batch_horizons(B: int, seed: int = 0, lo: int = 64, hi: int = 4096) -> np.ndarray:
    """T_b = round(exp(U[ln lo, ln hi])): log-uniform horizons."""
    r = np.random.default_rng(seed)
    return np.rint(np.exp(r.uniform(np.log(lo), np.log(hi), size=B))).astype(np.int32)


def uniform_horizons(B: int, seed: int = 0, lo: int = 1024, hi: int = 8192) -> np.ndarray:
    """T_b ~ U{lo, ..., hi}."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=B).astype(np.int32)


def cartpole_batch_x0(B: int, seed: int = 0) -> np.ndarray:
    """B initial states, instance b drawn from seed (seed, b)."""
    return np.stack([cartpole_x0(np.random.SeedSequence([seed, b]).generate_state(1)[0])
                     for b in range(B)])


# ---------------------------------------------------------------- the paper's own settings
# Sec. IV prints the model constants, Euler integration, the barrier schedule (mu from 0.1,
# times 0.2 until mu <= 1e-4, i.e. a last level of 0.1 * 0.2^5), the ADMM penalties and
# stopping rule, and the closed-loop experiment (4 s at 100 Hz, N = 60, |tau| < 5 Nm,
# |F| < 60 N).  It prints no cost weights, horizon length in seconds or trajectory-
# optimisation bounds: those are the readings of pendulum() and cartpole() above.
PAPER_IP = {"mu0": 0.1, "zeta": 0.2, "mu_stop": 1e-4, "mu_final": 0.1 * 0.2 ** 5}
PAPER_ADMM = {"pendulum_rho": 1.0, "cartpole_rho": 0.5, "tol": 1e-2}
PAPER_MPC = {"duration_s": 4.0, "rate_hz": 100, "horizon": 60, "torque_limit": 5.0, "force_limit": 60.0}


def pendulum_paper(dt: float = 1.0 / PAPER_MPC["rate_hz"]) -> Problem:
    """The paper's pendulum (Sec. IV-A): g=9.81, l=1, m=1, b=1e-3, Euler step dt, with the
    closed-loop experiment's torque limit |tau| <= 5 (Sec. IV-C); weights as pendulum()."""
    t = PAPER_MPC["torque_limit"]
    return pendulum(dt=dt, b=1e-3).replace(ulo=_f([-t]), uhi=_f([t]), name="pendulum_paper")


def cartpole_paper(dt: float = 1.0 / PAPER_MPC["rate_hz"]) -> Problem:
    """The paper's cart-pole (Sec. IV-B): m_c=10, m_p=1, l=0.5, g=9.81, Euler step dt, with
    the closed-loop experiment's force limit |F| <= 60 (Sec. IV-C) and no cart-position
    bound.  Q and Qf as cartpole(); R = 1e-4, so that the force limit rather than the force
    weight bounds the 10 kg cart (at R = 0.01 the loop leaves the cart 2.6 m from the
    origin after 4 s)."""
    f = PAPER_MPC["force_limit"]
    return cartpole(dt=dt).replace(integrator=EULER, prm=_f([10.0, 1.0, 0.5, 9.81]), R=np.array([[1e-4]]),
                                   ulo=_f([-f]), uhi=_f([f]), xlo=np.full(4, -INF), xhi=np.full(4, INF),
                                   name="cartpole_paper")


def pendulum_upright_x0(seed: int) -> np.ndarray:
    """theta ~ U[pi-0.3, pi+0.3], omega 0: near upright (the closed-loop experiment
    stabilises the upright position, Sec. IV-C)."""
    r = np.random.default_rng(seed)
    return _f([r.uniform(np.pi - 0.3, np.pi + 0.3), 0.0])


# ---------------------------------------------------------------- quadrotor
QUAD_MASS = 0.5
QUAD_G = 9.81


def quadrotor(waypoint=None, dt: float = 0.01) -> Problem:
    """12-state quadrotor (position, ZYX Euler angles, world velocity, body rates),
    4 rotor thrusts, mass 0.5, inertia diag(2.3e-3, 2.3e-3, 4e-3), arm 0.17,
    yaw-moment coefficient 0.01, Euler step.  Hover-to-waypoint tracking,
    Q=diag(1,1,1,.1,.1,.1,.1,.1,.1,.01,.01,.01), R=0.1 I around hover thrust,
    Qf=10 Q, thrust box [0, 4] per rotor."""
    wp = np.zeros(3) if waypoint is None else _f(waypoint)
    q = np.array([1.0] * 3 + [0.1] * 3 + [0.1] * 3 + [0.01] * 3)
    xref = np.zeros(12)
    xref[:3] = wp
    hover = QUAD_MASS * QUAD_G / 4.0
    return Problem(model=QUADROTOR, nx=12, nu=4, dt=dt, integrator=EULER,
                   prm=_f([QUAD_MASS, 2.3e-3, 2.3e-3, 4e-3, 0.17, 0.01, QUAD_G]),
                   Q=np.diag(q), R=0.1 * np.eye(4), Qf=10.0 * np.diag(q),
                   xref=xref, uref=np.full(4, hover),
                   xlo=np.full(12, -INF), xhi=np.full(12, INF),
                   ulo=np.zeros(4), uhi=np.full(4, 4.0), name="quadrotor")


def quadrotor_hover_u() -> float:
    """Hover thrust per rotor, m g / 4 (a strictly feasible start inside [0, 4])."""
    return QUAD_MASS * QUAD_G / 4.0


def quadrotor_waypoints(B: int, seed: int = 0) -> np.ndarray:
    """Waypoints uniform in the 2 m cube [-1, 1]^3 around the hover point (origin)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(B, 3))


# ---------------------------------------------------------------- synthetic
def _haar(r: np.random.Generator, n: int) -> np.ndarray:
    q, rr = np.linalg.qr(r.normal(size=(n, n)))
    return q * np.sign(np.diag(rr))


def synth(seed: int = 0, nx: int = 32, nu: int = 8) -> Problem:
    """x+ = A x + B u + 0.1 tanh(W x): A = 0.98 * Haar orthogonal, B ~ N(0, 1/nu),
    W ~ N(0, 1/nx), Q = U diag(U[0.1, 10]) U^T, R = 0.1 I, Qf = Q, |u| <= 1, target 0."""
    r = np.random.default_rng(seed)
    A = 0.98 * _haar(r, nx)
    B = r.normal(0.0, np.sqrt(1.0 / nu), size=(nx, nu))
    W = r.normal(0.0, np.sqrt(1.0 / nx), size=(nx, nx))
    U = _haar(r, nx)
    Q = U @ np.diag(r.uniform(0.1, 10.0, size=nx)) @ U.T
    Q = 0.5 * (Q + Q.T)
    return Problem(model=SYNTH, nx=nx, nu=nu, dt=1.0, integrator=EULER, prm=_f([0.1]),
                   Q=Q, R=0.1 * np.eye(nu), Qf=Q.copy(), xref=np.zeros(nx), uref=np.zeros(nu),
                   xlo=np.full(nx, -INF), xhi=np.full(nx, INF),
                   ulo=-np.ones(nu), uhi=np.ones(nu), A=A, B=B, W=W, name="synth")


def synth_x0(seed: int, nx: int = 32) -> np.ndarray:
    """x0 ~ N(0, I)."""
    return np.random.default_rng(seed + 1000).normal(size=nx)
