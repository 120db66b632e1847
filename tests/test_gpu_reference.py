"""Time-varying tracking targets (ptn_set_reference: the stage cost l_t of Sec. II-A with
targets x*_t, u*_t that change with t) on the GPU against the oracle with the same
trajectories: the narrow tiers in FP64 and FP32, a ragged batch, the wide tier, and the
adjoint.  Tolerances as in test_gpu_parity (FP64 1e-6; FP32 1e-4 with both sides solved to
max|d| <= 1e-7)."""
import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
FP32_TOL = 1e-4


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


@pytest.fixture(scope="module")
def ptn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_20027_gb300 import build, ptn as P
    build.build()
    P.load()
    return P


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def check(info, ref, x, u, lam, tol, with_lam=True):
    assert info["status"] == 0, info
    assert ref["info"]["status"] == 0, ref["info"]
    e = dict(x=rel(x.cpu().numpy(), ref["x"]), u=rel(u.cpu().numpy(), ref["u"]),
             lam=rel(lam.cpu().numpy(), ref["lam"]) if with_lam else 0.0,
             J=abs(info["J"] - ref["info"]["J"]) / max(1.0, abs(ref["info"]["J"])))
    assert max(e.values()) <= tol, e
    assert info["r_stat"] <= 1e-6 and info["r_dyn"] <= 1e-6 and info["r_feas"] == 0.0


def cartpole_targets(T, phase=0.0):
    # the cart follows a slow sine around the origin with the pole upright
    t = np.arange(T + 1) / T
    xr = np.zeros((T + 1, 4))
    xr[:, 0] = 0.4 * np.sin(2 * np.pi * t + phase)
    xr[:, 1] = np.pi
    xr[:, 2] = 0.4 * 2 * np.pi / 2.56 * np.cos(2 * np.pi * t + phase)
    ur = 0.1 * np.cos(2 * np.pi * t[:T])[:, None]
    return xr, ur


@pytest.mark.parametrize("T,prec,opts", [(256, 0, {}), (1024, 1, {"grid_min_T": 512}), (1024, 1, {"grid_min_T": 0})],
                         ids=["fp64-cta", "fp32-cluster", "fp32-cta"])
def test_cartpole_time_varying_targets_match_oracle(ptn, T, prec, opts):
    p = W.cartpole(T=T, horizon=2.56)
    xr, ur = cartpole_targets(T)
    x0 = W.cartpole_x0(2)
    tol = 1e-7 if prec else 1e-6
    s = ptn.Solver(p, max_T=T, precision=prec, tol_final=tol, **opts)
    s.set_reference(dev(xr), dev(ur))
    x, u, lam, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p.replace(xref_traj=xr, uref_traj=ur), x0, T, opts=O.Options(tol_final=tol))
    check(info, ref, x, u, lam, FP64_TOL if prec == 0 else FP32_TOL, with_lam=prec == 0)
    # the same handle with the targets cleared solves the constant-target problem
    s.set_reference(None, None)
    x2, u2, lam2, info2 = s.solve_ip(dev(x0), T)
    ref2 = O.solve_ip(p, x0, T, opts=O.Options(tol_final=tol))
    check(info2, ref2, x2, u2, lam2, FP64_TOL if prec == 0 else FP32_TOL, with_lam=prec == 0)


def test_ragged_batch_time_varying_targets_match_oracle(ptn):
    Tb = [96, 64]
    p = W.cartpole(T=96, horizon=0.96)  # dt = 0.01
    parts = [cartpole_targets(T, phase=0.7 * b) for b, T in enumerate(Tb)]
    xr = np.concatenate([a for a, _ in parts]); ur = np.concatenate([b for _, b in parts])
    x0s = np.stack([W.cartpole_x0(3), W.cartpole_x0(5)])
    s = ptn.Solver(p, max_T=96, max_batch=2, precision=0)
    s.set_reference(dev(xr), dev(ur))
    X, U, Lm, infos = s.solve_batch(dev(x0s), Tb)
    xo = uo = 0
    for b, T in enumerate(Tb):
        ref = O.solve_ip(p.replace(xref_traj=parts[b][0], uref_traj=parts[b][1]), x0s[b], T)
        check(infos[b], ref, X[xo:xo + T + 1], U[uo:uo + T], Lm[xo:xo + T + 1], FP64_TOL)
        xo += T + 1
        uo += T


def test_quadrotor_time_varying_targets_match_oracle(ptn):
    # the wide tier: the waypoint moves along a line during the horizon
    T = 48
    p = W.quadrotor(W.quadrotor_waypoints(1, 2)[0])
    xr = np.tile(p.xref, (T + 1, 1))
    xr[:, 0] += np.linspace(-0.3, 0.3, T + 1)
    x0 = np.zeros(12)
    hov = np.full((T, 4), W.quadrotor_hover_u())
    s = ptn.Solver(p, max_T=T, precision=0)
    s.set_reference(dev(xr), None)
    x, u, lam, info = s.solve_ip(dev(x0), T, u_init=dev(hov))
    ref = O.solve_ip(p.replace(xref_traj=xr), x0, T, u_init=hov)
    check(info, ref, x, u, lam, FP64_TOL)


@pytest.mark.parametrize("with_traj", [False, True], ids=["J_only", "J_and_traj"])
def test_adjoint_with_time_varying_targets_matches_oracle(ptn, with_traj):
    p = W.pendulum()
    T = 64
    t = np.arange(T + 1)
    xr = np.stack([np.pi * np.minimum(1.0, 2.0 * t / T), np.zeros(T + 1)], axis=1)
    x0 = W.pendulum_x0(1)
    s = ptn.Solver(p, max_T=T, precision=0, block_threads=64)
    s.set_reference(dev(xr), None)
    x, u, lam, info = s.solve_ip(dev(x0), T)
    assert info["status"] == 0
    rng = np.random.default_rng(2)
    gx = rng.standard_normal((T + 1, 2)) if with_traj else None
    gu = rng.standard_normal((T, 1)) if with_traj else None
    got = s.adjoint([T], dev(x0).reshape(1, -1), x, u, info["mu"], 0.8, None if gx is None else dev(gx),
                    None if gu is None else dev(gu))
    ref = O.adjoint(p.replace(xref_traj=xr), info["mu"], x.cpu().numpy(), u.cpu().numpy(), 0.8, gx, gu)
    assert ref["status"] == 0
    for k in ["x0", "Qd", "Rd", "Qfd", "prm"]:
        assert rel(got[k][0].cpu().numpy(), ref[k]) <= FP64_TOL, k
