"""Adjoint (gradients of a loss of the solution w.r.t. x0, diag Q, diag R, diag Qf and the
model constants) on the GPU against the oracle's adjoint at the same solution, and the
autograd wrapper built on it."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2409_20027_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ptn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_20027_gb300 import ptn as m
    m.load()
    return m


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda:0")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


KEYS = ["x0", "Qd", "Rd", "Qfd", "prm"]

CASES = [
    # name, problem, x0 list, T_b, solve precision, tolerance (the adjoint itself runs in
    # FP64 in every mode, so both compare at the FP64 tolerance)
    ("pendulum_fp64", W.pendulum, [W.pendulum_x0(0), W.pendulum_x0(1)], [64, 40], 0, 1e-6),
    ("cartpole_fp32", lambda: W.cartpole(T=256, horizon=2.56), [W.cartpole_x0(0), W.cartpole_x0(2)], [256, 256], 1,
     1e-6),
]


def solve(ptn, p, x0s, Tb, prec):
    s = ptn.Solver(p, max_T=max(Tb), max_batch=len(Tb), precision=prec, block_threads=64)
    x0 = dev(np.stack(x0s))
    x, u, lam, infos = s.solve_batch(x0, Tb)
    assert all(i["status"] == 0 for i in infos)
    return s, x0, x, u, infos


@pytest.mark.parametrize("name,mk,x0s,Tb,prec,tol", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("with_traj", [False, True], ids=["J_only", "J_and_traj"])
def test_adjoint_matches_oracle(ptn, name, mk, x0s, Tb, prec, tol, with_traj):
    p = mk()
    s, x0, x, u, infos = solve(ptn, p, x0s, Tb, prec)
    mu = infos[0]["mu"]
    rng = np.random.default_rng(11)
    S = sum(Tb)
    gx = rng.standard_normal((S + len(Tb), p.nx)) if with_traj else None
    gu = rng.standard_normal((S, p.nu)) if with_traj else None
    gJ = 0.7
    out = s.adjoint(Tb, x0, x, u, mu, gJ, None if gx is None else dev(gx), None if gu is None else dev(gu))
    xs, us = x.cpu().numpy(), u.cpu().numpy()
    xo = uo = 0
    for b, T in enumerate(Tb):
        ref = O.adjoint(p, mu, xs[xo:xo + T + 1], us[uo:uo + T], gJ,
                        None if gx is None else gx[xo:xo + T + 1], None if gu is None else gu[uo:uo + T])
        assert ref["status"] == 0
        for k in KEYS:
            got = out[k][b].cpu().numpy()
            assert rel(got, ref[k]) <= tol, (b, k, got, ref[k])
        xo += T + 1
        uo += T


def test_autograd_wrapper(ptn):
    p = W.pendulum()
    Tb = [48, 64]
    s = ptn.Solver(p, max_T=64, max_batch=2, precision=0, block_threads=64)
    x0 = dev(np.stack([W.pendulum_x0(2), W.pendulum_x0(3)])).requires_grad_(True)
    theta = dev(ptn.theta_of(p)).requires_grad_(True)
    x, u, J = ptn.solve_ip_autograd(s, x0, Tb, theta)
    rng = np.random.default_rng(5)
    cx = dev(rng.standard_normal(tuple(x.shape)))
    cu = dev(rng.standard_normal(tuple(u.shape)))
    wJ = dev([0.3, 1.7])
    loss = (wJ * J).sum() + (cx * x).sum() + (cu * u).sum()
    loss.backward()
    xs, us = x.detach().cpu().numpy(), u.detach().cpu().numpy()
    mu = 1e-6
    gth = np.zeros_like(ptn.theta_of(p))
    xo = uo = 0
    for b, T in enumerate(Tb):
        ref = O.adjoint(p, mu, xs[xo:xo + T + 1], us[uo:uo + T], float(wJ[b]),
                        cx[xo:xo + T + 1].cpu().numpy(), cu[uo:uo + T].cpu().numpy())
        assert rel(x0.grad[b].cpu().numpy(), ref["x0"]) <= 1e-6
        gth += np.concatenate([ref["Qd"], ref["Rd"], ref["Qfd"], ref["prm"]])
        xo += T + 1
        uo += T
    assert rel(theta.grad.cpu().numpy(), gth) <= 1e-6


@pytest.mark.parametrize("with_traj", [False, True], ids=["J_only", "J_and_traj"])
def test_grid_adjoint_long_horizon_matches_oracle(ptn, with_traj):
    # one long instance (cart-pole, T = 4096 on the 2.56 s horizon): the adjoint on the
    # cooperative grid against the one-CTA adjoint at the same solution and against the
    # oracle's adjoint, in every output, with J* alone and with trajectory gradients too
    T = 4096
    p = W.cartpole(T=T, horizon=2.56)
    s = ptn.Solver(p, max_T=T, precision=0, grid_min_T=512, cluster_max_blocks=0)
    x0 = dev(W.cartpole_x0(3)).reshape(1, -1)
    x, u, _, infos = s.solve_batch(x0, [T])
    assert infos[0]["status"] == 0
    mu = infos[0]["mu"]
    rng = np.random.default_rng(13)
    gx = rng.standard_normal((T + 1, 4)) if with_traj else None
    gu = rng.standard_normal((T, 1)) if with_traj else None
    gJ = 0.7
    args = ([T], x0, x, u, mu, gJ, None if gx is None else dev(gx), None if gu is None else dev(gu))
    grid = s.adjoint(*args)
    s.set_options(grid_min_T=0)
    cta = s.adjoint(*args)
    ref = O.adjoint(p, mu, x.cpu().numpy(), u.cpu().numpy(), gJ, gx, gu)
    assert ref["status"] == 0
    for k in KEYS:
        g, c = grid[k][0].cpu().numpy(), cta[k][0].cpu().numpy()
        assert rel(g, ref[k]) <= 1e-6, (k, g, ref[k])
        assert rel(g, c) <= 1e-9, (k, g, c)


@pytest.mark.parametrize("T,seg,grid_min_T,with_traj", [(300, 64, 0, True), (300, 64, 0, False),
                                                         (4096, 1000, 512, True)],
                         ids=["cta-traj", "cta-J_only", "grid-traj"])
def test_checkpointed_adjoint_matches_oracle(ptn, T, seg, grid_min_T, with_traj):
    # a horizon that does not fit the handle's workspace (seg_len steps): segments of
    # seg_len steps with a shorter last one, linearisations recomputed from the trajectory
    # in each sweep; against the oracle's adjoint and the whole-horizon GPU adjoint
    p = W.cartpole(T=T, horizon=2.56)
    x0 = W.cartpole_x0(4)
    whole = ptn.Solver(p, max_T=T, precision=0, cluster_max_blocks=0)
    x, u, _, infos = whole.solve_batch(dev(x0).reshape(1, -1), [T])
    assert infos[0]["status"] == 0
    mu = infos[0]["mu"]
    rng = np.random.default_rng(5)
    gx = rng.standard_normal((T + 1, 4)) if with_traj else None
    gu = rng.standard_normal((T, 1)) if with_traj else None
    gJ = 0.7
    s = ptn.Solver(p, max_T=seg, precision=0, grid_min_T=grid_min_T, cluster_max_blocks=0)
    got = s.adjoint_checkpointed(T, seg, dev(x0), x, u, mu, gJ, None if gx is None else dev(gx),
                                 None if gu is None else dev(gu))
    one = whole.adjoint([T], dev(x0).reshape(1, -1), x, u, mu, gJ, None if gx is None else dev(gx),
                        None if gu is None else dev(gu))
    ref = O.adjoint(p, mu, x.cpu().numpy(), u.cpu().numpy(), gJ, gx, gu)
    assert ref["status"] == 0
    for k in KEYS:
        g, w = got[k][0].cpu().numpy(), one[k][0].cpu().numpy()
        assert rel(g, ref[k]) <= 1e-6, (k, g, ref[k])
        assert rel(g, w) <= 1e-9, (k, g, w)


def test_checkpointed_adjoint_refuses_bad_segments(ptn):
    p = W.cartpole(T=64, horizon=2.56)
    s = ptn.Solver(p, max_T=32, precision=0)
    x = torch.zeros((65, 4), dtype=torch.float64, device="cuda:0")
    u = torch.zeros((64, 1), dtype=torch.float64, device="cuda:0")
    for seg in [0, 33]:
        with pytest.raises(ptn.PtnError):
            s.adjoint_checkpointed(64, seg, x[0], x, u, 1e-3)
