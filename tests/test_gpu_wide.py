"""Wide tier (n >= 8: one warp per time chunk, elements in shared memory) on the
quadrotor (n = 12, m = 4) against the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2409_20027_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4  # FP32 LQR data with FP64 solves; gradients, rollouts and merits are FP64


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


def hover(T):
    return np.full((T, 4), W.quadrotor_hover_u())


def check(info, ref, x, u, tol=TOL):
    assert info["status"] == 0, info
    assert ref["info"]["status"] == 0
    assert rel(x, ref["x"]) <= tol
    assert rel(u, ref["u"]) <= tol
    assert abs(info["J"] - ref["info"]["J"]) / max(1.0, abs(ref["info"]["J"])) <= tol
    assert info["r_stat"] <= 1e-6 and info["r_dyn"] <= 1e-6 and info["r_feas"] == 0.0


@pytest.mark.parametrize("threads,grid_min_T", [(128, 512), (256, 512), (128, 0)])
def test_quadrotor_batch_matches_oracle(ptn, threads, grid_min_T):
    # ragged horizons, including ones shorter than the number of warps (empty chunks);
    # a CTA range per instance of one cooperative launch (grid_min_T > 0), or one CTA each
    Tb = np.array([32, 3, 64, 17], dtype=np.int32)
    B = len(Tb)
    wps = W.quadrotor_waypoints(B, 1)
    base = W.quadrotor()
    xrefs = np.stack([W.quadrotor(wps[b]).xref for b in range(B)])
    s = ptn.Solver(base, max_T=int(Tb.max()), max_batch=B, block_threads=threads, grid_min_T=grid_min_T)
    u0 = np.concatenate([hover(int(T)) for T in Tb])
    X, U, Lm, infos = s.solve_batch(dev(np.zeros((B, 12))), Tb, xref=dev(xrefs), u_init=dev(u0))
    X, U = X.cpu().numpy(), U.cpu().numpy()
    xo = uo = 0
    for b in range(B):
        T = int(Tb[b])
        ref = O.solve_ip(W.quadrotor(wps[b]), np.zeros(12), T, u_init=hover(T))
        check(infos[b], ref, X[xo:xo + T + 1], U[uo:uo + T])
        xo += T + 1
        uo += T


def test_quadrotor_single_solve(ptn):
    T = 96
    p = W.quadrotor(W.quadrotor_waypoints(1, 4)[0])
    s = ptn.Solver(p, max_T=T)
    x, u, lam, info = s.solve_ip(dev(np.zeros(12)), T, u_init=dev(hover(T)))
    ref = O.solve_ip(p, np.zeros(12), T, u_init=hover(T))
    check(info, ref, x.cpu().numpy(), u.cpu().numpy())
    assert rel(lam.cpu().numpy(), ref["lam"]) <= TOL


def test_quadrotor_admm_fixed_iterations(ptn):
    T = 24
    p = W.quadrotor(W.quadrotor_waypoints(1, 2)[0])
    s = ptn.Solver(p, max_T=T, admm_fixed_iters=4)
    x, u, lam, z, v, info = s.solve_admm(dev(np.zeros(12)), T, u_init=dev(hover(T)), with_zv=True)
    ref = O.solve_admm(p, np.zeros(12), T, u_init=hover(T), opts=O.Options(admm_fixed_iters=4))
    assert info["status"] == 0 and ref["info"]["status"] == 0
    assert rel(x.cpu().numpy(), ref["x"]) <= TOL
    assert rel(u.cpu().numpy(), ref["u"]) <= TOL
    assert rel(z.cpu().numpy(), ref["z"]) <= TOL
    assert rel(v.cpu().numpy(), ref["v"]) <= TOL


def test_quadrotor_fp64_mode_matches_oracle(ptn):
    T = 16
    p = W.quadrotor(W.quadrotor_waypoints(1, 6)[0])
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64)
    x, u, lam, info = s.solve_ip(dev(np.zeros(12)), T, u_init=dev(hover(T)))
    ref = O.solve_ip(p, np.zeros(12), T, u_init=hover(T))
    check(info, ref, x.cpu().numpy(), u.cpu().numpy(), tol=1e-6)


@pytest.mark.parametrize("with_traj", [False, True], ids=["J_only", "J_and_traj"])
def test_quadrotor_adjoint_matches_oracle(ptn, with_traj):
    Tb = [24, 40]
    B = len(Tb)
    wps = W.quadrotor_waypoints(B, 3)
    xrefs = np.stack([W.quadrotor(wps[b]).xref for b in range(B)])
    s = ptn.Solver(W.quadrotor(), max_T=max(Tb), max_batch=B)
    u0 = np.concatenate([hover(T) for T in Tb])
    x0 = dev(np.zeros((B, 12)))
    X, U, Lm, infos = s.solve_batch(x0, Tb, xref=dev(xrefs), u_init=dev(u0))
    assert all(i["status"] == 0 for i in infos)
    mu = infos[0]["mu"]
    rng = np.random.default_rng(21)
    S = sum(Tb)
    gx = rng.standard_normal((S + B, 12)) if with_traj else None
    gu = rng.standard_normal((S, 4)) if with_traj else None
    out = s.adjoint(Tb, x0, X, U, mu, 0.6, None if gx is None else dev(gx), None if gu is None else dev(gu),
                    xref=dev(xrefs))
    Xs, Us = X.cpu().numpy(), U.cpu().numpy()
    xo = uo = 0
    for b, T in enumerate(Tb):
        ref = O.adjoint(W.quadrotor(wps[b]), mu, Xs[xo:xo + T + 1], Us[uo:uo + T], 0.6,
                        None if gx is None else gx[xo:xo + T + 1], None if gu is None else gu[uo:uo + T])
        assert ref["status"] == 0
        for k in ["x0", "Qd", "Rd", "Qfd", "prm"]:
            assert rel(out[k][b].cpu().numpy(), ref[k]) <= 1e-6, (b, k)
        xo += T + 1
        uo += T
