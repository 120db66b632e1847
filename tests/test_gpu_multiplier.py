"""GPU parity of the multiplier form of the co-states (option costate_mode = 1; a variant
of the method: dynamics multipliers moved to the LQR duals instead of the co-state scan
of Alg. 1) against the oracle's multiplier form, and against the co-state form's KKT
point.

Tolerances as in test_gpu_parity: FP64 1e-6 relative in x, u, lam (= the multipliers)
and the cost; FP32 LQR with FP64 solves 1e-4 with both sides solved to 1e-7.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-6
FP32_TOL = 1e-4
MULT = O.Options(costate_mode=1)


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
    assert ref["info"]["status"] == 0
    assert rel(x.cpu().numpy(), ref["x"]) <= tol
    assert rel(u.cpu().numpy(), ref["u"]) <= tol
    if with_lam:
        assert rel(lam.cpu().numpy(), ref["lam"]) <= tol
    assert abs(info["J"] - ref["info"]["J"]) / max(1.0, abs(ref["info"]["J"])) <= tol
    assert info["r_stat"] <= 1e-6 and info["r_dyn"] <= 1e-6 and info["r_feas"] == 0.0


CASES = {
    "pendulum-64": (W.pendulum(), W.pendulum_x0(0), 64, 64),
    "cartpole-128": (W.cartpole(), W.cartpole_x0(1), 128, 128),
    "cartpole-256-fixed-horizon": (W.cartpole(T=256, horizon=2.56), W.cartpole_x0(2), 256, 128),
    "cartpole-200-ragged": (W.cartpole(), W.cartpole_x0(3), 200, 64),
}


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("case", list(CASES))
def test_fp64_cta_matches_oracle_multiplier_form(ptn, case, mode):
    p, x0, T, threads = CASES[case]
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, block_threads=threads, grid_min_T=0,
                   cluster_max_blocks=0, costate_mode=mode)
    x, u, lam, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p, x0, T, opts=O.Options(costate_mode=mode))
    check(info, ref, x, u, lam, FP64_TOL)
    # and it is the co-state form's KKT point
    ref0 = O.solve_ip(p, x0, T)
    check(info, ref0, x, u, lam, FP64_TOL)


def test_fp64_follows_the_oracle_iteration_path(ptn):
    p, x0, T = W.pendulum(), W.pendulum_x0(1), 64
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, block_threads=64, costate_mode=1)
    _, _, _, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p, x0, T, opts=MULT)
    assert info["newton_iters"] == ref["info"]["newton_iters"]


TIERS = {
    "cta": dict(grid_min_T=0, cluster_max_blocks=0),
    "cluster": dict(grid_min_T=0, cluster_max_blocks=16),
    "grid": dict(grid_min_T=512, cluster_max_blocks=0),
}


@pytest.mark.parametrize("T,tier,mode", [(1024, "cluster", 1), (1024, "grid", 1), (1024, "grid", 2)])
def test_fp64_multi_cta_tiers(ptn, T, tier, mode):
    p = W.cartpole(T=T, horizon=2.56)
    x0 = W.cartpole_x0(1)
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, costate_mode=mode, **TIERS[tier])
    x, u, lam, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p, x0, T, opts=O.Options(costate_mode=mode))
    check(info, ref, x, u, lam, FP64_TOL)


@pytest.mark.parametrize("T,tier,prec,mode", [(256, "cta", 1, 1), (1024, "cluster", 1, 1), (4096, "grid", 1, 1),
                                              (4096, "cluster", 2, 1), (1024, "cluster", 1, 2), (4096, "grid", 1, 2)])
def test_fp32_matches_oracle(ptn, T, tier, prec, mode):
    # both sides solved to 1e-7, as in the co-state form's FP32 parity tests
    p = W.cartpole(T=T, horizon=2.56)
    x0 = W.cartpole_x0(1)
    s = ptn.Solver(p, max_T=T, precision=prec, tol_final=1e-7, costate_mode=mode, **TIERS[tier])
    x, u, lam, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p, x0, T, opts=O.Options(tol_final=1e-7, costate_mode=mode))
    check(info, ref, x, u, lam, FP32_TOL, with_lam=False)
    assert info["r_stat"] <= 1e-7


def test_batch_ragged_matches_oracle(ptn):
    p = W.cartpole()
    Tb = np.array([1, 5, 17, 64, 100, 3, 40], dtype=np.int32)
    B = len(Tb)
    x0s = W.cartpole_batch_x0(B, 6)
    s = ptn.Solver(p, max_T=int(Tb.max()), max_batch=B, precision=ptn.PTN_FP64, block_threads=64,
                   costate_mode=1)
    X, U, Lm, infos = s.solve_batch(dev(x0s), Tb)
    xo = uo = 0
    for b in range(B):
        T = int(Tb[b])
        ref = O.solve_ip(p, x0s[b], T, opts=MULT)
        check(infos[b], ref, X[xo:xo + T + 1], U[uo:uo + T], Lm[xo:xo + T + 1], FP64_TOL)
        xo += T + 1
        uo += T


def test_hybrid_form_on_batch_instances_where_the_pure_form_stalls(ptn):
    # batch workload instances (1.28 s horizon at dt_b = 1.28 / T_b): in mode 2 the GPU
    # batch matches the oracle's mode 2, which reaches the co-state form's KKT point
    Tb_all = W.batch_horizons(1024, seed=0)
    ks = [310, 236, 519, 58]
    Tb = Tb_all[ks].astype(np.int32)
    dtb = 1.28 / Tb
    x0s = W.cartpole_batch_x0(1024, seed=0)[ks]
    base = W.cartpole()
    s = ptn.Solver(base, max_T=int(Tb.max()), max_batch=len(ks), precision=ptn.PTN_FP64, block_threads=64,
                   costate_mode=2)
    X, U, Lm, infos = s.solve_batch(dev(x0s), Tb, dt_b=dtb)
    xo = uo = 0
    for b in range(len(ks)):
        T = int(Tb[b])
        sc = float(dtb[b]) / base.dt
        p = base.replace(dt=float(dtb[b]), Q=base.Q * sc, R=base.R * sc)
        ref = O.solve_ip(p, x0s[b], T, opts=O.Options(costate_mode=2))
        check(infos[b], ref, X[xo:xo + T + 1], U[uo:uo + T], Lm[xo:xo + T + 1], FP64_TOL)
        ref0 = O.solve_ip(p, x0s[b], T)
        assert rel(U[uo:uo + T].cpu().numpy(), ref0["u"]) <= FP64_TOL
        xo += T + 1
        uo += T


@pytest.mark.parametrize("tier", ["cta", "grid"])
def test_admm_fixed_outer_count(ptn, tier):
    p = W.cartpole()
    x0, T, K = W.cartpole_x0(3), 600, 6
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, admm_fixed_iters=K, tol_final=1e-9, costate_mode=1,
                   **TIERS[tier])
    x, u, lam, z, v, info = s.solve_admm(dev(x0), T, with_zv=True)
    ref = O.solve_admm(p, x0, T, opts=O.Options(admm_fixed_iters=K, tol_final=1e-9, costate_mode=1))
    assert info["status"] == 0 and info["outer_iters"] == K
    for a, b in [(x, ref["x"]), (u, ref["u"]), (z, ref["z"]), (v, ref["v"])]:
        assert rel(a.cpu().numpy(), b) <= FP64_TOL


def test_static_entry_point_is_the_handle_solve(ptn):
    p, x0, T = W.cartpole(), W.cartpole_x0(4), 150
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, block_threads=128, costate_mode=1)
    x, u, lam, info = s.solve_ip(dev(x0), T)
    xs, us, ls, infos = ptn.solve_ip_static(p, dev(x0), T, precision=ptn.PTN_FP64, block_threads=128,
                                            costate_mode=1)
    assert info["status"] == 0 and infos["status"] == 0
    assert torch.equal(x, xs) and torch.equal(u, us) and torch.equal(lam, ls)


@pytest.mark.parametrize("mode", [1, 2])
def test_wide_tier_multiplier_form_matches_oracle(ptn, mode):
    # the wide tier (nx >= 8, one warp per chunk) in the multiplier forms: the quadrotor in
    # FP64 against the oracle's form of the same mode; the static entry point runs the same
    # kernel with the same launch shape (identical results)
    p = W.quadrotor(W.quadrotor_waypoints(1, seed=0)[0])
    T = 64
    x0 = np.zeros(12)
    ui = np.full((T, 4), W.quadrotor_hover_u())
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, costate_mode=mode, grid_min_T=0)
    x, u, lam, info = s.solve_ip(dev(x0), T, u_init=dev(ui))
    ref = O.solve_ip(p, x0, T, u_init=ui, opts=O.Options(costate_mode=mode))
    check(info, ref, x, u, lam, FP64_TOL)
    xs, us, ls, infs = ptn.solve_ip_static(p, dev(x0), T, u_init=dev(ui), precision=ptn.PTN_FP64, costate_mode=mode)
    assert infs["status"] == 0
    assert torch.equal(x, xs) and torch.equal(u, us) and torch.equal(lam, ls)


def test_sequential_tier(ptn):
    # one thread per instance: the serial recursions with the multiplier form's terms
    p, x0, T = W.pendulum(), W.pendulum_x0(2), 64
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64, sequential=1, costate_mode=1)
    x, u, lam, info = s.solve_ip(dev(x0), T)
    ref = O.solve_ip(p, x0, T, opts=MULT)
    check(info, ref, x, u, lam, FP64_TOL)
