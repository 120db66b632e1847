"""Allocation-free entry point ptn_solve_ip_static against the handle's ptn_solve_ip.

Collected last on purpose: it must pass both on its own and after every other GPU test
has run in the same process (the static array then holds whatever earlier work left).
Two calls in a row check that nothing is carried over from one call to the next."""
import numpy as np
import pytest
import torch

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


CASES = [
    # (problem, x0 sequence, T, options, initial controls or None)
    ("pendulum", lambda: W.pendulum(), [W.pendulum_x0(0), W.pendulum_x0(1)], 64,
     dict(precision=0, block_threads=64), None),
    ("cartpole", lambda: W.cartpole(T=256, horizon=2.56), [W.cartpole_x0(0), W.cartpole_x0(3)], 256,
     dict(precision=1, block_threads=128), None),
    # the multiplier forms place four more arrays in the static array
    ("cartpole_mult1", lambda: W.cartpole(T=256, horizon=2.56), [W.cartpole_x0(0), W.cartpole_x0(3)], 256,
     dict(precision=1, block_threads=128, costate_mode=1), None),
    ("cartpole_mult2", lambda: W.cartpole(T=256, horizon=2.56), [W.cartpole_x0(0), W.cartpole_x0(3)], 256,
     dict(precision=0, block_threads=128, costate_mode=2), None),
    # the quadrotor runs the wide tier (one warp per chunk) from the same entry point
    ("quadrotor", lambda: W.quadrotor(W.quadrotor_waypoints(1, seed=0)[0]), [np.zeros(12), np.zeros(12) + 0.01], 64,
     dict(precision=0, block_threads=128), lambda T: np.full((T, 4), W.quadrotor_hover_u())),
]


@pytest.mark.parametrize("name,mk,x0s,T,opt,uinit", CASES, ids=[c[0] for c in CASES])
def test_static_matches_handle_two_calls(ptn, name, mk, x0s, T, opt, uinit):
    p = mk()
    s = ptn.Solver(p, max_T=T, grid_min_T=0, cluster_max_blocks=0, **opt)
    u0 = None if uinit is None else dev(uinit(T))
    for x0 in x0s:  # two calls in a row on the same static array
        xs, us, ls, infs = ptn.solve_ip_static(p, dev(x0), T, u_init=u0, **opt)
        xh, uh, lh, infh = s.solve_ip(dev(x0), T, u_init=u0)
        torch.cuda.synchronize()
        assert infs["status"] == infh["status"] == 0
        assert infs["newton_iters"] == infh["newton_iters"]
        # same kernel, same launch shape, same inputs: identical results
        assert torch.equal(xs, xh) and torch.equal(us, uh) and torch.equal(ls, lh)
        assert infs["J"] == infh["J"]


def test_static_without_costate_output(ptn):
    # lam_out = NULL: the co-states stay in the static array; x and u are unchanged
    import ctypes as C
    p = W.cartpole(T=256, horizon=2.56)
    T, x0 = 256, dev(W.cartpole_x0(2))
    o = ptn.default_options(precision=1)
    xh, uh, _, infh = ptn.Solver(p, max_T=T, options=ptn.default_options(precision=1)).solve_ip(x0, T)
    lib = ptn.load()
    P, keep = ptn._make_problem(p)
    for _ in range(2):
        xs = torch.empty((T + 1, 4), dtype=torch.float64, device="cuda:0")
        us = torch.empty((T, 1), dtype=torch.float64, device="cuda:0")
        info, err = ptn.Info(), C.create_string_buffer(256)
        rc = lib.ptn_solve_ip_static(C.byref(P), C.byref(o), C.c_void_p(x0.data_ptr()), None, T,
                                     C.c_void_p(xs.data_ptr()), C.c_void_p(us.data_ptr()), None, C.byref(info), err,
                                     256, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, err.value
        assert info.newton_iters == infh["newton_iters"]
        assert torch.equal(xs, xh) and torch.equal(us, uh)
    del keep


def test_static_rejects_sequential_baseline(ptn):
    p = W.pendulum()
    with pytest.raises(ptn.PtnError, match="sequential"):
        ptn.solve_ip_static(p, dev(W.pendulum_x0(0)), 64, precision=0, sequential=1)


def test_static_rejects_oversize_horizon(ptn):
    p = W.cartpole(T=65536, horizon=2.56)
    T = 65536  # about 0.7 KB per step: far beyond the 4 MiB array
    x0 = dev(W.cartpole_x0(0))
    with pytest.raises(ptn.PtnError, match="bytes of static scratch"):
        ptn.solve_ip_static(p, x0, T)  # full-size outputs, so a missed check could not write out of bounds
