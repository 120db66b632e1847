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
    # (problem, x0 sequence, T, options)
    ("pendulum", lambda: W.pendulum(), [W.pendulum_x0(0), W.pendulum_x0(1)], 64,
     dict(precision=0, block_threads=64)),
    ("cartpole", lambda: W.cartpole(T=256, horizon=2.56), [W.cartpole_x0(0), W.cartpole_x0(3)], 256,
     dict(precision=1, block_threads=128)),
]


@pytest.mark.parametrize("name,mk,x0s,T,opt", CASES, ids=[c[0] for c in CASES])
def test_static_matches_handle_two_calls(ptn, name, mk, x0s, T, opt):
    p = mk()
    s = ptn.Solver(p, max_T=T, **opt)
    for x0 in x0s:  # two calls in a row on the same static array
        xs, us, ls, infs = ptn.solve_ip_static(p, dev(x0), T, **opt)
        xh, uh, lh, infh = s.solve_ip(dev(x0), T)
        torch.cuda.synchronize()
        assert infs["status"] == infh["status"] == 0
        assert infs["newton_iters"] == infh["newton_iters"]
        # same kernel, same launch shape, same inputs: identical results
        assert torch.equal(xs, xh) and torch.equal(us, uh) and torch.equal(ls, lh)
        assert infs["J"] == infh["J"]


def test_static_rejects_oversize_horizon(ptn):
    p = W.cartpole(T=65536, horizon=2.56)
    T = 65536  # about 0.7 KB per step: far beyond the 4 MiB array
    x0 = dev(W.cartpole_x0(0))
    with pytest.raises(ptn.PtnError, match="bytes of static scratch"):
        ptn.solve_ip_static(p, x0, T)  # full-size outputs, so a missed check could not write out of bounds
