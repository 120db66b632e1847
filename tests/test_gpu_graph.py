"""Graph-capturable batch solves (ptn_batch_prepare + ptn_solve_batch_async).

The asynchronous entry point launches the same kernels as the synchronous one on the
same launch shape, so its results must be bit-identical to ptn_solve_batch on the same
inputs, whether it runs eagerly or is replayed from a captured CUDA graph; the
synchronous path is itself compared with the oracle, and one case here checks against
the oracle directly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def same(a, b):
    return torch.equal(a, b)


def report(infos):
    """The solve reports without the per-phase clock counters (timings differ run to run)."""
    return [{k: v for k, v in i.items() if k != "cycles"} for i in infos]


def test_async_batch_is_the_synchronous_solve(ptn):
    p = W.cartpole()
    Tb = np.array([1, 17, 64, 40, 3], dtype=np.int32)
    B = len(Tb)
    x0s = dev(W.cartpole_batch_x0(B, 11))
    s = ptn.Solver(p, max_T=int(Tb.max()), max_batch=B, precision=ptn.PTN_FP64, block_threads=64)
    X, U, L, infos = s.solve_batch(x0s, Tb)
    s.prepare_batch(Tb)
    Xa, Ua, La, info_dev = s.solve_batch_async(x0s)
    torch.cuda.synchronize()
    ia = ptn.infos_from_device(info_dev, B)
    assert same(X, Xa) and same(U, Ua) and same(L, La)
    assert report(infos) == report(ia)
    # one instance against the oracle directly
    T, xo, uo = int(Tb[2]), int(Tb[0] + Tb[1] + 2), int(Tb[0] + Tb[1])
    ref = O.solve_ip(p, W.cartpole_batch_x0(B, 11)[2], T)
    assert ia[2]["status"] == 0 and ref["info"]["status"] == 0
    assert rel(Xa[xo:xo + T + 1].cpu().numpy(), ref["x"]) <= 1e-6
    assert rel(Ua[uo:uo + T].cpu().numpy(), ref["u"]) <= 1e-6
    assert ia[2]["newton_iters"] == ref["info"]["newton_iters"]


def test_graph_replay_follows_inputs_updated_in_place(ptn):
    p = W.cartpole()
    Tb = np.array([30, 64, 45, 12], dtype=np.int32)
    B = len(Tb)
    s = ptn.Solver(p, max_T=int(Tb.max()), max_batch=B, precision=ptn.PTN_FP64, block_threads=64)
    s.prepare_batch(Tb)
    x0 = dev(W.cartpole_batch_x0(B, 0))
    X = torch.empty((int(Tb.sum()) + B, 4), dtype=torch.float64, device="cuda:0")
    U = torch.empty((int(Tb.sum()), 1), dtype=torch.float64, device="cuda:0")
    L = torch.empty_like(X)
    info = s.new_info_buffer(B)
    s.solve_batch_async(x0, x_out=X, u_out=U, lam_out=L, info_dev=info)  # loads the kernel
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s.solve_batch_async(x0, x_out=X, u_out=U, lam_out=L, info_dev=info)
    for seed in [1, 2, 3]:
        x0.copy_(dev(W.cartpole_batch_x0(B, seed)))
        info.zero_()
        g.replay()
        torch.cuda.synchronize()
        Xs, Us, Ls, infos = s.solve_batch(x0, Tb)
        assert same(X, Xs) and same(U, Us) and same(L, Ls), seed
        assert report(ptn.infos_from_device(info, B)) == report(infos)
        assert all(i["status"] == 0 for i in infos)
        assert ptn.status_view(info, B).cpu().tolist() == [[0, i["newton_iters"]] for i in infos]


@pytest.mark.parametrize("tier", ["cluster", "grid"])
def test_graph_replay_single_instance_multi_cta_tiers(ptn, tier):
    # one instance over several CTAs: a thread-block cluster, or the cooperative grid
    # (its barrier counters are reset by memset nodes of the same graph)
    T = 1024
    opts = {"cluster": dict(grid_min_T=0, cluster_max_blocks=16),
            "grid": dict(grid_min_T=512, cluster_max_blocks=0)}[tier]
    p = W.cartpole(T=T, horizon=2.56)
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, **opts)
    s.prepare_batch([T])
    x0 = dev(W.cartpole_x0(1)).reshape(1, 4)
    X = torch.empty((T + 1, 4), dtype=torch.float64, device="cuda:0")
    U = torch.empty((T, 1), dtype=torch.float64, device="cuda:0")
    info = s.new_info_buffer(1)
    s.solve_batch_async(x0, x_out=X, u_out=U, info_dev=info)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s.solve_batch_async(x0, x_out=X, u_out=U, info_dev=info)
    for seed in [2, 3]:
        x0.copy_(dev(W.cartpole_x0(seed)).reshape(1, 4))
        g.replay()
        torch.cuda.synchronize()
        Xs, Us, _, ii = s.solve_ip(x0.reshape(4), T)
        ia = ptn.infos_from_device(info, 1)[0]
        assert ii["status"] == 0 and ia["status"] == 0
        assert same(X, Xs) and same(U, Us), seed
        assert ia["newton_iters"] == ii["newton_iters"]


def test_prepared_layout_survives_synchronous_solves(ptn):
    p = W.pendulum()
    Tb = np.array([20, 64, 7], dtype=np.int32)
    B = len(Tb)
    s = ptn.Solver(p, max_T=64, max_batch=B, precision=ptn.PTN_FP64, block_threads=32)
    x0 = dev(np.stack([W.pendulum_x0(k) for k in range(B)]))
    s.prepare_batch(Tb)
    Xa, Ua, _, ia = s.solve_batch_async(x0)
    # a synchronous solve with another layout and other options in between
    s.set_options(tol_final=1e-7)
    s.solve_batch(x0[:2].contiguous(), [64, 64])
    Xb, Ub, _, ib = s.solve_batch_async(x0)
    torch.cuda.synchronize()
    assert same(Xa, Xb) and same(Ua, Ub)
    assert report(ptn.infos_from_device(ia, B)) == report(ptn.infos_from_device(ib, B))


def test_async_argument_errors(ptn):
    p = W.pendulum()
    s = ptn.Solver(p, max_T=16, max_batch=2, precision=ptn.PTN_FP64)
    x0 = dev(np.zeros((2, 2)))
    with pytest.raises(ptn.PtnError):
        s.solve_batch_async(x0)  # nothing prepared
    s.prepare_batch([16, 16])
    with pytest.raises(ptn.PtnError):
        s.prepare_batch([16, 0])  # empty horizon
    with pytest.raises(ptn.PtnError):
        s.prepare_batch([16, 16, 16])  # more instances than the handle holds
    with pytest.raises(ptn.PtnError):
        s.prepare_batch([16, 17])  # beyond the workspace
    with pytest.raises(ptn.PtnError):
        s.prepare_batch([16, 16], dt_b=[0.05, -1.0])
    # a failed prepare leaves no usable layout behind, in the library as in the binding
    with pytest.raises(ptn.PtnError):
        s.solve_batch_async(x0)
    s._prepared = (2, 32)
    with pytest.raises(ptn.PtnError, match="no batch prepared"):
        s.solve_batch_async(x0)


def test_graph_replay_survives_smaller_launches_of_the_same_kernel(ptn):
    # a kernel's dynamic shared-memory limit only grows: a solve with fewer threads per CTA
    # after the capture must leave the captured, larger launch valid
    p = W.cartpole()
    Tb = np.array([40, 64], dtype=np.int32)
    s = ptn.Solver(p, max_T=64, max_batch=2, precision=ptn.PTN_FP64, block_threads=256)
    s.prepare_batch(Tb)
    x0 = dev(W.cartpole_batch_x0(2, 1))
    X = torch.empty((int(Tb.sum()) + 2, 4), dtype=torch.float64, device="cuda:0")
    U = torch.empty((int(Tb.sum()), 1), dtype=torch.float64, device="cuda:0")
    info = s.new_info_buffer(2)
    s.solve_batch_async(x0, x_out=X, u_out=U, info_dev=info)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        s.solve_batch_async(x0, x_out=X, u_out=U, info_dev=info)
    small = ptn.Solver(p, max_T=64, max_batch=2, precision=ptn.PTN_FP64, block_threads=32)
    _, _, _, si = small.solve_batch(x0, Tb)  # the same kernel with less shared memory
    assert all(i["status"] == 0 for i in si)
    X.zero_()
    g.replay()
    torch.cuda.synchronize()
    Xs, Us, _, infos = s.solve_batch(x0, Tb)
    assert all(i["status"] == 0 for i in infos)
    assert same(X, Xs) and same(U, Us)
    assert report(ptn.infos_from_device(info, 2)) == report(infos)
