"""Closed-loop MPC with warm starts: the shift is host logic (CPU); the loop on the GPU
must follow the same loop run with oracle solves."""
import numpy as np
import pytest

from paper_2409_20027_gb300 import workloads as W


def test_shift_controls_drops_the_applied_control():
    torch = pytest.importorskip("torch")
    from paper_2409_20027_gb300 import mpc
    u = torch.arange(12, dtype=torch.float64).reshape(6, 2)  # B = 2 loops, T = 3, m = 2
    v = mpc.shift_controls(u, 3)
    assert v.tolist() == [[2, 3], [4, 5], [4, 5], [8, 9], [10, 11], [10, 11]]


@pytest.mark.gpu
def test_closed_loop_follows_oracle_loop():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle as O
    from paper_2409_20027_gb300 import mpc, ptn
    p = W.pendulum()
    T, steps, B = 30, 6, 3
    x0 = np.stack([W.pendulum_x0(s) for s in range(B)])
    s = ptn.Solver(p, max_T=T, max_batch=B, precision=ptn.PTN_FP64, block_threads=32)
    res = mpc.closed_loop(s, torch.tensor(x0, device="cuda:0"), T, steps)
    assert (res["status"] == 0).all()
    X = res["x"].cpu().numpy()
    for b in range(B):
        x, ui = x0[b], None
        for k in range(steps):
            r = O.solve_ip(p, x, T, u_init=ui)
            assert r["info"]["status"] == 0
            x = r["x"][1]
            ui = np.concatenate([r["u"][1:], r["u"][-1:]])
            assert np.abs(X[k + 1, b] - x).max() <= 1e-6 * max(1.0, np.abs(x).max()), (b, k)


@pytest.mark.gpu
def test_closed_loop_graph_replays_the_same_loop():
    # each period replayed from one captured CUDA graph: the same states, controls and
    # iteration counts as the loop that calls the synchronous batched solve
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_20027_gb300 import mpc, ptn
    p = W.cartpole()
    T, steps, B = 40, 8, 6
    x0 = torch.tensor(W.cartpole_batch_x0(B, 4), device="cuda:0")
    s = ptn.Solver(p, max_T=T, max_batch=B, precision=ptn.PTN_FP32_FP64SOLVE, block_threads=32)
    a = mpc.closed_loop(s, x0, T, steps)
    b = mpc.closed_loop_graph(s, x0, T, steps)
    assert (a["status"] == 0).all() and (b["status"] == 0).all()
    assert torch.equal(a["x"], b["x"]) and torch.equal(a["u"], b["u"])
    assert (a["iters"] == b["iters"]).all()


@pytest.mark.gpu
def test_paper_cartpole_loop_follows_oracle_loop():
    # the paper's closed-loop experiment (Sec. IV-C): its cart-pole (m_c = 10, m_p = 1,
    # Euler), |F| <= 60, N = 60 at 100 Hz, from near upright; the first periods use the
    # force limit, so the barrier terms are active
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle as O
    from paper_2409_20027_gb300 import mpc, ptn
    p = W.cartpole_paper()
    T, steps, B = W.PAPER_MPC["horizon"], 10, 3
    x0 = W.cartpole_batch_x0(B, seed=1)
    s = ptn.Solver(p, max_T=T, max_batch=B, precision=ptn.PTN_FP64, block_threads=64)
    res = mpc.closed_loop(s, torch.tensor(x0, device="cuda:0"), T, steps)
    assert (res["status"] == 0).all()
    X = res["x"].cpu().numpy()
    U = res["u"].cpu().numpy()
    for b in range(B):
        x, ui = x0[b], None
        for k in range(steps):
            r = O.solve_ip(p, x, T, u_init=ui)
            assert r["info"]["status"] == 0
            assert np.abs(U[k, b] - r["u"][0]).max() <= 1e-6 * max(1.0, np.abs(r["u"][0]).max()), (b, k)
            x = r["x"][1]
            ui = np.concatenate([r["u"][1:], r["u"][-1:]])
            assert np.abs(X[k + 1, b] - x).max() <= 1e-6 * max(1.0, np.abs(x).max()), (b, k)
