"""Pins for the associative elements and operators of Alg. 1-3.

The operators are checked to be associative, to have the identities they should,
and -- folded in a balanced-tree order unlike any sequential loop -- to reproduce
the sequential recursions they stand for: the co-state recursion eq. co-state-eq,
the Riccati recursion (pinned itself against a dense KKT solve in
test_oracle_newton.py) and the forward state recursion.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

RNG = np.random.default_rng(7)


def tree_fold(elems, combine, lo, hi):
    """Combine elems[lo:hi] in balanced-tree order (left half before right half)."""
    if hi - lo == 1:
        return elems[lo]
    mid = (lo + hi) // 2
    return combine(tree_fold(elems, combine, lo, mid), tree_fold(elems, combine, mid, hi))


# ---------------------------------------------------------------- co-state scan (Alg. 1)

def test_costate_scan_equals_backward_recursion():
    n, N = 4, 37
    F = [np.eye(n) + 0.2 * RNG.normal(size=(n, n)) for _ in range(N)]
    q = [RNG.normal(size=n) for _ in range(N)]
    lamT = RNG.normal(size=n)
    # sequential definition eq. co-state-eq / co-state-final
    lam = [None] * (N + 1)
    lam[N] = lamT
    for t in range(N - 1, -1, -1):
        lam[t] = q[t] + F[t].T @ lam[t + 1]
    # elements eq. co-state-elem-init and co-state-final-elem-init
    el = [(q[t], F[t].T) for t in range(N - 1)]
    el.append((q[N - 1] + F[N - 1].T @ lamT, np.zeros((n, n))))
    comb = lambda a, b: O.costate_combine(a[0], a[1], b[0], b[1])
    for t in range(N):
        g, Ft = tree_fold(el, comb, t, N)
        assert np.allclose(g, lam[t], rtol=1e-12, atol=1e-12)
        assert np.abs(Ft).max() == 0.0


def test_costate_operator_associative():
    n = 3
    e = [(RNG.normal(size=n), RNG.normal(size=(n, n))) for _ in range(3)]
    c = lambda a, b: O.costate_combine(a[0], a[1], b[0], b[1])
    l = c(c(e[0], e[1]), e[2]); r = c(e[0], c(e[1], e[2]))
    assert np.allclose(l[0], r[0]) and np.allclose(l[1], r[1])


# ---------------------------------------------------------------- value scan (Alg. 2)

def _random_elem(n, m, rng):
    F = np.eye(n) + 0.3 * rng.normal(size=(n, n))
    G = rng.normal(size=(n, m))
    L = rng.normal(size=(n, n)); P = L @ L.T + 0.5 * np.eye(n)
    M = 0.1 * rng.normal(size=(n, m))
    Lr = rng.normal(size=(m, m)); R = Lr @ Lr.T + np.eye(m)
    d = rng.normal(size=m)
    return F, G, P, M, R, d


def test_value_init_pinv_free_form_equals_printed_form():
    # eq. value-fun-elem-init with q_t, r_t (needs P^{-1}) vs the P^{-1}-free form
    for n, m in [(2, 1), (4, 1), (6, 3)]:
        for _ in range(5):
            F, G, P, M, R, d = _random_elem(n, m, RNG)
            a = O.value_init(F, G, P, M, R, d, 0.3)
            b = O.value_init(F, G, P, M, R, d, 0.3, pinv=True)
            for x, y in zip(a, b):
                assert np.allclose(x, y, rtol=1e-10, atol=1e-11)


def _identity(n):
    return (np.eye(n), np.zeros(n), np.zeros((n, n)), np.zeros(n), np.zeros((n, n)))


def test_value_operator_identity_and_associativity():
    n, m = 4, 2
    els = [O.value_init(*_random_elem(n, m, RNG), 0.1) for _ in range(3)]
    I = _identity(n)
    for e in els:
        for x, y in zip(O.value_combine(I, e), e):
            assert np.allclose(x, y, atol=1e-13)
        for x, y in zip(O.value_combine(e, I), e):
            assert np.allclose(x, y, atol=1e-13)
    l = O.value_combine(O.value_combine(els[0], els[1]), els[2])
    r = O.value_combine(els[0], O.value_combine(els[1], els[2]))
    for x, y in zip(l, r):
        assert np.allclose(x, y, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("prob,T,alpha", [(W.cartpole(T=33, horizon=0.33), 33, 1e-2),
                                          (W.pendulum(), 24, 0.0),
                                          (W.quadrotor(waypoint=[0.5, 0.2, -0.3]), 9, 1e-3)])
def test_value_scan_equals_riccati(prob, T, alpha):
    # Alg. 2: S_t = J_{t,<|}, s_t = -eta_{t,<|} with V*_t = nu_t (x) ... (x) nu_{N+1}
    n, m = prob.nx, prob.nu
    if prob.model == W.QUADROTOR:
        x0 = np.zeros(12); u = np.full((T, 4), W.quadrotor_hover_u()) + 0.05 * RNG.normal(size=(T, 4))
    elif prob.model == W.CARTPOLE:
        x0 = W.cartpole_x0(3); u = 0.5 * RNG.normal(size=(T, 1))
    else:
        x0 = W.pendulum_x0(3); u = RNG.normal(size=(T, 1))
    x = O.rollout(prob, x0, u)
    nd = O.newton_direction(prob, x, u, alpha, "barrier", 0.1)
    assert nd["status"] == 0
    el = [O.value_init(nd["F"][t], nd["G"][t], nd["P"][t], nd["M"][t], nd["R"][t], nd["d"][t], alpha)
          for t in range(T)]
    el.append((np.zeros((n, n)), np.zeros(n), np.zeros((n, n)), np.zeros(n), nd["P"][T]))
    for t in range(T + 1):
        A, b, Cm, eta, J = tree_fold(el, O.value_combine, t, T + 1)
        scale = max(1.0, np.abs(nd["S"][t]).max())
        assert np.allclose(J, nd["S"][t], rtol=1e-9, atol=1e-9 * scale)
        assert np.allclose(-eta, nd["s"][t], rtol=1e-9, atol=1e-9 * max(1.0, np.abs(nd["s"][t]).max()))
        assert np.abs(A).max() == 0 and np.abs(Cm).max() == 0 and np.abs(b).max() == 0


# ---------------------------------------------------------------- state scan (Alg. 3)

def test_state_scan_equals_forward_recursion():
    n, N = 4, 29
    Fc = [np.eye(n) + 0.2 * RNG.normal(size=(n, n)) for _ in range(N)]
    e = [RNG.normal(size=n) for _ in range(N)]
    dx = [np.zeros(n)]
    for t in range(N):
        dx.append(Fc[t] @ dx[t] + e[t])
    # eq. state-prop-elem-init; the first element has F = 0 and e = F_1 dx_1 + e_1
    el = [(np.zeros((n, n)), Fc[0] @ dx[0] + e[0])] + [(Fc[t], e[t]) for t in range(1, N)]
    comb = lambda a, b: O.state_combine(a[0], a[1], b[0], b[1])
    for t in range(1, N + 1):
        F, v = tree_fold(el, comb, 0, t)
        assert np.allclose(v, dx[t], rtol=1e-12, atol=1e-12)
        assert np.abs(F).max() == 0.0


def test_state_operator_associative():
    n = 3
    e = [(RNG.normal(size=(n, n)), RNG.normal(size=n)) for _ in range(3)]
    c = lambda a, b: O.state_combine(a[0], a[1], b[0], b[1])
    l = c(c(e[0], e[1]), e[2]); r = c(e[0], c(e[1], e[2]))
    assert np.allclose(l[0], r[0]) and np.allclose(l[1], r[1])
