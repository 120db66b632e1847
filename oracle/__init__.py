"""Serial FP64 CPU oracle for the parallel-in-time Newton method (arXiv 2409.20027).

TEST INFRASTRUCTURE ONLY: this package may be imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``, and by
nothing else.  It shares no code with the CUDA implementation; it links only
``ptn_oracle.c`` (plain C, compiled with gcc).

Each function cites the part of the paper it restates; the C source carries the
formulas.  Arrays are numpy float64, row-major, time-major:
``x`` is (T+1, nx), ``u`` is (T, nu), ``lam`` is (T+1, nx).

Parity pins (see tests/test_oracle_*.py) tie every function here to something
other than itself: closed-form LQR, dense KKT solves, finite differences,
physical invariants of the models, and brute-force minimisation on tiny horizons.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptn_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "libptn_oracle.so")

MAXN, MAXM, MAXP = 32, 8, 8
PENDULUM, CARTPOLE, QUADROTOR, SYNTH = 0, 1, 2, 3
EULER, RK4 = 0, 1
STATUS = {0: "ok", -1: "invalid argument", -2: "infeasible start", -3: "not converged",
          -4: "numerical failure"}
INFO_KEYS = ["status", "newton_iters", "outer_iters", "mu", "alpha", "r_stat", "r_dyn",
             "r_feas", "r_kkt", "J", "J_c", "r_p", "r_d", "ls_rejects", "factor_fails"]


def build(force: bool = False) -> str:
    """Compile ptn_oracle.c into oracle/_build/libptn_oracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_P = C.POINTER(C.c_double)


# callbacks of user-written terms (orc_ustage_fn, orc_uterm_fn, orc_ucons_fn)
_USTAGE = C.CFUNCTYPE(C.c_double, C.c_void_p, C.c_int, _P, _P, _P, _P)
_UTERM = C.CFUNCTYPE(C.c_double, C.c_void_p, _P, _P, _P)
_UCONS = C.CFUNCTYPE(None, C.c_void_p, C.c_int, _P, _P, _P, _P, _P)


class _Problem(C.Structure):
    _fields_ = [("model", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("integrator", C.c_int),
                ("dt", C.c_double), ("prm", C.c_double * MAXP),
                ("A", _P), ("B", _P), ("W", _P), ("Q", _P), ("R", _P), ("Qf", _P),
                ("xref", _P), ("uref", _P), ("xref_traj", _P), ("uref_traj", _P), ("T_traj", C.c_int),
                ("ustage", _USTAGE), ("uterm", _UTERM), ("ucons", _UCONS), ("nc", C.c_int),
                ("uctx", C.c_void_p),
                ("xlo", _P), ("xhi", _P), ("ulo", _P), ("uhi", _P)]


class _Options(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ["mu0", "zeta", "mu_final", "tol_inner", "tol_final", "rho", "admm_tol",
                 "alpha0", "alpha_min", "alpha_max", "ls_beta", "armijo_c1", "armijo_eps"]] + \
               [(k, C.c_int) for k in ["max_newton", "max_outer", "ls_count", "admm_fixed_iters",
                                       "costate_mode", "update_mode"]]


class _Aug(C.Structure):
    _fields_ = [("kind", C.c_int), ("nw", C.c_int), ("mu", C.c_double), ("rho", C.c_double),
                ("z", _P), ("v", _P)]


@dataclass
class Options:
    """Solver settings (the paper fixes none of these; values are readings):
    mu 1e-1 -> 1e-6 by x0.1, inner tolerance 1e-4 (1e-6 at the last mu), at most 500
    Newton iterations per barrier level, ten step sizes 1, 1/2, ..., Armijo c1 = 1e-4,
    Marquardt-type alpha update from alpha0 = 1e-6."""
    mu0: float = 1e-1
    zeta: float = 0.1
    mu_final: float = 1e-6
    tol_inner: float = 1e-4
    tol_final: float = 1e-6
    rho: float = 1.0
    admm_tol: float = 1e-2
    alpha0: float = 1e-6
    alpha_min: float = 1e-10
    alpha_max: float = 1e10
    ls_beta: float = 0.5
    armijo_c1: float = 1e-4
    armijo_eps: float = 1e-12
    max_newton: int = 500
    max_outer: int = 2000
    ls_count: int = 10
    admm_fixed_iters: int = 0
    # 0: co-states by the backward recursion (Sec. III-B); 1: multiplier form, a variant
    # that updates multipliers of the dynamics by the LQR duals (no recursion through F^T);
    # 2: the multiplier form restarted from the recursion's co-states at every sub-problem
    costate_mode: int = 0
    # 0: steps accepted on the closed-loop nonlinear rollout (line search); 1: the update
    # of Alg. 4 as printed, x <- x + dx, u <- u + du (taken when its cost is finite)
    update_mode: int = 0

    def _c(self) -> _Options:
        o = _Options()
        for k, _ in _Options._fields_:
            setattr(o, k, getattr(self, k))
        return o


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
    return _lib


def _arr(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_P)


class _Bound:
    """Keeps the numpy arrays referenced by a C problem struct alive.  T: the horizon of
    a call that evaluates costs (time-varying targets, (T+1) x nx and T x nu, are bound
    and checked against it); without T they are not bound (model-only calls)."""

    def __init__(self, prob, T=None):
        self.keep = []
        c = _Problem()
        c.model, c.nx, c.nu = int(prob.model), int(prob.nx), int(prob.nu)
        c.integrator = int(prob.integrator)
        c.dt = float(prob.dt)
        prm = np.zeros(MAXP)
        prm[: len(prob.prm)] = prob.prm
        for i in range(MAXP):
            c.prm[i] = prm[i]
        for name in ["A", "B", "W", "Q", "R", "Qf", "xref", "uref", "xlo", "xhi", "ulo", "uhi"]:
            v = getattr(prob, name, None)
            if v is None:
                setattr(c, name, None)
            else:
                a = _arr(v).ravel().copy()
                self.keep.append(a)
                setattr(c, name, _ptr(a))
        xt, ut = getattr(prob, "xref_traj", None), getattr(prob, "uref_traj", None)
        c.xref_traj = c.uref_traj = None
        c.T_traj = 0
        if (xt is not None or ut is not None) and T is not None:
            c.T_traj = int(T)
            for name, v, rows, cols in [("xref_traj", xt, T + 1, c.nx), ("uref_traj", ut, T, c.nu)]:
                if v is None:
                    continue
                a = _arr(v).reshape(-1).copy()
                if a.size != rows * cols:
                    raise ValueError(f"{name} must have {rows} x {cols} entries")
                self.keep.append(a)
                setattr(c, name, _ptr(a))
        self._bind_user_terms(prob, c)
        self.c = c
        self.n, self.m = c.nx, c.nu

    def _bind_user_terms(self, prob, c):
        # user-written stage cost, terminal cost and inequality rows (Problem.user_terms: an
        # object with stage(t, x, u) -> (l, grad_z, hess_z), terminal(x) -> (l, grad, hess),
        # constraints(t, x, u) -> (g, jac_z, hess_z) and nc; any of them may be None)
        ut = getattr(prob, "user_terms", None)
        c.nc = 0
        if ut is None:
            return
        n, m = int(prob.nx), int(prob.nu)
        K = n + m

        def put(ptr, a):
            if ptr:
                a = np.asarray(a, dtype=np.float64).ravel()
                for i, v in enumerate(a):
                    ptr[i] = v

        if getattr(ut, "stage", None) is not None:
            def stage(ctx, t, x, u, gz, Hz):
                xa = np.ctypeslib.as_array(x, shape=(n,)).copy()
                ua = np.ctypeslib.as_array(u, shape=(m,)).copy()
                l, g, H = ut.stage(int(t), xa, ua)
                put(gz, g); put(Hz, np.asarray(H).reshape(K, K))
                return float(l)
            cb = _USTAGE(stage); self.keep.append(cb); c.ustage = cb
        if getattr(ut, "terminal", None) is not None:
            def term(ctx, x, gx, Hx):
                xa = np.ctypeslib.as_array(x, shape=(n,)).copy()
                l, g, H = ut.terminal(xa)
                put(gx, g); put(Hx, np.asarray(H).reshape(n, n))
                return float(l)
            cb = _UTERM(term); self.keep.append(cb); c.uterm = cb
        if getattr(ut, "constraints", None) is not None and int(ut.nc) > 0:
            nc = int(ut.nc)

            def cons(ctx, t, x, u, g, Jz, Hz):
                xa = np.ctypeslib.as_array(x, shape=(n,)).copy()
                ua = np.ctypeslib.as_array(u, shape=(m,)).copy()
                gv, J, H = ut.constraints(int(t), xa, ua)
                put(g, gv); put(Jz, np.asarray(J).reshape(nc, K)); put(Hz, np.asarray(H).reshape(nc, K, K))
            cb = _UCONS(cons); self.keep.append(cb); c.ucons = cb
            c.nc = nc

    def ref(self):
        return C.byref(self.c)


def _aug(kind="none", mu=0.0, rho=1.0, z=None, v=None, nw=0):
    a = _Aug()
    a.kind = {"none": 0, "barrier": 1, "admm": 2}[kind]
    a.nw, a.mu, a.rho = nw, mu, rho
    keep = []
    if z is not None:
        z = _arr(z).copy(); v = _arr(v).copy(); keep += [z, v]
        a.z, a.v = _ptr(z), _ptr(v)
    return a, keep


# ---------------- models (Sec. IV; BASELINE configurations) ----------------

def step(prob, x, u):
    """x+ = f(x, u): Euler or RK4 step of the model, or the synthetic map."""
    b = _Bound(prob); x = _arr(x); u = _arr(u); out = np.zeros(b.n)
    lib().orc_step(b.ref(), _ptr(x), _ptr(u), _ptr(out))
    return out


def rhs(prob, x, u):
    """Continuous-time right-hand side (pendulum, cart-pole, quadrotor)."""
    b = _Bound(prob); x = _arr(x); u = _arr(u); out = np.zeros(b.n)
    lib().orc_rhs(b.ref(), _ptr(x), _ptr(u), _ptr(out))
    return out


def jac(prob, x, u):
    """(F, G) = (df/dx, df/du) by hyper-dual differentiation."""
    b = _Bound(prob); x = _arr(x); u = _arr(u)
    F = np.zeros((b.n, b.n)); G = np.zeros((b.n, b.m))
    lib().orc_jac(b.ref(), _ptr(x), _ptr(u), _ptr(F), _ptr(G))
    return F, G


def hess(prob, x, u, lam):
    """lam . f_zz blocks (Sec. III-C tensor contraction): (Hxx, Hxu, Huu)."""
    b = _Bound(prob); x = _arr(x); u = _arr(u); lam = _arr(lam)
    Hxx = np.zeros((b.n, b.n)); Hxu = np.zeros((b.n, b.m)); Huu = np.zeros((b.m, b.m))
    lib().orc_hess(b.ref(), _ptr(x), _ptr(u), _ptr(lam), _ptr(Hxx), _ptr(Hxu), _ptr(Huu))
    return Hxx, Hxu, Huu


def param_jac(prob, x, u):
    """df/dprm, shape (nx, 8)."""
    b = _Bound(prob); x = _arr(x); u = _arr(u); out = np.zeros((b.n, MAXP))
    lib().orc_param_jac(b.ref(), _ptr(x), _ptr(u), _ptr(out))
    return out


def param_hess(prob, x, u, lam):
    """d2 (lam . f) / dz dprm with z = (x, u), shape (nx + nu, 8)."""
    b = _Bound(prob); x = _arr(x); u = _arr(u); lam = _arr(lam)
    out = np.zeros((b.n + b.m, MAXP))
    lib().orc_param_hess(b.ref(), _ptr(x), _ptr(u), _ptr(lam), _ptr(out))
    return out


def rollout(prob, x0, u):
    b = _Bound(prob); x0 = _arr(x0); u = _arr(u)
    T = u.shape[0]
    x = np.zeros((T + 1, b.n))
    lib().orc_rollout(b.ref(), _ptr(x0), _ptr(u), C.c_int(T), _ptr(x))
    return x


def num_rows(prob):
    """Number of constraint rows w = [g; h] (finite box bounds)."""
    return int(lib().orc_num_rows(_Bound(prob).ref()))


def constraints(prob, x, u):
    b = _Bound(prob); nw = num_rows(prob); w = np.zeros(nw)
    lib().orc_constraints(b.ref(), _ptr(_arr(x)), _ptr(_arr(u)), _ptr(w))
    return w


def cost(prob, x, u, aug="none", mu=0.0, rho=1.0, z=None, v=None):
    """(J_c, J): augmented cost of Sec. III-A and the plain cost of eq. ocp."""
    x = _arr(x); u = _arr(u); T = u.shape[0]; b = _Bound(prob, T)
    a, keep = _aug(aug, mu, rho, z, v, num_rows(prob))
    Jp = C.c_double(0.0)
    lib().orc_cost.restype = C.c_double
    Jc = lib().orc_cost(b.ref(), C.byref(a), C.c_int(T), _ptr(x), _ptr(u), C.byref(Jp))
    return float(Jc), float(Jp.value)


def newton_direction(prob, x, u, alpha, aug="barrier", mu=0.1, rho=1.0, z=None, v=None):
    """One Newton step at the nominal (x, u) (Sec. III): dict with lam, d, S, s, Gam, gam,
    dx, du, P, M, R, F, G, G1, G2 and status (1 = R~ or Q not positive definite)."""
    x = _arr(x); u = _arr(u); T = u.shape[0]; b = _Bound(prob, T); n, m = b.n, b.m
    a, keep = _aug(aug, mu, rho, z, v, num_rows(prob))
    out = dict(lam=np.zeros((T + 1, n)), d=np.zeros((T, m)), S=np.zeros((T + 1, n, n)),
               s=np.zeros((T + 1, n)), Gam=np.zeros((T, m, n)), gam=np.zeros((T, m)),
               dx=np.zeros((T + 1, n)), du=np.zeros((T, m)), P=np.zeros((T + 1, n, n)),
               M=np.zeros((T, n, m)), R=np.zeros((T, m, m)), F=np.zeros((T, n, n)),
               G=np.zeros((T, n, m)))
    g12 = np.zeros(2)
    keys = ["lam", "d", "S", "s", "Gam", "gam", "dx", "du", "P", "M", "R", "F", "G"]
    st = lib().orc_newton_direction(b.ref(), C.byref(a), C.c_int(T), _ptr(x), _ptr(u),
                                    C.c_double(alpha), *[_ptr(out[k]) for k in keys], _ptr(g12))
    out["G1"], out["G2"], out["status"] = g12[0], g12[1], int(st)
    return out


def newton_direction_mult(prob, x, u, nu, alpha, aug="barrier", mu=0.1, rho=1.0, z=None, v=None):
    """One Newton step of the multiplier form (a variant, not in the paper: multipliers nu
    of the dynamics instead of the co-state recursion of Sec. III-B) at (x, u, nu): dict
    with q, d, dx, du, dnu (dual step S_t dx_t + s_t), G1, G2 and status."""
    x = _arr(x); u = _arr(u); T = u.shape[0]; b = _Bound(prob, T); n, m = b.n, b.m
    nu = _arr(nu, (T + 1, n))
    a, keep = _aug(aug, mu, rho, z, v, num_rows(prob))
    out = dict(q=np.zeros((T + 1, n)), d=np.zeros((T, m)), dx=np.zeros((T + 1, n)),
               du=np.zeros((T, m)), dnu=np.zeros((T + 1, n)))
    g12 = np.zeros(2)
    st = lib().orc_newton_direction_mult(b.ref(), C.byref(a), C.c_int(T), _ptr(x), _ptr(u), _ptr(nu),
                                         C.c_double(alpha), _ptr(out["q"]), _ptr(out["d"]),
                                         _ptr(out["dx"]), _ptr(out["du"]), _ptr(out["dnu"]), _ptr(g12))
    out["G1"], out["G2"], out["status"] = g12[0], g12[1], int(st)
    return out


# ---------------- associative elements and operators (Alg. 1-3) ----------------

def costate_combine(g1, Ft1, g2, Ft2):
    """eq. co-states-comb-rule: (g, F^T)_{j,i} from (j,t) then (t,i)."""
    g1, Ft1, g2, Ft2 = map(_arr, (g1, Ft1, g2, Ft2)); n = g1.shape[0]
    g = np.zeros(n); Ft = np.zeros((n, n))
    lib().orc_costate_combine(C.c_int(n), _ptr(g1), _ptr(Ft1), _ptr(g2), _ptr(Ft2), _ptr(g), _ptr(Ft))
    return g, Ft


def value_init(F, G, P, M, R, d, alpha, pinv=False):
    """eq. value-fun-elem-init; pinv=True uses the printed q_t, r_t form (needs P^{-1}).
    Returns (A, b, C, eta, J) or None when a factorisation fails."""
    F, G, P, M, R, d = map(_arr, (F, G, P, M, R, d)); n, m = G.shape
    A = np.zeros((n, n)); b = np.zeros(n); Cm = np.zeros((n, n)); eta = np.zeros(n); J = np.zeros((n, n))
    fn = lib().orc_value_init_pinv if pinv else lib().orc_value_init
    st = fn(C.c_int(n), C.c_int(m), _ptr(F), _ptr(G), _ptr(P), _ptr(M), _ptr(R), _ptr(d),
            C.c_double(alpha), _ptr(A), _ptr(b), _ptr(Cm), _ptr(eta), _ptr(J))
    return None if st else (A, b, Cm, eta, J)


def value_combine(e1, e2):
    """eq. value-fun-param (element 1 earlier in time); None if I + CJ is singular."""
    e1 = [_arr(a) for a in e1]; e2 = [_arr(a) for a in e2]; n = e1[1].shape[0]
    A = np.zeros((n, n)); b = np.zeros(n); Cm = np.zeros((n, n)); eta = np.zeros(n); J = np.zeros((n, n))
    st = lib().orc_value_combine(C.c_int(n), *[_ptr(a) for a in e1], *[_ptr(a) for a in e2],
                                 _ptr(A), _ptr(b), _ptr(Cm), _ptr(eta), _ptr(J))
    return None if st else (A, b, Cm, eta, J)


def state_combine(F1, e1, F2, e2):
    """eq. state-prop-comb-rule (element 1 earlier in time)."""
    F1, e1, F2, e2 = map(_arr, (F1, e1, F2, e2)); n = e1.shape[0]
    F = np.zeros((n, n)); e = np.zeros(n)
    lib().orc_state_combine(C.c_int(n), _ptr(F1), _ptr(e1), _ptr(F2), _ptr(e2), _ptr(F), _ptr(e))
    return F, e


# ---------------- solvers ----------------

def _info(a):
    d = {k: float(a[i]) for i, k in enumerate(INFO_KEYS)}
    d["status"] = int(d["status"])
    d["newton_iters"] = int(d["newton_iters"]); d["outer_iters"] = int(d["outer_iters"])
    return d


def solve_ip(prob, x0, T, u_init=None, opts: Options | None = None):
    """Primal log-barrier IP (eq. lb-min, lb-step-2) with Newton sub-solves (Alg. 4)."""
    opts = opts or Options()
    b = _Bound(prob, T); n, m = b.n, b.m; x0 = _arr(x0)
    ui = None if u_init is None else _arr(u_init, (T, m))
    x = np.zeros((T + 1, n)); u = np.zeros((T, m)); lam = np.zeros((T + 1, n)); info = np.zeros(16)
    o = opts._c()
    lib().orc_solve_ip(b.ref(), C.byref(o), _ptr(x0), _ptr(ui), C.c_int(T), _ptr(x), _ptr(u),
                       _ptr(lam), _ptr(info))
    return dict(x=x, u=u, lam=lam, info=_info(info))


def solve_fixed_mu(prob, x0, T, mu, tol, u_init, opts: Options | None = None):
    """Newton on the barrier problem at a single mu, warm-started from u_init."""
    opts = opts or Options()
    b = _Bound(prob, T); n, m = b.n, b.m; x0 = _arr(x0); ui = _arr(u_init, (T, m))
    x = np.zeros((T + 1, n)); u = np.zeros((T, m)); lam = np.zeros((T + 1, n)); info = np.zeros(16)
    o = opts._c()
    lib().orc_solve_fixed_mu(b.ref(), C.byref(o), C.c_double(mu), C.c_double(tol), _ptr(x0),
                             _ptr(ui), C.c_int(T), _ptr(x), _ptr(u), _ptr(lam), _ptr(info))
    return dict(x=x, u=u, lam=lam, info=_info(info))


def solve_admm(prob, x0, T, u_init=None, opts: Options | None = None):
    """ADMM (eq. admm-min ... admm-step-5) with Newton sub-solves (Alg. 4)."""
    opts = opts or Options()
    b = _Bound(prob, T); n, m = b.n, b.m; x0 = _arr(x0); nw = num_rows(prob)
    ui = None if u_init is None else _arr(u_init, (T, m))
    x = np.zeros((T + 1, n)); u = np.zeros((T, m)); lam = np.zeros((T + 1, n)); info = np.zeros(16)
    z = np.zeros((T, nw)); v = np.zeros((T, nw))
    o = opts._c()
    lib().orc_solve_admm(b.ref(), C.byref(o), _ptr(x0), _ptr(ui), C.c_int(T), _ptr(z), _ptr(v),
                         _ptr(x), _ptr(u), _ptr(lam), _ptr(info))
    return dict(x=x, u=u, lam=lam, z=z, v=v, info=_info(info))


def adjoint(prob, mu, x, u, gJ=1.0, gx=None, gu=None):
    """Gradients of gJ*J* + <gx, x*> + <gu, u*> w.r.t. x0, diag Q, diag R, diag Qf, prm."""
    x = _arr(x); u = _arr(u); T = u.shape[0]; b = _Bound(prob, T); n, m = b.n, b.m
    gx = None if gx is None else _arr(gx, (T + 1, n))
    gu = None if gu is None else _arr(gu, (T, m))
    out = dict(x0=np.zeros(n), Qd=np.zeros(n), Rd=np.zeros(m), Qfd=np.zeros(n), prm=np.zeros(MAXP))
    st = lib().orc_adjoint(b.ref(), C.c_double(mu), C.c_int(T), _ptr(x), _ptr(u), C.c_double(gJ),
                           _ptr(gx), _ptr(gu), _ptr(out["x0"]), _ptr(out["Qd"]), _ptr(out["Rd"]),
                           _ptr(out["Qfd"]), _ptr(out["prm"]))
    out["status"] = int(st)
    return out
