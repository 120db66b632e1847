"""The kernels' model code and scan operators on the host: ptn_models.cuh and ptn_ops.cuh
are written __host__ __device__, so a host build of the same templates
(tests/host_models/*.cu, compiled with nvcc, run on the CPU) gives the GPU path's step
map and its increment (FP64 and FP32), its forward-mode and closed-loop Jacobians, its
lam-contracted Hessians and the adjoint's parameter derivatives.  They must agree with the oracle's models, which are separate
code (hyper-dual numbers, pinned by finite differences in test_oracle_models), for every
model and integrator the kernels use -- without a GPU.  Likewise the kernels' value,
co-state and state combines and the value-element initialisation against the oracle's
operators (pinned by the scan identities in test_oracle_scans), in FP64 and in the FP32
form with FP64 solves."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_models", "ptn_host_models.cu")
SRC_OPS = os.path.join(ROOT, "tests", "host_models", "ptn_host_ops.cu")
SRC_SYN = os.path.join(ROOT, "tests", "host_models", "ptn_host_synth.cu")
CSRC = os.path.join(ROOT, "paper_2409_20027_gb300", "csrc")
EXE = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "host_models")
EXE_OPS = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "host_ops")
EXE_SYN = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "host_synth")
SRC_ARITH = os.path.join(ROOT, "tests", "host_models", "ptn_host_arith.cu")
EXE_ARITH = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "host_arith")


def _harness(src=SRC, exe=EXE):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    if not os.path.exists(exe) or any(os.path.getmtime(d) > os.path.getmtime(exe) for d in deps):
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        tmp = exe + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", CSRC, src, "-o", tmp], check=True, capture_output=True)
        os.replace(tmp, exe)
    return exe


def _cases():
    rng = np.random.default_rng(31)
    out = []
    for prob in [W.pendulum(), W.cartpole(), W.cartpole(T=4096, horizon=2.56), W.quadrotor()]:
        n, m = prob.nx, prob.nu
        for _ in range(4):
            if prob.model == W.QUADROTOR:
                x = rng.normal(scale=0.3, size=n)
                u = W.quadrotor_hover_u() + rng.normal(scale=0.2, size=m)
            else:
                x = rng.normal(scale=1.0, size=n)
                u = rng.normal(scale=2.0, size=m)
            lam = rng.normal(scale=5.0, size=n)
            out.append((prob, x, u, lam))
    return out


def test_model_code_of_the_kernels_matches_the_oracle_models():
    exe = _harness()
    cases = _cases()
    lines = []
    for prob, x, u, lam in cases:
        prm = np.zeros(8)
        prm[:len(prob.prm)] = prob.prm
        vals = [prob.model, prob.integrator, repr(float(prob.dt))] + [repr(float(v)) for v in
                                                                          np.concatenate([prm, x, u, lam])]
        lines.append(" ".join(str(v) for v in vals))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(cases)
    for (prob, x, u, lam), line in zip(cases, outs):
        n, m = prob.nx, prob.nu
        npm = {W.PENDULUM: 4, W.CARTPOLE: 4, W.QUADROTOR: 7}[prob.model]  # model constants used
        v = np.array([float(t) for t in line.split()])
        sizes = [n, n * n, n * m, n * n, n * m, m * m, n * npm, (n + m) * npm, n, n, n * n]
        parts = np.split(v, np.cumsum(sizes)[:-1])
        xn, F, G, Hxx, Hxu, Huu, fp, Hzp, d64, d32, Fcl = parts
        F0, G0 = O.jac(prob, x, u)
        H0 = O.hess(prob, x, u, lam)
        ref = [O.step(prob, x, u), F0.ravel(), G0.ravel(), H0[0].ravel(), H0[1].ravel(), H0[2].ravel(),
               O.param_jac(prob, x, u)[:, :npm].ravel(), O.param_hess(prob, x, u, lam)[:, :npm].ravel()]
        for name, a, b in zip(["x+", "F", "G", "Hxx", "Hxu", "Huu", "df/dprm", "d2(lam.f)/dz dprm"],
                              [xn, F, G, Hxx, Hxu, Huu, fp, Hzp], ref):
            scale = max(1.0, float(np.abs(b).max()))
            assert np.abs(a - b).max() <= 1e-12 * scale, (prob.name, name, a, b)
        # the increment f - x: FP64 to rounding of x+, FP32 to FP32 precision of the
        # increment itself (evaluated at the FP32-rounded point, as the mixed rollouts do)
        inc = O.step(prob, x, u) - x
        assert np.abs(d64 - inc).max() <= 1e-13 * max(1.0, float(np.abs(x).max()))
        xf = x.astype(np.float32).astype(np.float64)
        uf = u.astype(np.float32).astype(np.float64)
        inc32 = O.step(prob, xf, uf) - xf
        assert np.abs(d32 - inc32).max() <= 2e-5 * max(1e-3, float(np.abs(inc32).max())), (prob.name, d32, inc32)
        # closed-loop Jacobian F + G Gam
        Gam = np.array([[0.1 * lam[j] / (i + 1) for j in range(n)] for i in range(m)])
        assert np.abs(Fcl - (F0 + G0 @ Gam).ravel()).max() <= 1e-12 * max(1.0, float(np.abs(F0).max()))


def _val(rng):
    """A well-conditioned value element (A, b, C, eta, J): C, J symmetric PSD."""
    X = rng.normal(size=(4, 4)); Y = rng.normal(size=(4, 4))
    return (np.eye(4) + 0.2 * rng.normal(size=(4, 4)), rng.normal(size=4), 0.3 * X @ X.T,
            rng.normal(size=4), 0.3 * Y @ Y.T)


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 3e-5)], ids=["fp64", "fp32_fp64solve"])
def test_scan_operators_of_the_kernels_match_the_oracle_operators(prec, tol):
    exe = _harness(SRC_OPS, EXE_OPS)
    rng = np.random.default_rng(41 + prec)
    rnd = _f32 if prec else (lambda a: np.asarray(a, dtype=np.float64))
    lines, refs = [], []
    for _ in range(6):
        e1 = tuple(rnd(z) for z in _val(rng))
        e2 = tuple(rnd(z) for z in _val(rng))
        lines.append("V %d " % prec + " ".join(repr(float(v)) for z in e1 + e2 for v in np.ravel(z)))
        refs.append(np.concatenate([np.ravel(z) for z in O.value_combine(e1, e2)]))
        F = rnd(np.eye(4) + 0.1 * rng.normal(size=(4, 4))); G = rnd(rng.normal(size=(4, 1)))
        Pq = rng.normal(size=(4, 4)); P = rnd(Pq @ Pq.T + np.eye(4)); M = rnd(0.1 * rng.normal(size=(4, 1)))
        R = rnd(np.array([[0.5 + rng.random()]])); d = rng.normal(size=1)
        lines.append("I %d " % prec + " ".join(repr(float(v)) for v in
                                              np.concatenate([F.ravel(), G.ravel(), P.ravel(), M.ravel(), R.ravel(),
                                                              d, [1e-3]])))
        refs.append(np.concatenate([np.ravel(z) for z in O.value_init(F, G, P, M, R, d, 1e-3)]))
    for _ in range(4):
        g1, g2 = rng.normal(size=4), rng.normal(size=4)
        A1, A2 = np.eye(4) + 0.2 * rng.normal(size=(4, 4)), np.eye(4) + 0.2 * rng.normal(size=(4, 4))
        lines.append("C 0 " + " ".join(repr(float(v)) for v in np.concatenate([g1, A1.ravel(), g2, A2.ravel()])))
        g, Ft = O.costate_combine(g1, A1, g2, A2)
        refs.append(np.concatenate([np.ravel(g), np.ravel(Ft)]))
        lines.append("S 0 " + " ".join(repr(float(v)) for v in np.concatenate([A1.ravel(), g1, A2.ravel(), g2])))
        F, e = O.state_combine(A1, g1, A2, g2)
        refs.append(np.concatenate([np.ravel(e), np.ravel(F)]))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(refs)
    for line, ref, inp in zip(outs, refs, lines):
        assert "FAIL" not in line, inp[:2]
        got = np.array([float(t) for t in line.split()])
        t = tol if inp[0] in "VI" else 1e-12
        assert np.abs(got - ref).max() <= t * max(1.0, float(np.abs(ref).max())), (inp[:2], got, ref)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 3e-5)], ids=["fp64", "fp32_fp64solve"])
def test_step_fold_of_the_kernels_matches_init_then_combine(prec, tol):
    # the chunk fold's Woodbury form (one step's element combined with a later element)
    # against the oracle's element initialisation followed by its value combination, for
    # random later elements and the two starts of a fold: the identity element and the
    # terminal element (A = 0, C = 0, b = 0, eta = 0, J = P_{N+1})
    exe = _harness(SRC_OPS, EXE_OPS)
    rng = np.random.default_rng(57 + prec)
    rnd = _f32 if prec else (lambda a: np.asarray(a, dtype=np.float64))
    Z = np.zeros((4, 4))
    lines, refs = [], []
    for k in range(12):
        F = rnd(np.eye(4) + 0.1 * rng.normal(size=(4, 4))); G = rnd(rng.normal(size=(4, 1)))
        Pq = rng.normal(size=(4, 4)); P = rnd(Pq @ Pq.T + np.eye(4)); M = rnd(0.1 * rng.normal(size=(4, 1)))
        R = rnd(np.array([[0.5 + rng.random()]])); d = rng.normal(size=1)
        if k % 3 == 0:
            e = (np.eye(4), np.zeros(4), Z, np.zeros(4), Z)
        elif k % 3 == 1:
            Y = rng.normal(size=(4, 4))
            e = (Z, np.zeros(4), Z, np.zeros(4), rnd(Y @ Y.T))
        else:
            e = tuple(rnd(z) for z in _val(rng))
        step = np.concatenate([F.ravel(), G.ravel(), P.ravel(), M.ravel(), R.ravel(), d, [1e-3]])
        lines.append("W %d " % prec + " ".join(repr(float(v)) for v in
                                              np.concatenate([step] + [np.ravel(z) for z in e])))
        refs.append(np.concatenate([np.ravel(z) for z in O.value_combine(O.value_init(F, G, P, M, R, d, 1e-3), e)]))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(refs)
    for line, ref in zip(outs, refs):
        assert "FAIL" not in line
        got = np.array([float(t) for t in line.split()])
        assert np.abs(got - ref).max() <= tol * max(1.0, float(np.abs(ref).max())), (got, ref)


def test_riccati_step_of_the_kernels_matches_the_oracle_recursion():
    # one backward step of the kernels' sweep from the oracle's (S, s)_{t+1} reproduces the
    # oracle's Gam_t, gam_t and (S, s)_t (eq. value-fun-feedback with M^T), on the
    # cart-pole's Newton step at a barrier weight where the LQR has curvature from all terms
    exe = _harness(SRC_OPS, EXE_OPS)
    p = W.cartpole()
    T = 6
    rng = np.random.default_rng(9)
    u = rng.normal(scale=0.5, size=(T, 1))
    x = O.rollout(p, W.cartpole_x0(2), u)
    alpha = 1e-3
    nd = O.newton_direction(p, x, u, alpha, "barrier", mu=1e-2)
    assert nd["status"] == 0
    lines, refs = [], []
    for t in range(T):
        vals = np.concatenate([nd["F"][t].ravel(), nd["G"][t].ravel(), nd["P"][t].ravel(), nd["M"][t].ravel(),
                               nd["R"][t].ravel(), nd["d"][t].ravel(), [alpha], nd["S"][t + 1].ravel(),
                               nd["s"][t + 1]])
        lines.append("R 0 " + " ".join(repr(float(v)) for v in vals))
        refs.append(np.concatenate([nd["Gam"][t].ravel(), nd["gam"][t].ravel(), nd["S"][t].ravel(), nd["s"][t]]))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == T
    for t, (line, ref) in enumerate(zip(outs, refs)):
        assert "FAIL" not in line, t
        got = np.array([float(v) for v in line.split()])
        assert np.abs(got - ref).max() <= 1e-10 * max(1.0, float(np.abs(ref).max())), (t, got, ref)


@pytest.mark.parametrize("n,m", [(32, 8), (6, 2)])
def test_synthetic_map_closed_forms_match_the_oracle(n, m):
    # x+ = A x + B u + c tanh(W x) (the n = 32, m = 8 workload's model): step, F, G and
    # lam . f_xx in closed form (ptn_synth.cuh) against the oracle's hyper-dual evaluation
    exe = _harness(SRC_SYN, EXE_SYN)
    rng = np.random.default_rng(7 + n)
    lines, refs = [], []
    for seed in range(3):
        p = W.synth(seed, nx=n, nu=m)
        x = rng.normal(size=n)
        u = rng.normal(size=m)
        lam = rng.normal(scale=3.0, size=n)
        vals = np.concatenate([p.A.ravel(), p.B.ravel(), p.W.ravel(), x, u, lam])
        lines.append(f"{n} {m} {float(p.prm[0])!r} " + " ".join(repr(float(v)) for v in vals))
        F0, G0 = O.jac(p, x, u)
        Hxx, Hxu, Huu = O.hess(p, x, u, lam)
        assert np.abs(Hxu).max() == 0.0 and np.abs(Huu).max() == 0.0
        refs.append(np.concatenate([O.step(p, x, u), F0.ravel(), G0.ravel(), Hxx.ravel()]))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(refs)
    for line, ref in zip(outs, refs):
        got = np.array([float(t) for t in line.split()])
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, float(np.abs(ref).max()))


def test_pivot_keys_and_the_fp64_inverse():
    # the integer pivot key orders by magnitude (doubles: by the high word, so monotone with
    # ties below 2^-20 relative and among subnormals; floats: strictly), and the Gauss-Jordan
    # inverse of the value
    # combine matches numpy's inverse, with pivoting exercised and a singular matrix refused
    exe = _harness(SRC_OPS, EXE_OPS)
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.normal(size=40) * 10.0 ** rng.integers(-30, 30, size=40),
                         [0.0, -0.0, 1.0, -1.0, 1.0 + 2.0 ** -40, 5e-324, -5e-324, 3e38, -3e38]])
    lines = ["K 0 %r" % float(v) for v in xs]
    mats = [rng.normal(size=(4, 4)) for _ in range(6)]
    mats.append(np.array([[1e-9, 1, 2, 3], [4, 5, 6, 7.5], [8, 9.5, 10, 11], [12, 13, 14.5, 16]]))  # pivoting
    mats.append(np.diag([1e-6, 1.0, 1e3, 5.0]) + 1e-3 * rng.normal(size=(4, 4)))  # ill-scaled
    lines += ["G 0 " + " ".join(repr(float(v)) for v in A.ravel()) for A in mats]
    lines.append("G 0 " + " ".join(["1.0", "2.0", "3.0", "4.0"] * 4))  # singular
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(lines)
    kd = np.array([int(o.split()[0]) for o in outs[:len(xs)]])
    kf = np.array([int(o.split()[1]) for o in outs[:len(xs)]])
    a = np.abs(xs)
    af = np.abs(xs.astype(np.float32).astype(np.float64))
    for i in range(len(xs)):
        for j in range(len(xs)):
            if a[i] < a[j]:
                assert kd[i] <= kd[j], (xs[i], xs[j])
            if a[i] < a[j] * (1.0 - 2.0 ** -19) and a[j] >= np.finfo(np.float64).tiny:
                # strict between normal magnitudes (the high word resolves 2^-20 relative;
                # below the normal range all keys are 0)
                assert kd[i] < kd[j], (xs[i], xs[j])
            if af[i] < af[j]:
                assert kf[i] < kf[j], (xs[i], xs[j])
    for A, o in zip(mats, outs[len(xs):len(xs) + len(mats)]):
        got = np.array([float(t) for t in o.split()]).reshape(4, 4)
        ref = np.linalg.inv(A)
        tol = 1e-15 * np.linalg.cond(A) * 16
        assert np.abs(got - ref).max() <= tol * max(1.0, float(np.abs(ref).max())), (A, got, ref)
    assert outs[-1].strip() == "FAIL" or "FAIL" in outs[-1]


def test_ldlt_factorisation_and_solve():
    # LDL^T with reciprocal pivots (R~ and Q_uu of the value pass): solves SPD systems like
    # numpy's solver, ill-conditioned ones to the conditioning bound, and refuses a matrix
    # that is not positive definite
    exe = _harness(SRC_OPS, EXE_OPS)
    rng = np.random.default_rng(17)
    cases = []
    for k in range(5):
        Xq = rng.normal(size=(4, 4))
        A = Xq @ Xq.T + (10.0 ** -k) * np.eye(4)  # conditioning up to ~1e5
        cases.append((A, rng.normal(size=(4, 3))))
    indef = np.diag([1.0, 2.0, -0.5, 3.0])
    lines = ["L 0 " + " ".join(repr(float(v)) for v in np.concatenate([A.ravel(), Bm.ravel()])) for A, Bm in cases]
    lines.append("L 0 " + " ".join(repr(float(v)) for v in np.concatenate([indef.ravel(), np.ones(12)])))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(lines)
    for (A, Bm), o in zip(cases, outs):
        got = np.array([float(t) for t in o.split()]).reshape(4, 3)
        ref = np.linalg.solve(A, Bm)
        tol = 1e-15 * np.linalg.cond(A) * 32
        assert np.abs(got - ref).max() <= tol * max(1.0, float(np.abs(ref).max()))
    assert "FAIL" in outs[-1]


def test_element_operators_refuse_singular_and_indefinite_inputs():
    # value combine with I + C1 J2 singular (C1 J2 = -I), and element init with R~ < 0:
    # both report failure (the solver then raises alpha) instead of returning garbage
    exe = _harness(SRC_OPS, EXE_OPS)
    eye = np.eye(4)
    e1 = (eye, np.zeros(4), eye, np.zeros(4), eye)      # C1 = I
    e2 = (eye, np.zeros(4), eye, np.zeros(4), -eye)     # J2 = -I
    v = "V 0 " + " ".join(repr(float(x)) for z in e1 + e2 for x in np.ravel(z))
    i = "I 0 " + " ".join(repr(float(x)) for x in np.concatenate(
        [eye.ravel(), np.ones(4), eye.ravel(), np.zeros(4), [-1.0], [0.5], [1e-3]]))
    r = subprocess.run([exe], input=v + "\n" + i + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == 2 and "FAIL" in outs[0] and "FAIL" in outs[1]


def test_mixed_costate_operator_matches_the_oracle_combine():
    # the FP32-increment co-state element (g, I + D) of the mixed mode: composition as the
    # oracle's co-state combine of (g, I + D), to FP32 precision in the increment terms
    exe = _harness(SRC_OPS, EXE_OPS)
    rng = np.random.default_rng(23)
    lines, refs = [], []
    for _ in range(6):
        ga, gb = rng.normal(size=4) * 10, rng.normal(size=4) * 10
        Da = (0.05 * rng.normal(size=(4, 4))).astype(np.float32).astype(np.float64)
        Db = (0.05 * rng.normal(size=(4, 4))).astype(np.float32).astype(np.float64)
        lines.append("D 0 " + " ".join(repr(float(v)) for v in np.concatenate([ga, Da.ravel(), gb, Db.ravel()])))
        g, Ft = O.costate_combine(ga, np.eye(4) + Da, gb, np.eye(4) + Db)
        refs.append((g, Ft - np.eye(4)))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    outs = r.stdout.strip().splitlines()
    assert len(outs) == len(refs)
    for o, (g, D) in zip(outs, refs):
        v = np.array([float(t) for t in o.split()])
        assert np.abs(v[:4] - g).max() <= 1e-6 * max(1.0, float(np.abs(g).max()))
        assert np.abs(v[4:] - D.ravel()).max() <= 1e-6 * max(1e-3, float(np.abs(D).max()))


def test_solve_conversions_match_ieee_on_every_fp32_pattern():
    """The integer FP32 -> FP64 widening of the FP64 solves equals the host's conversion on
    all 2^32 bit patterns (FP32 subnormals become signed zeros; NaNs keep their payload,
    quieted), and the FP64 -> FP32 rounding equals the host's round-to-nearest-even on
    random doubles, exact ties and their neighbours and the overflow threshold."""
    exe = _harness(SRC_ARITH, EXE_ARITH)
    r = subprocess.run([exe, "F"], capture_output=True, text=True, check=True, timeout=600)
    bad, n = (int(t) for t in r.stdout.split())
    assert n == 2 ** 32 and bad == 0, r.stderr
    r = subprocess.run([exe, "D", "4000000", "7"], capture_output=True, text=True, check=True, timeout=600)
    bad, n = (int(t) for t in r.stdout.split())
    assert n > 4000000 and bad == 0, r.stderr
