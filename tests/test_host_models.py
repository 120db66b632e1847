"""The kernels' model code on the host: ptn_models.cuh is written __host__ __device__, so a
host build of the same templates (tests/host_models/ptn_host_models.cu, compiled with
nvcc, run on the CPU) gives the GPU path's step map, its forward-mode Jacobians and its
lam-contracted Hessians.  They must agree with the oracle's models, which are separate
code (hyper-dual numbers, pinned by finite differences in test_oracle_models), for every
model and integrator the kernels use -- without a GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2409_20027_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_models", "ptn_host_models.cu")
CSRC = os.path.join(ROOT, "paper_2409_20027_gb300", "csrc")
EXE = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "host_models")


def _harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    deps = [SRC] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    if not os.path.exists(EXE) or any(os.path.getmtime(d) > os.path.getmtime(EXE) for d in deps):
        os.makedirs(os.path.dirname(EXE), exist_ok=True)
        tmp = EXE + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", CSRC, SRC, "-o", tmp], check=True, capture_output=True)
        os.replace(tmp, EXE)
    return EXE


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
        v = np.array([float(t) for t in line.split()])
        sizes = [n, n * n, n * m, n * n, n * m, m * m]
        parts = np.split(v, np.cumsum(sizes)[:-1])
        xn, F, G, Hxx, Hxu, Huu = parts
        F0, G0 = O.jac(prob, x, u)
        H0 = O.hess(prob, x, u, lam)
        ref = [O.step(prob, x, u), F0.ravel(), G0.ravel(), H0[0].ravel(), H0[1].ravel(), H0[2].ravel()]
        for name, a, b in zip(["x+", "F", "G", "Hxx", "Hxu", "Huu"], [xn, F, G, Hxx, Hxu, Huu], ref):
            scale = max(1.0, float(np.abs(b).max()))
            assert np.abs(a - b).max() <= 1e-12 * scale, (prob.name, name, a, b)
