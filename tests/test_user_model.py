"""Models supplied from outside the library (ptn_user_model.cuh): a user unit is compiled
and linked into a library of its own, registers its launchers at load, and is then
solved like a built-in model.  One unit declares the pendulum of Sec. IV-A again as model
64, so the GPU solve must reproduce the built-in pendulum's solve bit for bit and the
oracle's pendulum within the FP64 tolerance; the other (model 65) adds user-written stage
and terminal costs and an inequality row, compared with the oracle given the same terms
as callbacks."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
UNIT = os.path.join(ROOT, "tests", "user_models", "ptn_user_pendulum.cu")
UNIT_COST = os.path.join(ROOT, "tests", "user_models", "ptn_user_cost.cu")
OUT = os.path.join(ROOT, "paper_2409_20027_gb300", "_build", "user_models_test")


def _user_lib():
    from paper_2409_20027_gb300 import build
    return build.build(extra=[UNIT, UNIT_COST], out=OUT)


def test_user_model_is_registered_when_the_library_loads():
    lib = ctypes.CDLL(_user_lib())
    nx, nu = ctypes.c_int(), ctypes.c_int()
    assert lib.ptn_model_dims(64, ctypes.byref(nx), ctypes.byref(nu)) == 0
    assert (nx.value, nu.value) == (2, 1)
    # built-in models are still there; unknown ids are refused
    assert lib.ptn_model_dims(1, ctypes.byref(nx), ctypes.byref(nu)) == 0 and (nx.value, nu.value) == (4, 1)
    assert lib.ptn_model_dims(65, ctypes.byref(nx), ctypes.byref(nu)) == 0 and (nx.value, nu.value) == (2, 1)
    assert lib.ptn_model_dims(66, ctypes.byref(nx), ctypes.byref(nu)) != 0


def test_default_library_does_not_know_the_user_model():
    from paper_2409_20027_gb300 import build, ptn
    build.build()  # up to date before the first load in this process
    assert ptn.model_dims(64) is None
    assert ptn.model_dims(0) == (2, 1) and ptn.model_dims(2) == (12, 4)


CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2409_20027_gb300 import ptn, workloads as W
T = 64
p = W.pendulum()
x0 = torch.tensor(W.pendulum_x0(0), dtype=torch.float64, device="cuda:0")
out = {}
for name, prob in [("builtin", p), ("user", p.replace(model=64))]:
    s = ptn.Solver(prob, max_T=T, precision=ptn.PTN_FP64, block_threads=64)
    x, u, lam, info = s.solve_ip(x0, T)
    out[name] = {"x": x.cpu().numpy().tolist(), "u": u.cpu().numpy().tolist(),
                 "lam": lam.cpu().numpy().tolist(), "status": info["status"],
                 "iters": info["newton_iters"], "J": info["J"]}
    s.close()
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_user_model_solves_like_the_builtin_model():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    lib = _user_lib()
    env = dict(os.environ, PTN_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    a, b = res["builtin"], res["user"]
    assert a["status"] == 0 and b["status"] == 0
    for k in ["x", "u", "lam"]:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    assert a["iters"] == b["iters"]
    ref = O.solve_ip(W.pendulum(), W.pendulum_x0(0), 64)
    rel = np.abs(np.asarray(b["u"]) - ref["u"]).max() / max(1.0, np.abs(ref["u"]).max())
    assert rel <= 1e-6 and abs(b["J"] - ref["info"]["J"]) <= 1e-6 * max(1.0, abs(ref["info"]["J"]))


CHILD_COST = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2409_20027_gb300 import ptn, workloads as W
T = 64
p = W.pendulum().replace(model=65)
x0 = torch.tensor(W.pendulum_x0(0), dtype=torch.float64, device="cuda:0")
out = {}
for name, prec, tol in [("fp64", ptn.PTN_FP64, 1e-6), ("fp32", ptn.PTN_FP32_FP64SOLVE, 1e-7)]:
    s = ptn.Solver(p, max_T=T, precision=prec, block_threads=64, tol_final=tol)
    x, u, lam, info = s.solve_ip(x0, T)
    out[name] = {"x": x.cpu().numpy().tolist(), "u": u.cpu().numpy().tolist(),
                 "lam": lam.cpu().numpy().tolist(), "status": info["status"], "J": info["J"],
                 "r_feas": info["r_feas"], "r_stat": info["r_stat"]}
    if name == "fp64":
        try:
            s.solve_admm(x0, T)
            out["admm"] = "ran"
        except ptn.PtnError as e:
            out["admm"] = str(e)
    s.close()
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_user_costs_and_rows_match_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    from test_oracle_user_terms import pendulum_user_problem
    lib = _user_lib()
    env = dict(os.environ, PTN_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD_COST, ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert "interior point only" in res["admm"]
    x0 = W.pendulum_x0(0)
    for name, tol, otol in [("fp64", 1e-6, 1e-6), ("fp32", 1e-4, 1e-7)]:
        g = res[name]
        assert g["status"] == 0 and g["r_feas"] == 0.0 and g["r_stat"] <= 1e-6, (name, g["status"])
        ref = O.solve_ip(pendulum_user_problem(), x0, 64, opts=O.Options(tol_final=otol))
        assert ref["info"]["status"] == 0
        for k in ["x", "u"] + (["lam"] if name == "fp64" else []):
            a, b = np.asarray(g[k]), ref[k]
            assert np.abs(a - b).max() <= tol * max(1.0, np.abs(b).max()), (name, k)
        assert abs(g["J"] - ref["info"]["J"]) <= tol * max(1.0, abs(ref["info"]["J"])), name
