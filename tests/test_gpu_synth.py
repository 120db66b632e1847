"""GPU parity of the synthetic scaling workload x+ = A x + B u + 0.1 tanh(W x) (n = 32,
m = 8, matrices from seed 0) on the wide tier, against the FP64 CPU oracle.

- T = 256 in the three co-state forms (0: the co-state scan of Alg. 1; 1: the multiplier
  form; 2: the multiplier form restarted from the co-states at every barrier level), one
  CTA of two warps;
- T = 1024 in the multiplier form, where at this seed the co-state recursion fails (the
  products of A + 0.1 W grow like 1.0167^T): one CTA, and the cooperative grid tier
  (every warp of the grid on the one instance);
- a batch of two instances of different horizons and initial states (T = 256 from
  synth_x0(0), T = 200 from synth_x0(4)).

FP32 LQR data with FP64 solves, compared at 1e-4 relative with both sides solved to
max|d| <= 1e-7.  The oracle's solves at n = 32 take tens of seconds, so the module starts
all of them at once in a pool of worker processes (spawn) and the tests wait for theirs.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2409_20027_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
TOL = 1e-7
REFS = [("s256", 256, 0, 0), ("s256", 256, 0, 1), ("s256", 256, 0, 2), ("s1024", 1024, 0, 1),
        ("b", 200, 4, 1)]


def _ref(job):
    """Oracle solve of the synthetic workload (runs in a worker process)."""
    import oracle as O
    from paper_2409_20027_gb300 import workloads as W
    _, T, k, mode = job
    return O.solve_ip(W.synth(0), W.synth_x0(k), T, opts=O.Options(costate_mode=mode, tol_final=TOL))


@pytest.fixture(scope="module")
def refs():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import oracle as O
    O.build()
    pool = mp.get_context("spawn").Pool(processes=min(len(REFS), os.cpu_count() or 1))
    pending = {job: pool.apply_async(_ref, (job,)) for job in REFS}
    pool.close()
    yield lambda job: pending[job].get(timeout=1800)
    pool.terminate()


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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))


def check(info, ref, x, u, lam, tol):
    assert info["status"] == 0, info
    assert ref["info"]["status"] == 0, ref["info"]
    e = dict(x=rel(x.cpu().numpy(), ref["x"]), u=rel(u.cpu().numpy(), ref["u"]),
             lam=rel(lam.cpu().numpy(), ref["lam"]),
             J=abs(info["J"] - ref["info"]["J"]) / max(1.0, abs(ref["info"]["J"])))
    assert max(e.values()) <= tol, e
    assert info["r_stat"] <= 1e-6 and info["r_dyn"] <= 1e-6 and info["r_feas"] == 0.0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_synth_T256_cta_matches_oracle(ptn, refs, mode):
    p, T = W.synth(0), 256
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=mode, tol_final=TOL, grid_min_T=0)
    x, u, lam, info = s.solve_ip(dev(W.synth_x0(0)), T)
    check(info, refs(("s256", T, 0, mode)), x, u, lam, FP32_TOL)


@pytest.mark.parametrize("tier", ["cta", "grid"])
def test_synth_T1024_multiplier_form_matches_oracle(ptn, refs, tier):
    p, T = W.synth(0), 1024
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1, tol_final=TOL,
                   grid_min_T=0 if tier == "cta" else 512)
    x, u, lam, info = s.solve_ip(dev(W.synth_x0(0)), T)
    check(info, refs(("s1024", T, 0, 1)), x, u, lam, FP32_TOL)


@pytest.mark.parametrize("grid_min_T", [0, 512], ids=["cta_per_instance", "cta_ranges"])
def test_synth_batch_matches_oracle(ptn, refs, grid_min_T):
    # one CTA per instance, or the cooperative launch with a CTA range per instance
    Tb = np.array([256, 200], dtype=np.int32)
    ks = [0, 4]
    s = ptn.Solver(W.synth(0), max_T=256, max_batch=2, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1,
                   tol_final=TOL, grid_min_T=grid_min_T)
    X, U, Lm, infos = s.solve_batch(dev(np.stack([W.synth_x0(k) for k in ks])), Tb)
    xo = uo = 0
    for b, (T, k) in enumerate(zip(Tb.tolist(), ks)):
        job = ("s256", T, k, 1) if T == 256 else ("b", T, k, 1)
        check(infos[b], refs(job), X[xo:xo + T + 1], U[uo:uo + T], Lm[xo:xo + T + 1], FP32_TOL)
        xo += T + 1
        uo += T


def test_synth_refused_where_not_built(ptn):
    # the static entry point (the matrices live in a handle's device memory) and the adjoint
    p = W.synth(0)
    with pytest.raises(ptn.PtnError, match="synthetic model"):
        ptn.solve_ip_static(p, dev(W.synth_x0(0)), 8, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1)
    s = ptn.Solver(p, max_T=8, precision=ptn.PTN_FP32_FP64SOLVE, costate_mode=1)
    x, u, _, info = s.solve_ip(dev(W.synth_x0(0)), 8)
    with pytest.raises(ptn.PtnError, match="synthetic model"):
        s.adjoint([8], dev(W.synth_x0(0)).reshape(1, -1), x, u, info["mu"])
