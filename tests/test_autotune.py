"""Launch-shape autotuner: the table lookup is host logic (CPU); the sweep times real
solves (GPU) and the tuned solve must still match the oracle."""
import numpy as np
import pytest

from paper_2409_20027_gb300 import autotune as A


def test_bucket_bounds():
    assert A.bucket_of(1) == 64 and A.bucket_of(64) == 64 and A.bucket_of(65) == 256
    assert A.bucket_of(16384) == 16384 and A.bucket_of(10 ** 6) == A.BUCKETS[-1]
    with pytest.raises(ValueError):
        A.bucket_of(0)


def test_lookup_save_load_and_apply(tmp_path):
    table = {A.key(1, 1): {"1024": {"options": {"block_threads": 64}, "ms": 1.0, "T": 1000}}}
    assert A.tuned_options(table, 1, 1, 700) == {"block_threads": 64}
    assert A.tuned_options(table, 1, 1, 2000) == {}   # no entry for the 4096 bucket
    assert A.tuned_options(table, 0, 1, 700) == {}    # other model
    p = str(tmp_path / "t.json")
    A.save(table, p)
    assert A.load(p) == table

    class FakeSolver:
        class prob:
            model = 1

        class options:
            precision = 1

        def __init__(self):
            self.set = {}

        def set_options(self, **kw):
            self.set.update(kw)

    s = FakeSolver()
    assert A.apply(s, table, 1024) == {"block_threads": 64} and s.set == {"block_threads": 64}


@pytest.mark.gpu
def test_sweep_then_tuned_solve_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle as O
    from paper_2409_20027_gb300 import ptn, workloads as W
    p = W.pendulum()
    T = 40
    x0 = W.pendulum_x0(3)
    x0d = torch.tensor(x0, dtype=torch.float64, device="cuda:0")
    cands = [{"block_threads": 32, "grid_steps_per_thread": 2, "cluster_max_blocks": 16},
             {"block_threads": 64, "grid_steps_per_thread": 2, "cluster_max_blocks": 16}]
    table = A.sweep(p, x0d, [T], ptn.PTN_FP64, candidates=cands, reps=1)
    ent = table[A.key(p.model, ptn.PTN_FP64)][str(A.bucket_of(T))]
    assert ent["options"] in cands and ent["ms"] > 0
    s = ptn.Solver(p, max_T=T, precision=ptn.PTN_FP64)
    assert A.apply(s, table, T) == ent["options"]
    x, u, lam, info = s.solve_ip(x0d, T)
    ref = O.solve_ip(p, x0, T)
    assert info["status"] == 0
    assert np.abs(x.cpu().numpy() - ref["x"]).max() <= 1e-6 * max(1.0, np.abs(ref["x"]).max())
