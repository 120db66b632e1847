"""The workload generators reproduce the constants the paper prints (Sec. IV)."""
import json
import os

import numpy as np

from paper_2409_20027_gb300 import workloads as W

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_pendulum_constants_match_paper():
    c = G["pendulum_constants"]
    p = W.pendulum(b=c["b"])
    assert np.allclose(p.prm[:4], [c["g"], c["l"], c["m"], c["b"]])


def test_cartpole_constants_match_paper():
    c = G["cartpole_constants"]
    p = W.cartpole().replace(prm=np.array([c["m_c"], c["m_p"], c["l"], c["g"]]))
    assert np.allclose(p.prm[:4], [10.0, 1.0, 0.5, 9.81])


def test_runtime_table_shape():
    r = G["runtime_seconds_A100_JAX"]
    for k, v in r.items():
        if k not in ("cite", "N"):
            assert len(v) == len(r["N"])
            assert all(a < b for a, b in zip(v[:1], v[-1:]))
