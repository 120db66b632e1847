"""The paper-protocol workload generators carry the constants the paper prints (Sec. IV).

Each test reads a generator's actual fields (model constants, integrator, bounds,
schedules) and compares them with the values in tests/golden/paper_values.json, which are
copied from the paper's text with their sections cited there.  A change to a generator
that drifts from the paper fails here.
"""
import json
import os

import numpy as np

from paper_2409_20027_gb300 import workloads as W

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_pendulum_paper_model_constants():
    # Sec. IV-A: g, l, m, b of the torque-limited pendulum, Euler integration
    c = G["pendulum_constants"]
    p = W.pendulum_paper()
    assert p.model == W.PENDULUM and p.integrator == W.EULER
    assert p.prm[:4].tolist() == [c["g"], c["l"], c["m"], c["b"]]


def test_cartpole_paper_model_constants():
    # Sec. IV-B: prm is ordered [m_c, m_p, l, g]; Euler integration
    c = G["cartpole_constants"]
    p = W.cartpole_paper()
    assert p.model == W.CARTPOLE and p.integrator == W.EULER
    assert p.prm[:4].tolist() == [c["m_c"], c["m_p"], c["l"], c["g"]]


def test_paper_barrier_schedule():
    # Sec. IV-A/B: mu starts at 0.1 and is multiplied by 0.2 until mu <= 1e-4; the last
    # level is the first power that reaches the threshold
    for sysname in ("pendulum_constants", "cartpole_constants"):
        c = G[sysname]
        assert W.PAPER_IP["mu0"] == c["ip_mu0"] and W.PAPER_IP["zeta"] == c["ip_zeta"]
        assert W.PAPER_IP["mu_stop"] == c["ip_mu_stop"]
    mus = [W.PAPER_IP["mu0"]]
    while mus[-1] > W.PAPER_IP["mu_stop"]:
        mus.append(mus[-1] * W.PAPER_IP["zeta"])
    assert np.isclose(W.PAPER_IP["mu_final"], mus[-1], rtol=1e-12, atol=0.0)
    assert mus[-2] > G["pendulum_constants"]["ip_mu_stop"] >= mus[-1]


def test_paper_admm_settings():
    # Sec. IV-A/B: rho 1 (pendulum), 0.5 (cart-pole); both residuals to 1e-2
    assert W.PAPER_ADMM["pendulum_rho"] == G["pendulum_constants"]["admm_rho"]
    assert W.PAPER_ADMM["cartpole_rho"] == G["cartpole_constants"]["admm_rho"]
    assert W.PAPER_ADMM["tol"] == G["pendulum_constants"]["admm_tol"] == G["cartpole_constants"]["admm_tol"]


def test_paper_mpc_experiment():
    # Sec. IV-C: 4 s at 100 Hz with N = 60, |tau| < 5 Nm and |F| < 60 N
    c = G["mpc_simulation"]
    m = W.PAPER_MPC
    assert (m["duration_s"], m["rate_hz"], m["horizon"]) == (c["duration_s"], c["rate_hz"], c["horizon"])
    pp, cp = W.pendulum_paper(), W.cartpole_paper()
    assert pp.dt == cp.dt == 1.0 / c["rate_hz"]
    assert pp.uhi.tolist() == [c["torque_limit"]] and pp.ulo.tolist() == [-c["torque_limit"]]
    assert cp.uhi.tolist() == [c["force_limit"]] and cp.ulo.tolist() == [-c["force_limit"]]
    # no state bounds in the paper's experiments
    assert np.isinf(cp.xlo).all() and np.isinf(cp.xhi).all()
