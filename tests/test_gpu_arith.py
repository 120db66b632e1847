"""The FP64 solves' own arithmetic (ptn_arith_check): the pivot reciprocal that replaces the
division in Gauss-Jordan and LDL^T pivots, and the integer-pipe FP32 <-> FP64 conversions
of the mixed modes' solves, against IEEE-754 arithmetic on the host (numpy)."""
import numpy as np
import pytest
import torch

from paper_2409_20027_gb300 import ptn

pytestmark = pytest.mark.gpu


def _ulp_err(a, b):
    # distance in units in the last place of b
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_pivot_reciprocal_within_one_ulp():
    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, 200000)
    expo = rng.integers(-1000, 1001, 200000)
    p = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 200000)
    extra = np.array([1.0, -1.0, 2.0, 0.5, 3.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, np.ldexp(1.0, 1000),
                      np.ldexp(1.0, -1000), np.ldexp(1.9999999999999998, 1000), 1e-300, 1e300, 7.0, 1.0 / 3.0])
    p = np.concatenate([p, extra, -extra])
    rcp, _, _ = ptn.arith_check(p=torch.tensor(p, device="cuda:0"))
    r = rcp.cpu().numpy()
    err = _ulp_err(r, 1.0 / p)
    assert err.max() <= 1.0, (err.max(), p[err.argmax()])
    # most results are the correctly rounded quotient
    assert np.mean(r == 1.0 / p) > 0.9


def test_pivot_reciprocal_singular_pivots():
    p = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, np.ldexp(1.0, -1001), np.ldexp(1.0, 1002), 5e-324, 1.7e308,
                  np.ldexp(1.0, -1023)])
    rcp, _, _ = ptn.arith_check(p=torch.tensor(p, device="cuda:0"))
    assert (rcp.cpu().numpy() == 0.0).all()


def test_f32_to_f64_exact():
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, 300000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.finfo(np.float32).max, np.finfo(np.float32).tiny, 1.0,
                        -1.0, 3.0e-39, -1.0e-45, np.nan], dtype=np.float32)
    f = np.concatenate([f, special])
    _, f2d, _ = ptn.arith_check(f=torch.tensor(f, device="cuda:0"))
    g = f2d.cpu().numpy()
    ref = f.astype(np.float64)
    nan = np.isnan(f)
    sub = (np.abs(f) < np.finfo(np.float32).tiny) & ~nan
    assert np.isnan(g[nan]).all()
    # FP32 subnormals become signed zeros
    assert (g[sub] == 0.0).all() and (np.signbit(g[sub]) == np.signbit(f[sub])).all()
    ok = ~nan & ~sub
    assert np.array_equal(g[ok], ref[ok])
    assert np.array_equal(np.signbit(g[ok]), np.signbit(ref[ok]))


def test_f64_to_f32_round_to_nearest_even():
    rng = np.random.default_rng(2)
    # doubles across the FP32 range, exact FP32 midpoints (ties) and their neighbours
    mant = rng.uniform(1.0, 2.0, 200000)
    d = np.ldexp(mant, rng.integers(-130, 130, 200000)) * rng.choice([-1.0, 1.0], 200000)
    fl = rng.uniform(-1e3, 1e3, 50000).astype(np.float32)
    half = np.spacing(np.abs(fl)).astype(np.float64) / 2.0
    ties = fl.astype(np.float64) + half
    fmax = float(np.finfo(np.float32).max)
    # fmax + 2^103 is the tie between FLT_MAX and 2^128: it rounds to inf
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e39, -1e39, fmax, fmax + 2.0 ** 103,
                        fmax * (1 + 2 ** -30), 1e-40, -1e-42, 2.0 ** -126, 2.0 ** -126 * (1 - 2 ** -30), 1e300, 1e-300])
    d = np.concatenate([d, ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf), special])
    _, _, d2f = ptn.arith_check(d=torch.tensor(d, device="cuda:0"))
    g = d2f.cpu().numpy()
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)
    nan = np.isnan(d)
    sub = (np.abs(d) < 2.0 ** -126) & ~nan
    assert np.isnan(g[nan]).all()
    assert (g[sub] == 0.0).all() and (np.signbit(g[sub]) == np.signbit(d[sub])).all()
    ok = ~nan & ~sub
    assert np.array_equal(g[ok], ref[ok]), d[ok][g[ok] != ref[ok]][:5]
    assert np.array_equal(np.signbit(g[ok]), np.signbit(ref[ok]))
