"""Pins for the oracle's analytic field descriptors beyond the Fourier rows.

The diffusion order s(x) and log kappa(x) of the paper's experiments are
smooth closed-form fields (Sec. 2 assumes s and kappa analytic; Sec. 7 uses
bumps and sigmoid-shaped orders).  The oracle's field evaluation
(field_analytic in oracle/vfd_oracle.c) sums Fourier rows, Gaussian bumps and
tensor bumps and may squash the sum into (lo, hi).  The Fourier rows are
pinned in test_oracle_quadrature.py; these tests pin the other branches by
properties that fix them without restating their formulas:

* Gaussian bump amp exp(-c |x - x0|^2): value amp at the centre; isotropic;
  log(value / amp) is linear in |x - x0|^2 with slope -c (the semigroup law
  g(r1) g(r2) = amp g(sqrt(r1^2 + r2^2))); 1D, 2D and 3D.
* tensor bump: zero outside the box of side ell; at the centre amp e^-d; a
  product of one-dimensional profiles (the 2x2 minors of the value table on
  a grid vanish); even in each coordinate; along one axis the factor at
  r = 1/2 is e^(-4/3), i.e. e^(-1/3) times its centre value e^-1.
* squash lo + (hi - lo) sigmoid(v): the logit of the squashed value recovers
  the unsquashed sum v computed by the oracle itself from the same rows;
  v = 0 gives the midpoint; reflection v -> -v gives lo + hi - value; every
  value lies strictly in (lo, hi).
A planted mistake in any branch (a sign, a missing factor 2, squaring the
wrong quantity, a dropped centre offset) breaks one of these.
"""
import math

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(123)


def _val(d, f, x):
    return oracle.field(d, f, np.asarray(x, dtype=np.float64))


@pytest.mark.parametrize("d", [1, 2, 3])
def test_gauss_bump_centre_isotropy_and_semigroup(d):
    x0 = np.array([0.3, -0.2, 0.1])[:d]
    amp, c = 0.7, 3.5
    f = synth.gauss_bump_field(0.0, x0, amp, c)
    assert abs(_val(d, f, x0) - amp) <= 1e-15
    # isotropy: equal distance in random directions gives equal values
    r = 0.37
    vals = []
    for _ in range(6):
        u = RNG.standard_normal(d)
        u /= np.linalg.norm(u)
        vals.append(_val(d, f, x0 + r * u))
    assert np.ptp(vals) <= 1e-15
    # semigroup: g(r1) g(r2) = amp g(sqrt(r1^2 + r2^2)) along any direction
    u = RNG.standard_normal(d)
    u /= np.linalg.norm(u)
    for r1, r2 in [(0.1, 0.2), (0.25, 0.4), (0.6, 0.05)]:
        g1 = _val(d, f, x0 + r1 * u)
        g2 = _val(d, f, x0 + r2 * u)
        g12 = _val(d, f, x0 + math.hypot(r1, r2) * u)
        assert abs(g1 * g2 - amp * g12) <= 1e-14
    # the slope of log(g/amp) against r^2 is -c
    r1, r2 = 0.2, 0.5
    slope = (math.log(_val(d, f, x0 + r2 * u) / amp) - math.log(_val(d, f, x0 + r1 * u) / amp)) / (r2 ** 2 - r1 ** 2)
    assert abs(slope + c) <= 1e-12


def test_gauss_bump_offset_adds():
    f0 = synth.gauss_bump_field(0.0, [0.1, 0.2], 0.5, 2.0)
    f1 = synth.gauss_bump_field(0.25, [0.1, 0.2], 0.5, 2.0)
    for _ in range(5):
        x = RNG.uniform(-1, 1, 2)
        assert abs(_val(2, f1, x) - _val(2, f0, x) - 0.25) <= 1e-15


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tensor_bump_support_centre_and_separability(d):
    xc = np.array([0.1, -0.3, 0.2])[:d]
    amp, ell = 1.3, 0.8
    f = synth.tensor_bump_field(0.0, xc, amp, ell)
    # centre: every factor at r = 0 is e^-1
    assert abs(_val(d, f, xc) - amp * math.exp(-d)) <= 1e-15
    # outside the box of side ell (|x_i - xc_i| >= ell/2 in some coordinate): zero
    for _ in range(10):
        x = xc + RNG.uniform(-0.3, 0.3, d) * ell
        i = RNG.integers(d)
        x[i] = xc[i] + (0.5 + RNG.uniform(0.0, 0.5)) * ell * (1 if RNG.random() < 0.5 else -1)
        assert _val(d, f, x) == 0.0
    # even in each coordinate
    for _ in range(5):
        y = RNG.uniform(-0.45, 0.45, d) * ell
        for i in range(d):
            z = y.copy()
            z[i] = -z[i]
            assert abs(_val(d, f, xc + y) - _val(d, f, xc + z)) <= 1e-15
    # 1D profile along an axis: at r = 2 (x - xc)/ell = 1/2 the factor is e^(-4/3)
    e = np.zeros(d)
    e[0] = 0.25 * ell
    assert abs(_val(d, f, xc + e) / _val(d, f, xc) - math.exp(-4.0 / 3.0 + 1.0)) <= 1e-14
    if d >= 2:
        # rank one in (x_0, x_1): the 2x2 minors of the table g(a_i, b_j) vanish
        a = RNG.uniform(-0.45, 0.45, 4) * ell
        b = RNG.uniform(-0.45, 0.45, 4) * ell
        G = np.empty((4, 4))
        for i in range(4):
            for j in range(4):
                x = xc.copy()
                x[0] += a[i]
                x[1] += b[j]
                G[i, j] = _val(d, f, x)
        for i in range(3):
            for j in range(3):
                assert abs(G[i, j] * G[i + 1, j + 1] - G[i, j + 1] * G[i + 1, j]) <= 1e-15


def _squashed(base, lo, hi):
    return synth.sigmoid_field(base, lo, hi)


@pytest.mark.parametrize("base", [
    synth.random_fourier_field(3001, 1.0),
    synth.gauss_bump_field(-0.4, [0.2, 0.1], 1.5, 2.0),
    synth.tensor_bump_field(0.3, [0.0, 0.1], -2.0, 1.2),
])
def test_squash_is_the_logit_inverse_of_the_sum(base):
    lo, hi = 0.1, 0.9
    f = _squashed(base, lo, hi)
    for _ in range(20):
        x = RNG.uniform(-1.0, 1.0, 2)
        v = _val(2, base, x)                # the unsquashed sum (pinned separately)
        y = _val(2, f, x)
        assert lo < y < hi
        assert abs(math.log((y - lo) / (hi - y)) - v) <= 1e-12 * max(1.0, abs(v))


def test_squash_midpoint_and_reflection():
    lo, hi = 0.1, 0.9
    mid = _squashed(synth.const_field(0.0), lo, hi)
    assert abs(_val(2, mid, [0.3, 0.4]) - 0.5 * (lo + hi)) <= 1e-15
    for v in (0.3, 1.7, -2.2):
        fp = _squashed(synth.const_field(v), lo, hi)
        fm = _squashed(synth.const_field(-v), lo, hi)
        x = [0.1, -0.2]
        assert abs(_val(2, fp, x) + _val(2, fm, x) - (lo + hi)) <= 1e-15
        assert (_val(2, fp, x) - 0.5 * (lo + hi)) * v > 0.0   # increasing in v


def test_config3_and_config5_fields_in_range():
    # the squashed order field of the many-mesh workload and the Gaussian-bump
    # order field of the 3D ball stay inside the admissible range of s
    W = synth.batch_workload(n_mesh=3, n_min=300, ratio=2.0)
    for m, s, _k, _n in W:
        v = np.array([_val(2, s, x) for x in m.coords[:200]])
        assert v.min() > 0.1 - 1e-15 and v.max() < 0.9 + 1e-15
    s5 = synth.gauss_bump_field(0.2, [0.1, -0.2, 0.3], 0.6, 4.0)
    pts = RNG.uniform(-1.1, 1.1, (200, 3))
    v = np.array([_val(3, s5, x) for x in pts])
    assert v.min() >= 0.2 and v.max() <= 0.8 + 1e-15
