"""Pins of the surrogate oracle (CPU only): backprop against finite
differences, the overlap coefficient against its closed forms and numerical
integration, Adam against its textbook first step, insertion and seeding."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import surrogate as sg


def test_backprop_matches_finite_differences():
    p = sg.init_params(3)
    for k in p:
        p[k] = p[k] + np.random.default_rng(1).normal(0, 0.1, p[k].shape)
    rng = np.random.default_rng(2)
    lam = rng.uniform(1.3, 3.3, 37)
    x = lam - 0.05 + 0.07 * rng.standard_normal(37)
    cache = sg.forward(p, lam)
    g = sg.backward(p, cache, x)
    h = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in np.random.default_rng(4).choice(flat.size, min(flat.size, 12), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = sg.nll(sg.forward(p, lam)["out"], x)
            flat[idx] = old - h
            lm = sg.nll(sg.forward(p, lam)["out"], x)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].ravel()[idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, idx)


def test_nll_minimum_is_the_sample_gaussian():
    """For a constant prediction the NLL is minimised by the sample mean and
    the log of the plug-in variance."""
    rng = np.random.default_rng(5)
    x = rng.normal(2.0, 0.3, 5000)
    mu, s = x.mean(), math.log(x.var())
    base = sg.nll(np.tile([mu, s], (x.size, 1)), x)
    for dmu, ds in ((0.01, 0), (-0.01, 0), (0, 0.05), (0, -0.05)):
        assert sg.nll(np.tile([mu + dmu, s + ds], (x.size, 1)), x) > base


def test_silu_grad():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(sg.silu_grad(z), (sg.silu(z + h) - sg.silu(z - h)) / (2 * h), rtol=1e-6, atol=1e-9)


def test_adam_first_step_is_signed_lr():
    """With bias correction the first Adam step moves each weight by
    lr * g / (|g| + eps) = lr * sign(g)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    sg.adam_step(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["w"], [0.99, -1.99, 0.49], rtol=0, atol=1e-7)


@pytest.mark.parametrize("m1,s1,m2,s2", [(0, 1, 0, 1), (0, 1, 1, 1), (0, 1, 3, 1), (0, 1, 0.5, 2),
                                         (1.3, 0.07, 1.4, 0.05), (2.0, 0.3, 1.1, 0.1)])
def test_overlap_coefficient(m1, s1, m2, s2):
    want = integrate.quad(lambda x: min(stats.norm.pdf(x, m1, s1), stats.norm.pdf(x, m2, s2)),
                          min(m1, m2) - 12 * max(s1, s2), max(m1, m2) + 12 * max(s1, s2),
                          limit=400, points=[m1, m2])[0]
    assert sg.gaussian_overlap(m1, s1, m2, s2) == pytest.approx(want, abs=1e-7)
    assert sg.gaussian_overlap(m2, s2, m1, s1) == pytest.approx(want, abs=1e-7)
    if s1 == s2:
        assert sg.gaussian_overlap(m1, s1, m2, s2) == pytest.approx(
            2 * stats.norm.cdf(-abs(m1 - m2) / (2 * s1)), abs=1e-12)


def test_insert_and_seed():
    lam = np.array([1.0, 1.2, 1.4, 1.6])
    mu = np.array([1.0, 1.2, 1.5, 1.6])
    lv = np.log(np.array([0.05, 0.05, 0.05, 0.05]) ** 2)
    new = sg.insert_windows(lam, mu, lv, 0.3)
    # gaps: 0.2/0.05 = 4 sd (OVL 0.046), 0.3 -> 6 sd, 0.1 -> 2 sd (OVL 0.317)
    np.testing.assert_allclose(new, [1.1, 1.3])
    order = sg.seed_order([1.5, 1.31, 1.29, 1.1, 1.31], 1.3)
    assert list(order) == [1, 2, 4, 0, 3]
