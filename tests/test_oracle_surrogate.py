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


@pytest.mark.parametrize("c,h", [(0.0, 1.0), (2.3, 1.0), (2.3, 0.25), (23.0, 10.0), (-1.0, 3.7)])
def test_normalised_density_maps_to_physical(c, h):
    """A Gaussian predicted in normalised units (mu', s' = log sigma'^2) over
    x' = (x - c) / h is, in physical units, the density p'(x') / h (change of
    variables): to_physical must give the N(mu, exp(log sigma^2)) with that
    pdf at every x, so a wrong scaling of the log-variance fails."""
    out = np.array([[0.3, -2.1], [-1.2, 0.4]])
    mu, lv = sg.to_physical(out, c, h)
    x = np.linspace(-5.0, 5.0, 41) * h + c
    for q in range(out.shape[0]):
        xp = sg.normalise(np.zeros_like(x), x, c, h)[1]
        want = stats.norm.pdf(xp, out[q, 0], math.exp(0.5 * out[q, 1])) / h
        got = stats.norm.pdf(x, mu[q], math.exp(0.5 * lv[q]))
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-300)
    # normalise is the inverse map of the mean: lambda' = 0 at c, 1 at c + h
    lp, xp = sg.normalise([c, c + h], [c - h, c], c, h)
    np.testing.assert_allclose(lp, [0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(xp, [-1.0, 0.0], atol=1e-15)


def test_minibatch_indices_from_philox_words():
    """Index j of Adam step t comes from Philox4x32-10 block (j, t, 0, 3):
    (word1 * 2^32 + word0) mod total, recomputed here for single blocks with
    the oracle's one-block generator; every index is in range and the draws
    are uniform (chi-square over 16 cells)."""
    from oracle import _clib

    seed, step, batch, total = 0x1234ABCD5678EF01, 17, 4096, 1000003
    idx = sg.minibatch(_clib.philox_bulk, seed, step, batch, total)
    assert idx.shape == (batch,) and idx.min() >= 0 and idx.max() < total
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for j in (0, 1, 977, batch - 1):
        w = _clib.philox(np.array([j, step, 0, 3], dtype=np.uint32), key)
        assert idx[j] == ((int(w[1]) << 32) | int(w[0])) % total
    big = sg.minibatch(_clib.philox_bulk, seed, step + 1, 1 << 16, 16)
    counts = np.bincount(big, minlength=16)
    assert stats.chisquare(counts).pvalue > 1e-4
    assert not np.array_equal(sg.minibatch(_clib.philox_bulk, seed, step + 1, batch, total), idx)


def test_training_recovers_a_linear_gaussian_model():
    """Adam training on per-window Gaussian samples whose mean is linear in
    lambda and whose width is constant (the Gaussian model of x of Sec. II)
    recovers both, in physical units with h != 1: the predicted mean within
    0.4 sigma and sigma within 20 % across the trained range, and the loss on
    the whole store within 0.03 of the model's own minimum
    0.5 [log (sigma/h)^2 + 1]."""
    from oracle import _clib

    rng = np.random.default_rng(7)
    lam = np.linspace(13.0, 33.0, 11)
    a, b, sig = -1.0, 0.9, 0.5
    R, T = 8, 200
    store = np.concatenate([a + b * l + sig * rng.standard_normal(R * T) for l in lam])
    off = np.arange(lam.size) * R * T
    c, h = 23.0, 10.0
    p = sg.init_params(2)
    p, _, _ = sg.train(p, store, off, lam, 3000, 256, 3e-3, 5, c, h, _clib.philox_bulk)
    lt = np.linspace(13.0, 33.0, 21)
    mu, lv = sg.to_physical(sg.forward(p, sg.normalise(lt, lt, c, h)[0])["out"], c, h)
    assert np.max(np.abs(mu - (a + b * lt))) < 0.4 * sig
    sd = np.exp(0.5 * lv)
    assert np.all(np.abs(sd / sig - 1.0) < 0.2), sd
    lam_all = np.repeat(lam, R * T)
    ln, xn = sg.normalise(lam_all, store, c, h)
    loss = sg.nll(sg.forward(p, ln)["out"], xn)
    assert abs(loss - 0.5 * (math.log((sig / h) ** 2) + 1.0)) < 0.03


def test_gate_on_measured_overlaps():
    """Samples mu +- sigma (equal counts) have mean mu and population
    variance sigma^2 exactly, so the measured OVL of two such windows is
    the equal-width closed form 2 Phi(-|d| / (2 sigma)); the gate opens
    exactly when that value is below the threshold."""
    from scipy.stats import norm

    sigma = 0.25
    def win(mu):
        return np.array([[mu - sigma, mu + sigma], [mu + sigma, mu - sigma]])

    for d in (0.1, 0.5, 1.0):
        xw = [win(0.0), win(d), win(2 * d)]
        mu, var = sg.window_moments(xw)
        np.testing.assert_allclose(mu, [0.0, d, 2 * d], atol=1e-15)
        np.testing.assert_allclose(var, sigma ** 2, rtol=1e-14)
        want = 2.0 * norm.cdf(-d / (2.0 * sigma))
        np.testing.assert_allclose(sg.measured_overlaps(xw), [want, want], rtol=1e-12)
        for thr in (want - 1e-6, want + 1e-6):
            assert sg.needs_training(xw, thr) == (want < thr)
