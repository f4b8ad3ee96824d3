"""Pins of the App. C work-distribution oracle (CPU)."""
import itertools
import math

import numpy as np

from oracle import estimators as est
from oracle import histograms as hist
from paper_1105_4840_gb300 import inputs


def test_convolution_equals_brute_force_over_tuples():
    """Omega_s is the distribution of the summed per-step bin shifts over
    every tuple (x_1, ..., x_{s-1}), one sample per window, each tuple weighted
    1 / prod n_i: brute force over all 4 x 3 x 5 tuples."""
    rng = np.random.default_rng(1)
    lam = np.array([0.0, 0.3, 0.7, 1.0])
    k, kT, x_lo, dx, K, dW, M = 40.0, 1.0, -1.0, 0.01, 400, 0.05, 400
    samples = [lam[0] + 0.1 * rng.standard_normal(4), lam[1] + 0.1 * rng.standard_normal(3),
               lam[2] + 0.1 * rng.standard_normal(5), lam[3] + 0.1 * rng.standard_normal(2)]
    for left_edge in (False, True):
        omega, _, _, _ = hist.work_distributions(samples, lam, k, kT, x_lo, dx, K, dW, M, left_edge)
        want = np.zeros(2 * M + 1)
        per = []
        for i in range(3):
            j = np.floor((np.asarray(samples[i]) - x_lo) / dx).astype(int)
            sh = hist.shifts(lam[i], lam[i + 1], k, x_lo, dx, K, dW, left_edge)
            per.append(sh[j])
        for tup in itertools.product(*per):
            want[M + sum(tup)] += 1.0 / (4 * 3 * 5)
        if not left_edge:
            np.testing.assert_allclose(omega[3], want, atol=1e-15)
        else:  # the printed rule also smooths the W = 0 bin after every step
            w2 = want.copy()
            w2[M] = omega[3][M]
            np.testing.assert_allclose(omega[3], w2, atol=1e-15)


def test_fine_bins_converge_to_the_factorised_estimator():
    """With bin centres, dF^JE from Omega approaches the exact factorised
    all-combinations estimate (Eq. (12)) as dx, dW -> 0."""
    lam = inputs.lambda_grid(1.3, 1.9, 7)
    k, kT = 500.0, inputs.kT_of(300.0)
    x = inputs.gaussian_x_samples(lam, k, kT, 4, 250, seed=5).astype(np.float64)
    exact = est.free_energy_profile([x[i] for i in range(lam.size)], lam, k, kT)["dF_JE"]
    errs = []
    for dx, dW in ((2e-3, 0.2), (5e-4, 0.05), (1e-4, 0.01)):
        K = int(round(1.5 / dx))
        M = int(round(150.0 / dW))
        _, dF, _, lost = hist.work_distributions([x[i] for i in range(lam.size)], lam, k, kT, 0.8, dx, K, dW, M)
        assert lost.max() < 1e-12
        errs.append(np.abs(dF - exact).max())
    assert errs[2] < errs[0] and errs[2] < 0.02 * kT


def test_printed_floor_rule_drifts_by_half_a_bin_per_step():
    """The printed rule (left edges, floor) shifts the mean work of Omega_i by
    about -dW/2 per step relative to bin centres (plus the x left-edge
    offset k Delta dx)."""
    lam = inputs.lambda_grid(1.3, 1.9, 7)
    k, kT = 500.0, inputs.kT_of(300.0)
    x = inputs.gaussian_x_samples(lam, k, kT, 4, 250, seed=6).astype(np.float64)
    dx, dW, K, M = 1e-3, 0.1, 1500, 600
    W = (np.arange(2 * M + 1) - M) * dW
    means = []
    for left in (False, True):
        om, _, _, _ = hist.work_distributions([x[i] for i in range(lam.size)], lam, k, kT, 0.8, dx, K, dW, M, left)
        means.append([(o * W).sum() / o.sum() for o in om])
    d = np.diff(np.array(means[1]) - np.array(means[0]))
    step_shift = -0.5 * dW + 0.5 * k * 0.1 * 2 * 0.5 * dx  # floor bias, and left-edge x = centre - dx/2
    assert np.all(np.abs(d - step_shift) < 0.3 * dW)
