"""Pins of the oracle's estimators (CPU only): Eq. (9) algebra, the
all-combinations average by brute force, closed forms for Gaussian, flat and
harmonic wells, the jackknife, and the paper's worked variance example."""
import json
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import estimators as est

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_eq9_equals_hamiltonian_difference():
    """Eq. (9) factorised form equals H(lambda_{i+1}, x) - H(lambda_i, x) of Eq. (B.1)."""
    rng = np.random.default_rng(0)
    x = rng.normal(1.7, 0.2, 1000)
    for lam_i, lam_n, k in ((1.3, 1.4, 500.0), (-0.4, -0.55, 20.0), (2.0, 2.0, 3.0)):
        w = est.work_increment(x, lam_i, lam_n, k)
        h = 0.5 * k * (x - lam_n) ** 2 - 0.5 * k * (x - lam_i) ** 2
        np.testing.assert_allclose(w, h, rtol=1e-12, atol=1e-12)


def test_all_combinations_brute_force():
    """s = 4 windows, 5 samples each: averaging exp(-beta W_mech) over all 125
    tuples equals the factorised estimator."""
    rng = np.random.default_rng(1)
    lam = np.array([0.0, 0.3, 0.7, 0.9])
    samples = [rng.normal(l - 0.05, 0.15, (1, 5)) for l in lam]
    k, kT = 30.0, 1.3
    brute = est.je_all_tuples([s.ravel() for s in samples], lam, k, kT)
    prof = est.free_energy_profile(samples, lam, k, kT)
    assert prof["dF_JE"][-1] == pytest.approx(brute, rel=1e-13, abs=1e-13)
    # and the per-window pieces add up: s=3 prefix equals the brute force on 3 windows
    brute3 = est.je_all_tuples([s.ravel() for s in samples[:3]], lam[:3], k, kT)
    assert prof["dF_JE"][2] == pytest.approx(brute3, rel=1e-13, abs=1e-13)


def _stratified_normal(mu, sd, n):
    """Deterministic 'samples' at the midpoint quantiles of N(mu, sd^2)."""
    u = (np.arange(n) + 0.5) / n
    return mu + sd * math.sqrt(2.0) * special.erfinv(2.0 * u - 1.0)


def test_gaussian_x_reproduces_closed_form_B5():
    """For Gaussian x_i the JE average has the closed form of Eq. (B.5):
    dF = sum k Delta^2/2 (1 - gamma_i^2) + k Delta (lambda_i - <x_i>)."""
    # increments keep beta k Delta sigma <= ~1 so that midpoint-quantile
    # samples resolve the exponential tail to ~1e-5
    lam = np.array([1.3, 1.35, 1.39, 1.45, 1.48])
    k, kT = 500.0, 2.494
    mu = lam - np.array([0.05, 0.02, 0.08, 0.0, 0.03])
    g2 = np.array([1.1, 1.3, 1.2, 0.9, 1.4])
    sd = np.sqrt(g2 * kT / k)
    samples = [_stratified_normal(mu[i], sd[i], 400000)[None, :] for i in range(lam.size)]
    prof = est.free_energy_profile(samples, lam, k, kT)
    d = np.diff(lam)
    want = np.concatenate([[0.0], np.cumsum(k * d * d / 2 * (1 - g2[:-1]) + k * d * (lam[:-1] - mu[:-1]))])
    np.testing.assert_allclose(prof["dF_JE"], want, atol=2e-4 * kT)
    # the Gaussian estimator on the same samples gives the same numbers
    np.testing.assert_allclose(prof["dF_G"], want, atol=2e-4 * kT)


def test_flat_and_harmonic_wells():
    """Equilibrium samples in a flat well: dF = 0.  In a harmonic well
    kappa/2 x^2 the trap-biased free energy changes by
    kappa k / (2 (kappa + k)) (lambda_j^2 - lambda_1^2)."""
    k, kT = 20.0, 1.0
    lam = np.linspace(-1.5, 1.5, 21)
    for kappa in (0.0, 8.0):
        mu = k * lam / (kappa + k)
        sd = math.sqrt(kT / (kappa + k))
        samples = [_stratified_normal(m, sd, 200000)[None, :] for m in mu]
        prof = est.free_energy_profile(samples, lam, k, kT)
        exact = kappa * k / (2 * (kappa + k)) * (lam ** 2 - lam[0] ** 2)
        np.testing.assert_allclose(prof["dF_JE"], exact, atol=1e-4)
        # Eq. (14) is the left Riemann sum of dF/dlambda = k (lambda - <x>)
        riemann = np.concatenate([[0.0], np.cumsum(k * np.diff(lam) * (lam[:-1] - mu[:-1]))])
        np.testing.assert_allclose(prof["dF_fluct"], riemann, atol=1e-6)


def test_gaussian_estimator_is_mean_minus_half_variance():
    """Eq. (13) increment equals <w_i> - beta var(w_i) / 2 computed directly
    from the work samples."""
    rng = np.random.default_rng(5)
    lam = np.array([0.2, 0.5, 0.65])
    k, kT = 40.0, 0.8
    samples = [rng.normal(l + 0.1, 0.2, (3, 700)) for l in lam]
    prof = est.free_energy_profile(samples, lam, k, kT)
    want = 0.0
    for i in range(2):
        w = est.work_increment(samples[i], lam[i], lam[i + 1], k).ravel()
        want += w.mean() - w.var() / (2 * kT)
        assert prof["dF_G"][i + 1] == pytest.approx(want, rel=1e-10, abs=1e-10)
        assert prof["W_mean"][i + 1] == pytest.approx(
            sum(est.work_increment(samples[m], lam[m], lam[m + 1], k).mean() for m in range(i + 1)),
            rel=1e-12)


def test_jackknife_of_linear_estimator_is_standard_error():
    """For Eq. (14) (linear in <x>) with equal replica sizes the
    delete-one-replica jackknife equals the standard error of the replica
    means, times k |Delta|."""
    rng = np.random.default_rng(7)
    lam = np.array([1.0, 1.2])
    k, kT = 50.0, 2.0
    x = rng.normal(1.05, 0.1, (9, 40))
    prof = est.free_energy_profile([x, x], lam, k, kT)
    rm = x.mean(axis=1)
    want = k * 0.2 * rm.std(ddof=1) / math.sqrt(rm.size)
    assert prof["se_fluct"][1] == pytest.approx(want, rel=1e-10)


def test_combined_estimate_and_accumulating_force():
    rng = np.random.default_rng(9)
    lam = np.array([1.0, 1.1, 1.2, 1.3])
    k, kT = 500.0, 2.5
    samples = [rng.normal(l - 0.02, 0.07, (4, 50)) for l in lam]
    prof = est.free_energy_profile(samples, lam, k, kT)
    np.testing.assert_allclose(prof["dF_com"], (prof["dF_JE"] + prof["dF_fluct"]) / 2)
    np.testing.assert_allclose(prof["uncertainty"], (prof["dF_JE"] - prof["dF_fluct"]) / 2)
    assert prof["acc_force"][0] == 0.0
    np.testing.assert_allclose(prof["acc_force"][1:], prof["dF_fluct"][1:] / (lam[1:] - lam[0]))
    np.testing.assert_allclose(prof["gamma2"], k * np.array([s.var() for s in samples]) / kT,
                               rtol=1e-12)


def test_zw_variance_worked_example():
    """App. C worked example: sigma_W ~ 10 kcal/mol, Q ~ 20000, T = 300 K give
    a variance of about 0.7 and a standard deviation of about 0.8."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        g = json.load(fh)["zw_variance_example"]
    kT = g["R_kcal_per_mol_K"] * g["T_K"]
    var = est.zw_variance(g["sigma_w_kcal"], g["Q"], kT)
    assert round(var, 1) == g["variance_kcal2"]
    assert round(math.sqrt(var), 1) == g["sd_kcal"]


def test_je_increment_is_shift_invariant_and_exact():
    rng = np.random.default_rng(2)
    w = rng.normal(3.0, 2.0, 10000)
    kT = 1.7
    direct = -kT * math.log(np.mean(np.exp(-w / kT)))
    assert est.je_increment(w, kT) == pytest.approx(direct, rel=1e-12)
    assert est.je_increment(w + 1000.0, kT) == pytest.approx(direct + 1000.0, rel=1e-12)


def test_partials_merge_equals_direct_profile():
    """Shards' per-replica partials, concatenated along the replica axis and
    combined with the log-sum-exp merge, reproduce every estimator computed
    from the union of the samples (a second, independent route through the
    same definitions: one replica dominating exp(-w/kT) included)."""
    rng = np.random.default_rng(12)
    lam = np.array([0.0, 0.4, 0.7, 1.3, 1.5])
    k, kT = 30.0, 0.8
    samples = [lam[i] - 0.05 + 0.2 * rng.standard_normal((6, 40)) for i in range(lam.size)]
    samples[1][2, 5] = 3.0  # a far-out sample: its replica dominates the exponential sum
    direct = est.free_energy_profile(samples, lam, k, kT)
    shard_a = est.window_partials([x[:4] for x in samples], lam, k, kT)
    shard_b = est.window_partials([x[4:] for x in samples], lam, k, kT)
    merged = est.free_energy_from_partials(np.concatenate([shard_a, shard_b], axis=1), lam, k, kT)
    for key in ("dF_JE", "dF_fluct", "dF_G", "W_mean", "dF_com", "uncertainty", "acc_force", "mean_x",
                "var_x", "gamma2", "se_JE", "se_fluct", "var_ZW"):
        np.testing.assert_allclose(merged[key], direct[key], rtol=1e-10, atol=1e-12, err_msg=key)
    # partials of a single replica: the window's plain sums
    P = est.window_partials([samples[0][:1]], lam[:1], k, kT)
    assert P.shape == (1, 1, 5) and P[0, 0, 2] == 40
    np.testing.assert_allclose(P[0, 0, 3], np.sum(samples[0][0] - lam[0]), rtol=1e-12)
