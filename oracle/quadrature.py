"""Exact trap-biased free energies by quadrature (test infrastructure).

F(lambda, k) = -kT ln Z(lambda, k) with Z(lambda, k) the configurational
partition function of H(lambda, x) = H_o + k/2 (x - lambda)^2 (Sec. II, Eq. (3)
and the definition under Eq. (5)); the JE estimate of Eq. (12) converges to
F(lambda_s, k) - F(lambda_1, k), the free energy of the trap-biased system.
"""
from __future__ import annotations

import math

import numpy as np


def _trapz(y, x):
    return float(np.sum(0.5 * (y[1:] + y[:-1]) * np.diff(x)))


def od1d_free_energy(lam: float, k: float, a: float = 2.0, kT: float = 1.0,
                     half_width: float = 6.0, n: int = 60001) -> float:
    """-kT ln int exp(-(a (x^2 - 1)^2 + k/2 (x - lambda)^2)/kT) dx."""
    x = np.linspace(-half_width, half_width, n)
    e = (a * (x * x - 1.0) ** 2 + 0.5 * k * (x - lam) ** 2) / kT
    e0 = e.min()
    return e0 * kT - kT * math.log(_trapz(np.exp(-(e - e0)), x))


def od1d_moments(lam: float, k: float, a: float = 2.0, kT: float = 1.0,
                 half_width: float = 6.0, n: int = 60001):
    """Mean and variance of x under exp(-H(lambda, x)/kT)."""
    x = np.linspace(-half_width, half_width, n)
    e = (a * (x * x - 1.0) ** 2 + 0.5 * k * (x - lam) ** 2) / kT
    p = np.exp(-(e - e.min()))
    z = _trapz(p, x)
    m = _trapz(p * x, x) / z
    v = _trapz(p * (x - m) ** 2, x) / z
    return m, v


def od1d_unbiased_free_energy(a: float = 2.0, kT: float = 1.0, half_width: float = 6.0,
                              n: int = 60001) -> float:
    """F_0 = -kT ln int exp(-a (x^2 - 1)^2 / kT) dx (no trap)."""
    x = np.linspace(-half_width, half_width, n)
    e = a * (x * x - 1.0) ** 2 / kT
    return -kT * math.log(_trapz(np.exp(-e), x))


def gaussian_chain_free_energy(lam: float, k: float, s2: float, kT: float,
                               n: int = 200001) -> float:
    """Trap on x = |R| of an isotropic Gaussian end-to-end vector R with
    per-axis variance s2: -kT ln int_0^inf 4 pi x^2 (2 pi s2)^{-3/2}
    exp(-x^2/(2 s2)) exp(-k (x - lambda)^2 / (2 kT)) dx (relative to the free
    chain; additive constants cancel in differences)."""
    hi = max(lam, 0.0) + 14.0 * math.sqrt(s2)  # the chain density is < e^-90 beyond
    x = np.linspace(0.0, hi, n)
    log_p = (2.0 * np.log(np.maximum(x, 1e-300)) + math.log(4.0 * math.pi)
             - 1.5 * math.log(2.0 * math.pi * s2) - x * x / (2.0 * s2)
             - 0.5 * k * (x - lam) ** 2 / kT)
    m = log_p.max()
    return -kT * (m + math.log(_trapz(np.exp(log_p - m), x)))


def gaussian_chain_mean_x(lam: float, k: float, s2: float, kT: float, n: int = 200001) -> float:
    hi = max(lam, 0.0) + 14.0 * math.sqrt(s2)  # the chain density is < e^-90 beyond
    x = np.linspace(0.0, hi, n)
    log_p = 2.0 * np.log(np.maximum(x, 1e-300)) - x * x / (2.0 * s2) - 0.5 * k * (x - lam) ** 2 / kT
    p = np.exp(log_p - log_p.max())
    return _trapz(p * x, x) / _trapz(p, x)
