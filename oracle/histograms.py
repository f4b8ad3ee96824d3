"""Work distributions from binned reaction-coordinate distributions (App. C),
FP64 numpy (test infrastructure).

For each window i the samples of x_i are counted into K bins of width dx
(rho_i, normalised to probabilities).  The distribution of the accumulated
mechanical work after the first i - 1 pulling steps, Omega_i, lives on the
bins W = b dW, b = -M..M.  Omega_1 is all at W = 0 (no work before the first
step, Eq. (9)); each further step adds the increment of Eq. (9),
w_i(x) = k/2 (lambda_{i+1} - lambda_i)(lambda_{i+1} + lambda_i - 2 x),
at every x bin of window i, weighted by rho_i:
    Omega_{i+1}(b') = sum_j rho_i(j) Omega_i(b' - shift_i(j)).
Readings (App. C is garbled in places): the recursion runs through Omega_s
(the printed loop stops one window early); with `left_edge` False (the
default reading) a bin stands for its centre, x_j = x_lo + (j + 1/2) dx, and
a shifted work value goes to the nearest bin, shift = round(w / dW); with
`left_edge` True the rule as printed, x_j = x_lo + j dx and shift =
floor(w / dW), with its smoothing Omega_i(0) = (Omega_i(-1) + Omega_i(1)) / 2.
From Omega_i: dF^JE(lambda_i) = -kT ln sum_b Omega_i(b) exp(-b dW / kT)
(Eq. (12)), and the variance formula of App. C with sigma_W the standard
deviation of Omega_i and Q its number of non-zero bins.
"""
from __future__ import annotations

import math

import numpy as np


def rho(samples, x_lo, dx, K):
    """Counts of x in bins [x_lo + j dx, x_lo + (j + 1) dx), j = 0..K-1,
    divided by the sample count; also the count falling outside."""
    x = np.asarray(samples, dtype=np.float64).ravel()
    j = np.floor((x - x_lo) / dx).astype(np.int64)
    inside = (j >= 0) & (j < K)
    r = np.bincount(j[inside], minlength=K).astype(np.float64) / x.size
    return r, int((~inside).sum())


def shifts(lam_i, lam_next, k, x_lo, dx, K, dW, left_edge=False):
    """Work-bin shift of every x bin for the step lambda_i -> lambda_{i+1}."""
    j = np.arange(K, dtype=np.float64)
    x = x_lo + (j if left_edge else j + 0.5) * dx
    w = 0.5 * k * (lam_next - lam_i) * (lam_next + lam_i - 2.0 * x)
    return (np.floor(w / dW) if left_edge else np.floor(w / dW + 0.5)).astype(np.int64)


def work_distributions(samples, lambdas, k, kT, x_lo, dx, K, dW, M, left_edge=False):
    """Omega_i for i = 1..s ([s, 2M + 1], bin b at index b + M), the JE profile,
    the App. C variance and the probability lost outside the W range."""
    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    nb = 2 * M + 1
    omega = np.zeros((s, nb))
    omega[0, M] = 1.0
    lost = np.zeros(s)
    for i in range(s - 1):
        r, _ = rho(samples[i], x_lo, dx, K)
        sh = shifts(lam[i], lam[i + 1], k, x_lo, dx, K, dW, left_edge)
        nxt = np.zeros(nb)
        for j in np.nonzero(r)[0]:
            d = sh[j]
            src = omega[i]
            # nxt[b + d] += r[j] * src[b] for every b with b + d inside the range
            lo, hi = max(0, -d), min(nb, nb - d)
            if lo < hi:
                nxt[lo + d:hi + d] += r[j] * src[lo:hi]
        if left_edge:
            nxt[M] = 0.5 * (nxt[M - 1] + nxt[M + 1])
        omega[i + 1] = nxt
        lost[i + 1] = max(0.0, 1.0 - math.fsum(nxt.tolist()))
    W = (np.arange(nb) - M) * dW
    dF = np.zeros(s)
    var = np.zeros(s)
    for i in range(s):
        p = omega[i]
        tot = math.fsum(p.tolist())
        nz = p > 0
        m = W[nz].min()
        dF[i] = m - kT * math.log(math.fsum((p[nz] * np.exp(-(W[nz] - m) / kT)).tolist()) / tot)
        mean = math.fsum((p * W).tolist()) / tot
        sw2 = math.fsum((p * (W - mean) ** 2).tolist()) / tot
        Q = int(nz.sum())
        var[i] = sw2 / Q + sw2 * sw2 / (2.0 * kT * kT * (Q - 1)) if Q > 1 else 0.0
    return omega, dF, var, lost
