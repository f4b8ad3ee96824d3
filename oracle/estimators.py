"""Free-energy estimators of the paper, plain FP64 numpy (test infrastructure).

Every function states the passage it follows.  Readings of ambiguous points:
  * Delta lambda.  Eqs. (13), (14) and App. B write (lambda_s - lambda_1)/s for
    the increment, but the paper's grids (13, 14, ..., 33 A with s = 21) have
    increment (lambda_s - lambda_1)/(s - 1).  Here every sum uses the actual
    increment Delta_i = lambda_{i+1} - lambda_i, which is what Eq. (9) and the
    B.5 derivation need and what a non-uniform grid needs.
  * Profile points.  F(lambda_j) - F(lambda_1) uses windows 1..j-1 (Eq. (9)
    sums to s-1); the value at lambda_1 is 0 (Fig. 4b sets the s = 1 force to 0).
  * All-combinations average.  The windows are independent (Sec. II: rho(W_mech)
    is proportional to rho(x_1)...rho(x_{s-1})), so the average of
    exp(-beta W_mech) over every tuple (x_1, ..., x_{s-1}) of samples factorises
    into the product of the per-window averages of exp(-beta w_i).
  * gamma_i^2 = k sigma_i^2 / kT (Eq. (13) text) with the plug-in variance
    (divisor n).
  * Standard error: delete-one-replica jackknife inside each window, variances
    added over windows.
  * Zuckerman-Woolf variance (Sec. IV A, App. C): sigma_W^2 is the variance of
    W_mech = sum of the independent increments; Q is the number of independent
    work tuples, min_i n_i.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def work_increment(x, lam_i: float, lam_next: float, k: float):
    """Eq. (9) / Eq. (B.1): work of moving the trap centre from lambda_i to
    lambda_{i+1} with the reaction coordinate at x_i,
    w_i = k/2 (lambda_{i+1} - lambda_i)(lambda_{i+1} + lambda_i - 2 x_i)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * k * (lam_next - lam_i) * (lam_next + lam_i - 2.0 * x)


def je_increment(w, kT: float) -> float:
    """Eq. (12) for one window: -kT ln((1/n) sum_a exp(-w_a / kT)), evaluated
    as m - kT ln((1/n) sum_a exp(-(w_a - m)/kT)) with m = min w and an exactly
    rounded sum (math.fsum)."""
    w = np.asarray(w, dtype=np.float64).ravel()
    if w.size == 0:
        return math.nan
    m = float(w.min())
    s = math.fsum(np.exp(-(w - m) / kT).tolist())
    return m - kT * math.log(s / w.size)


def zw_variance(sigma_w: float, Q: float, kT: float) -> float:
    """Variance of the JE estimate (Sec. IV A, App. C; Zuckerman & Woolf):
    sigma_W^2 / Q + beta^2 sigma_W^4 / (2 (Q - 1))."""
    beta = 1.0 / kT
    return sigma_w ** 2 / Q + beta ** 2 * sigma_w ** 4 / (2.0 * (Q - 1.0))


def _window_terms(x2d, lam_i, lam_next, k, kT):
    """Per-window JE increment, mean and plug-in variance of x."""
    x = np.asarray(x2d, dtype=np.float64)
    w = work_increment(x, lam_i, lam_next, k)
    mean = math.fsum(x.ravel().tolist()) / x.size
    var = math.fsum(((x.ravel() - mean) ** 2).tolist()) / x.size
    return je_increment(w, kT), mean, var, w


def _jackknife_var(values):
    v = np.asarray(values, dtype=np.float64)
    R = v.size
    if R < 2:
        return math.nan
    return (R - 1) / R * float(np.sum((v - v.mean()) ** 2))


def free_energy_profile(samples, lambdas, k: float, kT: float) -> dict:
    """All estimators of the paper on per-window samples.

    samples[i] : array [R_i, T_i] of x samples of window i (lambda_i).
    Returns arrays over the s windows (index j = profile point lambda_j):
      dF_JE     Eq. (12) with the all-combinations average (factorised)
      dF_fluct  Eq. (14) with increments Delta_i: sum_{i<j} k Delta_i (lambda_i - <x_i>)
      dF_G      Eq. (13)/(B.5): sum_{i<j} [k Delta_i^2/2 (1 - gamma_i^2) + k Delta_i (lambda_i - <x_i>)]
      dF_com    (dF_JE + dF_fluct)/2   (Sec. IV B, Sec. V)
      uncertainty (dF_JE - dF_fluct)/2
      W_mean    <W_mech> = sum_{i<j} <w_i>   (Fig. 3b)
      acc_force dF_fluct / (lambda_j - lambda_1), 0 at j = 0   (Fig. 4b)
      mean_x, var_x, gamma2 per window
      se_JE, se_fluct  jackknife standard errors
      var_ZW    Zuckerman-Woolf variance of dF_JE
    """
    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    if len(samples) != s:
        raise ValueError("one sample block per window")
    out = {name: np.zeros(s) for name in ("dF_JE", "dF_fluct", "dF_G", "W_mean", "se_JE",
                                          "se_fluct", "var_ZW", "acc_force")}
    mean_x = np.zeros(s)
    var_x = np.zeros(s)
    inc_je = np.zeros(max(s - 1, 0))
    inc_fl = np.zeros(max(s - 1, 0))
    inc_g = np.zeros(max(s - 1, 0))
    inc_w = np.zeros(max(s - 1, 0))
    jk_je = np.zeros(max(s - 1, 0))
    jk_fl = np.zeros(max(s - 1, 0))
    var_w = np.zeros(max(s - 1, 0))
    n_w = np.zeros(max(s - 1, 0))
    for i in range(s):
        x = np.asarray(samples[i], dtype=np.float64)
        if x.ndim == 1:
            x = x[None, :]
        mean_x[i] = math.fsum(x.ravel().tolist()) / x.size
        var_x[i] = math.fsum(((x.ravel() - mean_x[i]) ** 2).tolist()) / x.size
        if i == s - 1:
            break
        d = lam[i + 1] - lam[i]
        je, mu, var, w = _window_terms(x, lam[i], lam[i + 1], k, kT)
        g2 = k * var / kT
        inc_je[i] = je
        inc_fl[i] = k * d * (lam[i] - mu)
        inc_g[i] = k * d * d / 2.0 * (1.0 - g2) + k * d * (lam[i] - mu)
        inc_w[i] = math.fsum(w.ravel().tolist()) / w.size
        var_w[i] = math.fsum(((w.ravel() - inc_w[i]) ** 2).tolist()) / w.size
        n_w[i] = w.size
        R = x.shape[0]
        if R >= 2:
            loo_je, loo_fl = [], []
            for r in range(R):
                rest = np.delete(x, r, axis=0)
                loo_je.append(je_increment(work_increment(rest, lam[i], lam[i + 1], k), kT))
                loo_fl.append(k * d * (lam[i] - math.fsum(rest.ravel().tolist()) / rest.size))
            jk_je[i] = _jackknife_var(loo_je)
            jk_fl[i] = _jackknife_var(loo_fl)
        else:
            jk_je[i] = jk_fl[i] = math.nan
    for j in range(1, s):
        out["dF_JE"][j] = math.fsum(inc_je[:j].tolist())
        out["dF_fluct"][j] = math.fsum(inc_fl[:j].tolist())
        out["dF_G"][j] = math.fsum(inc_g[:j].tolist())
        out["W_mean"][j] = math.fsum(inc_w[:j].tolist())
        out["se_JE"][j] = math.sqrt(math.fsum(jk_je[:j].tolist()))
        out["se_fluct"][j] = math.sqrt(math.fsum(jk_fl[:j].tolist()))
        sw2 = math.fsum(var_w[:j].tolist())
        Q = float(n_w[:j].min())
        out["var_ZW"][j] = zw_variance(math.sqrt(sw2), Q, kT) if Q > 1 else math.nan
        out["acc_force"][j] = out["dF_fluct"][j] / (lam[j] - lam[0])
    out["dF_com"] = 0.5 * (out["dF_JE"] + out["dF_fluct"])
    out["uncertainty"] = 0.5 * (out["dF_JE"] - out["dF_fluct"])
    out["mean_x"] = mean_x
    out["var_x"] = var_x
    out["gamma2"] = k * var_x / kT
    out["lambda"] = lam.copy()
    return out


def je_all_tuples(samples_1d, lambdas, k, kT) -> float:
    """Eq. (12) literally: average exp(-beta W_mech) over every tuple
    (x_1, ..., x_{s-1}), one sample per window, with W_mech from Eq. (9).
    Exponential in s; for small brute-force checks only."""
    import itertools

    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    terms = []
    for tup in itertools.product(*[np.asarray(samples_1d[i], dtype=np.float64).ravel()
                                   for i in range(s - 1)]):
        W = math.fsum(0.5 * k * (lam[i + 1] - lam[i]) * (lam[i + 1] + lam[i] - 2.0 * tup[i])
                      for i in range(s - 1))
        terms.append(W)
    W = np.asarray(terms)
    return je_increment(W, kT)


def window_partials(samples, lambdas, k: float, kT: float):
    """Per-replica partial sums of every window, the quantities a shard of
    replicas contributes to the estimators above: [s][R][5] =
    {m = min_t w_i, S = sum_t exp(-(w_i - m)/kT), n, sum_t (x - lambda_i),
    sum_t (x - lambda_i)^2} with w_i of Eq. (9) (0 in the last window)."""
    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    out = []
    for i in range(s):
        x = np.asarray(samples[i], dtype=np.float64)
        if x.ndim == 1:
            x = x[None, :]
        ln = lam[i + 1] if i + 1 < s else lam[i]
        rows = []
        for r in range(x.shape[0]):
            w = work_increment(x[r], lam[i], ln, k)
            m = float(w.min())
            d = x[r] - lam[i]
            rows.append([m, math.fsum(np.exp(-(w - m) / kT).tolist()), float(x.shape[1]),
                         math.fsum(d.tolist()), math.fsum((d * d).tolist())])
        out.append(rows)
    return np.asarray(out)


def free_energy_from_partials(P, lambdas, k: float, kT: float) -> dict:
    """The estimators of free_energy_profile from per-replica partials
    (window_partials), e.g. the union of several shards' partials
    concatenated along the replica axis.  Exponential sums of different
    replicas are brought to the window's common shift m = min_r m_r before
    they are added (log-sum-exp merge); the jackknife leaves out one
    replica's partials."""
    P = np.asarray(P, dtype=np.float64)
    lam = np.asarray(lambdas, dtype=np.float64)
    s, R = P.shape[0], P.shape[1]
    names = ("dF_JE", "dF_fluct", "dF_G", "W_mean", "se_JE", "se_fluct", "var_ZW", "acc_force")
    out = {n: np.zeros(s) for n in names}
    mean_x, var_x = np.zeros(s), np.zeros(s)
    inc = {n: np.zeros(max(s - 1, 0)) for n in ("je", "fl", "g", "w", "jje", "jfl", "vw", "n")}
    for i in range(s):
        m_r, S_r, n_r, a_r, b_r = (P[i, :, c] for c in range(5))
        n = math.fsum(n_r.tolist())
        a = math.fsum(a_r.tolist())
        b = math.fsum(b_r.tolist())
        mean_x[i] = lam[i] + a / n
        var_x[i] = b / n - (a / n) ** 2
        if i == s - 1:
            break
        d = lam[i + 1] - lam[i]
        m = float(m_r.min())
        E = S_r * np.exp(-(m_r - m) / kT)
        inc["je"][i] = m - kT * math.log(math.fsum(E.tolist()) / n)
        inc["fl"][i] = -k * d * a / n
        inc["g"][i] = k * d * d / 2.0 * (1.0 - k * var_x[i] / kT) + inc["fl"][i]
        inc["w"][i] = 0.5 * k * d * (lam[i + 1] + lam[i] - 2.0 * mean_x[i])
        inc["vw"][i] = k * k * d * d * var_x[i]
        inc["n"][i] = n
        if R >= 2:
            # each leave-one-out sum exact in rational arithmetic, rounded
            # once (the same value as fsum over the other R - 1 terms)
            Ef = [Fraction(float(e)) for e in E]
            tot = sum(Ef, Fraction(0))
            loo_je = [m - kT * math.log(float(tot - Ef[r]) / (n - n_r[r])) for r in range(R)]
            loo_fl = [-k * d * (a - a_r[r]) / (n - n_r[r]) for r in range(R)]
            inc["jje"][i] = _jackknife_var(loo_je)
            inc["jfl"][i] = _jackknife_var(loo_fl)
        else:
            inc["jje"][i] = inc["jfl"][i] = math.nan
    for j in range(1, s):
        out["dF_JE"][j] = math.fsum(inc["je"][:j].tolist())
        out["dF_fluct"][j] = math.fsum(inc["fl"][:j].tolist())
        out["dF_G"][j] = math.fsum(inc["g"][:j].tolist())
        out["W_mean"][j] = math.fsum(inc["w"][:j].tolist())
        out["se_JE"][j] = math.sqrt(math.fsum(inc["jje"][:j].tolist()))
        out["se_fluct"][j] = math.sqrt(math.fsum(inc["jfl"][:j].tolist()))
        sw2 = math.fsum(inc["vw"][:j].tolist())
        Q = float(inc["n"][:j].min())
        out["var_ZW"][j] = zw_variance(math.sqrt(sw2), Q, kT) if Q > 1 else math.nan
        out["acc_force"][j] = out["dF_fluct"][j] / (lam[j] - lam[0])
    out["dF_com"] = 0.5 * (out["dF_JE"] + out["dF_fluct"])
    out["uncertainty"] = 0.5 * (out["dF_JE"] - out["dF_fluct"])
    out["mean_x"] = mean_x
    out["var_x"] = var_x
    out["gamma2"] = k * var_x / kT
    out["lambda"] = lam.copy()
    return out


def turn_on_free_energy(x_first, lam1: float, k: float, kT: float) -> float:
    """Eq. (5): the free energy of turning the trap on at lambda_1,
    dF(lambda_1, k) = F(lambda_1, k) - F_0 = kT ln < exp(k/2 (x_1 - lambda_1)^2 / kT) >
    over the trapped ensemble (the samples of the first window), evaluated as
    M + kT ln((1/n) sum exp((u - M)/kT)) with u = k/2 (x_1 - lambda_1)^2,
    M = max u and an exactly rounded sum."""
    x = np.asarray(x_first, dtype=np.float64).ravel()
    if x.size == 0:
        return math.nan
    u = 0.5 * k * (x - lam1) ** 2
    M = float(u.max())
    return M + kT * math.log(math.fsum(np.exp((u - M) / kT).tolist()) / x.size)


def state_free_energy(samples, lambdas, k: float, kT: float) -> dict:
    """Eq. (15): the state free energy G(lambda_j, lambda_1) =
    dF^JE(lambda_j, lambda_1, k) - dF(lambda_1, k) for every profile point j
    (dF^JE of Eq. (12) as in free_energy_profile, dF(lambda_1, k) of Eq. (5)
    on the first window's samples), so G(lambda_1, lambda_1) = -dF(lambda_1, k).
    Standard error: delete-one-replica jackknife.  The first window's samples
    enter both its JE increment and the turn-on average, so replica r of that
    window is left out of both together; the jackknife variances of the other
    windows' JE increments are added.  Returns {"G", "se_G", "dF_turn_on"}."""
    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    xs = []
    for i in range(s):
        x = np.asarray(samples[i], dtype=np.float64)
        xs.append(x[None, :] if x.ndim == 1 else x)
    prof = free_energy_profile(xs, lam, k, kT)
    on = turn_on_free_energy(xs[0], lam[0], k, kT)
    G = prof["dF_JE"] - on
    se = np.full(s, math.nan)

    def je_inc(x, i):
        return je_increment(work_increment(x, lam[i], lam[i + 1], k), kT)

    def loo(x):
        return [np.delete(x, r, axis=0) for r in range(x.shape[0])]

    if xs[0].shape[0] >= 2:
        jk = [_jackknife_var([je_inc(x, i) for x in loo(xs[i])]) for i in range(1, s - 1)]
        se[0] = math.sqrt(_jackknife_var([turn_on_free_energy(x, lam[0], k, kT) for x in loo(xs[0])]))
        if s > 1:
            v0 = _jackknife_var([je_inc(x, 0) - turn_on_free_energy(x, lam[0], k, kT) for x in loo(xs[0])])
            for j in range(1, s):
                se[j] = math.sqrt(v0 + math.fsum(jk[: j - 1]))
    return {"G": G, "se_G": se, "dF_turn_on": on}
