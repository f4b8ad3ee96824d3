"""FP64 oracle of the learned window-placement part (test infrastructure).

The paper asks that adjacent x distributions overlap comparably to their
spread (Sec. III after Eq. (9); Sec. IV B: increments no larger than the
fluctuation of x; Sec. V criterion (iii)) and models each window's x
distribution as a Gaussian with mean <x_i> and variance gamma_i^2 kT / k
(Sec. II, text before Eq. (13)).  The surrogate turns that into a procedure:

  * an MLP lambda -> (mu, log sigma^2) of x, 1 -> 64 -> 64 -> 2 with SiLU,
    trained on (lambda_i, x) samples by the Gaussian negative log-likelihood
    0.5 [log sigma^2 + (x - mu)^2 / sigma^2] with Adam;
  * the overlap coefficient OVL = int min(p_1, p_2) of two Gaussians;
  * insertion of the midpoint of every adjacent pair whose predicted OVL is
    below a threshold, and seeding of each new window's replicas from the
    stored end states whose final x is closest to the predicted mean;
  * optionally, a gate before training: the measured moments of every
    window's samples give the adjacent OVLs, and only a pair below the
    threshold makes the round train and insert.

Plain numpy, FP64, written to be read against the definitions above.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

H = 64  # hidden width


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(seed: int, scale_in: float = 1.0):
    """He-style initial weights from the shared seeded input generator (the
    CUDA side is given the same arrays)."""
    from paper_1105_4840_gb300.inputs import mlp_init_params

    return mlp_init_params(seed, H, scale_in)


def forward(p, lam):
    """lam [B] -> dict with z1, h1, z2, h2, out [B, 2] = (mu, log sigma^2)."""
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 1)
    z1 = lam @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    out = h2 @ p["W3"].T + p["b3"]
    return {"lam": lam, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "out": out}


def nll(out, x):
    """Mean Gaussian negative log-likelihood 0.5 [s + (x - mu)^2 e^{-s}]
    (without the constant 0.5 log 2 pi)."""
    mu, s = out[:, 0], out[:, 1]
    x = np.asarray(x, dtype=np.float64).ravel()
    return float(np.mean(0.5 * (s + (x - mu) ** 2 * np.exp(-s))))


def backward(p, cache, x):
    """Gradients of the mean NLL with respect to every parameter."""
    x = np.asarray(x, dtype=np.float64).ravel()
    B = x.size
    mu, s = cache["out"][:, 0], cache["out"][:, 1]
    e = np.exp(-s)
    dout = np.stack([-(x - mu) * e, 0.5 * (1.0 - (x - mu) ** 2 * e)], axis=1) / B
    g = {"W3": dout.T @ cache["h2"], "b3": dout.sum(axis=0)}
    dh2 = dout @ p["W3"]
    dz2 = dh2 * silu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * silu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["lam"]
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def gaussian_overlap(mu1, s1, mu2, s2) -> float:
    """OVL = int min(p1, p2) dx of N(mu1, s1^2) and N(mu2, s2^2): the pdfs
    cross where their log-densities are equal (a quadratic in x); between
    crossings the smaller pdf is integrated with the normal CDF."""
    mu1, s1, mu2, s2 = float(mu1), float(s1), float(mu2), float(s2)
    Phi = lambda z: 0.5 * special.erfc(-z / math.sqrt(2.0))
    if abs(s1 - s2) < 1e-12 * max(s1, s2):
        return 2.0 * Phi(-abs(mu1 - mu2) / (2.0 * s1))
    # a x^2 + b x + c = 0 from log p1 = log p2
    a = 1.0 / (2 * s2 ** 2) - 1.0 / (2 * s1 ** 2)
    b = mu1 / s1 ** 2 - mu2 / s2 ** 2
    c = mu2 ** 2 / (2 * s2 ** 2) - mu1 ** 2 / (2 * s1 ** 2) + math.log(s2 / s1)
    disc = max(b * b - 4 * a * c, 0.0)
    r1, r2 = sorted(((-b - math.sqrt(disc)) / (2 * a), (-b + math.sqrt(disc)) / (2 * a)))
    cdf = lambda x, m, s: Phi((x - m) / s)
    # the wider Gaussian is the smaller pdf outside [r1, r2]
    wide, narrow = ((mu1, s1), (mu2, s2)) if s1 > s2 else ((mu2, s2), (mu1, s1))
    inside = cdf(r2, *wide) - cdf(r1, *wide)
    outside = cdf(r1, *narrow) + (1.0 - cdf(r2, *narrow))
    return inside + outside


def insert_windows(lambdas, mu, log_var, threshold):
    """Midpoints of every adjacent pair (lambda_i, lambda_{i+1}) whose
    predicted x distributions N(mu, exp(log_var)) overlap less than
    `threshold`."""
    lam = np.asarray(lambdas, dtype=np.float64)
    sd = np.exp(0.5 * np.asarray(log_var, dtype=np.float64))
    new = []
    for i in range(lam.size - 1):
        if gaussian_overlap(mu[i], sd[i], mu[i + 1], sd[i + 1]) < threshold:
            new.append(0.5 * (lam[i] + lam[i + 1]))
    return np.array(new)


def window_moments(x_windows):
    """Mean and population variance of each window's samples (all replicas
    pooled): the measured Gaussian of the window."""
    mu = np.array([math.fsum(np.ravel(x).tolist()) / np.size(x) for x in x_windows])
    var = np.array([math.fsum(((np.ravel(x).astype(np.float64) - m) ** 2).tolist()) / np.size(x)
                    for x, m in zip(x_windows, mu)])
    return mu, var


def measured_overlaps(x_windows):
    """OVL of each adjacent pair of windows from their measured moments."""
    mu, var = window_moments(x_windows)
    sd = np.sqrt(var)
    return np.array([gaussian_overlap(mu[i], sd[i], mu[i + 1], sd[i + 1]) for i in range(mu.size - 1)])


def needs_training(x_windows, threshold) -> bool:
    """The gate of a round: train the surrogate (and so consider inserting
    windows) only if some adjacent pair's measured overlap is below the
    threshold."""
    return bool(np.any(measured_overlaps(x_windows) < threshold))


def seed_order(final_x, target):
    """Indices of the candidate end states ordered by |x_final - target|
    (stable for ties); replica r of a new window starts from candidate
    order[r mod len]."""
    final_x = np.asarray(final_x, dtype=np.float64)
    return np.argsort(np.abs(final_x - target), kind="stable")


def normalise(lam, x, c, h):
    """lambda' = (lambda - c) / h, x' = (x - c) / h."""
    return (np.asarray(lam, dtype=np.float64) - c) / h, (np.asarray(x, dtype=np.float64) - c) / h


def to_physical(out, c, h):
    """(mu', s') -> (mu, log sigma^2) = (c + h mu', s' + 2 log h)."""
    return c + h * out[:, 0], out[:, 1] + 2.0 * math.log(h)


def minibatch(philox_bulk, seed, step, batch, total):
    """Sample indices of one Adam step: Philox4x32-10 block j of counter
    (j, step, 0, 3) gives index (word1 * 2^32 + word0) mod total."""
    raw, _ = philox_bulk(seed, 0, step, 0, 3, batch)
    r = (raw[:, 1].astype(np.uint64) << np.uint64(32)) | raw[:, 0].astype(np.uint64)
    return (r % np.uint64(total)).astype(np.int64)


def train(p, x_store, offsets, lambdas, steps, batch, lr, seed, c, h, philox_bulk, state=None, t0=0):
    """Adam on mini-batches drawn from a run's sample store (layout
    [window][replica][sample]; offsets[w] = first sample of window w)."""
    state = {} if state is None else state
    offsets = np.asarray(offsets, dtype=np.int64)
    lam_w = np.asarray(lambdas, dtype=np.float64)
    x_store = np.asarray(x_store, dtype=np.float64)
    loss = math.nan
    for step in range(steps):
        idx = minibatch(philox_bulk, seed, t0 + step, batch, x_store.size)
        w = np.searchsorted(offsets, idx, side="right") - 1
        lam_n, x_n = normalise(lam_w[w], x_store[idx], c, h)
        cache = forward(p, lam_n)
        loss = nll(cache["out"], x_n)
        g = backward(p, cache, x_n)
        adam_step(p, g, state, lr)
    return p, state, loss
