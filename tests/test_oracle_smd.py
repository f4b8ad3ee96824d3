"""Pins of the constant-velocity pulling oracle (CPU)."""
import math

import numpy as np

from oracle import _clib
from oracle import estimators as est
from paper_1105_4840_gb300 import inputs


def test_zero_velocity_is_a_window_run():
    """With the trap standing still the work stays 0 and the x records are
    the samples of the parallel protocol's window run (same noise)."""
    p = inputs.chain_params(14, 2)
    start = inputs.chain_start(p, 3)
    ch = _clib.Chain(p)
    x, w, _, _ = ch.smd(start, 1.1, 0.0, 500.0, 2.49, 0.001, 5.0, 300, 100, 20, 7, 4)
    xs, _, _ = ch.run(start, 1.1, 500.0, 2.49, 0.001, 5.0, 300, 100, 20, 7, 4)
    np.testing.assert_array_equal(x, xs)
    assert np.all(w == 0.0)
    x1, w1 = _clib.od1d_smd(2.0, -0.5, 0.0, 20.0, 1.0, 1.0, 1e-3, 400, 100, 10, 3, 2, -1.0)
    x2, _ = _clib.od1d_run(2.0, -0.5, 20.0, 1.0, 1.0, 1e-3, 400, 100, 10, 3, 2, -1.0)
    np.testing.assert_array_equal(x1, x2)
    assert np.all(w1 == 0.0)


def test_moving_harmonic_trap_work_mean_and_jarzynski():
    """A free overdamped particle (U = 0) in a trap moving at constant
    velocity: the mean work follows the exact mean of the discrete dynamics
    (a linear recursion), and since F(lambda, k) does not depend on lambda,
    Jarzynski's average of the work gives 0."""
    k, kT, gamma, dt, vdt = 20.0, 1.0, 1.0, 1e-3, 5e-4  # ~0.5 kT dissipated: JE converges
    n_steps, n_equil, stride, R = 3000, 1000, 250, 600
    rng = np.random.default_rng(0)
    x0 = rng.normal(0.0, math.sqrt(kT / k), R)  # equilibrated in the trap at lambda1 = 0
    W = np.array([_clib.od1d_smd(0.0, 0.0, vdt, k, kT, gamma, dt, n_steps, n_equil, stride, 11, r, x0[r])[1]
                  for r in range(R)])
    # exact mean of the discrete process: <x> starts at 0 and relaxes under
    # the moving trap; the work increment is linear in x
    m, lam, wm = 0.0, 0.0, 0.0
    means = []
    for step in range(n_steps):
        if step > n_equil:
            new = vdt * (step - n_equil)
            wm += 0.5 * k * (new - lam) * (new + lam - 2.0 * m)
            lam = new
        m = m - k * (m - lam) * dt / gamma
        done = step + 1
        if done > n_equil and (done - n_equil) % stride == 0:
            means.append(wm)
    means = np.array(means)
    se = W.std(axis=0, ddof=1) / math.sqrt(R)
    assert np.all(np.abs(W.mean(axis=0) - means) <= 4.0 * se + 1e-12)
    assert means[-1] > 0.0  # dissipated work
    for j in range(W.shape[1]):
        assert abs(est.je_increment(W[:, j], kT)) < 4.0 * se[j] + 0.05
