"""Sequential pulling protocol (Sec. III (i)), FP64 oracle (test infrastructure).

One simulation visits the windows in order: the trap centre is set to
lambda_1, the system relaxes for tau steps while x is recorded, then the
centre moves to lambda_2 and the run continues from the state reached, and so
on to lambda_s.  The time steps are numbered continuously over the whole
simulation (window i covers steps i*tau .. (i+1)*tau - 1), which fixes the
Philox noise of every step; equilibration and sampling count from each
window's first step.  Several independent simulations (replica r, uid
uid_base + r) give the per-window sample blocks [R, T] the estimators take.
"""
from __future__ import annotations

import numpy as np

from . import _clib


def chain_spp(params, start, lambdas, run, uid_base=0):
    """Samples [s][R, T] and final positions [R][N, 3] of R sequential pulls
    of a chain (run: k, kT, dt, gamma, n_steps = tau, n_equil, stride,
    replicas, seed)."""
    ch = _clib.Chain(params)
    tau = run.n_steps
    samples = [[] for _ in lambdas]
    finals = []
    for r in range(run.replicas):
        pos = np.array(start, dtype=np.float64)
        vel = None
        for i, lam in enumerate(lambdas):
            x, pos, vel = ch.run(pos, lam, run.k, run.kT, run.dt, run.gamma, tau, run.n_equil, run.stride,
                                 run.seed, uid_base + r, v0=vel, step0=i * tau)
            samples[i].append(x)
        finals.append(pos)
    return [np.array(b) for b in samples], finals


def od1d_spp(a, x0, lambdas, run, uid_base=0):
    """Samples [s][R, T] and final x [R] of R sequential pulls of the 1D model."""
    tau = run.n_steps
    samples = [[] for _ in lambdas]
    finals = []
    for r in range(run.replicas):
        x = x0
        for i, lam in enumerate(lambdas):
            xs, x = _clib.od1d_run(a, lam, run.k, run.kT, run.gamma, run.dt, tau, run.n_equil, run.stride,
                                   run.seed, uid_base + r, x, step0=i * tau)
            samples[i].append(xs)
        finals.append(x)
    return [np.array(b) for b in samples], np.array(finals)
