"""Sweep drivers over the pulling protocols (the experiments of Sec. IV B-D on
synthetic systems): coarser window grids taken out of a finer run, spring
constants, and relaxation times.  Host logic only: every simulation and every
estimate runs through the C ABI (`pmf`)."""
from __future__ import annotations

import time

import numpy as np

from . import pmf


def _settings(run, **kw):
    """A copy of a RunSettings with fields replaced."""
    import copy

    r = copy.copy(run)
    for k, v in kw.items():
        setattr(r, k, v)
    return r


def subsample(run_handle, lambdas, k, kT, every: int):
    """Estimates from every `every`-th window of a finished run (windows 0,
    every, 2 every, ... and always the last one): the coarser grid of Sec. IV B
    (Delta lambda doubled when every = 2) evaluated on the same samples."""
    lam = np.asarray(lambdas, dtype=np.float64)
    idx = list(range(0, lam.size, every))
    if idx[-1] != lam.size - 1:
        idx.append(lam.size - 1)
    xs = run_handle.x_samples()
    R = xs[0].shape[0]
    sub = [xs[i] for i in idx]
    flat = np.concatenate([a.ravel() for a in sub]).astype(np.float32)
    res = pmf.pmf_free_energy_from_samples(flat, lam[idx], R, [a.shape[1] for a in sub], k, kT)
    res["windows"] = np.array(idx)
    return res


def _timed_run(system, lambdas, settings, sequential=False, chain=0):
    p = pmf.make_params(settings, chain=chain)
    t0 = time.perf_counter()
    if sequential:
        rr = pmf.pmf_run_prepare_sequential(system, lambdas, p)
        rr.launch()
        rr.wait()
    else:
        rr = pmf.pmf_run_windows(system, lambdas, p)
    res = rr.free_energy()
    return rr, res, time.perf_counter() - t0


def k_sweep(system, lambdas, settings, ks, sequential=False):
    """One run per spring constant (Sec. IV C); returns, per k, the estimates
    and the wall time of run + reduction."""
    out = []
    for k in ks:
        rr, res, el = _timed_run(system, lambdas, _settings(settings, k=float(k)), sequential)
        out.append({"k": float(k), "result": res, "seconds": el})
        rr.close()
    return out


def tau_sweep(system, lambdas, settings, taus_steps, at_lambda=None, sequential=False):
    """One run per relaxation time (Sec. IV D, Fig. 6a): dF_JE, dF_fluct,
    dF_com and the uncertainty at the window nearest `at_lambda` (the last
    one if None) as functions of tau; the equilibration discard stays 10 %."""
    lam = np.asarray(lambdas, dtype=np.float64)
    j = lam.size - 1 if at_lambda is None else int(np.argmin(np.abs(lam - at_lambda)))
    out = []
    for n in taus_steps:
        n = int(n)
        rr, res, el = _timed_run(system, lam, _settings(settings, n_steps=n, n_equil=n // 10), sequential)
        out.append({"n_steps": n, "lambda": float(lam[j]), "dF_JE": float(res["dF_JE"][j]),
                    "dF_fluct": float(res["dF_fluct"][j]), "dF_com": float(res["dF_com"][j]),
                    "uncertainty": float(res["uncertainty"][j]), "se_JE": float(res["se_JE"][j]),
                    "seconds": el})
        rr.close()
    return out
