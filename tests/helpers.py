"""Shared test helpers: seeded workloads and parallel oracle runs.

Oracle runs go through ctypes (which releases the GIL), so a thread pool runs
independent replicas on all host cores."""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

from oracle import _clib


def f32(a):
    """Round to FP32 and back: the state the FP32 path actually holds."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def oracle_chain_samples(params, start, lambdas, run, threads=None, uid_base=0):
    """Oracle x samples [s][R, T] of the PPP on a chain (uid = w * R + r)."""
    ch = _clib.Chain(params)
    jobs = [(w, r) for w in range(len(lambdas)) for r in range(run.replicas)]
    threads = threads or min(32, os.cpu_count() or 1)

    def one(job):
        w, r = job
        x, _, _ = ch.run(start, lambdas[w], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                         run.stride, run.seed, uid_base + w * run.replicas + r)
        return x

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, jobs))
    out = []
    for w in range(len(lambdas)):
        out.append(np.array(res[w * run.replicas:(w + 1) * run.replicas]))
    return out


def oracle_od1d_samples(a, x0, run, uid_base=0):
    out = []
    for w, lam in enumerate(run.lambdas):
        rows = []
        for r in range(run.replicas):
            x, _ = _clib.od1d_run(a, lam, run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil,
                                  run.stride, run.seed, uid_base + w * run.replicas + r, x0)
            rows.append(x)
        out.append(np.array(rows))
    return out
