"""FP32 vs FP64 integration (the precision study on the 104-bead workload):
per window pair, the JE increment of the FP32 GPU run, the FP64 GPU run and
the FP64 oracle on a subset of the same replicas (same Philox streams) must
agree within their combined jackknife standard errors; so must the whole
path.  Trajectories themselves diverge over thousands of steps (chaotic
dynamics), so the comparison is statistical."""
import concurrent.futures as cf
import math
import os

import numpy as np
import pytest

from oracle import _clib
from oracle import estimators as est
from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS, R_GPU, R_ORACLE = 4000, 64, 6


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def _increments(res):
    return np.diff(res["dF_JE"]), np.sqrt(np.maximum(np.diff(res["se_JE"] ** 2), 0.0))


def test_fp32_fp64_oracle_agree_per_window_pair(pmf):
    w = inputs.chain_workload(n_steps=STEPS, replicas=R_GPU)
    p, start, run = w["params"], w["start"], w["run"]
    lam = run.lambdas
    res = {}
    for prec in (0, 1):
        sysh = pmf.pmf_create_system_chain([p], [start], precision=prec)
        rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
        res[prec] = rr.free_energy()
    ch = _clib.Chain(p)

    def one(job):
        wi, r = job
        return ch.run(start, lam[wi], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil, run.stride,
                      run.seed, wi * run.replicas + r)[0]

    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        xs = list(ex.map(one, [(wi, r) for wi in range(lam.size) for r in range(R_ORACLE)]))
    ores = est.free_energy_profile([np.array(xs[i * R_ORACLE:(i + 1) * R_ORACLE]) for i in range(lam.size)],
                                   lam, run.k, run.kT)
    j32, s32 = _increments(res[0])
    j64, s64 = _increments(res[1])
    jor, sor = _increments(ores)
    z64 = (j32 - j64) / np.hypot(s32, s64)
    zor = (j32 - jor) / np.hypot(s32, sor)
    print("window-pair z (FP32-FP64):", np.round(z64, 2))
    print("window-pair z (FP32-oracle):", np.round(zor, 2))
    assert np.all(np.isfinite(z64)) and np.all(np.isfinite(zor))
    assert np.max(np.abs(z64)) < 4.5 and np.max(np.abs(zor)) < 4.5
    for ref in (res[1], ores):
        zp = (res[0]["dF_JE"][-1] - ref["dF_JE"][-1]) / math.hypot(res[0]["se_JE"][-1], ref["se_JE"][-1])
        assert abs(zp) < 4.0, zp
