"""GPU tests of constant-velocity pulling against its oracle: records of x
and of the accumulated work per replica (1D and chain, FP32 and FP64),
bit-identity over persistent segment sizes, and the per-record estimators
against the oracle's on the same work values."""
import math

import numpy as np
import pytest

from oracle import _clib
from oracle import estimators as est
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def test_smd_1d_matches_oracle(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.stride, run.replicas = 6000, 1000, 100, 4
    v = 0.5  # length per time unit: 2.5 length units over the pull
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_prepare_smd(sysh, -1.2, v, pmf.make_params(run, uid_base=3))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()[0]
    W = rr.smd_work()
    for r in range(4):
        xo, wo = _clib.od1d_smd(w["a"], -1.2, v * run.dt, run.k, run.kT, run.gamma, run.dt, run.n_steps,
                                run.n_equil, run.stride, run.seed, 3 + r, w["x0"])
        np.testing.assert_allclose(xs[r], xo, atol=2e-6, rtol=0)
        np.testing.assert_allclose(W[r], wo, atol=1e-9, rtol=0)
    res = rr.smd_free_energy()
    np.testing.assert_allclose(res["lambda"], -1.2 + v * run.dt * run.stride * np.arange(1, W.shape[1] + 1),
                               rtol=0, atol=1e-12)
    for j in range(W.shape[1]):
        assert math.isclose(res["dF_JE"][j], est.je_increment(W[:, j], run.kT), rel_tol=1e-12, abs_tol=1e-12)
        assert math.isclose(res["W_mean"][j], W[:, j].mean(), rel_tol=1e-12, abs_tol=1e-12)
        assert math.isclose(res["W_var"][j], W[:, j].var(), rel_tol=1e-10, abs_tol=1e-12)
        assert math.isclose(res["dF_cumulant"][j], W[:, j].mean() - W[:, j].var() / (2 * run.kT),
                            rel_tol=1e-10, abs_tol=1e-12)
        assert math.isclose(res["mean_x"][j], xs[:, j].astype(np.float64).mean(), rel_tol=1e-12, abs_tol=1e-12)


@pytest.mark.parametrize("prec,tx,tw", [(0, 1e-4, 2e-3), (1, 1e-9, 1e-8)])
def test_smd_chain_matches_oracle(pmf, prec, tx, tw):
    p = inputs.chain_params(30, 9)
    start = f32(inputs.chain_start(p, 19, target_x=1.0))
    x0 = float(np.linalg.norm(start[-1] - start[0]))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=400, n_equil=100,
                             stride=50, replicas=3, seed=6)
    v = 1.0  # nm / ps
    sysh = pmf.pmf_create_system_chain([p], [start], precision=prec)
    rr = pmf.pmf_run_prepare_smd(sysh, x0, v, pmf.make_params(run))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()[0]
    W = rr.smd_work()
    ch = _clib.Chain(p)
    for r in range(3):
        xo, wo, _, _ = ch.smd(start, x0, v * run.dt, run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                              run.stride, run.seed, r)
        np.testing.assert_allclose(xs[r], xo, atol=max(tx, 2e-7), rtol=0)
        np.testing.assert_allclose(W[r], wo, atol=tw, rtol=0)


def test_smd_segments_are_bit_identical(pmf):
    p = inputs.chain_params(30, 9)
    start = f32(inputs.chain_start(p, 19, target_x=1.0))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=400, n_equil=100,
                             stride=50, replicas=5, seed=6)
    sysh = pmf.pmf_create_system_chain([p], [start])
    out = []
    for ctas, seg in ((0, 1000), (2, 37), (-1, 0)):
        pmf.pmf_chain_set_grid(sysh, 0, ctas, seg)
        rr = pmf.pmf_run_prepare_smd(sysh, 1.0, 1.0, pmf.make_params(run))
        rr.launch()
        rr.wait()
        out.append((rr.smd_work(), rr.x_samples()[0]))
    for W, x in out[1:]:
        assert np.array_equal(W, out[0][0]) and np.array_equal(x, out[0][1])
