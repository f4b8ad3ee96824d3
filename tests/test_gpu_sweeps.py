"""GPU tests of the sweep drivers: the coarse-grid estimate equals the oracle
on the same subset of samples; spring-constant and relaxation-time sweeps of
the 1D model agree with quadrature at each setting."""
import numpy as np
import pytest

from oracle import estimators as est
from oracle import quadrature as quad
from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1105_4840_gb300 import pmf, sweeps
    return pmf, sweeps


def test_subsample_matches_oracle(mods):
    pmf, sweeps = mods
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    got = sweeps.subsample(rr, run.lambdas, run.k, run.kT, every=2)
    xs = rr.x_samples()
    idx = list(range(0, 21, 2))
    assert list(got["windows"]) == idx
    want = est.free_energy_profile([xs[i].astype(np.float64) for i in idx], run.lambdas[idx], run.k, run.kT)
    for key in ("dF_JE", "dF_fluct", "dF_G", "dF_com"):
        np.testing.assert_allclose(got[key], want[key], rtol=1e-11, atol=1e-12, err_msg=key)
    got3 = sweeps.subsample(rr, run.lambdas, run.k, run.kT, every=3)  # 0, 3, ..., 18 and the last
    assert list(got3["windows"]) == list(range(0, 21, 3)) + [20]


def test_k_sweep_matches_quadrature(mods):
    pmf, sweeps = mods
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    out = sweeps.k_sweep(sysh, run.lambdas, run, [10.0, 20.0, 40.0])
    for o in out:
        exact = np.array([quad.od1d_free_energy(l, o["k"]) for l in run.lambdas])
        exact -= exact[0]
        res = o["result"]
        assert np.all(np.abs(res["dF_JE"] - exact) <= 4.0 * res["se_JE"] + 0.08), o["k"]
        assert o["seconds"] > 0


def test_tau_sweep_converges(mods):
    pmf, sweeps = mods
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    out = sweeps.tau_sweep(sysh, run.lambdas, run, [2000, 8000, 20000], at_lambda=0.6)
    assert [o["n_steps"] for o in out] == [2000, 8000, 20000]
    exact = quad.od1d_free_energy(0.6, run.k) - quad.od1d_free_energy(run.lambdas[0], run.k)
    last = out[-1]
    assert abs(last["lambda"] - 0.6) < 1e-12
    assert abs(last["dF_JE"] - exact) <= 4.0 * last["se_JE"] + 0.05
    assert abs(last["dF_com"] - 0.5 * (last["dF_JE"] + last["dF_fluct"])) < 1e-12
