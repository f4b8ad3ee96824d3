"""GPU tests of the App. C work distributions against the oracle on the same
samples (both binning rules), and of their convergence to the factorised
estimator."""
import numpy as np
import pytest

from oracle import histograms as hist
from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


@pytest.fixture(scope="module")
def od1d_run(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    return rr, run, sysh


@pytest.mark.parametrize("left_edge", [False, True])
def test_work_distributions_match_oracle(pmf, od1d_run, left_edge):
    rr, run, _ = od1d_run
    xs = [a.astype(np.float64) for a in rr.x_samples()]
    x_lo, dx, K, dW, M = -2.5, 1e-3, 5000, 0.01, 3000
    g = rr.work_distributions(x_lo, dx, K, dW, M, left_edge=left_edge)
    om, dF, var, lost = hist.work_distributions(xs, run.lambdas, run.k, run.kT, x_lo, dx, K, dW, M, left_edge)
    np.testing.assert_allclose(g["omega"], om, rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(g["dF_JE"], dF, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(g["var_ZW"], var, rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(g["lost"], lost, atol=1e-12)
    if not left_edge:  # (the printed rule's smoothing of the W = 0 bin changes the total by itself)
        assert g["lost"].max() < 1e-9


def test_fine_bins_approach_the_factorised_estimate(pmf, od1d_run):
    rr, run, _ = od1d_run
    exact = rr.free_energy()["dF_JE"]
    g = rr.work_distributions(-2.5, 2e-4, 25000, 2e-3, 15000, with_omega=False)
    assert np.max(np.abs(g["dF_JE"] - exact)) < 0.005 * run.kT


def test_sequential_run_and_range_errors(pmf, od1d_run):
    _, run, sysh = od1d_run
    r2 = pmf.pmf_run_prepare_sequential(sysh, run.lambdas, pmf.make_params(run))
    r2.launch()
    r2.wait()
    g = r2.work_distributions(-2.5, 1e-3, 5000, 0.01, 3000, with_omega=False)
    exact = r2.free_energy()["dF_JE"]
    assert np.max(np.abs(g["dF_JE"] - exact)) < 0.02 * run.kT
    with pytest.raises(pmf.PmfError) as e:  # no window has a sample in [5, 6)
        r2.work_distributions(5.0, 1e-3, 1000, 0.01, 100)
    assert e.value.status == pmf.PMF_EINVAL
