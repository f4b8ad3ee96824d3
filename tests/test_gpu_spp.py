"""GPU tests of the sequential pulling protocol (Sec. III (i)) against its
oracle: per-sample parity for the 1D model and the chain across window
changes, bit-identity over segment sizes, and the 1D free energy against
quadrature."""
import numpy as np
import pytest

from oracle import spp
from oracle import quadrature as quad
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def test_spp_1d_matches_oracle(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.replicas = 3002, 302, 3
    lam = np.linspace(-1.5, 1.5, 5)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_prepare_sequential(sysh, lam, pmf.make_params(run, uid_base=9))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()
    xo, xf = spp.od1d_spp(w["a"], w["x0"], lam, run, uid_base=9)
    for i in range(lam.size):
        np.testing.assert_allclose(xs[i], xo[i], atol=2e-6, rtol=0)
    np.testing.assert_allclose(rr.final_state()[0], xf, atol=2e-6, rtol=0)


@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 1e-9)])
def test_spp_chain_matches_oracle(pmf, prec, tol):
    p = inputs.chain_params(40, 8)
    start = f32(inputs.chain_start(p, 18, target_x=1.0))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=150, n_equil=50,
                             stride=50, replicas=3, seed=4)
    lam = np.array([1.0, 1.2, 1.4])
    sysh = pmf.pmf_create_system_chain([p], [start], precision=prec)
    rr = pmf.pmf_run_prepare_sequential(sysh, lam, pmf.make_params(run))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()
    pos = rr.final_state()[0].reshape(3, 40, 3)
    xo, fo = spp.chain_spp(p, start, lam, run)
    for i in range(lam.size):  # samples are stored in FP32 on both integration paths
        np.testing.assert_allclose(xs[i], xo[i], atol=max(tol, 2e-7), rtol=0)
    for r in range(3):
        assert np.abs(pos[r] - fo[r]).max() <= tol


def test_spp_segments_are_bit_identical(pmf):
    """Windows split into several persistent segments (38-step pieces of a
    150-step window) give the same samples as one segment per window."""
    p = inputs.chain_params(40, 8)
    start = f32(inputs.chain_start(p, 18, target_x=1.0))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=150, n_equil=50,
                             stride=25, replicas=5, seed=4)
    lam = np.array([1.0, 1.2, 1.4, 1.6])
    sysh = pmf.pmf_create_system_chain([p], [start])
    out = []
    for ctas, seg in ((0, 1000), (2, 40), (7, 1)):
        pmf.pmf_chain_set_grid(sysh, 0, ctas, seg)
        rr = pmf.pmf_run_prepare_sequential(sysh, lam, pmf.make_params(run))
        rr.launch()
        rr.wait()
        out.append(np.concatenate([a.ravel() for a in rr.x_samples()]))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_spp_1d_workload_matches_quadrature(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_prepare_sequential(sysh, run.lambdas, pmf.make_params(run))
    rr.launch()
    rr.wait()
    res = rr.free_energy()
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in run.lambdas])
    exact -= exact[0]
    assert np.all(np.abs(res["dF_JE"] - exact) <= 4.0 * res["se_JE"] + 0.05)


def test_spp_rejects_per_window_steps(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_run_prepare_sequential(sysh, run.lambdas, pmf.make_params(run, n_steps_per_window=[20000] * 21))
    assert e.value.status == pmf.PMF_EINVAL
