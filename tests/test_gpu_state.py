"""Eq. (15) state free energy and the Eq. (5) turn-on free energy on the GPU
against the FP64 oracle: identical samples (<= 1e-12 relative, jackknife
<= 1e-8), and a whole 1D run with the same noise streams as the oracle's,
which both match the quadrature."""
import numpy as np
import pytest

from oracle import _clib, estimators as est, quadrature as quad
from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


@pytest.mark.parametrize("s,R,T", [(21, 32, 3600), (1, 5, 40), (4, 300, 129), (3, 1, 20)])
def test_state_free_energy_parity(pmf, s, R, T):
    k, kT = 500.0, inputs.kT_of(300.0)
    lam = inputs.lambda_grid(1.3, 3.3, s) if s > 1 else np.array([1.3])
    x = inputs.gaussian_x_samples(lam, k, kT, R, T, seed=7 * s + R)
    g = pmf.pmf_state_free_energy_from_samples(x.ravel(), lam, R, [T] * s, k, kT)
    o = est.state_free_energy([x[i].astype(np.float64) for i in range(s)], lam, k, kT)
    assert abs(g["dF_turn_on"] - o["dF_turn_on"]) <= 1e-12 * max(abs(o["dF_turn_on"]), kT)
    assert np.all(np.abs(g["G"] - o["G"]) <= 1e-12 * np.maximum(np.abs(o["G"]), kT))
    np.testing.assert_allclose(g["se_G"], o["se_G"], rtol=1e-8, equal_nan=True)


def test_state_free_energy_of_a_1d_run(pmf):
    """A soft trap (k = 2) pulled -0.6 -> 0.6 over the double well: the GPU
    run's G matches the oracle's on the oracle's own trajectories (same
    streams, FP64 on both sides) and the quadrature."""
    k, kT, a = 2.0, 1.0, 2.0
    lam = np.linspace(-0.6, 0.6, 4)
    run = inputs.RunSettings(k=k, kT=kT, dt=1e-3, gamma=1.0, n_steps=200000, n_equil=2000, stride=20,
                             replicas=8, seed=31, lambdas=lam)
    sysh = pmf.pmf_create_system_1d(a, -0.6)
    rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    g = rr.state_free_energy()
    xo = [np.array([_clib.od1d_run(a, l, k, kT, 1.0, 1e-3, run.n_steps, run.n_equil, run.stride, run.seed,
                                   w * run.replicas + r, -0.6)[0] for r in range(run.replicas)])
          for w, l in enumerate(lam)]
    o = est.state_free_energy(xo, lam, k, kT)
    np.testing.assert_allclose(g["G"], o["G"], atol=1e-4)
    np.testing.assert_allclose(g["se_G"], o["se_G"], rtol=1e-3)
    F = np.array([quad.od1d_free_energy(l, k) for l in lam])
    exact = (F - F[0]) - (F[0] - quad.od1d_unbiased_free_energy())
    assert np.max(np.abs(g["G"] - exact)) < 0.1
    # the run's ordinary profile is unchanged by the extra call
    fe = rr.free_energy()
    np.testing.assert_allclose(g["G"] + g["dF_turn_on"], fe["dF_JE"], rtol=0, atol=1e-12)


def test_state_free_energy_rejects_batches_and_pulls(pmf):
    p = inputs.chain_params(40, 3)
    start = inputs.chain_start(p, 7)
    run = inputs.RunSettings(k=300.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=400, n_equil=40,
                             stride=40, replicas=2, seed=4)
    sysh = pmf.pmf_create_system_chain([p, p], [start, start])
    rb = pmf.pmf_run_batch_prepare(sysh, [(0, [1.0, 1.1]), (1, [1.0, 1.2])], pmf.make_params(run))
    rb.launch()
    rb.wait()
    with pytest.raises(pmf.PmfError) as e:
        rb.state_free_energy()
    assert e.value.status == pmf.PMF_EINVAL
