"""Pins of the sequential pulling protocol oracle (Sec. III (i)), CPU only."""
import numpy as np

from oracle import _clib, spp
from oracle import estimators as est
from oracle import quadrature as quad
from paper_1105_4840_gb300 import inputs


def test_spp_with_a_fixed_trap_is_one_continuous_run():
    """Two windows with the same centre and no equilibration discard are one
    run of 2 tau steps cut in two: the samples and the final state agree
    exactly (chain and 1D)."""
    p = inputs.chain_params(12, 3)
    start = inputs.chain_start(p, 4)
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=60, n_equil=0,
                             stride=10, replicas=2, seed=5)
    lam = np.array([1.0, 1.0])
    xs, finals = spp.chain_spp(p, start, lam, run, uid_base=7)
    ch = _clib.Chain(p)
    for r in range(2):
        x, rf, _ = ch.run(start, 1.0, run.k, run.kT, run.dt, run.gamma, 120, 0, 10, run.seed, 7 + r)
        np.testing.assert_array_equal(np.concatenate([xs[0][r], xs[1][r]]), x)
        np.testing.assert_array_equal(finals[r], rf)
    w = inputs.od1d_workload()
    r1 = w["run"]
    r1.n_steps, r1.n_equil, r1.stride, r1.replicas = 1002, 0, 3, 2  # tau not a multiple of 4
    xs, xf = spp.od1d_spp(w["a"], w["x0"], np.array([0.2, 0.2]), r1)
    for r in range(2):
        x, f = _clib.od1d_run(w["a"], 0.2, r1.k, r1.kT, r1.gamma, r1.dt, 2004, 0, 3, r1.seed, r, w["x0"])
        np.testing.assert_array_equal(np.concatenate([xs[0][r], xs[1][r]]), x)
        assert xf[r] == f


def test_spp_one_window_is_the_parallel_protocol():
    w = inputs.od1d_workload()
    run = w["run"]
    run.replicas = 3
    xs, _ = spp.od1d_spp(w["a"], w["x0"], np.array([0.4]), run, uid_base=11)
    for r in range(3):
        x, _ = _clib.od1d_run(w["a"], 0.4, run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil,
                              run.stride, run.seed, 11 + r, w["x0"])
        np.testing.assert_array_equal(xs[0][r], x)


def test_spp_double_well_matches_quadrature():
    """The 1D workload pulled sequentially: Eq. (12) on the SPP samples agrees
    with the quadrature within 4 jackknife errors plus 0.05 kT."""
    w = inputs.od1d_workload()
    run = w["run"]
    xs, _ = spp.od1d_spp(w["a"], w["x0"], run.lambdas, run)
    res = est.free_energy_profile(xs, run.lambdas, run.k, run.kT)
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in run.lambdas])
    exact -= exact[0]
    assert np.all(np.abs(res["dF_JE"] - exact) <= 4.0 * res["se_JE"] + 0.05)
