"""Edge cases of the CUDA path: the longest chains that fit in shared memory
(forces and a short trajectory against the oracle, one bead more refused),
a single window, a window grid pulled backwards, the largest window counts
of a run and of a batch, and degenerate arguments."""
import math

import numpy as np
import pytest

from oracle import _clib
from oracle import quadrature as quad
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def _largest_chain(pmf, precision):
    """Largest N accepted for this precision (shared memory of one replica)."""
    lo, hi = 32, 1024
    while lo < hi:  # the first refused length
        mid = (lo + hi + 1) // 2
        p = inputs.chain_params(mid, 5)
        try:
            pmf.pmf_create_system_chain([p], [np.zeros((mid, 3))], precision=precision).close()
            lo = mid
        except pmf.PmfError as e:
            assert e.status == pmf.PMF_EINVAL
            hi = mid - 1
    return lo


@pytest.mark.parametrize("precision", [0, 1])
def test_longest_chain_forces_and_trajectory(pmf, precision):
    n = _largest_chain(pmf, precision)
    assert n >= (700 if precision == 0 else 500)
    p = inputs.chain_params(n, 5)
    start = f32(inputs.chain_start(p, 77, tries=1))
    hot = f32(start + np.random.default_rng(n).normal(0.0, 0.005, start.shape))
    sysh = pmf.pmf_create_system_chain([p], [hot], precision=precision)
    fg = pmf.pmf_chain_forces(sysh, 0, hot, 2.0, 500.0)
    fo = _clib.Chain(p).forces(hot, 2.0, 500.0)
    rel = np.linalg.norm(fg - fo) / np.linalg.norm(fo)
    assert rel <= (1e-5 if precision == 0 else 1e-12), rel
    assert np.abs(fg - fo).max() <= (1e-5 if precision == 0 else 1e-12) * np.abs(fo).max()
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=60, n_equil=30,
                             stride=30, replicas=2, seed=2)
    x0 = float(np.linalg.norm(hot[-1] - hot[0]))  # trap centred on the start: no violent pull
    lam = np.array([x0])
    rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    pos = rr.final_state()[0].reshape(2, n, 3)
    for r in range(2):
        _, ro, _ = _clib.Chain(p).run(hot, x0, run.k, run.kT, run.dt, run.gamma, 60, 30, 30, 2, r)
        assert np.abs(pos[r] - ro).max() <= (1e-4 if precision == 0 else 1e-9)
    q = inputs.chain_params(n + 1, 5)
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([q], [np.zeros((n + 1, 3))], precision=precision)
    assert e.value.status == pmf.PMF_EINVAL


def test_single_window(pmf):
    """One window: every profile value is 0 and the window's moments are the
    samples' own."""
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, np.array([0.3]), pmf.make_params(run))
    res = rr.free_energy()
    x = rr.x_samples()[0].astype(np.float64)
    for key in ("dF_JE", "dF_fluct", "dF_G", "dF_com", "uncertainty", "W_mean", "acc_force"):
        assert res[key][0] == 0.0, key
    np.testing.assert_allclose(res["mean_x"][0], x.mean(), rtol=1e-12)
    np.testing.assert_allclose(res["var_x"][0], x.var(), rtol=1e-9)


def test_reverse_pull_matches_quadrature(pmf):
    """The same grid pulled backwards (lambda decreasing): the profile is
    F(lambda_j) - F(lambda_1) of the reversed path and agrees with the
    quadrature at every point; its end value is minus the forward one's."""
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], 1.0)  # start in the right minimum
    lam = run.lambdas[::-1].copy()
    res = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run)).free_energy()
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in lam])
    exact -= exact[0]
    # within 4 jackknife standard errors plus the protocol's finite-relaxation
    # bias (of order 0.05 kT on this workload)
    assert np.all(np.abs(res["dF_JE"] - exact) <= 4.0 * res["se_JE"] + 0.05)
    fwd = np.array([quad.od1d_free_energy(l, run.k) for l in run.lambdas])
    assert math.isclose(exact[-1], -(fwd[-1] - fwd[0]), abs_tol=1e-12)


def test_largest_window_counts(pmf):
    """1024 windows in one run and 4096 in a batch run; one more is refused."""
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.stride, run.replicas = 40, 20, 10, 2
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    lam = np.linspace(-1.5, 1.5, 1024)
    rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    res = rr.free_energy()
    assert res["dF_JE"].size == 1024 and np.all(np.isfinite(res["dF_JE"]))
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_run_prepare(sysh, np.linspace(-1.5, 1.5, 1025), pmf.make_params(run))
    assert e.value.status == pmf.PMF_EINVAL
    items = [(0, np.linspace(-1.5, 1.5, 1024) + 0.001 * i) for i in range(4)]
    rb = pmf.pmf_run_batch_prepare(sysh, items, pmf.make_params(run))
    rb.launch()
    rb.wait()
    assert rb.info()["n_windows"] == 4096
    r3 = rb.free_energy_item(3, 1024)
    assert np.all(np.isfinite(r3["dF_JE"]))
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_run_batch_prepare(sysh, items + [(0, np.array([0.0]))], pmf.make_params(run))
    assert e.value.status == pmf.PMF_EINVAL


def test_degenerate_arguments(pmf):
    w = inputs.od1d_workload()
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    lam = np.array([0.0, 0.5])

    def bad(**kw):
        run = inputs.RunSettings(k=20.0, kT=1.0, dt=1e-3, gamma=1.0, n_steps=100, n_equil=10, stride=10,
                                 replicas=2, seed=0)
        for key, v in kw.items():
            setattr(run, key, v)
        with pytest.raises(pmf.PmfError) as e:
            pmf.pmf_run_prepare(sysh, lam, pmf.make_params(run))
        assert e.value.status == pmf.PMF_EINVAL

    bad(stride=200)        # no sample after the equilibration
    bad(n_equil=100)       # n_equil must be below n_steps
    bad(replicas=0)
    bad(k=0.0)
    bad(kT=-1.0)
    bad(dt=0.0)
    bad(gamma=0.0)         # the overdamped model needs friction
    with pytest.raises(pmf.PmfError):
        pmf.pmf_run_prepare(sysh, np.array([]), pmf.make_params(w["run"]))
    with pytest.raises(pmf.PmfError):
        pmf.pmf_free_energy_from_samples(np.zeros(3, dtype=np.float32), [0.0], 1, [3], 1.0, 1.0)
