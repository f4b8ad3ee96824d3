"""GPU tests of batched runs: many independent PPP paths (chains of uneven
length, uneven window counts) in one CUDA graph of concurrent per-chain
launches.  Sampled replicas are checked against the FP64 oracle from the
same start and Philox stream; every item must equal the same path run alone
(bit for bit: the same kernel on the same CTA work); per-item free energies
must equal the reduction of the item's own samples."""
import concurrent.futures as cf
import os

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


def _small_batch():
    lengths, n_win = (40, 57, 75), (2, 3, 2)
    params = [inputs.chain_params(n, 30 + i) for i, n in enumerate(lengths)]
    starts = [f32(inputs.chain_start(p, 60 + i)) for i, p in enumerate(params)]
    lams = [np.linspace(1.0, 1.6, s) + 0.1 * i for i, s in enumerate(n_win)]
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=200, n_equil=100,
                             stride=50, replicas=2, seed=9)
    return params, starts, lams, run


def _final_positions(rr, params, lams, R):
    pos, _ = rr.final_state()
    out, o = [], 0
    for p, l in zip(params, lams):
        n = l.size * R * p.n * 3
        out.append(pos[o:o + n].reshape(l.size, R, p.n, 3))
        o += n
    assert o == pos.size
    return out


def test_batch_matches_oracle(pmf):
    """Every replica of a 3-chain batch (N = 40, 57, 75) after 200 steps
    within 1e-4 nm of the oracle, samples within 1e-4 nm; uids continue
    across items."""
    params, starts, lams, run = _small_batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.launch()
    rr.wait()
    pos = _final_positions(rr, params, lams, run.replicas)
    xs = rr.x_samples()
    w0 = 0
    for m, (p, l) in enumerate(zip(params, lams)):
        ch = _clib.Chain(p)
        for w in range(l.size):
            for r in range(run.replicas):
                uid = (w0 + w) * run.replicas + r
                xo, ro, _ = ch.run(starts[m], l[w], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                                   run.stride, run.seed, uid)
                assert np.abs(pos[m][w, r] - ro).max() <= 1e-4, (m, w, r)
                np.testing.assert_allclose(xs[w0 + w][r], xo, atol=1e-4, rtol=0)
        w0 += l.size


def test_batch_items_equal_single_runs(pmf):
    """Item m of a batch is bit-identical to the same windows run alone with
    uid_base = its first global window x replicas; repeat launches of the
    captured graph are bit-identical too."""
    params, starts, lams, run = _small_batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.launch()
    rr.wait()
    xb = np.concatenate([a.ravel() for a in rr.x_samples()])
    rr.launch()
    rr.wait()
    assert np.array_equal(xb, np.concatenate([a.ravel() for a in rr.x_samples()]))
    w0, o = 0, 0
    for m, l in enumerate(lams):
        single = pmf.pmf_run_windows(sysh, l, pmf.make_params(run, chain=m, uid_base=w0 * run.replicas))
        xm = np.concatenate([a.ravel() for a in single.x_samples()])
        assert np.array_equal(xb[o:o + xm.size], xm), m
        o += xm.size
        w0 += l.size
    assert o == xb.size


def test_batch_free_energy_per_item(pmf):
    """pmf_free_energy_item = the reduction of the item's own samples (the
    same kernels on the same data); the whole-run calls refuse a batch."""
    params, starts, lams, run = _small_batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()
    w0 = 0
    for m, l in enumerate(lams):
        g = rr.free_energy_item(m, l.size)
        x = np.concatenate([xs[w0 + i].ravel() for i in range(l.size)])
        T = xs[w0].shape[1]
        h = pmf.pmf_free_energy_from_samples(x, l, run.replicas, [T] * l.size, run.k, run.kT)
        for key in h:
            np.testing.assert_array_equal(g[key], h[key], err_msg=key)
        o = est.free_energy_profile([xs[w0 + i].astype(np.float64) for i in range(l.size)], l, run.k, run.kT)
        np.testing.assert_allclose(g["dF_JE"], o["dF_JE"], atol=1e-10 * max(1.0, np.abs(o["dF_JE"]).max()))
        w0 += l.size
    with pytest.raises(pmf.PmfError) as e:
        rr.free_energy()
    assert e.value.status == pmf.PMF_EINVAL
    with pytest.raises(pmf.PmfError):
        rr.work_samples()


def test_batch_recaptures_after_warp_change(pmf):
    """Changing a chain's warps per replica between launches re-captures the
    graph; results stay within FP32 summation-order differences."""
    params, starts, lams, run = _small_batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.launch()
    rr.wait()
    p4, _ = rr.final_state()
    pmf.pmf_chain_set_warps(sysh, 1, 8)
    rr.launch()
    rr.wait()
    p8, _ = rr.final_state()
    assert np.abs(p8 - p4).max() <= 1e-4
    pmf.pmf_chain_set_warps(sysh, 1, 4)
    rr.launch()
    rr.wait()
    assert np.array_equal(rr.final_state()[0], p4)


def test_batch_1d_matches_oracle(pmf):
    """Two 1D paths with different grids in one batch, against the oracle."""
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.replicas = 3000, 300, 2
    lams = [np.array([-1.2, -0.6, 0.0]), np.array([0.3, 0.9])]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_batch_prepare(sysh, [(0, l) for l in lams], pmf.make_params(run))
    rr.launch()
    rr.wait()
    xs = rr.x_samples()
    lam_all = np.concatenate(lams)
    for wi in range(lam_all.size):
        for r in range(2):
            x, _ = _clib.od1d_run(w["a"], lam_all[wi], run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil,
                                  run.stride, run.seed, 2 * wi + r, w["x0"])
            np.testing.assert_allclose(xs[wi][r], x, atol=2e-6, rtol=0)


def test_batch_rejects_bad_items(pmf):
    params, starts, lams, run = _small_batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    for items in ([(3, lams[0])], [(0, np.array([1.0, 1.0]))], [(0, np.array([1.0, np.nan]))]):
        with pytest.raises(pmf.PmfError) as e:
            pmf.pmf_run_batch_prepare(sysh, items, pmf.make_params(run))
        assert e.value.status == pmf.PMF_EINVAL
    too_many = [(0, np.linspace(1.0, 2.0, 1000))] * 5
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_run_batch_prepare(sysh, too_many, pmf.make_params(run))
    assert e.value.status == pmf.PMF_EINVAL


@pytest.mark.parametrize("policy", [0, 1])
def test_full_batch_sampled_replicas(pmf, policy):
    """The 64-chain batch (N 40-400, 21-61 windows, 16 replicas; 2669
    windows, 42,704 replicas) in the launch configuration the benchmark
    times (one packed launch; policy 0 is the default, 1 the one the
    benchmark's autotuner picks), shortened to 200 steps: sampled replicas
    of the shortest, longest and four other chains against the oracle."""
    bw = inputs.batch_workload()
    run = bw["run"]
    run.n_steps, run.n_equil, run.stride = 200, 100, 100
    params, lams = bw["params"], bw["lambdas"]
    starts = [f32(s) for s in bw["starts"]]
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.set_batch_launch(pmf.PMF_BATCH_PACKED, policy)
    rr.launch()
    rr.wait()
    pos = _final_positions(rr, params, lams, run.replicas)
    n = np.array([p.n for p in params])
    pick = sorted({int(n.argmin()), int(n.argmax()), 5, 17, 33, 63})
    w0s = np.concatenate([[0], np.cumsum([l.size for l in lams])])
    jobs = []
    for m in pick:
        for w, r in ((0, 0), (lams[m].size - 1, run.replicas - 1), (lams[m].size // 2, 7)):
            jobs.append((m, w, r))

    def one(job):
        m, w, r = job
        ch = _clib.Chain(params[m])
        _, ro, _ = ch.run(starts[m], lams[m][w], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                          run.stride, run.seed, (w0s[m] + w) * run.replicas + r)
        return np.abs(pos[m][w, r] - ro).max()

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        errs = list(ex.map(one, jobs))
    assert max(errs) <= 1e-4, list(zip(jobs, errs))
