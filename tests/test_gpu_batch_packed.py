"""The packed persistent launch of batched runs: one kernel launch per
1e5-step chunk for the whole batch, CTAs of 16 warps taking (segment, pack)
items, a pack being up to 16 / G replicas of one item simulated by teams of
G warps.  Every replica runs the force schedule of G warps, so a packed
batch is bit-identical to the per-item launches with G warps per replica;
every packing policy agrees with the FP64 oracle per replica."""
import time

import numpy as np
import pytest

from oracle import _clib
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def _batch(lengths=(40, 57, 75, 104, 150), n_win=(2, 3, 2, 2, 1), replicas=3, n_steps=300):
    params = [inputs.chain_params(n, 70 + i) for i, n in enumerate(lengths)]
    starts = [f32(inputs.chain_start(p, 90 + i)) for i, p in enumerate(params)]
    lams = [np.linspace(1.0, 1.6, s) + 0.1 * i for i, s in enumerate(n_win)]
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=n_steps,
                             n_equil=n_steps // 2, stride=50, replicas=replicas, seed=13)
    return params, starts, lams, run


def test_packed_is_the_default_and_equals_graph_with_the_same_teams(pmf):
    """Under policy 2 every chain of this batch gets teams of 8 warps; the
    graph of per-item launches with 8 warps per replica gives the same
    samples bit for bit, and so does a repeat of the packed launch."""
    params, starts, lams, run = _batch()
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    info = rr.batch_launch()
    assert info["mode"] == pmf.PMF_BATCH_PACKED and info["policy"] == 0
    assert np.all(info["teams"] >= 4) and info["packs"] >= 1 and info["ctas"] >= 1
    rr.set_batch_launch(pmf.PMF_BATCH_PACKED, 2)
    info = rr.batch_launch()
    assert np.all(info["teams"] == 8), info
    rr.launch()
    rr.wait()
    xp = np.concatenate([a.ravel() for a in rr.x_samples()])
    rr.launch()
    rr.wait()
    assert np.array_equal(xp, np.concatenate([a.ravel() for a in rr.x_samples()]))
    for m in range(len(params)):
        pmf.pmf_chain_set_warps(sysh, m, 8)
    rg = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rg.set_batch_launch(pmf.PMF_BATCH_GRAPH)
    assert rg.batch_launch()["mode"] == pmf.PMF_BATCH_GRAPH
    rg.launch()
    rg.wait()
    assert np.array_equal(xp, np.concatenate([a.ravel() for a in rg.x_samples()]))


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_every_policy_matches_oracle(pmf, policy):
    """Teams of 2, 4, 8 and 16 warps (the policies pick different ones per
    chain length): every replica's final state within 1e-4 nm of the oracle
    after 200 steps (the trajectory tolerance), x samples within 1e-4 nm."""
    params, starts, lams, run = _batch(lengths=(40, 104, 260), n_win=(2, 2, 1), replicas=2, n_steps=200)
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    rr.set_batch_launch(pmf.PMF_BATCH_PACKED, policy)
    rr.launch()
    rr.wait()
    pos, _ = rr.final_state()
    xs = rr.x_samples()
    o, w0 = 0, 0
    for m, (p, l) in enumerate(zip(params, lams)):
        ch = _clib.Chain(p)
        n = l.size * run.replicas * p.n * 3
        pm = pos[o:o + n].reshape(l.size, run.replicas, p.n, 3)
        o += n
        for w in range(l.size):
            for r in range(run.replicas):
                uid = (w0 + w) * run.replicas + r
                xo, ro, _ = ch.run(starts[m], l[w], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                                   run.stride, run.seed, uid)
                assert np.abs(pm[w, r] - ro).max() <= 1e-4, (policy, m, w, r)
                np.testing.assert_allclose(xs[w0 + w][r], xo, atol=1e-4, rtol=0)
        w0 += l.size


def test_autotune_keeps_a_working_launch(pmf):
    params, starts, lams, run = _batch(n_steps=2000)
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    ms = rr.batch_autotune(500)
    assert ms > 0
    info = rr.batch_launch()
    assert info["mode"] in (pmf.PMF_BATCH_GRAPH, pmf.PMF_BATCH_PACKED)
    rr.launch()
    rr.wait()
    ref = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run))
    ref.set_batch_launch(info["mode"], info["policy"])
    ref.launch()
    ref.wait()
    for a, b in zip(rr.x_samples(), ref.x_samples()):
        np.testing.assert_array_equal(a, b)


def test_packed_refusals_and_fp64_default(pmf):
    params, starts, lams, run = _batch(lengths=(40, 57), n_win=(2, 2))
    s64 = pmf.pmf_create_system_chain(params, starts, precision=pmf.PMF_FP64)
    r64 = pmf.pmf_run_batch_prepare(s64, list(enumerate(lams)), pmf.make_params(run))
    assert r64.batch_launch()["mode"] == pmf.PMF_BATCH_GRAPH
    with pytest.raises(pmf.PmfError) as e:
        r64.set_batch_launch(pmf.PMF_BATCH_PACKED, 0)
    assert e.value.status == pmf.PMF_EINVAL
    s32 = pmf.pmf_create_system_chain(params, starts)
    r32 = pmf.pmf_run_batch_prepare(s32, list(enumerate(lams)), pmf.make_params(run))
    for bad in ((7, 0), (pmf.PMF_BATCH_PACKED, 3)):
        with pytest.raises(pmf.PmfError) as e:
            r32.set_batch_launch(*bad)
        assert e.value.status == pmf.PMF_EINVAL


def test_packed_host_timeout_stops_the_launch(pmf):
    """The packed kernel polls the host-mapped stop flag between work items:
    a long batch with a 0.2 s limit returns PMF_ETIMEOUT long before it
    would have ended."""
    params, starts, lams, run = _batch(replicas=8, n_steps=2000000)
    sysh = pmf.pmf_create_system_chain(params, starts)
    rr = pmf.pmf_run_batch_prepare(sysh, list(enumerate(lams)), pmf.make_params(run, timeout_s=0.2))
    assert rr.batch_launch()["mode"] == pmf.PMF_BATCH_PACKED
    rr.launch()
    t0 = time.perf_counter()
    with pytest.raises(pmf.PmfError) as e:
        rr.wait()
    assert e.value.status == pmf.PMF_ETIMEOUT
    assert time.perf_counter() - t0 < 2.0
