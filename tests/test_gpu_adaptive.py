"""GPU tests of the learned window placement: the overlap kernel against the
oracle's closed form, seeded runs against oracle runs from the same starts,
and the adaptive protocol on the 1D model against quadrature."""
import numpy as np
import pytest

from oracle import _clib, quadrature as quad, surrogate as sg
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def test_overlap_kernel_matches_oracle(pmf):
    rng = np.random.default_rng(3)
    mu = np.cumsum(rng.uniform(0.0, 0.3, 200))
    sd = rng.uniform(0.03, 0.2, 200)
    sd[50] = sd[51]  # equal widths: the closed form's special case
    got = pmf.pmf_overlap(mu, np.log(sd ** 2))
    want = np.array([sg.gaussian_overlap(mu[i], sd[i], mu[i + 1], sd[i + 1]) for i in range(199)])
    np.testing.assert_allclose(got, want, atol=1e-12, rtol=0)


def test_seeded_chain_run_matches_oracle(pmf):
    """Every replica from its own start state: 200 steps vs the oracle."""
    n = 40
    p = inputs.chain_params(n, 21)
    starts = [f32(inputs.chain_start(p, 50 + q)) for q in range(4)]
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=200, n_equil=100,
                             stride=100, replicas=2, seed=4)
    lam = np.array([1.1, 1.3])
    sysh = pmf.pmf_create_system_chain([p], [starts[0]])
    rr = pmf.pmf_run_prepare_seeded(sysh, lam, pmf.make_params(run), np.stack(starts))
    rr.launch()
    rr.wait()
    pos, _ = rr.final_state()
    pos = pos.reshape(2, 2, n, 3)
    ch = _clib.Chain(p)
    for w in range(2):
        for r in range(2):
            _, ro, _ = ch.run(starts[2 * w + r], lam[w], run.k, run.kT, run.dt, run.gamma, 200, 100, 100, 4,
                              2 * w + r)
            assert np.abs(pos[w, r] - ro).max() <= 1e-4


def test_seeded_1d_run_matches_oracle(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.replicas = 4000, 400, 3
    lam = np.array([-0.5, 0.2])
    starts = np.array([-1.0, -0.3, 0.4, 0.9, 1.2, -1.3])
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_prepare_seeded(sysh, lam, pmf.make_params(run), starts)
    rr.launch()
    rr.wait()
    xs = rr.x_samples()
    for wi in range(2):
        for r in range(3):
            x, _ = _clib.od1d_run(w["a"], lam[wi], run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil,
                                  run.stride, run.seed, 3 * wi + r, starts[3 * wi + r])
            np.testing.assert_allclose(xs[wi][r], x, atol=2e-6, rtol=0)


def test_adaptive_protocol_on_double_well(pmf):
    """From 6 coarse windows (spacing 0.6, about 3 standard deviations of x;
    overlaps 0.1 - 0.36) the surrogate inserts windows until neighbours
    overlap by at least 0.5; the resulting JE profile matches the quadrature
    at every final window."""
    w = inputs.od1d_workload()
    run = w["run"]
    lam0 = np.linspace(-1.5, 1.5, 6)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(sg.init_params(2))
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.5, max_rounds=4,
                                     max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5)
    assert meta["inserted"] > 0 and meta["n_windows"] == 6 + meta["inserted"]
    lam = meta["lambdas"]
    assert np.all(np.diff(lam) > 0)
    np.testing.assert_allclose(res["lambda"], lam)
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in lam])
    exact -= exact[0]
    err_adaptive = np.max(np.abs(res["dF_JE"] - exact))
    assert err_adaptive < 0.1
    # what the surrogate gains: the same 6 coarse windows without insertion
    plain = pmf.pmf_run_windows(sysh, lam0, pmf.make_params(run)).free_energy()
    exact0 = np.array([quad.od1d_free_energy(l, run.k) for l in lam0])
    exact0 -= exact0[0]
    err_plain = np.max(np.abs(plain["dF_JE"] - exact0))
    print(f"max |dF_JE - exact|: coarse grid {err_plain:.3f} kT, with learned insertion {err_adaptive:.3f} kT")
    assert err_plain > 2.0 * err_adaptive
    # neighbours now overlap (measured from the samples' own moments)
    sd = np.sqrt(res["var_x"])
    ovl = np.array([sg.gaussian_overlap(res["mean_x"][i], sd[i], res["mean_x"][i + 1], sd[i + 1])
                    for i in range(lam.size - 1)])
    assert np.median(ovl) > 0.4
    assert meta["gpu_seconds"] > 0


def test_adaptive_warp_choice_is_scoped(pmf):
    """The adaptive protocol may run its sparse launches with more warps per
    replica; the chain is back at its default afterwards, a warp count the
    caller chose is kept, and both runs give finite profiles on the same
    final grid size."""
    n = 40
    p = inputs.chain_params(n, 21)
    start = f32(inputs.chain_start(p, 50, target_x=1.0))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=400, n_equil=100,
                             stride=50, replicas=4, seed=3)
    lam0 = np.linspace(1.0, 1.6, 4)
    init = pmf.pack_mlp_params(sg.init_params(2))
    for chosen in (None, 6):
        sysh = pmf.pmf_create_system_chain([p], [start])
        if chosen is not None:
            pmf.pmf_chain_set_warps(sysh, 0, chosen)
        meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.3, max_rounds=1,
                                         max_windows=8, mlp_steps=50, mlp_batch=128, mlp_lr=3e-3, mlp_seed=1)
        assert pmf.pmf_chain_get_launch(sysh, 0)[0] == (4 if chosen is None else chosen)
        assert np.all(np.isfinite(res["dF_JE"])) and meta["gpu_seconds"] > 0
        sysh.close()


def _check_decisions(meta, threshold, max_windows, R):
    """Every round's inserted centres are the oracle's insert_windows on the
    round's own windows and surrogate predictions (its OVL values are the
    oracle's closed form to 1e-10), the next round starts from the union,
    and every replica of an inserted window started from the candidate the
    oracle's seed_order ranks at r mod (2 R)."""
    tr = meta["trace"]
    assert len(tr) >= 1
    for q, rd in enumerate(tr):
        lam, mu, lv = rd["lambdas"], rd["mu"], rd["log_var"]
        if rd["trained"] == 0:
            # the gate closed: no measured gap, no training, nothing inserted
            assert q == len(tr) - 1 and rd["inserted"].size == 0
            assert np.all(rd["data_ovl"] >= threshold) and np.all(np.isnan(mu))
            continue
        assert rd["trained"] == 1
        sd = np.exp(0.5 * lv)
        ovl_o = np.array([sg.gaussian_overlap(mu[i], sd[i], mu[i + 1], sd[i + 1]) for i in range(lam.size - 1)])
        np.testing.assert_allclose(rd["ovl"], ovl_o, rtol=0, atol=1e-10)
        want = sg.insert_windows(lam, mu, lv, threshold)[: max(0, max_windows - lam.size)]
        np.testing.assert_array_equal(rd["inserted"], want)
        for j, lam_new in enumerate(rd["inserted"]):
            i = int(np.searchsorted(lam, lam_new))  # between windows i - 1 and i
            assert lam[i - 1] < lam_new < lam[i]
            order = sg.seed_order(rd["cand_x"][j], rd["target"][j])
            np.testing.assert_array_equal(rd["seed"][j], order[np.arange(R) % order.size])
        if q + 1 < len(tr):
            np.testing.assert_array_equal(tr[q + 1]["lambdas"], np.sort(np.concatenate([lam, rd["inserted"]])))
    assert meta["inserted"] == sum(rd["inserted"].size for rd in tr)


def test_adaptive_decisions_match_oracle_1d(pmf):
    w = inputs.od1d_workload()
    run = w["run"]
    lam0 = np.linspace(-1.5, 1.5, 6)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(sg.init_params(2))
    meta, _ = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.5, max_rounds=4,
                                   max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5,
                                   trace=True)
    assert meta["inserted"] > 0
    _check_decisions(meta, 0.5, 64, run.replicas)
    # the final grid is the last round's windows plus its insertions
    last = meta["trace"][-1]
    np.testing.assert_array_equal(meta["lambdas"], np.sort(np.concatenate([last["lambdas"], last["inserted"]])))


def test_adaptive_decisions_match_oracle_chain(pmf):
    """A 40-bead chain on a coarse grid (and a window cap that bites): the
    seeding candidates are chain end states, their x the end-to-end
    distances."""
    n = 40
    p = inputs.chain_params(n, 21)
    start = f32(inputs.chain_start(p, 50, target_x=1.0))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=2000, n_equil=200,
                             stride=50, replicas=6, seed=3)
    lam0 = np.linspace(1.0, 1.9, 4)
    sysh = pmf.pmf_create_system_chain([p], [start])
    init = pmf.pack_mlp_params(sg.init_params(2))
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.3, max_rounds=2,
                                     max_windows=9, mlp_steps=300, mlp_batch=256, mlp_lr=3e-3, mlp_seed=2,
                                     trace=True)
    assert meta["inserted"] > 0
    _check_decisions(meta, 0.3, 9, run.replicas)
    assert np.all(np.isfinite(res["dF_JE"]))


def test_adaptive_decisions_with_continuation(pmf):
    """With continue_windows every round runs all windows in one launch; the
    decisions are still the oracle's."""
    w = inputs.od1d_workload()
    run = w["run"]
    lam0 = np.linspace(-1.5, 1.5, 6)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(sg.init_params(2))
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.5, max_rounds=3,
                                     max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5,
                                     trace=True, continue_windows=True)
    assert meta["inserted"] > 0
    _check_decisions(meta, 0.5, 64, run.replicas)
    last = meta["trace"][-1]
    np.testing.assert_array_equal(meta["lambdas"], np.sort(np.concatenate([last["lambdas"], last["inserted"]])))
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in meta["lambdas"]])
    exact -= exact[0]
    assert np.max(np.abs(res["dF_JE"] - exact)) < 0.1


def test_continued_windows_resume_their_replicas(pmf):
    """One round with continuation on the 1D model: each original window's
    replica r runs again from replica r's end state of the coarse run (fresh
    uids after the coarse run's), so its mean x equals the oracle's from that
    start with those uids."""
    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil = 6000, 600
    lam0 = np.linspace(-1.5, 1.5, 6)
    R = run.replicas
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    coarse = pmf.pmf_run_windows(sysh, lam0, pmf.make_params(run))
    x_end = coarse.final_state()[0].reshape(lam0.size, R)
    init = pmf.pack_mlp_params(sg.init_params(2))
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.5, max_rounds=1,
                                     max_windows=64, mlp_steps=200, mlp_batch=256, mlp_lr=3e-3, mlp_seed=5,
                                     trace=True, continue_windows=True)
    lam = meta["lambdas"]
    assert meta["inserted"] > 0 and lam.size == lam0.size + meta["inserted"]
    for i, l in enumerate(lam0):
        j = int(np.where(lam == l)[0][0])
        xs = [_clib.od1d_run(w["a"], l, run.k, run.kT, run.gamma, run.dt, run.n_steps, run.n_equil, run.stride,
                             run.seed, lam0.size * R + j * R + r, x_end[i, r])[0] for r in range(R)]
        want = float(np.mean(np.concatenate(xs).astype(np.float32).astype(np.float64)))
        assert abs(res["mean_x"][j] - want) < 1e-6, (i, res["mean_x"][j], want)


def _uniform_samples(pmf, sysh, lam0, run):
    """The coarse run a protocol starts with (uids from 0), run on its own."""
    return pmf.pmf_run_windows(sysh, lam0, pmf.make_params(run)).x_samples()


def test_gate_skips_training_without_a_gap(pmf):
    """11 windows on the 1D well (spacing 0.3): every measured neighbour
    overlap is above 0.3, so the gated protocol stops in round 0 without
    training; its measured overlaps are the oracle's from the same samples,
    and its final profile is the coarse run's."""
    w = inputs.od1d_workload()
    run = w["run"]
    lam0 = np.linspace(-1.5, 1.5, 11)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(sg.init_params(2))
    xs = _uniform_samples(pmf, sysh, lam0, run)
    want_ovl = sg.measured_overlaps(xs)
    assert not sg.needs_training(xs, 0.3)
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.3, max_rounds=3,
                                     max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5,
                                     trace=True, train_on_gap=True)
    tr = meta["trace"]
    assert len(tr) == 1 and tr[0]["trained"] == 0 and meta["inserted"] == 0 and meta["rounds"] == 0
    np.testing.assert_allclose(tr[0]["data_ovl"], want_ovl, rtol=0, atol=1e-10)
    plain = pmf.pmf_run_windows(sysh, lam0, pmf.make_params(run)).free_energy()
    np.testing.assert_allclose(res["dF_JE"], plain["dF_JE"], rtol=1e-12, atol=1e-12)
    _check_decisions(meta, 0.3, 64, run.replicas)
    # ungated, the same protocol trains in round 0 and takes longer
    meta2, _ = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, threshold=0.3, max_rounds=3,
                                    max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5,
                                    trace=True)
    assert meta2["trace"][0]["trained"] == 1
    assert meta["gpu_seconds"] < meta2["gpu_seconds"]


def test_gate_opens_on_a_gap_and_decides_as_ungated(pmf):
    """6 windows (spacing 0.6) with threshold 0.5: the measured overlaps
    (the oracle's, from the coarse run's samples) show a gap, so round 0
    trains and inserts exactly what the ungated protocol inserts; every
    later round either trains on a measured gap or ends the protocol."""
    w = inputs.od1d_workload()
    run = w["run"]
    lam0 = np.linspace(-1.5, 1.5, 6)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    init = pmf.pack_mlp_params(sg.init_params(2))
    xs = _uniform_samples(pmf, sysh, lam0, run)
    assert sg.needs_training(xs, 0.5)
    kw = dict(threshold=0.5, max_rounds=4, max_windows=64, mlp_steps=400, mlp_batch=512, mlp_lr=3e-3, mlp_seed=5,
              trace=True, continue_windows=True)
    meta, res = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, train_on_gap=True, **kw)
    ref, _ = pmf.pmf_run_adaptive(sysh, lam0, pmf.make_params(run), init, **kw)
    tr = meta["trace"]
    assert tr[0]["trained"] == 1
    np.testing.assert_allclose(tr[0]["data_ovl"], sg.measured_overlaps(xs), rtol=0, atol=1e-10)
    for key in ("mu", "log_var", "ovl", "inserted", "target", "seed"):
        np.testing.assert_array_equal(tr[0][key], ref["trace"][0][key])
    _check_decisions(meta, 0.5, 64, run.replicas)
    for rd in tr:
        assert rd["trained"] == int(np.any(rd["data_ovl"] < 0.5))
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in meta["lambdas"]])
    assert np.max(np.abs(res["dF_JE"] - (exact - exact[0]))) < 0.1
