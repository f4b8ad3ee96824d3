"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs."""
import math

import numpy as np
import pytest

from oracle import _clib, estimators as est, quadrature as quad
from paper_1105_4840_gb300 import inputs
from tests.helpers import f32, oracle_chain_samples, oracle_od1d_samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


# ---------------------------------------------------------------- Philox

def test_philox_bitwise_and_normals(pmf):
    for seed, c0, c1, c2, c3 in ((0, 0, 0, 0, 0), (0xDEADBEEF12345678, 0xFFFFFF00, 17, 400000, 1)):
        n = 100000
        raw_g, nor_g = pmf.pmf_philox(seed, c0, c1, c2, c3, n)
        raw_o, nor_o = _clib.philox_bulk(seed, c0, c1, c2, c3, n)
        np.testing.assert_array_equal(raw_g, raw_o)
        # FP32 Box-Muller error bound.  u = (b + 1/2) 2^-32 rounded to FP32:
        # du/u <= 2^-23.  __logf: abs error <= 2^-21.41 on [0.5, 2], else 3 ulp,
        # so d(r^2) <= 9.6e-7 + 3.6e-7 r^2 with r^2 = -2 ln u, and
        # dr <= min(d(r^2) / 2r, sqrt(d(r^2))) + 1 ulp.  The angle
        # 2 pi (u - 1/2) is off by <= 1.2e-6 and __sincosf adds <= 2^-21.19,
        # so the cos/sin factor is off by <= 1.7e-6.
        u = (raw_o.astype(np.float64) + 0.5) / 2.0 ** 32
        r = np.sqrt(-2.0 * np.log(u[:, [0, 0, 2, 2]]))
        dr2 = 9.6e-7 + 3.6e-7 * r * r
        dr = np.minimum(dr2 / (2.0 * np.maximum(r, 1e-30)), np.sqrt(dr2)) + 1.2e-7 * r
        bound = 1.25 * (1.7e-6 * r + dr + 1.2e-7 * np.abs(nor_o))
        assert np.all(np.abs(nor_g - nor_o) <= bound)


# ---------------------------------------------------------------- forces

@pytest.mark.parametrize("n", [4, 5, 8, 13, 31, 32, 33, 40, 63, 64, 100, 104, 110, 120, 128, 200, 333, 400])
def test_forces_match_oracle(pmf, n):
    p = inputs.chain_params(n, 100 + n)
    r = f32(inputs.chain_start(p, 7 + n) + np.random.default_rng(n).normal(0, 0.005, (n, 3)))
    lam, k = 1.7, 500.0
    sysh = pmf.pmf_create_system_chain([p], [r])
    fg = pmf.pmf_chain_forces(sysh, 0, r, lam, k)
    fo = _clib.Chain(p).forces(r, lam, k)
    rel = np.linalg.norm(fg - fo) / np.linalg.norm(fo)
    assert rel <= 1e-5, rel
    assert np.abs(fg - fo).max() <= 1e-5 * np.abs(fo).max()
    sys64 = pmf.pmf_create_system_chain([p], [r], precision=pmf.PMF_FP64)
    f64 = pmf.pmf_chain_forces(sys64, 0, r, lam, k)
    assert np.linalg.norm(f64 - fo) / np.linalg.norm(fo) <= 1e-12


@pytest.mark.parametrize("variant", range(6))
@pytest.mark.parametrize("n", [40, 104, 200])
def test_forces_every_schedule_variant(pmf, n, variant):
    """Every cost model of the FP32 schedule gives the oracle's forces (the
    variants only move pieces between warps)."""
    p = inputs.chain_params(n, 300 + n)
    r = f32(inputs.chain_start(p, 9 + n) + np.random.default_rng(n + variant).normal(0, 0.005, (n, 3)))
    sysh = pmf.pmf_create_system_chain([p], [r])
    pmf.pmf_chain_set_schedule(sysh, 0, variant)
    assert pmf.pmf_chain_get_schedule(sysh, 0) == variant
    fg = pmf.pmf_chain_forces(sysh, 0, r, 1.7, 500.0)
    fo = _clib.Chain(p).forces(r, 1.7, 500.0)
    assert np.linalg.norm(fg - fo) / np.linalg.norm(fo) <= 1e-5
    with pytest.raises(pmf.PmfError):
        pmf.pmf_chain_set_schedule(sysh, 0, 6)


def test_forces_without_nonbonded_and_angles(pmf):
    n = 37
    p = inputs.gaussian_chain_params(n, 80.0)
    r = f32(np.random.default_rng(3).normal(0, 0.5, (n, 3)))
    sysh = pmf.pmf_create_system_chain([p], [r])
    fg = pmf.pmf_chain_forces(sysh, 0, r, 1.0, 30.0)
    fo = _clib.Chain(p).forces(r, 1.0, 30.0)
    assert np.linalg.norm(fg - fo) / np.linalg.norm(fo) <= 1e-5


# ---------------------------------------------------------------- trajectory

def _run_chain(pmf, p, start, run, lambdas, precision=0, n_steps_per_window=None, timeout_s=0.0):
    sysh = pmf.pmf_create_system_chain([p], [start], precision=precision)
    run_ = pmf.pmf_run_windows(sysh, lambdas, pmf.make_params(run, n_steps_per_window=n_steps_per_window,
                                                              timeout_s=timeout_s))
    return sysh, run_


def test_trajectory_200_steps(pmf):
    """200 BAOAB steps from identical state and Philox noise: FP32 GPU within
    1e-4 nm of the FP64 oracle (FP64 GPU within 1e-9 nm)."""
    p = inputs.chain_params(104, 1)
    start = f32(inputs.chain_start(p, 1001, target_x=1.3))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=200,
                             n_equil=100, stride=100, replicas=2, seed=0)
    lam = np.array([1.3, 1.4])
    ch = _clib.Chain(p)
    for prec, tol in ((0, 1e-4), (1, 1e-9)):
        _, rr = _run_chain(pmf, p, start, run, lam, precision=prec)
        pos, vel = rr.final_state()
        pos = pos.reshape(2, 2, 104, 3)
        for w in range(2):
            for r in range(2):
                _, ro, _ = ch.run(start, lam[w], run.k, run.kT, run.dt, run.gamma, 200, 100, 100, 0, w * 2 + r)
                err = np.abs(pos[w, r] - ro).max()
                assert err <= tol, (prec, w, r, err)


# ---------------------------------------------------------------- reductions

def _compare_profiles(g, o, kT, rel=1e-12):
    for key in ("dF_JE", "dF_fluct", "dF_G", "dF_com", "uncertainty", "W_mean", "acc_force"):
        scale = np.maximum(np.abs(o[key]), kT)
        assert np.all(np.abs(g[key] - o[key]) <= rel * scale), key
    for key in ("mean_x", "var_x", "gamma2"):
        np.testing.assert_allclose(g[key], o[key], rtol=1e-10, err_msg=key)
    for key in ("se_JE", "se_fluct", "var_ZW"):
        np.testing.assert_allclose(g[key], o[key], rtol=1e-8, equal_nan=True, err_msg=key)


@pytest.mark.parametrize("s,R,T", [(21, 32, 3600), (5, 3, 1), (7, 1, 50), (4, 300, 129)])
def test_reduction_parity(pmf, s, R, T):
    """Eq. (9)/(12)/(13)/(14) reductions on identical samples: <= 1e-12 relative."""
    lam = inputs.lambda_grid(1.3, 3.3, s)
    k, kT = 500.0, inputs.kT_of(300.0)
    x = inputs.gaussian_x_samples(lam, k, kT, R, T, seed=s * 1000 + R)
    g = pmf.pmf_free_energy_from_samples(x.ravel(), lam, R, [T] * s, k, kT)
    o = est.free_energy_profile([x[i].astype(np.float64) for i in range(s)], lam, k, kT)
    _compare_profiles(g, o, kT)


@pytest.mark.parametrize("case", ["decreasing", "wide", "flat_step", "sign_change"])
def test_reduction_exponent_range(pmf, case):
    """The stage-1 exponential on the FP32 pipe against the oracle's FP64
    one, <= 1e-12 relative: a path pulled towards smaller lambda (the
    minimum of w at the smallest x), samples spread so far beyond the trap's
    width that exponents pass -80 (those terms are dropped), two equal
    neighbouring centres (w = 0 for every sample), and samples on both
    sides of zero."""
    g = np.random.default_rng(["decreasing", "wide", "flat_step", "sign_change"].index(case) + 77)
    R, T = 6, 700
    kT = inputs.kT_of(300.0)
    if case == "decreasing":
        lam, k, sd = inputs.lambda_grid(3.3, 1.3, 11), 500.0, 0.07
    elif case == "wide":
        lam, k, sd = inputs.lambda_grid(1.3, 2.3, 11), 20000.0, 0.05
    elif case == "flat_step":
        lam, k, sd = np.array([1.3, 1.5, 1.5, 1.7, 1.9]), 500.0, 0.07
    else:
        lam, k, kT, sd = inputs.lambda_grid(-1.5, 1.5, 9), 20.0, 1.0, 0.3
    x = (lam[:, None, None] + sd * g.standard_normal((lam.size, R, T))).astype(np.float32)
    gpu = pmf.pmf_free_energy_from_samples(x.ravel(), lam, R, [T] * lam.size, k, kT)
    o = est.free_energy_profile([x[i].astype(np.float64) for i in range(lam.size)], lam, k, kT)
    _compare_profiles(gpu, o, kT)


@pytest.mark.parametrize("R", [300, 16384, 20000])
def test_combination_many_replicas(pmf, R):
    """The per-window combination and its delete-one-replica jackknife on
    synthetic per-replica partials with one replica dominating the
    exponential sums (the leave-one-out sum then cancels almost all of the
    total): 16384 replicas keep their sums in shared memory, 20000 take the
    other branch.  Against the oracle's combination of the same partials."""
    s, k, kT = 3, 500.0, inputs.kT_of(300.0)
    lam = np.array([1.3, 1.4, 1.55])
    g = np.random.default_rng(R)
    P = np.zeros((s, R, 5))
    T = 50.0
    P[:, :, 0] = 1.0 + 0.5 * g.standard_normal((s, R))      # min w
    P[:, :, 1] = 1.0 + 10.0 * g.random((s, R))               # shifted exponential sum
    P[:, :, 2] = T
    P[:, :, 3] = T * 0.02 * g.standard_normal((s, R))        # sum (x - lambda)
    P[:, :, 4] = T * 0.003 + np.abs(P[:, :, 3]) ** 2 / T     # sum (x - lambda)^2
    P[0, R // 3, 0] -= 40.0 * kT                             # this replica's weight dominates window 0
    got = pmf.pmf_free_energy_from_partials(P, lam, k, kT)
    want = est.free_energy_from_partials(P, lam, k, kT)
    _compare_profiles(got, want, kT)


def test_reduction_ragged_and_device_pointer(pmf):
    torch = pytest.importorskip("torch")
    lam = np.array([-1.5, -1.2, -1.0, -0.2, 0.4, 1.5])
    k, kT = 20.0, 1.0
    R = 5
    T = [10, 333, 1, 77, 2048, 9]
    g = np.random.default_rng(4)
    blocks = [(l + 0.1 * g.standard_normal((R, t))).astype(np.float32) for l, t in zip(lam, T)]
    flat = np.concatenate([b.ravel() for b in blocks])
    o = est.free_energy_profile([b.astype(np.float64) for b in blocks], lam, k, kT)
    gh = pmf.pmf_free_energy_from_samples(flat, lam, R, T, k, kT)
    _compare_profiles(gh, o, kT)
    xd = torch.from_numpy(flat).cuda()
    gd = pmf.pmf_free_energy_from_samples(xd.data_ptr(), lam, R, T, k, kT, x_on_device=True)
    torch.cuda.synchronize()
    for key in gh:
        np.testing.assert_array_equal(gd[key], gh[key])


# ---------------------------------------------------------------- 1D model

def test_od1d_workload_parity_and_quadrature(pmf):
    """Full 1D workload: FP64 GPU samples equal the oracle's to FP32 storage
    rounding; the JE profile is within 0.1 kT of the quadrature."""
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    xg = rr.x_samples()
    xo = oracle_od1d_samples(w["a"], w["x0"], run)
    for i in range(len(xo)):
        np.testing.assert_allclose(xg[i], xo[i], atol=2e-6, rtol=0)
    g = rr.free_energy()
    o = est.free_energy_profile(xo, run.lambdas, run.k, run.kT)
    assert np.max(np.abs(g["dF_JE"] - o["dF_JE"])) < 1e-4
    exact = np.array([quad.od1d_free_energy(l, run.k) for l in run.lambdas])
    exact -= exact[0]
    assert np.max(np.abs(g["dF_JE"] - exact)) < 0.1
    # work samples of Eq. (9) against the oracle's work on its own samples
    wg = rr.work_samples(pmf.PMF_WORK_PER_WINDOW_INCREMENT)
    wo = np.concatenate([est.work_increment(xo[i], run.lambdas[i], run.lambdas[i + 1], run.k).ravel()
                         for i in range(len(xo) - 1)])
    np.testing.assert_allclose(wg, wo, atol=run.k * 0.15 * 2 * 2e-6 + 1e-12)
    wp = rr.work_samples(pmf.PMF_WORK_PAIRED_CUMULATIVE).reshape(len(xo) - 1, run.replicas, -1)
    cum = np.cumsum(np.stack([est.work_increment(xo[i], run.lambdas[i], run.lambdas[i + 1], run.k)
                              for i in range(len(xo) - 1)]), axis=0)
    np.testing.assert_allclose(wp, cum, atol=1e-4)


# ---------------------------------------------------------------- chain, statistics

def test_chain_free_energy_within_two_se_of_oracle(pmf):
    """104-bead chain, 3 windows x 8 replicas: GPU FP32 and oracle FP64 runs
    (same Philox streams) give dF within 2 combined standard errors."""
    p = inputs.chain_params(104, 1)
    start = inputs.chain_start(p, 1001, target_x=1.3)
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=3000,
                             n_equil=1000, stride=10, replicas=8, seed=0)
    lam = np.array([1.30, 1.35, 1.40])
    _, rr = _run_chain(pmf, p, f32(start), run, lam)
    g = rr.free_energy()
    xo = oracle_chain_samples(p, start, lam, run)
    o = est.free_energy_profile(xo, lam, run.k, run.kT)
    for key, sek in (("dF_JE", "se_JE"), ("dF_fluct", "se_fluct")):
        se = np.sqrt(g[sek] ** 2 + o[sek] ** 2)
        assert np.all(np.abs(g[key] - o[key])[1:] <= 2.0 * se[1:] + 1e-9), (key, g[key], o[key], se)


def test_chain_full_path_within_two_se_of_oracle(pmf):
    """The 104-bead workload's whole path (21 windows, 1.3 -> 3.3 nm) at 16
    replicas x 2e4 steps per window, same Philox streams on both sides: the
    FP32 GPU run's dF^JE(lambda_s) and dF_fluct(lambda_s) within 2 combined
    jackknife standard errors of the FP64 oracle's (trajectories decorrelate
    within a few thousand steps, so the comparison is statistical); every
    other profile point within 3."""
    w = inputs.chain_workload(n_steps=20000, replicas=16)
    p, start, run = w["params"], w["start"], w["run"]
    lam = run.lambdas
    assert lam.size == 21
    _, rr = _run_chain(pmf, p, f32(start), run, lam)
    g = rr.free_energy()
    xo = oracle_chain_samples(p, start, lam, run)
    o = est.free_energy_profile(xo, lam, run.k, run.kT)
    for key, sek in (("dF_JE", "se_JE"), ("dF_fluct", "se_fluct")):
        se = np.hypot(g[sek], o[sek])
        z = (g[key] - o[key])[1:] / se[1:]
        print(key, "end", g[key][-1], o[key][-1], "z", np.round(z, 2))
        assert abs(z[-1]) <= 2.0, (key, g[key][-1], o[key][-1], se[-1])
        assert np.all(np.abs(z) <= 3.0), (key, z)


def test_gaussian_chain_matches_radial_quadrature(pmf):
    """Bond-only chain (r0 = 0): <x> in each window equals the radial
    quadrature of the Gaussian end-to-end distribution in the trap."""
    n, kb, k = 6, 50.0, 20.0
    p = inputs.gaussian_chain_params(n, kb)
    kT = inputs.kT_of(300.0)
    start = np.zeros((n, 3))
    start[:, 0] = np.linspace(0, 1.0, n)
    run = inputs.RunSettings(k=k, kT=kT, dt=0.01, gamma=5.0, n_steps=40000, n_equil=2000, stride=10,
                             replicas=32, seed=5)
    lam = np.array([0.6, 1.0, 1.4])
    _, rr = _run_chain(pmf, p, start, run, lam)
    xs = rr.x_samples()
    s2 = (n - 1) * kT / kb
    for i, l in enumerate(lam):
        rm = xs[i].mean(axis=1)
        se = rm.std(ddof=1) / math.sqrt(rm.size)
        assert abs(rm.mean() - quad.gaussian_chain_mean_x(l, k, s2, kT)) < 4 * se + 1e-3


# ---------------------------------------------------------------- failure paths

def test_nonfinite_trajectory_sets_enumeric(pmf):
    p = inputs.chain_params(40, 2)
    start = inputs.chain_start(p, 3)
    start[20] = start[5]  # two beads on top of each other: infinite LJ force
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=500,
                             n_equil=0, stride=10, replicas=2, seed=0)
    with pytest.raises(pmf.PmfError) as e:
        _run_chain(pmf, p, start, run, np.array([1.0, 1.1]))
    assert e.value.status == pmf.PMF_ENUMERIC


def test_timeout_is_reported(pmf):
    p = inputs.chain_params(104, 1)
    start = inputs.chain_start(p, 1001, target_x=1.3)
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=200000,
                             n_equil=1000, stride=100, replicas=4, seed=0)
    with pytest.raises(pmf.PmfError) as e:
        _run_chain(pmf, p, start, run, np.array([1.3, 1.4]), timeout_s=1e-4)
    assert e.value.status == pmf.PMF_ETIMEOUT


def test_repeat_launch_is_bit_identical(pmf):
    p = inputs.chain_params(70, 4)
    start = inputs.chain_start(p, 5)
    run = inputs.RunSettings(k=300.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=2000,
                             n_equil=200, stride=20, replicas=3, seed=9)
    sysh, rr = _run_chain(pmf, p, start, run, np.array([1.5, 1.6, 1.8]))
    a = rr.x_samples()
    rr.launch()
    rr.wait()
    b = rr.x_samples()
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("warps", [4, 5, 6, 8])
@pytest.mark.parametrize("n", [13, 40, 104, 110, 333])
def test_forces_other_warp_counts(pmf, n, warps):
    """Same thermal-like states as test_forces_match_oracle (bonds off their
    rest length by ~0.005 nm): at exact rest lengths the FP32 rounding of a
    0.15 nm bond vector (~1.5e-8 nm) times k_b = 2.5e5 leaves an absolute
    floor of ~4e-3 kJ/mol/nm per bond that a norm-wise 1e-5 criterion on
    near-zero total forces cannot absorb."""
    p = inputs.chain_params(n, 300 + n)
    r = f32(inputs.chain_start(p, 17 + n) + np.random.default_rng(n + 1).normal(0, 0.005, (n, 3)))
    sysh = pmf.pmf_create_system_chain([p], [r])
    pmf.pmf_chain_set_warps(sysh, 0, warps)
    fg = pmf.pmf_chain_forces(sysh, 0, r, 2.0, 400.0)
    fo = _clib.Chain(p).forces(r, 2.0, 400.0)
    assert np.linalg.norm(fg - fo) / np.linalg.norm(fo) <= 1e-5


def test_autotune_picks_a_valid_count_and_runs(pmf):
    p = inputs.chain_params(104, 1)
    start = inputs.chain_start(p, 1001, target_x=1.3)
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=600, n_equil=100,
                             stride=50, replicas=4, seed=0)
    lam = inputs.lambda_grid(1.3, 1.6, 4)
    sysh = pmf.pmf_create_system_chain([p], [f32(start)])
    best, ms = pmf.pmf_chain_autotune(sysh, lam, pmf.make_params(run), probe_steps=200)
    assert best in (4, 5, 6, 8) and ms > 0
    rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    assert np.all(np.isfinite(rr.free_energy()["dF_JE"]))


@pytest.mark.parametrize("prec,per_window", [(0, False), (1, False), (0, True)])
def test_persistent_grid_is_bit_identical(pmf, prec, per_window):
    """Persistent launches (replicas migrating between CTAs in segments of a
    few steps, fewer CTAs than replicas) reproduce the one-CTA-per-replica
    trajectories and samples bit for bit, for FP32 and FP64 integration."""
    p = inputs.chain_params(70, 3)
    start = f32(inputs.chain_start(p, 1003, target_x=1.2))
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=330, n_equil=30,
                             stride=20, replicas=5, seed=11)
    lam = np.array([1.2, 1.5, 1.8, 2.1])
    sysh = pmf.pmf_create_system_chain([p], [start], precision=prec)
    out = []
    for ctas, seg in ((-1, 0), (7, 45), (0, 1000), (3, 1)):
        pmf.pmf_chain_set_grid(sysh, 0, ctas, seg)
        spw = [330, 200, 330, 60] if per_window else None
        rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run, n_steps_per_window=spw))
        out.append((np.concatenate([a.ravel() for a in rr.x_samples()]), rr.final_state()[0]))
    for x, pos in out[1:]:
        assert np.array_equal(x, out[0][0])
        assert np.array_equal(pos, out[0][1])


def test_partials_export_and_shard_merge(pmf):
    """pmf_run_partials against the oracle's partials of the same samples;
    combining a run's own partials reproduces pmf_free_energy bit for bit;
    two shards (disjoint uid blocks) merged by replica concatenation equal the
    reduction of their pooled samples."""
    from paper_1105_4840_gb300 import shard

    w = inputs.od1d_workload()
    run = w["run"]
    run.n_steps, run.n_equil, run.replicas = 4000, 400, 4
    lam = np.linspace(-1.5, 1.5, 9)
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    shards, xs = [], []
    for rank in range(2):
        base = shard.shard_uid_base(rank, lam.size, run.replicas)
        rr = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run, uid_base=base))
        P = rr.partials()
        x = rr.x_samples()
        Po = est.window_partials([a.astype(np.float64) for a in x], lam, run.k, run.kT)
        np.testing.assert_array_equal(P[:, :, 2], Po[:, :, 2])
        np.testing.assert_allclose(P, Po, rtol=1e-12, atol=1e-12)
        a = pmf.pmf_free_energy_from_partials(P, lam, run.k, run.kT)
        b = rr.free_energy()
        for key in a:
            np.testing.assert_array_equal(a[key], b[key], err_msg=key)
        shards.append(P)
        xs.append(x)
    merged = shard.merge_partials(shards)
    got = pmf.pmf_free_energy_from_partials(merged, lam, run.k, run.kT)
    pooled = np.concatenate([np.concatenate([xs[0][i], xs[1][i]], axis=0).ravel() for i in range(lam.size)])
    T = xs[0][0].shape[1]
    want = pmf.pmf_free_energy_from_samples(pooled.astype(np.float32), lam, 2 * run.replicas, [T] * lam.size,
                                            run.k, run.kT)
    _compare_profiles(got, want, run.kT, rel=1e-11)


@pytest.mark.parametrize("replicas,warps", [(32, 4), (32, 5), (32, 6), (1024, 4)])
def test_full_size_launch_sampled_replicas(pmf, replicas, warps):
    """The 104-bead workload at its full replica counts (21 x 32, and 21 x 1024
    of the precision study) in the benchmark's launch configuration
    (persistent grid, autotuned warp counts), shortened to 300 steps in
    100-step segments so two segment hand-overs occur while the FP32 and FP64
    trajectories still agree closely (chaos amplifies rounding differences
    by roughly e per 0.1 ps): sampled replicas of the first, middle and last
    windows against the oracle."""
    import concurrent.futures as cf
    import os

    w = inputs.chain_workload(n_steps=300, replicas=replicas)
    p, start, run = w["params"], w["start"], w["run"]
    run.n_equil, run.stride = 100, 50
    sysh = pmf.pmf_create_system_chain([p], [start])
    pmf.pmf_chain_set_warps(sysh, 0, warps)
    pmf.pmf_chain_set_grid(sysh, 0, 0, 100)
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    pos = rr.final_state()[0].reshape(21, replicas, 104, 3)
    xs = rr.x_samples()
    picks = [(0, 0), (10, replicas // 2), (20, replicas - 1), (5, 7 % replicas)]
    ch = _clib.Chain(p)

    def one(job):
        wi, r = job
        xo, ro, _ = ch.run(start, run.lambdas[wi], run.k, run.kT, run.dt, run.gamma, run.n_steps, run.n_equil,
                           run.stride, run.seed, wi * replicas + r)
        return np.abs(pos[wi, r] - ro).max(), np.abs(xs[wi][r] - xo).max()

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        errs = list(ex.map(one, picks))
    assert max(e[0] for e in errs) <= 2e-4, errs
    assert max(e[1] for e in errs) <= 1e-4, errs
