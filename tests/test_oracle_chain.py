"""Pins of the oracle's chain energy, forces and BAOAB integrator (CPU only)."""
import math

import numpy as np
import pytest

from oracle import _clib, quadrature
from paper_1105_4840_gb300 import inputs


def _params(n, seed=3):
    return inputs.chain_params(n, seed)


def test_forces_match_finite_differences():
    """Analytic forces equal -dU/dr by central differences (h = 1e-6 nm)."""
    p = _params(14)
    ch = _clib.Chain(p)
    r = inputs.chain_start(p, 5)
    r = r + np.random.default_rng(0).normal(0, 0.01, r.shape)
    lam, k = 1.1, 500.0
    f = ch.forces(r, lam, k)
    h = 1e-6
    fd = np.zeros_like(r)
    for i in range(p.n):
        for a in range(3):
            rp = r.copy(); rp[i, a] += h
            rm = r.copy(); rm[i, a] -= h
            fd[i, a] = -(ch.energy(rp, lam, k)[0] - ch.energy(rm, lam, k)[0]) / (2 * h)
    assert np.linalg.norm(f - fd) / np.linalg.norm(fd) < 1e-6


def test_forces_finite_differences_each_term():
    """Each term alone (bonds, angles, dihedrals with general phases, LJ +
    Coulomb, trap) is consistent with its energy."""
    base = _params(9, seed=11)
    r = inputs.chain_start(base, 2)
    r = r + np.random.default_rng(1).normal(0, 0.02, r.shape)
    variants = []
    for term in ("bond", "angle", "dih", "nb", "trap"):
        p = _params(9, seed=11)
        p.kb = 2.5e5 if term == "bond" else 0.0
        p.ktheta = 400.0 if term == "angle" else 0.0
        if term != "dih":
            p.dih_k = np.zeros_like(p.dih_k)
        else:
            p.dih_phase = np.random.default_rng(2).uniform(-math.pi, math.pi, p.dih_phase.shape)
        p.nonbonded = term == "nb"
        k = 300.0 if term == "trap" else 0.0
        variants.append((term, p, k))
    for term, p, k in variants:
        ch = _clib.Chain(p)
        f = ch.forces(r, 0.7, k)
        h = 1e-6
        fd = np.zeros_like(r)
        for i in range(p.n):
            for a in range(3):
                rp = r.copy(); rp[i, a] += h
                rm = r.copy(); rm[i, a] -= h
                fd[i, a] = -(ch.energy(rp, 0.7, k)[0] - ch.energy(rm, 0.7, k)[0]) / (2 * h)
        assert np.linalg.norm(fd) > 0, term
        assert np.linalg.norm(f - fd) / np.linalg.norm(fd) < 1e-6, term
        # Newton's third law: internal forces sum to zero
        assert np.abs(f.sum(axis=0)).max() < 1e-8 * np.abs(f).max(), term


def _four_beads(pos, **kw):
    p = inputs.chain_params(4, 0)
    p.kb = kw.get("kb", 0.0)
    p.r0 = kw.get("r0", 0.15)
    p.ktheta = kw.get("ktheta", 0.0)
    p.theta0 = kw.get("theta0", math.radians(109.5))
    p.dih_k = np.zeros((4, 3))
    p.dih_phase = np.zeros((4, 3))
    if "dih_k" in kw:
        p.dih_k[0] = kw["dih_k"]
        p.dih_phase[0] = kw["dih_phase"]
    p.nonbonded = kw.get("nonbonded", False)
    if "sigma" in kw:
        p.sigma[:] = kw["sigma"]
        p.epsilon[:] = kw["epsilon"]
        p.charge[:] = kw["charge"]
    return _clib.Chain(p), np.asarray(pos, dtype=np.float64)


def test_energy_special_cases():
    # bond stretched by 0.01 nm: kb/2 * 1e-4 per bond
    ch, r = _four_beads([[0, 0, 0], [0.16, 0, 0], [0.32, 0, 0], [0.48, 0, 0]], kb=1000.0)
    _, parts = ch.energy(r, 0.0, 0.0)
    assert parts[0] == pytest.approx(3 * 0.5 * 1000.0 * 0.01 ** 2, rel=1e-12)
    # right angles: ktheta/2 (pi/2 - theta0)^2 per angle
    ch, r = _four_beads([[1, 0, 0], [0, 0, 0], [0, 1, 0], [1, 1, 0]], ktheta=400.0)
    _, parts = ch.energy(r, 0.0, 0.0)
    assert parts[1] == pytest.approx(2 * 0.5 * 400.0 * (math.pi / 2 - math.radians(109.5)) ** 2,
                                     rel=1e-12)
    # planar cis (phi = 0) and trans (phi = pi) dihedrals
    K = np.array([0.7, 1.3, 0.4])
    dph = np.array([0.0, math.pi, 0.0])
    for d, phi in (([1, 1, 0], 0.0), ([1, -1, 0], math.pi)):
        ch, r = _four_beads([[0, 1, 0], [0, 0, 0], [1, 0, 0], d], dih_k=K, dih_phase=dph)
        _, parts = ch.energy(r, 0.0, 0.0)
        want = sum(K[m] * (1 + math.cos((m + 1) * phi - dph[m])) for m in range(3))
        assert parts[2] == pytest.approx(want, rel=1e-12, abs=1e-12)
    # the one nonbonded pair (0, 3) at the LJ minimum 2^(1/6) sigma_03
    sig = np.array([0.3, 0.2, 0.2, 0.34])
    eps = np.array([0.5, 0.1, 0.1, 0.2])
    q = np.array([0.3, 0.0, 0.0, -0.2])
    rmin = 2 ** (1 / 6) * 0.5 * (0.3 + 0.34)
    ch, r = _four_beads([[0, 0, 0], [0.1, 0.5, 0], [0.2, 0.5, 0], [rmin, 0, 0]],
                        nonbonded=True, sigma=sig, epsilon=eps, charge=q)
    _, parts = ch.energy(r, 0.0, 0.0)
    assert parts[3] == pytest.approx(-math.sqrt(0.5 * 0.2), rel=1e-12)
    assert parts[4] == pytest.approx(inputs.COULOMB_K * 0.3 * -0.2 / rmin, rel=1e-12)
    # the trap on the end-to-end distance
    _, parts = ch.energy(r, 0.5, 200.0)
    assert parts[5] == pytest.approx(0.5 * 200.0 * (rmin - 0.5) ** 2, rel=1e-12)
    assert ch.rc(r) == pytest.approx(rmin, rel=1e-14)


def _nve_max_dev(dt, n_seg=40, seg_time=0.05):
    p = _params(24)
    ch = _clib.Chain(p)
    r = inputs.chain_start(p, 9)
    kT = inputs.kT_of(300.0)
    v = ch.init_velocities(kT, 5, 0)
    e0 = ch.energy(r, 1.0, 500.0)[0] + ch.kinetic(v)
    steps = int(round(seg_time / dt))
    dev = 0.0
    for _ in range(n_seg):
        _, r, v = ch.run(r, 1.0, 500.0, kT, dt, 0.0, steps, steps, 1, 5, 0, v0=v)
        e = ch.energy(r, 1.0, 500.0)[0] + ch.kinetic(v)
        dev = max(dev, abs(e - e0))
    return dev


def test_nve_energy_conservation_second_order():
    """With friction off BAOAB is velocity Verlet: the energy error stays
    bounded and shrinks as dt^2."""
    d1 = _nve_max_dev(0.0005)
    d2 = _nve_max_dev(0.00025)
    assert d1 < 0.05 * inputs.kT_of(300.0) * 24
    assert 3.0 < d1 / d2 < 5.5


def test_initial_velocities_maxwell_boltzmann():
    p = _params(400)
    ch = _clib.Chain(p)
    kT = inputs.kT_of(300.0)
    ke = np.mean([ch.kinetic(ch.init_velocities(kT, 1, uid)) for uid in range(20)])
    assert ke == pytest.approx(1.5 * 400 * kT, rel=0.02)


def test_gaussian_chain_trap_matches_radial_quadrature():
    """Bond-only chain with r0 = 0: the end-to-end vector is Gaussian with
    per-axis variance (N-1) kT / kb; in the trap k/2 (x - lambda)^2 the mean
    of x equals the radial quadrature.  BAOAB samples harmonic configurations
    exactly at any stable dt."""
    n, kb, k, lam = 6, 50.0, 20.0, 1.0
    p = inputs.gaussian_chain_params(n, kb)
    ch = _clib.Chain(p)
    kT = inputs.kT_of(300.0)
    r0 = np.zeros((n, 3))
    r0[:, 0] = np.linspace(0, lam, n)
    means = []
    for uid in range(16):
        x, _, _ = ch.run(r0, lam, k, kT, 0.01, 5.0, 40000, 2000, 10, 123, uid)
        means.append(x.mean())
    means = np.array(means)
    se = means.std(ddof=1) / math.sqrt(means.size)
    want = quadrature.gaussian_chain_mean_x(lam, k, (n - 1) * kT / kb, kT)
    assert abs(means.mean() - want) < 4 * se + 1e-3
