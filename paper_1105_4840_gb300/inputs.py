"""Seeded synthetic inputs for the parallel step-wise pulling protocol.

This module only builds inputs: the parameters of a synthetic bead chain that
stands in for the deca-alanine molecule of Sec. IV (whose structure and
CHARMM22 force field are not available here), its common starting state x_o
(Sec. III (ii): every PPP window starts from the same state), the lambda grids
of the windows, the run settings of each workload, and synthetic reaction
coordinate samples for reduction tests.  It contains none of the method's
arithmetic (no forces, no integrator, no work or free-energy formula), so both
the CUDA path and the FP64 oracle may consume it.

Units of the chain: nm, ps, amu, kJ/mol, elementary charge.  The 1D model is
in reduced units (kT = 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Boltzmann constant times Avogadro's number, kJ mol^-1 K^-1 (CODATA 2018).
KB_KJ_PER_MOL_K = 0.0083144626181532
# Coulomb constant 1/(4 pi eps0) in kJ mol^-1 nm e^-2.
COULOMB_K = 138.935458


def kT_of(temperature_k: float) -> float:
    """k_B T in kJ/mol."""
    return KB_KJ_PER_MOL_K * temperature_k


@dataclass
class ChainParams:
    """Force-field parameters of one synthetic chain of `n` beads."""

    n: int
    sigma: np.ndarray      # [n] nm
    epsilon: np.ndarray    # [n] kJ/mol
    charge: np.ndarray     # [n] e, zero sum
    mass: np.ndarray       # [n] amu
    dih_k: np.ndarray      # [n, 3] K_1..K_3 (kJ/mol) of the dihedral starting at bead i
    dih_phase: np.ndarray  # [n, 3] delta_n in {0, pi}
    kb: float = 2.5e5      # bond stiffness kJ/mol/nm^2
    r0: float = 0.15       # bond length nm
    ktheta: float = 400.0  # angle stiffness kJ/mol/rad^2
    theta0: float = math.radians(109.5)
    ke: float = COULOMB_K
    nonbonded: bool = True


def chain_params(n_beads: int, param_seed: int, *, mass: float = 12.0) -> ChainParams:
    """Synthetic chain with the parameter distributions of the 104-bead workload:
    LJ sigma ~ U[0.25, 0.35] nm, epsilon ~ U[0.2, 0.6] kJ/mol, charges
    ~ U[-0.4, 0.4] e shifted to zero sum, three-term periodic dihedrals with
    K_n ~ U[0, 2] kJ/mol and delta_n in {0, pi}, all masses `mass` amu."""
    if n_beads < 4:
        raise ValueError("a chain needs at least 4 beads")
    g = np.random.Generator(np.random.PCG64(param_seed))
    sigma = g.uniform(0.25, 0.35, n_beads)
    eps = g.uniform(0.2, 0.6, n_beads)
    q = g.uniform(-0.4, 0.4, n_beads)
    q = q - q.mean()
    dih_k = g.uniform(0.0, 2.0, (n_beads, 3))
    dih_phase = np.where(g.random((n_beads, 3)) < 0.5, 0.0, math.pi)
    dih_k[n_beads - 3:] = 0.0  # no dihedral starts at the last three beads
    dih_phase[n_beads - 3:] = 0.0
    return ChainParams(n=n_beads, sigma=sigma, epsilon=eps, charge=q,
                       mass=np.full(n_beads, mass), dih_k=dih_k, dih_phase=dih_phase)


def gaussian_chain_params(n_beads: int, kb: float, *, mass: float = 12.0) -> ChainParams:
    """Bonds only (r0 = 0), no angles, dihedrals or nonbonded terms: the
    end-to-end vector is Gaussian with variance (N-1) kT / kb per axis."""
    z = np.zeros(n_beads)
    return ChainParams(n=n_beads, sigma=z.copy(), epsilon=z.copy(), charge=z.copy(),
                       mass=np.full(n_beads, mass), dih_k=np.zeros((n_beads, 3)),
                       dih_phase=np.zeros((n_beads, 3)), kb=kb, r0=0.0, ktheta=0.0,
                       theta0=0.0, nonbonded=False)


def _place(a, b, c, bond, angle, torsion):
    """Position of a new bead d with |cd| = bond, angle(b, c, d) = angle and
    torsion angle (a, b, c, d) = torsion (natural extension reference frame)."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    nrm = np.cross(b - a, bc)
    nrm /= np.linalg.norm(nrm)
    m = np.cross(nrm, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(torsion),
                   bond * math.sin(angle) * math.sin(torsion)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * nrm


def chain_start(p: ChainParams, seed: int, *, target_x: float | None = None,
                min_dist: float = 0.30, tries: int = 48) -> np.ndarray:
    """Common starting conformation x_o [n, 3]: a seeded self-avoiding walk
    with bond r0 (0.15 nm if r0 = 0) and angle theta0 (109.5 deg if unset),
    torsions drawn from {60, 180, 300} deg plus noise, no pair |i - j| >= 3
    closer than `min_dist`.  With `target_x`, the walk (of `tries`) whose
    end-to-end distance is closest to it is returned."""
    g = np.random.Generator(np.random.PCG64(seed))
    n = p.n
    bond = p.r0 if p.r0 > 0 else 0.15
    angle = p.theta0 if p.theta0 > 0 else math.radians(109.5)
    best, best_gap = None, math.inf
    for _ in range(tries):
        walk = _one_walk(g, n, bond, angle, min_dist)
        if walk is None:
            continue
        gap = 0.0 if target_x is None else abs(np.linalg.norm(walk[-1] - walk[0]) - target_x)
        if gap < best_gap:
            best, best_gap = walk, gap
        if target_x is None:
            break
    if best is None:
        raise RuntimeError("could not build a self-avoiding start conformation")
    return best - best.mean(axis=0)


def _one_walk(g, n, bond, angle, min_dist):
    r = np.zeros((n, 3))
    r[1] = [bond, 0.0, 0.0]
    r[2] = r[1] + bond * np.array([-math.cos(angle), math.sin(angle), 0.0])
    choices = np.radians([60.0, 180.0, 300.0])
    for i in range(3, n):
        for _attempt in range(64):
            tor = choices[g.integers(0, 3)] + g.normal(0.0, math.radians(12.0))
            cand = _place(r[i - 3], r[i - 2], r[i - 1], bond, angle, tor)
            if i >= 3:
                d = np.linalg.norm(r[: i - 2] - cand, axis=1)
                if d.size and d.min() < min_dist:
                    continue
            r[i] = cand
            break
        else:
            return None
    return r


def lambda_grid(lo: float, hi: float, s: int) -> np.ndarray:
    """s window centres lambda_1..lambda_s, uniform from lo to hi."""
    return np.linspace(lo, hi, s)


@dataclass
class RunSettings:
    """Per-workload run settings (the paper's problem statement: windows,
    trap stiffness k, relaxation per window, temperature)."""

    k: float
    kT: float
    dt: float
    gamma: float
    n_steps: int
    n_equil: int
    stride: int
    replicas: int
    seed: int
    lambdas: np.ndarray = field(default_factory=lambda: np.zeros(0))


def od1d_workload() -> dict:
    """1D double well U = 2 (x^2 - 1)^2 kT, k = 20 kT, 21 windows on
    [-1.5, 1.5], 8 replicas per window, dt = 1e-3, 2e4 steps, kT = 1, D = 1,
    every replica starts at the left minimum x_o = -1, Philox seed 0."""
    run = RunSettings(k=20.0, kT=1.0, dt=1e-3, gamma=1.0, n_steps=20000, n_equil=2000,
                      stride=10, replicas=8, seed=0, lambdas=lambda_grid(-1.5, 1.5, 21))
    return {"a": 2.0, "x0": -1.0, "run": run}


def chain_workload(n_beads: int = 104, replicas: int = 32, n_steps: int = 400_000,
                   windows: int = 21, lo: float = 1.3, hi: float = 3.3,
                   param_seed: int = 1, seed: int = 0) -> dict:
    """The 104-bead chain workload: x pulled 1.3 -> 3.3 nm in 21 windows,
    k = 500 kJ/mol/nm^2, 300 K, dt = 1 fs, gamma = 5/ps, 0.4 ns per window,
    32 replicas per window, x recorded every 0.1 ps after a 10% equilibration."""
    p = chain_params(n_beads, param_seed)
    start = chain_start(p, param_seed + 1000, target_x=lo)
    run = RunSettings(k=500.0, kT=kT_of(300.0), dt=0.001, gamma=5.0, n_steps=n_steps,
                      n_equil=n_steps // 10, stride=100, replicas=replicas, seed=seed,
                      lambdas=lambda_grid(lo, hi, windows))
    return {"params": p, "start": start, "run": run}


def batch_workload(n_chains: int = 64, n_min: int = 40, n_max: int = 400, w_min: int = 21, w_max: int = 61,
                   replicas: int = 16, n_steps: int = 100_000, seed: int = 0, lengths_seed: int = 7,
                   start_tries: int = 2) -> dict:
    """Many independent pulls at once: n_chains synthetic chains (the
    parameter distributions of chain_params, param seed 100 + m) with
    lengths uniform in [n_min, n_max] beads and window counts uniform in
    [w_min, w_max]; chain m is pulled from lo_m to hi_m = (1.3, 3.3) nm x
    sqrt(N_m / 104) (a random coil's size grows about as sqrt(N)), 16
    replicas per window, 0.1 ns per window, the 104-bead workload's
    temperature, trap and integrator settings.  Returns params, starts and
    the per-chain lambda grids."""
    g = np.random.Generator(np.random.PCG64(lengths_seed))
    lengths = g.integers(n_min, n_max + 1, n_chains)
    windows = g.integers(w_min, w_max + 1, n_chains)
    params, starts, lams = [], [], []
    for m in range(n_chains):
        n = int(lengths[m])
        p = chain_params(n, 100 + m)
        scale = math.sqrt(n / 104.0)
        lo, hi = 1.3 * scale, 3.3 * scale
        params.append(p)
        starts.append(chain_start(p, 2000 + m, target_x=lo, tries=start_tries))
        lams.append(lambda_grid(lo, hi, int(windows[m])))
    run = RunSettings(k=500.0, kT=kT_of(300.0), dt=0.001, gamma=5.0, n_steps=n_steps,
                      n_equil=n_steps // 10, stride=100, replicas=replicas, seed=seed)
    return {"params": params, "starts": starts, "lambdas": lams, "run": run}


def adaptive_workload(n_beads: int = 104, param_seed: int | None = None) -> dict:
    """Learned window placement against the uniform grid: an n-bead chain
    (parameter seed 1 for 104 beads, 2 otherwise) pulled from lo to hi =
    (1.3, 3.3) nm x sqrt(n / 104) with the 104-bead workload's trap,
    temperature and integrator; the adaptive protocol starts from 11 uniform
    windows, the uniform protocol uses 21.  Below 200 beads: 256 replicas per
    window, window relaxation times tau of 0.2, 0.4, 0.8, 1.6 ns (the
    uniform grid also at 3.2 ns), dynamics seeds 0..2; from 200 beads on:
    128 replicas, tau of 0.4, 0.8, 1.6 ns (uniform also 3.2 ns), seeds 0..1.
    The converged reference is 41 uniform windows with the same replica
    count, continued for 16 rounds of 0.4 ns, each round resuming every
    replica from its end state, averaged over its last 4 rounds
    (s_reference: the earlier single-run reference of 81 windows)."""
    ps = param_seed if param_seed is not None else (1 if n_beads == 104 else 2)
    p = chain_params(n_beads, ps)
    scale = math.sqrt(n_beads / 104.0)
    lo, hi = 1.3 * scale, 3.3 * scale
    start = chain_start(p, ps + 1000, target_x=lo)
    long_chain = n_beads >= 200
    R = 128 if long_chain else 256
    run = RunSettings(k=500.0, kT=kT_of(300.0), dt=0.001, gamma=5.0, n_steps=0, n_equil=0, stride=100,
                      replicas=R, seed=0)
    return {"params": p, "start": start, "lo": lo, "hi": hi, "run": run,
            "tau_ps": [400.0, 800.0, 1600.0] if long_chain else [200.0, 400.0, 800.0, 1600.0],
            "tau_uniform_extra": [3200.0], "seeds": [0, 1] if long_chain else [0, 1, 2],
            "s_uniform": 21, "s_adaptive0": 11, "s_reference": 81, "s_reference_cont": 41,
            "replicas_reference": R, "reference_round_ps": 400.0, "reference_rounds": 16, "reference_average": 4}


def mlp_init_params(seed: int, hidden: int = 64, scale_in: float = 1.0) -> dict:
    """Seeded He-style initial weights of the surrogate 1 -> hidden -> hidden
    -> 2 network (W1 [hidden, 1], b1, W2 [hidden, hidden], b2, W3 [2, hidden],
    b3), FP64; both the oracle and the CUDA side start from these arrays."""
    g = np.random.Generator(np.random.PCG64(seed))
    return {
        "W1": g.normal(0.0, math.sqrt(2.0) / scale_in, (hidden, 1)),
        "b1": np.zeros(hidden),
        "W2": g.normal(0.0, math.sqrt(2.0 / hidden), (hidden, hidden)),
        "b2": np.zeros(hidden),
        "W3": g.normal(0.0, math.sqrt(1.0 / hidden), (2, hidden)),
        "b3": np.zeros(2),
    }


def gaussian_x_samples(lambdas, k, kT, replicas, samples, seed, *, shift=0.3, gamma2=1.2):
    """Synthetic FP32 reaction-coordinate samples [s][R][T]: Gaussian around
    lambda_i - shift * (i % 3) / 3 with variance gamma2 * kT / k.  Used to feed
    identical samples to the reductions of both sides."""
    g = np.random.Generator(np.random.PCG64(seed))
    lam = np.asarray(lambdas, dtype=np.float64)
    s = lam.size
    sd = math.sqrt(gamma2 * kT / k)
    mu = lam - shift * (np.arange(s) % 3) / 3.0
    x = mu[:, None, None] + sd * g.standard_normal((s, replicas, samples))
    return x.astype(np.float32)
