"""Host-side pieces of bench.py that need no GPU: the exact reference of the
1D adaptive-vs-uniform ladder against the oracle's quadrature, the sample
count per replica, and the flop count of the roofline against the pair and
term counts of a chain, and the criterion of the adaptive-vs-uniform
ladders."""
import numpy as np

import bench
from oracle import quadrature as quad
from paper_1105_4840_gb300 import inputs


def test_od1d_exact_reference_matches_oracle_quadrature():
    w = inputs.od1d_workload()
    run = w["run"]
    lam = np.array([-1.5, -0.75, -0.1, 0.4, 1.05, 1.5])
    e = bench._od1d_exact(lam, w["a"], run.k, run.kT)
    o = np.array([quad.od1d_free_energy(l, run.k) for l in lam])
    np.testing.assert_allclose(e, o - o[0], atol=1e-9)
    # the double well is symmetric: the full path costs nothing
    assert abs(e[-1]) < 1e-9


def test_samples_per_replica():
    run = inputs.chain_workload()["run"]
    assert bench.samples_per_replica(run) == 3600  # (4e5 - 4e4) / 100


def test_flops_per_replica_step_counts_terms():
    n = 104
    pairs = sum(1 for i in range(n) for j in range(i + 3, n))
    expect = 36 * pairs + 20 * (n - 1) + 60 * (n - 2) + 110 * (n - 3) + 33 * n
    assert bench.flops_per_replica_step(n) == expect == 208158


def test_ladder_summary_criterion():
    """A seed reaches eps at the shortest tau from which every longer run
    stays within eps: a run inside eps followed by one outside does not
    count; the median is reported only when every seed got there."""
    kT, F = 2.0, 10.0
    rows = []
    for seed, devs in ((0, [-3.0, 0.1, 0.25, 0.1]), (1, [-3.0, -0.5, 0.25, -0.1]), (2, [0.0, 1.5, 0.9, 0.21])):
        for i, (tau, d) in enumerate(zip((100.0, 200.0, 400.0, 800.0), devs)):
            rows.append({"seed": seed, "tau_ps": tau, "gpu_s": float(2 ** i), "dF": F + d * kT, "se": 0.2})
    s = bench.ladder_summary(rows, [0, 1, 2], F, kT)
    # eps 0.2: seed 0 only at 800 (0.25 at 400 is out), seed 1 at 800, seed 2 never (0.21 at 800)
    assert [p["tau_ps"] if p else None for p in s["per_seed"]] == [800.0, 800.0, None]
    assert s["median_gpu_s"] is None and s["seeds_converged"] == 2
    eps = {e["eps_kT"]: e for e in s["by_eps"]}
    assert [p["tau_ps"] for p in eps[0.3]["per_seed"]] == [200.0, 400.0, 800.0]
    assert eps[0.3]["median_gpu_s"] == 4.0
    assert [p["tau_ps"] for p in eps[1.0]["per_seed"]] == [200.0, 200.0, 400.0]
    bt = {b["tau_ps"]: b for b in s["by_tau"]}
    np.testing.assert_allclose(bt[100.0]["bias_kT"], -2.0)
    np.testing.assert_allclose(bt[100.0]["sd_kT"], np.std([-3.0, -3.0, 0.0], ddof=1))
    np.testing.assert_allclose(bt[800.0]["mean_se_kT"], 0.1)
