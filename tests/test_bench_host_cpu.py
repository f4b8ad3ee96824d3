"""Host-side pieces of bench.py that need no GPU: the exact reference of the
1D adaptive-vs-uniform ladder against the oracle's quadrature, the sample
count per replica, and the flop count of the roofline against the pair and
term counts of a chain."""
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
