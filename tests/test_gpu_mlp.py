"""GPU parity of the surrogate MLP (BF16 tensor-core layer, FP32 elsewhere)
against the FP64 oracle: forward, gradients, and Adam training on identical
mini-batches."""
import math

import numpy as np
import pytest

from oracle import _clib, surrogate as sg
from paper_1105_4840_gb300 import inputs
from tests.helpers import oracle_od1d_samples

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def _params(seed, jitter=0.2):
    p = sg.init_params(seed)
    g = np.random.default_rng(seed + 1)
    for k in p:
        p[k] = p[k] + jitter * g.standard_normal(p[k].shape)
    # the GPU keeps FP32 masters: give the oracle the same rounded values
    return {k: np.asarray(v, dtype=np.float32).astype(np.float64) for k, v in p.items()}


def _bf(a):
    """Round to BF16 (round to nearest even) in FP64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_matches_oracle(pmf):
    p = _params(3)
    c, h = 2.3, 1.0
    lam = np.linspace(1.2, 3.4, 301)  # 3 tiles, the last ragged
    m = pmf.Mlp(pmf.pack_mlp_params(p), c, h)
    mu, lv = m.predict(lam)
    o = sg.forward(p, (lam - c) / h)
    mu_o, lv_o = sg.to_physical(o["out"], c, h)
    # bound from BF16 operands of the 64x64 layer: each product has relative
    # error <= 2^-8, so |dZ2_o| <= 2^-8 sum_i |W2_oi H1_i|; SiLU is 1.1-Lipschitz
    bound_z2 = 2.0 ** -8 * (np.abs(o["h1"]) @ np.abs(p["W2"]).T)
    bound_out = 1.1 * bound_z2 @ np.abs(p["W3"]).T + 1e-5 * (1 + np.abs(o["out"]))
    assert np.all(np.abs(mu - mu_o) <= h * bound_out[:, 0])
    assert np.all(np.abs(lv - lv_o) <= bound_out[:, 1])
    # and the BF16 rounding does matter at this level (the tensor cores ran)
    assert np.max(np.abs(mu - mu_o)) > 0


def test_gradient_matches_oracle(pmf):
    p = _params(5)
    c, h = 0.0, 1.5
    rng = np.random.default_rng(9)
    lam = rng.uniform(-1.5, 1.5, 384)
    x = (0.8 * lam + 0.2 * rng.standard_normal(384)).astype(np.float32)
    m = pmf.Mlp(pmf.pack_mlp_params(p), c, h)
    g, loss = m.gradient(lam, x)
    ln, xn = sg.normalise(lam, x.astype(np.float64), c, h)
    cache = sg.forward(p, ln)
    go = sg.backward(p, cache, xn)
    assert loss == pytest.approx(sg.nll(cache["out"], xn), rel=2e-2)
    off = 0
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        n = p[k].size
        gk = g[off:off + n].astype(np.float64)
        ok = go[k].ravel()
        rel = np.linalg.norm(gk - ok) / np.linalg.norm(ok)
        assert rel < 2e-2, (k, rel)
        off += n


@pytest.mark.parametrize("split", [1, 0])
def test_training_on_1d_run_matches_oracle_training(pmf, split):
    """Adam on identical Philox mini-batches of the 1D workload's samples:
    GPU and oracle surrogates agree, and both fit the window statistics
    (split: a CTA per tile and an update launch per step; else one CTA)."""
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    info = rr.info()
    xo = oracle_od1d_samples(w["a"], w["x0"], run)
    store = np.concatenate([b.ravel() for b in xo]).astype(np.float32).astype(np.float64)
    c, h = 0.0, 1.5
    p0 = _params(11, jitter=0.0)
    steps, batch, lr, seed = 300, 512, 3e-3, 7
    m = pmf.Mlp(pmf.pack_mlp_params(p0), c, h)
    m.set_split(split)
    loss_g = m.train(rr, steps, batch, lr, seed)
    po, _, loss_o = sg.train({k: v.copy() for k, v in p0.items()}, store, info["sample_offset"], run.lambdas,
                             steps, batch, lr, seed, c, h, _clib.philox_bulk)
    assert loss_g == pytest.approx(loss_o, abs=0.05)
    mu_g, lv_g = m.predict(run.lambdas)
    mu_o, lv_o = sg.to_physical(sg.forward(po, (run.lambdas - c) / h)["out"], c, h)
    sd = np.array([b.std() for b in xo])
    assert np.max(np.abs(mu_g - mu_o) / sd) < 0.25
    assert np.max(np.abs(lv_g - lv_o)) < 0.25
    mean = np.array([b.mean() for b in xo])
    assert np.median(np.abs(mu_g - mean) / sd) < 0.3


def test_split_training_matches_one_cta_step_by_step(pmf):
    """The same mini-batches, one Adam step: the split launch's weights equal
    the one-CTA kernel's up to FP32 summation order of the tile gradients
    (Adam's first step moves every weight by lr sign(g), so any difference
    beyond rounding is a wrong gradient); then 200 steps stay close."""
    w = inputs.od1d_workload()
    run = w["run"]
    sysh = pmf.pmf_create_system_1d(w["a"], w["x0"])
    rr = pmf.pmf_run_windows(sysh, run.lambdas, pmf.make_params(run))
    p0 = pmf.pack_mlp_params(_params(11, jitter=0.0))
    out = {}
    for split in (1, 0):
        m = pmf.Mlp(p0, 0.0, 1.5)
        m.set_split(split)
        m.train(rr, 1, 512, 3e-3, 7)
        one = m.params()
        m.train(rr, 199, 512, 3e-3, 8)
        out[split] = (one, m.params(), m.predict(run.lambdas))
        m.close()
    d1 = np.abs(out[1][0] - out[0][0])
    assert np.mean(d1 > 1e-6) < 0.01 and d1.max() <= 2 * 3e-3
    mu1, lv1 = out[1][2]
    mu0, lv0 = out[0][2]
    sd = np.array([b.std() for b in rr.x_samples()])
    assert np.max(np.abs(mu1 - mu0) / sd) < 0.1 and np.max(np.abs(lv1 - lv0)) < 0.1
    with pytest.raises(pmf.PmfError) as e:
        pmf.Mlp(p0, 0.0, 1.0).set_split(2)
    assert e.value.status == pmf.PMF_EINVAL
