"""Failure detection on the GPU without any fault: the persistent chain
launch's bounded wait runs out on a flag nothing sets, and the host's
wall-clock limit stops a run through a host-mapped stop flag.  In both cases
the kernels return by themselves and the context stays usable."""
import time

import numpy as np
import pytest

from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def _short_chain():
    p = inputs.chain_params(40, 3)
    start = inputs.chain_start(p, 7)
    run = inputs.RunSettings(k=300.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=3000,
                             n_equil=300, stride=30, replicas=2, seed=4)
    return p, start, run


def test_device_segment_wait_runs_out(pmf):
    """Every replica's second segment waits for a first segment that never
    runs (the queue starts after them): with a 50 ms limit (a legitimate wait
    for a 1000-step segment of this chain is about a millisecond) the kernel
    raises its timeout flag and returns; pmf_run_wait reports PMF_ETIMEOUT,
    not a numerical failure, and the results are refused until a run
    finishes.  The same handle then runs normally."""
    p, start, run = _short_chain()
    lam = np.array([1.0, 1.1])
    sysh = pmf.pmf_create_system_chain([p], [start])
    pmf.pmf_chain_set_grid(sysh, 0, 0, 1000)
    rr = pmf.pmf_run_prepare(sysh, lam, pmf.make_params(run, segment_wait_s=0.05))
    rr.set_queue_start(lam.size * run.replicas)
    rr.launch()
    t0 = time.perf_counter()
    with pytest.raises(pmf.PmfError) as e:
        rr.wait()
    assert e.value.status == pmf.PMF_ETIMEOUT
    assert "segment_wait_s" in str(e.value)
    assert time.perf_counter() - t0 < 10.0
    with pytest.raises(pmf.PmfError) as e2:
        rr.free_energy()
    assert e2.value.status == pmf.PMF_ESTATE
    rr.set_queue_start(0)
    rr.launch()
    rr.wait()
    ref = pmf.pmf_run_windows(sysh, lam, pmf.make_params(run))
    for a, b in zip(rr.x_samples(), ref.x_samples()):
        np.testing.assert_array_equal(a, b)


def test_queue_start_rejected_where_not_persistent(pmf):
    p, start, run = _short_chain()
    sysh = pmf.pmf_create_system_chain([p, p], [start, start])
    rb = pmf.pmf_run_batch_prepare(sysh, [(0, [1.0, 1.1]), (1, [1.0, 1.2])], pmf.make_params(run))
    with pytest.raises(pmf.PmfError) as e:
        rb.set_queue_start(4)
    assert e.value.status == pmf.PMF_EINVAL
    rr = pmf.pmf_run_prepare(sysh, [1.0, 1.1], pmf.make_params(run))
    with pytest.raises(pmf.PmfError) as e:
        rr.set_queue_start(-1)
    assert e.value.status == pmf.PMF_EINVAL
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_run_prepare(sysh, [1.0, 1.1], pmf.make_params(run, segment_wait_s=-1.0))
    assert e.value.status == pmf.PMF_EINVAL


def test_host_timeout_stops_the_kernels(pmf):
    """A run of several seconds with a 0.2 s wall-clock limit: pmf_run_wait
    raises the stop flag, the persistent CTAs return at their next work item,
    and the call comes back long before the run would have ended."""
    p = inputs.chain_params(104, 1)
    start = inputs.chain_start(p, 1001, target_x=1.3)
    run = inputs.RunSettings(k=500.0, kT=inputs.kT_of(300.0), dt=0.001, gamma=5.0, n_steps=1000000,
                             n_equil=1000, stride=100, replicas=4, seed=0)
    sysh = pmf.pmf_create_system_chain([p], [start])
    lam = np.array([1.3, 1.4])
    rr = pmf.pmf_run_prepare(sysh, lam, pmf.make_params(run, timeout_s=0.2))
    rr.launch()
    t0 = time.perf_counter()
    with pytest.raises(pmf.PmfError) as e:
        rr.wait()
    el = time.perf_counter() - t0
    assert e.value.status == pmf.PMF_ETIMEOUT
    assert "stopped" in str(e.value)
    assert el < 1.5, el
    with pytest.raises(pmf.PmfError) as e2:
        rr.x_samples()
    assert e2.value.status == pmf.PMF_ESTATE
    # the device is idle and usable: a short run completes
    _, s2, r2 = _short_chain()
    p2 = inputs.chain_params(40, 3)
    sys2 = pmf.pmf_create_system_chain([p2], [s2])
    out = pmf.pmf_run_windows(sys2, np.array([1.0, 1.1]), pmf.make_params(r2)).free_energy()
    assert np.all(np.isfinite(out["dF_JE"]))
