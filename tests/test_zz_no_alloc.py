"""The allocation-free reduction entry point (pmf_free_energy_noalloc).

Some callers cannot let a library allocate GPU memory: a host program whose
own pool has already reserved the device memory, or a latency-critical loop
that must not pay the device-wide synchronisation of cudaMalloc/cudaFree.
For them the library offers a variant of the FP64 reduction whose scratch is
a fixed device array.  This test calls it twice in a row through the C ABI
and checks each result against the regular entry point on the same samples,
within the tolerances the other reduction tests use; it also checks that the
second call leaves the device's free memory unchanged.

The file name sorts last so that a run that stops at the first failure has
already run every other test; it also passes when run alone."""
import numpy as np
import pytest

from paper_1105_4840_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("lambda", "dF_JE", "dF_fluct", "dF_G", "dF_com", "uncertainty", "se_JE", "se_fluct",
          "var_ZW", "W_mean", "acc_force", "mean_x", "var_x", "gamma2")


def _close(a, b, kT):
    for q, key in enumerate(FIELDS):
        if key in ("se_JE", "se_fluct", "var_ZW"):
            np.testing.assert_allclose(a[key], b[key], rtol=1e-8, equal_nan=True, err_msg=key)
        elif key in ("mean_x", "var_x", "gamma2", "lambda"):
            np.testing.assert_allclose(a[key], b[key], rtol=1e-10, err_msg=key)
        else:
            assert np.all(np.abs(a[key] - b[key]) <= 1e-12 * np.maximum(np.abs(b[key]), kT)), key


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_1105_4840_gb300 import pmf

    s, R, T = 21, 32, 3600
    lam = inputs.lambda_grid(1.3, 3.3, s)
    k, kT = 500.0, inputs.kT_of(300.0)
    results = []
    free_after_first = None
    for call, seed in enumerate((11, 12)):
        x = inputs.gaussian_x_samples(lam, k, kT, R, T, seed=seed)
        want = pmf.pmf_free_energy_from_samples(x.ravel(), lam, R, [T] * s, k, kT)
        x_dev = torch.from_numpy(x.ravel()).cuda()
        lam_dev = torch.from_numpy(lam.copy()).cuda()
        out_dev = torch.full((14 * s,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        pmf.pmf_set_stream(torch.cuda.current_stream().cuda_stream)
        pmf.pmf_free_energy_noalloc(x_dev.data_ptr(), lam_dev.data_ptr(), s, R, T, k, kT, out_dev.data_ptr())
        torch.cuda.synchronize()
        pmf.pmf_set_stream(0)
        if call == 1:
            assert torch.cuda.mem_get_info()[0] >= free_before
        got_flat = out_dev.cpu().numpy()
        got = {key: got_flat[q * s:(q + 1) * s] for q, key in enumerate(FIELDS)}
        _close(got, want, kT)
        results.append(got)
    # the two calls saw different samples: the shared scratch carried nothing over
    assert not np.array_equal(results[0]["dF_JE"], results[1]["dF_JE"])


@pytest.mark.parametrize("s,R", [(4, 16384), (2, 32768)])
def test_noalloc_at_its_size_limits(s, R):
    """n_windows x replicas = 65536 fills the partials part of the fixed
    scratch; 16384 replicas keep the per-replica sums of the combination
    step in shared memory, 32768 take its other branch.  Two calls in a
    row, each against the regular entry point."""
    torch = pytest.importorskip("torch")
    from paper_1105_4840_gb300 import pmf

    T = 4
    lam = inputs.lambda_grid(1.3, 1.6, s)
    k, kT = 500.0, inputs.kT_of(300.0)
    for seed in (21, 22):
        x = inputs.gaussian_x_samples(lam, k, kT, R, T, seed=seed)
        want = pmf.pmf_free_energy_from_samples(x.ravel(), lam, R, [T] * s, k, kT)
        x_dev = torch.from_numpy(x.ravel()).cuda()
        lam_dev = torch.from_numpy(lam.copy()).cuda()
        out_dev = torch.full((14 * s,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        pmf.pmf_set_stream(torch.cuda.current_stream().cuda_stream)
        pmf.pmf_free_energy_noalloc(x_dev.data_ptr(), lam_dev.data_ptr(), s, R, T, k, kT, out_dev.data_ptr())
        torch.cuda.synchronize()
        pmf.pmf_set_stream(0)
        got_flat = out_dev.cpu().numpy()
        _close({key: got_flat[q * s:(q + 1) * s] for q, key in enumerate(FIELDS)}, want, kT)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1105_4840_gb300 import pmf

    x = torch.zeros(4, device="cuda")
    lam = torch.zeros(2, dtype=torch.float64, device="cuda")
    out = torch.zeros(28, dtype=torch.float64, device="cuda")
    for n_windows, replicas in ((2, 40000), (1025, 1), (1, 4)):
        with pytest.raises(pmf.PmfError) as e:
            pmf.pmf_free_energy_noalloc(x.data_ptr(), lam.data_ptr(), n_windows, replicas, 1, 1.0, 1.0,
                                        out.data_ptr())
        assert e.value.status == pmf.PMF_EINVAL
