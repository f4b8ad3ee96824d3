"""The FP32 throughput probe that gives the integrator's roofline its
measured ceiling: scalar and packed FMA rates are positive, of the order
of SMs x 128 lanes x 2 flops x clock, and the packed form is not slower."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pmf():
    from paper_1105_4840_gb300 import pmf as m
    return m


def test_fp32_peak_scalar_and_packed(pmf):
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # loose bounds: 128 lanes x 2 flops per SM at 0.5-2.5 GHz
    lo, hi = sms * 256 * 0.5e9 / 1e12, sms * 256 * 2.5e9 / 1e12
    packed, ms_p = pmf.pmf_fp32_peak(packed=True, iters=1 << 14, reps=2)
    scalar, ms_s = pmf.pmf_fp32_peak(packed=False, iters=1 << 14, reps=2)
    assert lo < scalar < hi and lo < packed < hi, (scalar, packed)
    assert ms_p > 0 and ms_s > 0
    assert packed > 0.9 * scalar


def test_fp32_peak_arguments(pmf):
    for kw in (dict(iters=0), dict(reps=0), dict(ctas_per_sm=-1), dict(ctas_per_sm=65)):
        with pytest.raises(pmf.PmfError) as e:
            pmf.pmf_fp32_peak(**kw)
        assert e.value.status == pmf.PMF_EINVAL


def test_fp64_peak(pmf):
    """The FP64 probe runs and reports a positive rate below the FP32 one."""
    fp64, ms = pmf.pmf_fp64_peak(iters=1 << 10, reps=2)
    fp32, _ = pmf.pmf_fp32_peak(packed=False, iters=1 << 12, reps=2)
    assert ms > 0 and 0.0 < fp64 < fp32
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_fp64_peak(iters=0)
    assert e.value.status == pmf.PMF_EINVAL
