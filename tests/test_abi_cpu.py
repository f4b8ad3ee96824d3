"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point declared in include/pmf.h, rejects bad arguments with
PMF_EINVAL, and refuses to compute without a device (no CPU fallback)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "pmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pmf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1105_4840_gb300 import pmf

    names = _declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(pmf.lib, n)]
    assert not missing, missing
    # and the binding exposes the same names
    from paper_1105_4840_gb300 import pmf as b
    for n in ("pmf_run_windows", "pmf_run_prepare", "pmf_free_energy_from_samples", "pmf_philox",
              "pmf_chain_forces", "pmf_set_stream", "pmf_version"):
        assert hasattr(b, n) or hasattr(b.Run, n.replace("pmf_", "")), n


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_bad_arguments_are_rejected():
    from paper_1105_4840_gb300 import inputs, pmf

    p = inputs.chain_params(12, 1)
    s = inputs.chain_start(p, 2)
    bad = inputs.chain_params(12, 1)
    bad.mass[4] = 0.0
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([bad], [s])
    assert e.value.status == pmf.PMF_EINVAL
    bad = inputs.chain_params(12, 1)
    bad.dih_phase[2, 1] = 1.0  # only 0 or pi
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([bad], [s])
    assert e.value.status == pmf.PMF_EINVAL
    s_bad = s.copy()
    s_bad[3, 1] = np.nan
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([p], [s_bad])
    assert e.value.status == pmf.PMF_EINVAL
    tiny = inputs.chain_params(4, 1)
    tiny.n = 3
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([tiny], [np.zeros((3, 3))])
    assert e.value.status == pmf.PMF_EINVAL
    # warp counts outside {4, 5, 6, 8} and chain lengths outside [4, 1024]
    for nw, n in ((7, 104), (3, 104), (4, 3), (4, 1025)):
        with pytest.raises(pmf.PmfError) as e:
            pmf.pmf_chain_schedule(n, nw, pmf.PMF_FP32)
        assert e.value.status == pmf.PMF_EINVAL


@pytest.mark.skipif(_has_gpu(), reason="checks the no-device path")
def test_no_cpu_fallback_without_device():
    from paper_1105_4840_gb300 import inputs, pmf

    p = inputs.chain_params(12, 1)
    s = inputs.chain_start(p, 2)
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_create_system_chain([p], [s])
    assert e.value.status == pmf.PMF_ECUDA
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_philox(0, 0, 0, 0, 0, 4)
    assert e.value.status == pmf.PMF_ECUDA
    x = np.zeros(2 * 3 * 5, dtype=np.float32)
    with pytest.raises(pmf.PmfError) as e:
        pmf.pmf_free_energy_from_samples(x, [0.0, 1.0], 3, [5, 5], 1.0, 1.0)
    assert e.value.status == pmf.PMF_ECUDA


def test_binding_is_marshalling_only():
    """The binding never imports the oracle and has no numeric fallback."""
    src = open(os.path.join(ROOT, "paper_1105_4840_gb300", "pmf.py")).read()
    assert "oracle" not in src.replace("oracle", "", 0) or "import oracle" not in src
    assert "import oracle" not in src and "from oracle" not in src
