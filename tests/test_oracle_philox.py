"""Pins of the oracle's Philox4x32-10 and Box-Muller normals (CPU only).

The oracle implements Philox4x32-10 from its published definition (Salmon et
al., SC'11).  It is pinned to Triton's independent implementation, run on the
CPU by Triton's interpreter, on counters that exercise every word of the
counter and of the key, and its normals are checked against N(0, 1)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import _clib

HERE = os.path.dirname(os.path.abspath(__file__))


def _triton_ref(seed, c0, c1, c2, c3, n):
    pytest.importorskip("triton")
    out = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox_ref.py"),
                          str(seed), str(c0), str(c1), str(c2), str(c3), str(n)],
                         capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-300:])
    return np.array([[int(v) for v in line.split()] for line in out.stdout.strip().splitlines()],
                    dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("seed,c1,c2,c3", [
    (0, 0, 0, 0),
    (0x0123456789ABCDEF, 7, 123456, 1),
    (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 3),
])
def test_philox_matches_triton(seed, c1, c2, c3):
    n = 64
    c0 = 0xFFFFFFF0  # wraps around 2^32 inside the batch
    ref = _triton_ref(seed, c0, c1, c2, c3, n)
    raw, _ = _clib.philox_bulk(seed, c0, c1, c2, c3, n)
    np.testing.assert_array_equal(raw, ref)


def test_philox_bits_are_uniform():
    raw, _ = _clib.philox_bulk(42, 0, 3, 9, 0, 50000)
    bits = raw.ravel()
    # every bit position is set about half of the time
    frac = np.array([((bits >> b) & 1).mean() for b in range(32)])
    assert np.all(np.abs(frac - 0.5) < 0.01)
    # neighbouring counters are not correlated
    u = (raw[:, 0].astype(np.float64) + 0.5) / 2.0 ** 32
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.02


def test_box_muller_normals():
    from scipy import stats

    _, nor = _clib.philox_bulk(7, 0, 11, 5, 0, 100000)
    z = nor.ravel()
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the sine and cosine halves of one pair are uncorrelated
    assert abs(np.corrcoef(nor[:, 0], nor[:, 1])[0, 1]) < 0.02
