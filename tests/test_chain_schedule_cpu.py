"""CPU emulation of the chain kernel's nonbonded ring units (no GPU).

For every unit of the host schedule this replays the kernel's lane/step
index arithmetic and checks that (a) every pair i < j with j - i >= 3 is
evaluated exactly once and no excluded, self or padded pair contributes,
(b) the rotating j-force accumulators hold the bead the kernel assumes at
every step and at the flush, and (c) every shared-memory index stays inside
its buffer."""
import numpy as np
import pytest

NS = [4, 5, 6, 7, 8, 9, 13, 16, 17, 24, 31, 32, 33, 39, 40, 41, 48, 56, 63, 64, 65, 72, 96, 100, 104,
      110, 112, 120, 127, 128, 129, 200, 255, 256, 333, 400, 1000, 1024]


def _width(t, n_tiles, w_last):
    return w_last if t == n_tiles - 1 else 32


# kind: (ring width W, first step TB, steps NST, diagonal, packed offset D or 0)
# kind: (ring width W, first step TB, steps NST, diagonal, quad offset D or 0)
# scalar kinds step t by 1; quad kinds step t by 2 with two i-beads per lane
KINDS = {0: (32, 0, 8, 0, 0), 1: (32, 8, 8, 0, 0), 2: (32, 16, 8, 0, 0), 3: (32, 24, 8, 0, 0),
         4: (32, 1, 8, 1, 0), 5: (32, 9, 8, 1, 0), 6: (16, 0, 8, 0, 0), 7: (16, 8, 8, 0, 0),
         8: (16, 1, 8, 1, 0), 9: (8, 0, 8, 0, 0), 10: (8, 1, 4, 1, 0),
         21: (32, 1, 4, 0, 8), 22: (32, 17, 4, 0, 8), 23: (32, 2, 4, 1, 8), 24: (16, 1, 4, 0, 8),
         25: (8, 1, 2, 0, 4), 26: (32, 1, 8, 0, 8)}
SPLIT = {26}  # quad kinds whose ring steps jump by 10 halfway (t = 1..7, then 17..23)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("NW", [4, 5, 6, 8])
@pytest.mark.parametrize("N", NS)
def test_ring_pieces_cover_pairs_once(N, NW, precision, variant):
    from paper_1105_4840_gb300 import pmf

    if precision == 1 and variant:
        pytest.skip("FP64 schedules do not depend on the cost model")
    assert pmf.pmf_chain_schedule_variants() == 6
    units, Np = pmf.pmf_chain_schedule(N, NW, precision, variant)
    n_tiles = (N + 31) // 32
    rem = N % 32
    w_last = 32 if rem == 0 else (8 if rem <= 8 else (16 if rem <= 16 else 32))
    assert Np == (n_tiles - 1) * 32 + w_last
    count = np.zeros((Np, Np), dtype=np.int64)
    for (w, I1, I2, J, kind, near1, near2) in units:
        assert 0 <= w < NW and 0 <= I1 <= J < n_tiles and kind in KINDS
        W, TB, NST, DIAG, DP = KINDS[kind]
        assert (kind >= 21 or kind in (8, 10)) if precision == 0 else kind <= 10
        if DP:
            _quad_piece(count, N, Np, n_tiles, w_last, I1, J, near1, W, TB, NST, DIAG, DP, kind in SPLIT)
            continue
        assert W == _width(J, n_tiles, w_last)
        assert bool(DIAG) == (I1 == J)
        tiles = [(I1, near1)] + ([(I2, near2)] if I2 >= 0 else [])
        if I2 >= 0:
            assert not DIAG and I1 < I2 < J
        lanes = np.arange(32)
        lr = lanes & (W - 1)
        src = (lanes & ~(W - 1)) | ((lr + 1) & (W - 1))
        acc = (lr + TB) & (W - 1)  # j index whose force each lane carries
        for k in range(NST):
            t = TB + k
            assert np.all(acc == ((lr + t) & (W - 1)))
            jidx = lr + t
            assert jidx.max() < 2 * W <= 64  # duplicated tile copy
            j = J * 32 + (jidx & (W - 1))
            for I, near in tiles:
                assert bool(near) == (J - I == 1) or (DIAG and near)
                wI = _width(I, n_tiles, w_last)
                i = I * 32 + lanes
                ion = lanes < wI
                masked = np.zeros(32, dtype=bool)
                if t < 3 and near:
                    masked |= np.abs(i - j) <= 2
                if DIAG and 2 * t == W:
                    masked |= lr >= W // 2
                ok = ion & ~masked & (i < N) & (j < N)
                assert np.all(i[ok] != j[ok])
                assert np.all(np.abs(i[ok] - j[ok]) >= 3)
                for a, b in zip(i[ok], j[ok]):
                    count[min(a, b), max(a, b)] += 1
                assert I * 32 + wI <= Np
            if k + 1 < NST:
                acc = acc[src]
        flush = (lr + TB + NST - 1) & (W - 1)
        assert np.all(acc == flush)
        for g in range(32 // W):
            assert np.all(acc[g * W:(g + 1) * W] == acc[:W])
        assert (J * 32 + flush[:W]).max() < Np
    want = np.zeros_like(count)
    for a in range(N):
        want[a, a + 3:N] = 1
    np.testing.assert_array_equal(count, want)


def _quad_piece(count, N, Np, n_tiles, w_last, I, J, near, W, TB, NST, DIAG, D, split=False):
    """Replay of quad_piece: lane l holds i1 at ring index l and i2 at l + 1;
    step k (t = TB + 2k, plus 8 in the second half of a split piece) pairs
    both with ring positions l + t (stream a) and l + t + D (stream b); both
    j-force streams rotate by the step's increment of t."""
    assert D == (8 if W == 32 else W // 2)
    lanes = np.arange(32)
    lr = lanes & (W - 1)
    l2 = (lanes & ~(W - 1)) | ((lr + 1) & (W - 1))
    assert sorted(l2) == list(range(32))  # a permutation: the i2 flush hits distinct beads
    def t_of(k):
        return TB + 2 * k + (8 if split and 2 * k >= NST else 0)

    acc_a = (lr + TB) & (W - 1)
    acc_b = (lr + TB + D) & (W - 1)
    wI = _width(I, n_tiles, w_last)
    gi1, gi2 = I * 32 + lanes, I * 32 + l2
    on1, on2 = lanes < wI, l2 < wI
    for k in range(NST):
        t = t_of(k)
        assert (lr + t).max() < 2 * W  # packed entry index p = lr + t
        for stream, tt, acc in (("a", t, acc_a), ("b", t + D, acc_b)):
            assert np.all(acc == ((lr + tt) & (W - 1)))
            j = J * 32 + ((lr + tt) & (W - 1))
            for gi, on, first in ((gi1, on1, True), (gi2, on2, False)):
                masked = np.zeros(32, dtype=bool)
                if stream == "a" and near and TB < 4 and t < 4:
                    masked |= np.abs(gi - j) <= 2
                if stream == "b" and first and DIAG and k == NST - 1:
                    masked |= lr >= W // 2
                ok = on & ~masked & (gi < N) & (j < N)
                assert np.all(gi[ok] != j[ok])
                assert np.all(np.abs(gi[ok] - j[ok]) >= 3)
                for a, b in zip(gi[ok], j[ok]):
                    count[min(a, b), max(a, b)] += 1
        if k + 1 < NST:
            src = (lanes & ~(W - 1)) | ((lr + t_of(k + 1) - t) & (W - 1))
            acc_a, acc_b = acc_a[src], acc_b[src]
    tl = t_of(NST - 1)
    fa = (lr + tl) & (W - 1)
    fb = (lr + tl + D) & (W - 1)
    assert np.all(acc_a == fa) and np.all(acc_b == fb)
    for g in range(32 // W):
        assert np.all(acc_a[g * W:(g + 1) * W] == acc_a[:W])
        assert np.all(acc_b[g * W:(g + 1) * W] == acc_b[:W])
    assert max((J * 32 + fa[:W]).max(), (J * 32 + fb[:W]).max()) < Np
    assert I * 32 + wI <= Np


def test_schedule_is_balanced():
    from paper_1105_4840_gb300 import pmf

    for precision in (0, 1):
        units, _ = pmf.pmf_chain_schedule(104, 4, precision)
        load = np.zeros(4)
        for (w, I1, I2, J, kind, n1, n2) in units:
            load[w] += KINDS[kind][2] * (2 if (I2 >= 0 or KINDS[kind][4]) else 1)
        assert load.max() <= 1.5 * load.mean()
