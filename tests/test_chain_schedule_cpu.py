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


@pytest.mark.parametrize("NW", [4, 8])
@pytest.mark.parametrize("N", NS)
def test_ring_units_cover_pairs_once(N, NW):
    from paper_1105_4840_gb300 import pmf

    units, Np = pmf.pmf_chain_schedule(N, NW)
    n_tiles = (N + 31) // 32
    rem = N % 32
    w_last = 32 if rem == 0 else (8 if rem <= 8 else (16 if rem <= 16 else 32))
    assert Np == (n_tiles - 1) * 32 + w_last
    count = np.zeros((Np, Np), dtype=np.int64)
    for (w, I, J, tb, te, flags) in units:
        assert 0 <= w < NW and 0 <= I <= J < n_tiles and 0 <= tb < te
        W = _width(J, n_tiles, w_last)
        wI = _width(I, n_tiles, w_last)
        assert te <= (W // 2 + 1 if I == J else W)
        diag, near = bool(flags & 1), bool(flags & 2)
        assert diag == (I == J) and near == (J - I <= 1)
        lanes = np.arange(32)
        lr = lanes & (W - 1)
        src = (lanes & ~(W - 1)) | ((lr + 1) & (W - 1))
        acc = (lr + tb) & (W - 1)  # j index whose force each lane carries
        for t in range(tb, te):
            assert np.all(acc == ((lr + t) & (W - 1)))
            jidx = lr + t
            assert jidx.max() < 2 * W <= 64  # duplicated tile copy
            j = J * 32 + (jidx & (W - 1))
            i = I * 32 + lanes
            ion = lanes < wI
            masked = np.zeros(32, dtype=bool)
            if t < 3 and near:
                masked |= np.abs(i - j) <= 2
            if diag and 2 * t == W:
                masked |= lr >= W // 2
            ok = ion & ~masked & (i < N) & (j < N)
            assert np.all(i[ok] != j[ok])
            assert np.all(np.abs(i[ok] - j[ok]) >= 3)
            for a, b in zip(i[ok], j[ok]):
                count[min(a, b), max(a, b)] += 1
            if t + 1 < te:
                acc = acc[src]
        # flush: lanes < W write bead J*32 + ((lr + te - 1) & (W - 1)); groups of
        # W lanes (reduced by xor) must carry the same bead
        flush = (lr + te - 1) & (W - 1)
        assert np.all(acc == flush)
        for g in range(32 // W):
            assert np.all(acc[g * W:(g + 1) * W] == acc[:W])
        assert (J * 32 + flush[:W]).max() < Np
        assert I * 32 + wI <= Np
    want = np.zeros_like(count)
    for a in range(N):
        want[a, a + 3:N] = 1
    np.testing.assert_array_equal(count, want)


def test_schedule_is_balanced():
    from paper_1105_4840_gb300 import pmf

    units, _ = pmf.pmf_chain_schedule(104, 4)
    load = np.zeros(4)
    for (w, I, J, tb, te, flags) in units:
        load[w] += te - tb
    assert load.max() <= 1.25 * load.mean()
