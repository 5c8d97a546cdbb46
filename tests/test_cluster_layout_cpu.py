"""CPU checks of the cluster form's shared-memory layouts and data flow
(the cluster form of the Fourier step, Eq. 3 with F_c of Sec. II, for
64 x 64 and 128 x 128 frames): the index maps restated in numpy, checked for
being bijections, for bank-conflict freedom of every access pattern the
kernel makes, for the reduce-scatter ranges, and for the 8-lane line DFT with
its in-place exchange against numpy's FFT."""
import numpy as np
import pytest

SIZES = [64, 128]


def r1(n):
    """Values per lane of an n-point line (n = r1 x 8)."""
    return n // 8


def fidx(r, x, n):
    return (x >> 4) * (n * 16) + (r << 4) + (((((x & 15) >> 1) ^ (r & 7)) << 1) | (x & 1))


def nidx_strip(p, n):
    s = p // (2 * n)
    return s * (2 * n) + ((p % (2 * n)) ^ ((s & 1) << 4))


def nidx(q, x, n):
    return nidx_strip((x >> 1) * (2 * n) + (q << 1) + (x & 1), n)


def xslot(k1, t):
    return k1 * 8 + (t ^ (k1 & 7))


def group_row(g):
    return (g & ~7) | ((g & 1) << 2) | ((g >> 1) & 3)


def out_pos(t, d, k2, n):
    return t + 8 * d + r1(n) * k2


def banks8(idx):
    """Bank pair (of 16 per 128-byte wavefront) of float2 indices."""
    return [i % 16 for i in idx]


@pytest.mark.parametrize("n", SIZES)
def test_maps_are_bijections(n):
    groups = n // 2
    r, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    f = fidx(r, x, n)
    assert sorted(f.ravel().tolist()) == list(range(n * n))
    q = nidx(r, x, n)
    assert sorted(q.ravel().tolist()) == list(range(n * n))
    assert sorted(xslot(k1, t) for k1 in range(r1(n)) for t in range(8)) == list(range(n))
    assert sorted(group_row(g) for g in range(groups)) == list(range(groups))
    for g in range(0, groups, 2):
        assert group_row(g) ^ 4 == group_row(g + 1)
    assert sorted(out_pos(t, d, k2, n) for t in range(8) for d in range(r1(n) // 8) for k2 in range(8)) \
        == list(range(n))


def half_warps(n):
    """(group pair) of each half-warp: lanes 8 g + t, t < 8, for groups g, g + 1."""
    return [(g, g + 1) for g in range(0, n // 2, 2)]


def assert_conflict_free(idx16):
    assert len(set(banks8(idx16))) == 16, idx16


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("rho", [0, 1])
def test_row_pass_accesses_conflict_free(n, rho):
    D = r1(n) // 8
    for g0, g1 in half_warps(n):
        rows = [group_row(g0) + n // 2 * rho, group_row(g1) + n // 2 * rho]
        for i in range(r1(n)):   # pass-1 reads, x = t + 8 i
            assert_conflict_free([fidx(y, t + 8 * i, n) for y in rows for t in range(8)])
        for k1 in range(r1(n)):  # exchange writes
            assert_conflict_free([fidx(y, xslot(k1, t), n) for y in rows for t in range(8)])
        for d in range(D):       # exchange reads, k1 = t' + 8 d
            for tt in range(8):
                assert_conflict_free([fidx(y, xslot(tp + 8 * d, tt), n) for y in rows for tp in range(8)])
        for d in range(D):       # pass-2 writes
            for k2 in range(8):
                assert_conflict_free([fidx(y, out_pos(tp, d, k2, n), n) for y in rows for tp in range(8)])


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("rho", [0, 1])
def test_column_pass_accesses_conflict_free(n, rho):
    D = r1(n) // 8
    for g0, g1 in half_warps(n):
        cols = [g0 + n // 2 * rho, g1 + n // 2 * rho]
        for i in range(r1(n)):
            assert_conflict_free([fidx(t + 8 * i, c, n) for c in cols for t in range(8)])
        for k1 in range(r1(n)):
            assert_conflict_free([fidx(xslot(k1, t), c, n) for c in cols for t in range(8)])
        for d in range(D):
            for tt in range(8):
                assert_conflict_free([fidx(xslot(tp + 8 * d, tt), c, n) for c in cols for tp in range(8)])
        for d in range(D):
            for k2 in range(8):
                assert_conflict_free([fidx(out_pos(tp, d, k2, n), c, n) for c in cols for tp in range(8)])
        # the norm buffer (4-byte words, 32 banks): written after the forward
        # column pass, read before the inverse one, by a whole warp (4 columns)
        w0 = (g0 // 4) * 4
        wcols = [w0 + u + n // 2 * rho for u in range(4)]
        for d in range(D):
            for k2 in range(8):
                words = [nidx(out_pos(tp, d, k2, n), c, n) % 32 for c in wcols for tp in range(8)]
                assert len(set(words)) == 32
        for i in range(r1(n)):
            words = [nidx(t + 8 * i, c, n) % 32 for c in wcols for t in range(8)]
            assert len(set(words)) == 32


@pytest.mark.parametrize("n", SIZES)
def test_strip_order_runs_and_reduce_scatter_ranges(n):
    P = n * n
    # four consecutive strip-order pixels are four consecutive words
    for p in range(0, P, 4):
        base = nidx_strip(p, n)
        assert base % 4 == 0
        assert [nidx_strip(p + u, n) for u in range(4)] == [base + u for u in range(4)]
    # the pixels of steps 3 (fours) and 6 (pairs) partition the frame
    for M in range(1, 9):
        fours = [(4 * ((r * (P // 4)) // M), 4 * (((r + 1) * (P // 4)) // M)) for r in range(M)]
        pairs = [(((r * (P // 2)) // M), (((r + 1) * (P // 2)) // M)) for r in range(M)]
        for rng in (fours, [(2 * a, 2 * b) for a, b in pairs]):
            assert rng[0][0] == 0 and rng[-1][1] == P
            assert all(rng[i][1] == rng[i + 1][0] for i in range(M - 1))
    # a pixel pair (x even) is one 16-byte chunk of the frame
    for q in range(n):
        for x in range(0, n, 2):
            assert fidx(q, x, n) % 2 == 0 and fidx(q, x + 1, n) == fidx(q, x, n) + 1


def line_dft_emulated(line, inverse=False, read_slot=xslot):
    """The 8-lane line DFT with the in-place exchange, as the kernel runs it:
    pass 1 per lane t (an R1-point DFT over i of x[t + 8 i], twiddle
    W_n^(t k1)), the exchange through slots xslot(k1, t) of the line, pass 2
    per lane t' (8-point DFTs over the lanes for k1 = t' + 8 d), and the
    results written to positions t' + 8 d + R1 k2."""
    n = len(line)
    R1 = r1(n)
    sgn = 1.0 if inverse else -1.0
    w = lambda m, k: np.exp(sgn * 2j * np.pi * m / k)
    buf = np.array(line, np.complex128)
    y = np.zeros((8, R1), np.complex128)
    for t in range(8):
        xs = buf[[t + 8 * i for i in range(R1)]]
        for k1 in range(R1):
            y[t, k1] = sum(xs[i] * w(i * k1, R1) for i in range(R1)) * w(t * k1, n)
    for t in range(8):
        for k1 in range(R1):
            buf[xslot(k1, t)] = y[t, k1]
    out = np.zeros(n, np.complex128)
    for tp in range(8):
        for d in range(R1 // 8):
            k1 = tp + 8 * d
            u = [buf[read_slot(k1, tt)] for tt in range(8)]
            for k2 in range(8):
                out[out_pos(tp, d, k2, n)] = sum(u[tt] * w(tt * k2, 8) for tt in range(8))
    return out


@pytest.mark.parametrize("n", SIZES)
def test_line_dft_with_exchange_matches_numpy(n):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(line_dft_emulated(x), np.fft.fft(x), rtol=0, atol=1e-9 * np.abs(x).sum())
    np.testing.assert_allclose(line_dft_emulated(x, inverse=True), np.fft.ifft(x) * n, rtol=0,
                               atol=1e-9 * np.abs(x).sum())
    # a planted mistake in the exchange (each lane reads the slot of lane tt ^ 1) is caught
    wrong = line_dft_emulated(x, read_slot=lambda k1, tt: xslot(k1, tt ^ 1))
    assert np.abs(wrong - np.fft.fft(x)).max() > 1e-3 * np.abs(x).sum()
