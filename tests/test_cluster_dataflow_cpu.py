"""The cluster form's data flow (Eq. 3 with the constrained transform F_c of
Sec. II, and the object source of Eq. 5), restated on the CPU in FP64 through
the kernel's shared-memory index maps and checked against the oracle's
Fourier update (no GPU): per mode (one CTA each) the exit wave, the forward
row and column DFTs as 8-lane line DFTs with their in-place exchange, |X|^2
into the norm buffer in the intensities' strip order; per CTA r the factor
beta sqrt(I)/(N sqrt(S)) - 1/N^2 of its share of the pixels from every
mode's norms, pushed into every mode's buffer; the inverse column and row
DFTs of f X; psi' = (2 - beta) P O + G; and c_j = sum_k conj(P_k) psi'_k over
each CTA's share of pixel pairs, summed in mode order.  Planted mistakes in
the reduce-scatter and in the factor must be caught."""
import numpy as np
import pytest

from oracle import dm as odm
from synth import make_scan, initial_guess, random_exit_waves
from test_cluster_layout_cpu import fidx, nidx, nidx_strip, xslot, out_pos, r1


def line_dfts(lines, inverse=False):
    """The 8-lane line DFT of every row of `lines` [L, n] (unnormalised),
    through the exchange slots of the line itself, as the kernel runs it."""
    L, n = lines.shape
    R1 = r1(n)
    D = R1 // 8
    sgn = 1.0 if inverse else -1.0
    i = np.arange(R1)
    t = np.arange(8)
    # pass 1: lane t transforms x[t + 8 i] over i, then the twiddle W_n^(t k1)
    x = lines.reshape(L, R1, 8)                                       # [l][i][t]
    w1 = np.exp(sgn * 2j * np.pi * np.outer(i, i) / R1)               # [i][k1]
    y = np.einsum("lit,ik->ltk", x, w1) * np.exp(sgn * 2j * np.pi * np.outer(t, i) / n)[None]
    buf = np.empty_like(lines)
    slots = np.array([[xslot(k1, tt) for k1 in range(R1)] for tt in range(8)])   # [t][k1]
    buf[:, slots] = y
    # pass 2: lane t' takes k1 = t' + 8 d and transforms over the lanes tt
    out = np.empty_like(lines)
    w2 = np.exp(sgn * 2j * np.pi * np.outer(t, t) / 8)                # [tt][k2]
    for d in range(D):
        rd = np.array([[xslot(tp + 8 * d, tt) for tt in range(8)] for tp in range(8)])   # [t'][tt]
        u = buf[:, rd]                                                 # [l][t'][tt]
        z = np.einsum("lpt,tk->lpk", u, w2)                            # [l][t'][k2]
        pos = np.array([[out_pos(tp, d, k2, n) for k2 in range(8)] for tp in range(8)])
        out[:, pos] = z
    return out


def cluster_view(psi_j, probe, obj, pos_j, inten_j, beta, planted=None):
    """One view through the cluster form's steps; returns psi', c_j and the
    Fourier-error terms of every CTA."""
    M, n, _ = psi_j.shape
    P = n * n
    rr, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    fi = fidx(rr, xx, n)                  # frame index of (row, column)
    ni = nidx(rr, xx, n)                  # norm-buffer index of (row, column)
    po = odm.field_products(probe, obj, pos_j)
    F = np.zeros((M, P), np.complex128)   # one frame per CTA, in the swizzled layout
    NB = np.zeros((M, P))
    for k in range(M):
        phi = 2.0 * po[k] - psi_j[k]
        F[k, fi] = line_dfts(phi)                                   # 1: rows
        cols = line_dfts(F[k, fi].T.copy())                         # 2: columns (line = column)
        F[k, fi.T] = cols
        NB[k, ni.T] = np.abs(cols) ** 2
    # 3: the factors, CTA r over its pixels in strip order, in fours
    strip = (np.arange(P) // (2 * n), (np.arange(P) % (2 * n)) // 2, np.arange(P) % 2)
    i_strip = inten_j[strip[1], 2 * strip[0] + strip[2]]            # I in strip order
    ef = np.zeros(M)
    for r in range(M):
        lo, hi = 4 * ((r * (P // 4)) // M), 4 * (((r + 1) * (P // 4)) // M)
        p = np.arange(lo, hi)
        idx = np.array([nidx_strip(q, n) for q in p])
        S = np.zeros(len(p))
        for k in range(M):
            if planted == "own norms only" and k != r:
                continue
            S += NB[k, idx]
        iv = i_strip[p]
        sc = np.where(S > 0, np.sqrt(np.maximum(iv, 0)) / (n * np.sqrt(np.where(S > 0, S, 1))), 0.0)
        b = 1.0 if planted == "no beta" else beta
        f = b * sc - 1.0 / n ** 2
        ef[r] = np.sum((np.sqrt(S) / n - np.sqrt(np.maximum(iv, 0))) ** 2)
        for k in range(M):
            NB[k, idx] = f
    # 4, 5: inverse column and row DFTs of f X, psi' and conj(P_k) psi'
    psi_new = np.empty_like(psi_j)
    for k in range(M):
        cols = line_dfts((F[k, fi] * NB[k, ni]).T.copy(), inverse=True)
        F[k, fi.T] = cols
        g = line_dfts(F[k, fi], inverse=True)
        psi_new[k] = (2.0 - beta) * po[k] + g
        F[k, fi] = np.conj(probe[k]) * psi_new[k]
    # 6: c_j, CTA r over its pixel pairs in natural order, modes summed in order
    c = np.zeros(P, np.complex128)
    for r in range(M):
        lo, hi = (r * (P // 2)) // M, ((r + 1) * (P // 2)) // M
        px = np.arange(2 * lo, 2 * hi)
        acc = F[0, fi.ravel()[px]].copy()
        for k in range(1, M):
            acc += F[k, fi.ravel()[px]]
        c[px] = acc
    return psi_new, c.reshape(n, n), ef


def scan_case(n, m, seed):
    step = n // 8
    cfg = dict(n=n, modes=m, grid=(2, 2), step=step, jitter=1, obj=(n + step + 4,) * 2,
               probe="gauss" if m == 1 else "hg", fwhm=n / 2.0, photons=1e6, seed=seed)
    s = make_scan(cfg, noise=True)
    rng = np.random.default_rng(seed + 7)
    p0, o0 = initial_guess(s, rng, kind="perturbed")
    psi0 = random_exit_waves(p0, o0, s.pos, rng)
    return s, p0.astype(np.complex128), o0.astype(np.complex128), psi0.astype(np.complex128)


@pytest.mark.parametrize("n,m", [(64, 3), (64, 1), (128, 4)])
def test_cluster_dataflow_matches_the_oracle(n, m):
    s, p0, o0, psi0 = scan_case(n, m, 70 + m)
    inten = np.asarray(s.intensities, np.float64)
    beta = 0.8
    for j in range(s.views):
        psi_new, c, ef = cluster_view(psi0[j], p0, o0, s.pos[j], inten[j], beta)
        want, err_num, _ = odm.fourier_update_view(psi0[j], p0, o0, s.pos[j], inten[j], beta)
        assert np.abs(psi_new - want).max() <= 1e-9 * np.abs(want).max()
        c_want = np.sum(np.conj(p0) * want, axis=0)
        assert np.abs(c - c_want).max() <= 1e-9 * np.abs(c_want).max()
        assert abs(ef.sum() - err_num) <= 1e-9 * err_num


@pytest.mark.parametrize("mistake", ["own norms only", "no beta"])
def test_cluster_dataflow_catches_planted_mistakes(mistake):
    n, m = 64, 3
    s, p0, o0, psi0 = scan_case(n, m, 80)
    inten = np.asarray(s.intensities, np.float64)
    psi_new, _, _ = cluster_view(psi0[0], p0, o0, s.pos[0], inten[0], 0.8, planted=mistake)
    want, _, _ = odm.fourier_update_view(psi0[0], p0, o0, s.pos[0], inten[0], 0.8)
    assert np.abs(psi_new - want).max() > 1e-3 * np.abs(want).max()
