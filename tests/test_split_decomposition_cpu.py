"""The split-column form's arithmetic, restated on the CPU in the kernel's
data flow and checked against numpy's 2-D FFT (no GPU): the row DFT and the
first radix-16 stage of the column DFT per row residue n1 (with W^(n1 k1)),
the second stage per k1 on 128-byte-swizzled boxes of (n1, mode) rows read
by (column, mode) lanes, the mode sum as a reduce-scatter over the 8 mode
lanes followed by an all-gather of the factors, and the two inverse stages.
The result must equal beta Phi' - Phi of Eq. 3's constrained transform (the
quantity the kernel adds to (2 - beta) P O), and the Fourier-error terms the
lanes accumulate must add up to sum (sqrt(S)/N - sqrt(I))^2."""
import numpy as np

N, M, R = 256, 8, 16


def W(e):
    return np.exp(-2j * np.pi * e / N)


def swz(r, c):   # byte offset of (box row r, column c): 16-byte chunk ^ (r mod 8)
    return r * 128 + (((c >> 1) ^ (r & 7)) << 4) + ((c & 1) << 3)


def reduce_scatter(s):   # s[m][16] -> o[m][2]: lane m ends with k2 = 2m, 2m + 1
    cur, width = {m: np.asarray(s[m]) for m in range(8)}, 16
    for bit in (4, 2, 1):
        nxt, half = {}, width // 2
        for m in range(8):
            p = m ^ bit
            keep = cur[m][half:] if m & bit else cur[m][:half]
            got = cur[p][:half] if p & bit else cur[p][half:]
            nxt[m] = keep + got
        cur, width = nxt, half
    return cur


def all_gather(f2):   # f2[m][2] (k2 = 2m, 2m + 1) -> f[m][16]
    cur = {m: np.asarray(f2[m]) for m in range(8)}
    for bit in (1, 2, 4):
        cur = {m: (np.concatenate([cur[m ^ bit], cur[m]]) if m & bit else np.concatenate([cur[m], cur[m ^ bit]]))
               for m in range(8)}
    return cur


def test_split_form_data_flow_equals_the_constrained_transform():
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((M, N, N)) + 1j * rng.standard_normal((M, N, N))
    inten = rng.random((N, N)) * 50
    beta = 0.8
    # row tasks: row DFT, then the first column stage per residue n1
    T = np.fft.fft(phi, axis=2)
    Y = np.zeros((R, R, M, N), complex)          # scratch [k1][n1][mode][column]
    for n1 in range(R):
        w = np.fft.fft(T[:, n1::R, :], axis=1)    # over n2 -> k1
        for k1 in range(R):
            Y[k1, n1] = w[:, k1, :] * W(n1 * k1)
    # column tasks, item (k1, 16 columns): swizzled box, (column, mode) lanes
    ef = 0.0
    for k1 in range(R):
        for xb in range(16):
            box = np.zeros(2048, complex)
            for n1 in range(R):
                for m in range(M):
                    for cc in range(16):
                        box[swz(n1 * 8 + m, cc) // 8] = Y[k1, n1, m, 16 * xb + cc]
            for c in range(16):
                X = {m: np.fft.fft([box[(n1 * 1024 + swz(m, c)) // 8] for n1 in range(R)]) for m in range(M)}
                S2 = reduce_scatter({m: np.abs(X[m]) ** 2 for m in range(M)})
                f2 = {}
                for m in range(M):
                    I2 = inten[k1 + R * np.arange(2 * m, 2 * m + 2), 16 * xb + c]
                    ss, si = np.sqrt(S2[m]), np.sqrt(I2)
                    ef += np.sum((ss / N - si) ** 2)
                    f2[m] = beta * si / (N * ss) - 1.0 / N ** 2
                f = all_gather(f2)
                for m in range(M):
                    Z = np.fft.ifft(X[m] * f[m]) * R   # unnormalised inverse over k2 -> n1
                    for n1 in range(R):
                        box[(n1 * 1024 + swz(m, c)) // 8] = Z[n1]
            for n1 in range(R):
                for m in range(M):
                    for cc in range(16):
                        Y[k1, n1, m, 16 * xb + cc] = box[swz(n1 * 8 + m, cc) // 8]
    # inverse row tasks: the inverse first stage per residue, then the inverse row DFT
    U = np.zeros((M, N, N), complex)
    for n1 in range(R):
        w = np.stack([Y[k1, n1] * np.conj(W(n1 * k1)) for k1 in range(R)], axis=1)
        U[:, n1::R, :] = np.fft.ifft(w, axis=1) * R
    G = np.fft.ifft(U, axis=2) * N
    # Eq. 3's constrained transform: beta Phi' - Phi with Phi' = F^-1[sqrt(I) X / sqrt(S)] (orthonormal)
    X = np.fft.fft2(phi, norm="ortho")
    S = np.sum(np.abs(X) ** 2, axis=0)
    phi_p = np.fft.ifft2(np.sqrt(inten) * X / np.sqrt(S), norm="ortho")
    ref = beta * phi_p - phi
    assert np.linalg.norm(G - ref) <= 1e-12 * np.linalg.norm(ref)
    ef_ref = np.sum((np.sqrt(S) - np.sqrt(inten)) ** 2)
    assert abs(ef - ef_ref) <= 1e-10 * ef_ref


def test_the_swizzle_gives_each_half_warp_distinct_banks():
    # lanes m + 8 cc (cc < 4) of warp w read column 4 w + cc of mode m: each
    # half-warp's 16 eight-byte reads fall on 16 different 8-byte bank slots
    for w in range(4):
        for n1 in range(R):
            for half in (0, 1):
                slots = {(n1 * 1024 + swz(m, 4 * w + 2 * half + cc)) % 128 // 8
                         for m in range(8) for cc in range(2)}
                assert len(slots) == 16
