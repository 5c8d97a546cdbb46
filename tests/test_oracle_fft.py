"""Pins for the oracle's transform F (Eq. 1 / Eq. 3): the orthonormal 2-D DFT
with the zero frequency at [0, 0].

Each check ties ``oracle.dm.fft2`` / ``ifft2`` to something other than the
oracle itself: the DFT sum written out term by term, Parseval's identity, and
the transform of a delta and of a plane wave."""
import cmath
import math

import numpy as np
import pytest

from oracle import dm


def brute_dft2(x, sign):
    """(1/N) sum_{uy,ux} x[uy,ux] exp(sign * 2 pi i (qy uy + qx ux) / N), by loops."""
    n = x.shape[0]
    out = np.zeros((n, n), dtype=np.complex128)
    for qy in range(n):
        for qx in range(n):
            acc = 0j
            for uy in range(n):
                for ux in range(n):
                    acc += x[uy, ux] * cmath.exp(sign * 2j * math.pi * (qy * uy + qx * ux) / n)
            out[qy, qx] = acc / n
    return out


@pytest.mark.parametrize("n", [2, 4, 8])
def test_forward_and_inverse_match_brute_force(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n))
    f = dm.fft2(x)
    b = dm.ifft2(x)
    for m in range(3):
        np.testing.assert_allclose(f[m], brute_dft2(x[m], -1), rtol=0, atol=1e-13)
        np.testing.assert_allclose(b[m], brute_dft2(x[m], +1), rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [16, 64])
def test_parseval_and_round_trip(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((2, n, n)) + 1j * rng.standard_normal((2, n, n))
    f = dm.fft2(x)
    assert abs(np.sum(np.abs(f) ** 2) - np.sum(np.abs(x) ** 2)) < 1e-10 * np.sum(np.abs(x) ** 2)
    np.testing.assert_allclose(dm.ifft2(f), x, atol=1e-12)


def test_delta_maps_to_constant_and_plane_wave_to_delta():
    n = 8
    d = np.zeros((n, n), complex)
    d[0, 0] = 1.0
    np.testing.assert_allclose(dm.fft2(d), np.full((n, n), 1.0 / n), atol=1e-15)
    # A plane wave exp(+2 pi i (a uy + b ux)/N) lands on frequency (a, b)
    # with weight N (no fftshift, forward sign -).
    a, b = 3, 5
    uy, ux = np.mgrid[0:n, 0:n]
    pw = np.exp(2j * np.pi * (a * uy + b * ux) / n)
    f = dm.fft2(pw)
    expect = np.zeros((n, n), complex)
    expect[a, b] = n
    np.testing.assert_allclose(f, expect, atol=1e-12)
