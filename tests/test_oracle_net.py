"""Pins of the FP64 reference of the warm-start network (oracle/net.py):
one layer against a textbook correlation, the analytic gradient against
central finite differences, and the BF16 rounding against its definition."""
import numpy as np
import pytest

from oracle import net


def test_layer_table_and_parameter_count():
    ls = net.layers()
    assert [l[3] for l in ls] == [64, 32, 16, 8, 4, 8, 16, 32, 64, 64]
    assert ls[0][:2] == (1, 16) and ls[4][:2] == (128, 256) and ls[-1][:2] == (16, 2)
    assert net.param_count() == sum(co * ci * 9 + co for ci, co, *_ in ls)


def test_first_layer_is_a_strided_zero_padded_correlation():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    p = net.he_params(rng)
    x = rng.standard_normal((1, 1, 128, 128))
    acts = net.forward(p, x, bf16_weights=False)
    w, b = net.unpack(p)[0]
    for co in (0, 7, 15):
        full = scipy_signal.correlate2d(x[0, 0], w[co, 0], mode="same") + b[co]
        ref = np.maximum(full[::2, ::2], 0.0)
        assert np.allclose(acts[1][0, co], ref, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    p = net.he_params(rng) + 0.01 * rng.standard_normal(net.param_count())
    x = rng.standard_normal((2, 1, 128, 128))
    t = rng.standard_normal((2, 2, 64, 64))
    _, g = net.loss_and_gradients(p, x, t, bf16_weights=False)
    offs = np.cumsum([0] + [co * ci * 9 + co for ci, co, *_ in net.layers()])
    picks = [int(offs[i] + rng.integers(0, offs[i + 1] - offs[i])) for i in range(len(offs) - 1)]
    eps = 1e-6
    for i in picks:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp, _ = net.loss_and_gradients(pp, x, t, bf16_weights=False)
        lm, _ = net.loss_and_gradients(pm, x, t, bf16_weights=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_bf16_rounding_is_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.14159265], np.float32)
    r = net.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway, ties to even (mantissa ends in 0)
    assert r[2] == 1.0 + 2 ** -6       # halfway, rounds up to the even neighbour
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12
