"""Pins of the FP64 reference of the warm-start network (oracle/net.py):
one layer against a textbook correlation, the analytic gradient against
central finite differences, and the BF16 rounding against its definition."""
import numpy as np
import pytest

from oracle import net


def test_layer_table_and_parameter_count():
    ls = net.layers()
    assert [l[3] for l in ls] == [64, 32, 16, 8, 4, 2, 4, 8, 16, 32, 64, 64]
    assert ls[0][:2] == (1, 16) and ls[5][:2] == (256, 256) and ls[6][:2] == (256, 256) and ls[-1][:2] == (16, 2)
    assert net.param_count() == sum(co * ci * 9 + co for ci, co, *_ in ls)
    assert 1.9e6 < net.param_count() < 2.1e6


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


@pytest.mark.parametrize("loss", ["mse", "gauge"])
def test_gradient_matches_central_differences(loss):
    rng = np.random.default_rng(2)
    p = net.he_params(rng) + 0.01 * rng.standard_normal(net.param_count())
    x = rng.standard_normal((2, 1, 128, 128))
    t = rng.standard_normal((2, 2, 64, 64))
    if loss == "gauge":
        t[:, 0] = 0.5 + 0.5 * rng.random((2, 64, 64))
    _, g = net.loss_and_gradients(p, x, t, bf16_weights=False, loss=loss)
    offs = np.cumsum([0] + [co * ci * 9 + co for ci, co, *_ in net.layers()])
    picks = [int(offs[i] + rng.integers(0, offs[i + 1] - offs[i])) for i in range(len(offs) - 1)]
    eps = 1e-6
    for i in picks:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp, _ = net.loss_and_gradients(pp, x, t, bf16_weights=False, loss=loss)
        lm, _ = net.loss_and_gradients(pm, x, t, bf16_weights=False, loss=loss)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


# ---- the phase-gauge-invariant loss -----------------------------------------

def _outputs(rng, b=3, p=8):
    y = np.empty((b, 2, p, p))
    t = np.empty((b, 2, p, p))
    y[:, 0], t[:, 0] = 0.3 + rng.random((b, p, p)), 0.3 + rng.random((b, p, p))
    y[:, 1], t[:, 1] = rng.uniform(-3, 3, (b, p, p)), rng.uniform(-3, 3, (b, p, p))
    return y, t


def _brute_force_loss(y, t):
    """min over theta of mean |exp(i theta) z - t|^2 per sample, by a dense
    grid and golden-section refinement (no closed form used)."""
    z = y[:, 0] * np.exp(1j * y[:, 1])
    tc = t[:, 0] * np.exp(1j * t[:, 1])
    total = 0.0
    for b in range(y.shape[0]):
        f = lambda th: float(np.sum(np.abs(np.exp(1j * th) * z[b] - tc[b]) ** 2))
        grid = np.linspace(-np.pi, np.pi, 4001)
        k = int(np.argmin([f(th) for th in grid]))
        lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
        g = (np.sqrt(5) - 1) / 2
        for _ in range(80):
            m1, m2 = hi - g * (hi - lo), lo + g * (hi - lo)
            if f(m1) < f(m2):
                hi = m2
            else:
                lo = m1
        total += f(0.5 * (lo + hi))
    return total / (y.shape[0] * y.shape[2] * y.shape[3])


def test_gauge_loss_is_the_minimum_over_a_global_phase():
    y, t = _outputs(np.random.default_rng(20))
    loss, _ = net.gauge_loss(y, t)
    assert loss == pytest.approx(_brute_force_loss(y, t), rel=1e-10, abs=1e-14)


def test_gauge_loss_ignores_a_phase_factor_per_patch():
    rng = np.random.default_rng(21)
    y, t = _outputs(rng)
    loss, g = net.gauge_loss(y, t)
    y2, t2 = y.copy(), t.copy()
    y2[:, 1] += rng.uniform(-4, 4, 3)[:, None, None]
    t2[:, 1] += rng.uniform(-4, 4, 3)[:, None, None]
    loss2, g2 = net.gauge_loss(y2, t2)
    assert loss2 == pytest.approx(loss, rel=1e-12)
    assert np.allclose(g2, g, rtol=1e-9, atol=1e-15)


def test_gauge_loss_vanishes_on_a_turned_copy():
    rng = np.random.default_rng(22)
    _, t = _outputs(rng)
    y = t.copy()
    y[:, 1] += 1.234
    loss, g = net.gauge_loss(y, t)
    assert abs(loss) < 1e-13
    assert np.max(np.abs(g)) < 1e-13


def test_gauge_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(23)
    y, t = _outputs(rng)
    _, g = net.gauge_loss(y, t)
    eps = 1e-6
    for _ in range(24):
        idx = tuple(int(rng.integers(0, s)) for s in y.shape)
        yp, ym = y.copy(), y.copy()
        yp[idx] += eps
        ym[idx] -= eps
        fd = (net.gauge_loss(yp, t)[0] - net.gauge_loss(ym, t)[0]) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd)) + 1e-11, (idx, fd, g[idx])


def test_planted_mistakes_in_the_gauge_loss_fail_the_pins():
    """Without the fitted phase (Re S for |S|) the invariance pin fails; with
    the amplitude gradient's factor 2 dropped the finite-difference pin
    fails."""
    rng = np.random.default_rng(24)
    y, t = _outputs(rng)

    def no_fit(y, t):
        z = y[:, 0] * np.exp(1j * y[:, 1])
        tc = t[:, 0] * np.exp(1j * t[:, 1])
        s = np.sum(np.conj(z) * tc, axis=(1, 2))
        return float(np.sum(np.sum(np.abs(z) ** 2, axis=(1, 2)) + np.sum(np.abs(tc) ** 2, axis=(1, 2))
                            - 2 * s.real) / z.size)
    y2 = y.copy()
    y2[:, 1] += 0.7
    assert abs(no_fit(y2, t) - no_fit(y, t)) > 1e-3

    loss, g = net.gauge_loss(y, t)
    g_bad = g.copy()
    g_bad[:, 0] *= 0.5
    idx = (1, 0, 3, 4)
    eps = 1e-6
    yp, ym = y.copy(), y.copy()
    yp[idx] += eps
    ym[idx] -= eps
    fd = (net.gauge_loss(yp, t)[0] - net.gauge_loss(ym, t)[0]) / (2 * eps)
    assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd))
    assert abs(fd - g_bad[idx]) > 1e-3 * abs(fd)


def test_bf16_rounding_is_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.14159265], np.float32)
    r = net.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway, ties to even (mantissa ends in 0)
    assert r[2] == 1.0 + 2 ** -6       # halfway, rounds up to the even neighbour
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12
