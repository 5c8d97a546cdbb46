"""Pins for the two projections of the oracle.

Modulus (the constrained transform F_c of Sec. II): after projection the mode
sum of |.|^2 equals the measured intensity, each mode keeps its phase,
projecting twice equals projecting once, a single mode reduces to textbook
modulus replacement sqrt(I) x/|x|, and S = 0 maps to zero.

Overlap (Eq. 5 then Eq. 4): on consistent exit waves psi = P O both updates
return their inputs (fixed point / idempotence), and the floor delta has the
closed form of a single uniformly illuminated view."""
import numpy as np
import pytest

from oracle import dm


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("m", [1, 3])
def test_modulus_matches_intensity_and_keeps_phase(m):
    rng = np.random.default_rng(10 + m)
    x = rand_c(rng, (m, 8, 8))
    inten = rng.uniform(0.1, 5.0, (8, 8))
    y, s = dm.modulus_projection(x, inten)
    np.testing.assert_allclose(np.sum(np.abs(y) ** 2, axis=0), inten, rtol=1e-13)
    np.testing.assert_allclose(s, np.sum(np.abs(x) ** 2, axis=0), rtol=1e-14)
    # same phase: y = (positive real) * x, with one real factor shared by all modes
    ratio = y / x
    np.testing.assert_allclose(ratio.imag, 0, atol=1e-13)
    assert np.all(ratio.real > 0)
    np.testing.assert_allclose(ratio.real, np.broadcast_to(ratio.real[0], ratio.shape), rtol=1e-13)


def test_modulus_idempotent():
    rng = np.random.default_rng(2)
    x = rand_c(rng, (4, 8, 8))
    inten = rng.uniform(0.0, 3.0, (8, 8))
    y1, _ = dm.modulus_projection(x, inten)
    y2, _ = dm.modulus_projection(y1, inten)
    nz = inten > 0
    np.testing.assert_allclose(y2[:, nz], y1[:, nz], rtol=1e-13, atol=1e-14)


def test_single_mode_is_textbook_modulus_replacement():
    rng = np.random.default_rng(3)
    x = rand_c(rng, (1, 8, 8))
    inten = rng.uniform(0.0, 3.0, (8, 8))
    y, _ = dm.modulus_projection(x, inten)
    np.testing.assert_allclose(y[0], np.sqrt(inten) * x[0] / np.abs(x[0]), rtol=1e-13)


def test_zero_mode_sum_and_negative_intensity():
    x = np.zeros((2, 4, 4), complex)
    x[0, 1, 1] = 1 + 1j
    inten = np.full((4, 4), 2.0)
    inten[1, 1] = -3.0            # a negative (noisy) count is clamped to zero
    y, s = dm.modulus_projection(x, inten)
    assert np.all(y == 0)         # S = 0 everywhere except [1,1], where I -> 0
    assert s[1, 1] == pytest.approx(2.0)


def consistent_state(rng, m=2, n=8, grid=3, step=3):
    h = w = (grid - 1) * step + n + 2
    probe = rand_c(rng, (m, n, n))
    obj = rand_c(rng, (h, w))
    pos = np.array([[1 + a * step, 1 + b * step] for a in range(grid) for b in range(grid)], np.int32)
    psi = dm.init_exit_waves(probe, obj, pos)
    return probe, obj, pos, psi


def covered(shape, pos, n):
    cov = np.zeros(shape, bool)
    for r, c in pos:
        cov[r:r + n, c:c + n] = True
    return cov


def test_object_update_fixed_point_on_consistent_waves():
    rng = np.random.default_rng(4)
    probe, obj, pos, psi = consistent_state(rng)
    start = rand_c(rng, obj.shape)
    new = dm.object_update(psi, probe, start, pos, delta_rel=0.0)
    cov = covered(obj.shape, pos, probe.shape[-1])
    np.testing.assert_allclose(new[cov], obj[cov], rtol=1e-12)
    np.testing.assert_array_equal(new[~cov], start[~cov])     # uncovered pixels keep their value


def test_probe_update_fixed_point_on_consistent_waves():
    rng = np.random.default_rng(5)
    probe, obj, pos, psi = consistent_state(rng, m=3)
    new = dm.probe_update(psi, rand_c(rng, probe.shape), obj, pos, delta_rel=0.0)
    np.testing.assert_allclose(new, probe, rtol=1e-12)


def test_overlap_pass_idempotent():
    rng = np.random.default_rng(6)
    probe, obj, pos, _ = consistent_state(rng)
    psi = dm.init_exit_waves(probe, obj, pos) + 0.3 * rand_c(rng, (len(pos),) + probe.shape)
    o1 = dm.object_update(psi, probe, obj, pos, 0.0)
    p1 = dm.probe_update(psi, probe, o1, pos, 0.0)
    psi1 = dm.init_exit_waves(p1, o1, pos)
    o2 = dm.object_update(psi1, p1, o1, pos, 0.0)
    p2 = dm.probe_update(psi1, p1, o2, pos, 0.0)
    cov = covered(obj.shape, pos, probe.shape[-1])
    np.testing.assert_allclose(o2[cov], o1[cov], rtol=1e-11)
    np.testing.assert_allclose(p2, p1, rtol=1e-11)


def test_denominator_floor_closed_form():
    # One view covering the whole object, uniform probe p: every pixel has
    # den = |p|^2 = max den, so O = conj(p) psi / (|p|^2 (1 + delta_rel)).
    n = 4
    p = 0.6 - 0.8j
    probe = np.full((1, n, n), p)
    rng = np.random.default_rng(7)
    psi = rand_c(rng, (1, 1, n, n))
    pos = np.array([[0, 0]], np.int32)
    for d in (0.0, 1e-3, 0.5):
        o = dm.object_update(psi, probe, np.zeros((n, n), complex), pos, d)
        np.testing.assert_allclose(o, np.conj(p) * psi[0, 0] / (abs(p) ** 2 * (1 + d)), rtol=1e-14)
    # and the probe update with a uniform object o: P = conj(o) psi / (|o|^2 (1 + delta_rel))
    o = 0.3 + 0.4j
    obj = np.full((n, n), o)
    for d in (0.0, 0.25):
        pn = dm.probe_update(psi, probe, obj, pos, d)
        np.testing.assert_allclose(pn[0], np.conj(o) * psi[0, 0] / (abs(o) ** 2 * (1 + d)), rtol=1e-14)


def test_sampled_object_update_fixed_point_and_uncovered_pixels():
    # Eq. 5 at single pixels: consistent waves give back the object on
    # covered pixels; uncovered pixels keep the starting value.
    rng = np.random.default_rng(8)
    probe, obj, pos, psi = consistent_state(rng, m=3)
    start = rand_c(rng, obj.shape)
    n = probe.shape[-1]
    cov = covered(obj.shape, pos, n)
    pix = [tuple(p) for p in np.argwhere(cov)[::7]] + [tuple(p) for p in np.argwhere(~cov)]
    den = dm.object_denominator(probe, pos, obj.shape)
    got = dm.object_update_at(pix, lambda j: psi[j], probe, start, pos, 0.0, den.max())
    for (r, c), g in zip(pix, got):
        if cov[r, c]:
            assert g == pytest.approx(obj[r, c], rel=1e-12)
        else:
            assert g == start[r, c]


def test_sampled_object_update_closed_form_and_whole_array_agreement():
    # one uniform view: O = conj(p) psi / (|p|^2 (1 + delta_rel)) at every pixel
    n = 4
    p = 0.6 - 0.8j
    probe = np.full((1, n, n), p)
    rng = np.random.default_rng(9)
    psi = rand_c(rng, (1, 1, n, n))
    pos = np.array([[0, 0]], np.int32)
    pix = [(r, c) for r in range(n) for c in range(n)]
    got = dm.object_update_at(pix, lambda j: psi[j], probe, np.zeros((n, n), complex), pos, 0.5, abs(p) ** 2)
    np.testing.assert_allclose(got, (np.conj(p) * psi[0, 0] / (abs(p) ** 2 * 1.5)).ravel(), rtol=1e-14)
    # on a generic state it agrees with the whole-array update
    probe, obj, pos, _ = consistent_state(rng, m=2)
    psi = rand_c(rng, (len(pos),) + probe.shape)
    full = dm.object_update(psi, probe, obj, pos, 1e-3)
    den = dm.object_denominator(probe, pos, obj.shape)
    pix = [(r, c) for r in range(obj.shape[0]) for c in range(obj.shape[1])]
    got = dm.object_update_at(pix, lambda j: psi[j], probe, obj, pos, 1e-3, den.max())
    np.testing.assert_allclose(got, full.ravel(), rtol=1e-12)
