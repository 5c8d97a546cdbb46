"""Host-side pieces of the learned warm start (torch on the CPU): the
footprint gather and the stitching of per-view predictions whose global
phases are arbitrary (one view's intensities fix its patch only up to a
constant phase factor)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import warmstart as ws
from synth.scan import grf_object, raster_positions


def _scene(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    obj = grf_object((260, 260), rng)
    pos = raster_positions((8, 8), 16, 1, ws.N, (260, 260), rng)
    return rng, obj, pos


def test_footprints_are_the_slices_at_the_positions():
    _, obj, pos = _scene(1)
    fp = ws.footprints(torch.from_numpy(obj.astype(np.complex64)), pos).numpy()
    for j in (0, 17, len(pos) - 1):
        r, c = pos[j]
        assert np.array_equal(fp[j], obj[r:r + ws.N, c:c + ws.N].astype(np.complex64))


def _covered(pos, shape):
    cov = np.zeros(shape, bool)
    c = (ws.N - ws.PATCH) // 2
    for r, q in pos:
        cov[r + c:r + c + ws.PATCH, q + c:q + c + ws.PATCH] = True
    return cov


def _rel_up_to_phase(a, b):
    s = np.vdot(a, b)
    a = a * s / abs(s)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_aligned_stitch_recovers_patches_with_arbitrary_phases():
    """Exact central patches of a known object, each turned by a random
    global phase: the aligned stitch rebuilds the object on the covered
    pixels up to one global phase; plain averaging does not."""
    rng, obj, pos = _scene(2)
    t = ws.target_from_object(ws.footprints(torch.from_numpy(obj.astype(np.complex64)), pos))
    pred = t.clone()
    pred[:, 1] += torch.from_numpy(rng.uniform(-np.pi, np.pi, len(pos)).astype(np.float32))[:, None, None]
    cov = _covered(pos, obj.shape)
    aligned = ws.stitch(pred, pos, obj.shape, align=True).numpy()
    plain = ws.stitch(pred, pos, obj.shape, align=False).numpy()
    assert _rel_up_to_phase(aligned[cov], obj[cov]) < 1e-5
    assert _rel_up_to_phase(plain[cov], obj[cov]) > 0.3
    assert np.all(aligned[~cov] == 1)
    # the aligned patches share the phase reference of the uncovered pixels'
    # value 1: their sum is real and positive
    total = np.sum(aligned[cov])
    assert abs(np.angle(total)) < 0.05


def test_aligned_stitch_averages_noise_without_drift():
    """Noisy patches (complex white noise of 35 % of the mean amplitude) with
    random phases over a 30 x 30 scan: the stitched object's error is well
    below the noise, so the alignment does not drift along the scan."""
    rng = np.random.Generator(np.random.PCG64(4))
    obj = grf_object((420, 420), rng)
    pos = raster_positions((30, 30), 10, 1, ws.N, (420, 420), rng)
    t = ws.target_from_object(ws.footprints(torch.from_numpy(obj.astype(np.complex64)), pos))
    z = t[:, 0] * torch.exp(1j * t[:, 1])
    g = torch.Generator().manual_seed(5)
    noise = 0.35 * float(z.abs().mean()) * torch.complex(torch.randn(z.shape, generator=g),
                                                         torch.randn(z.shape, generator=g)) / np.sqrt(2)
    zn = (z + noise) * torch.exp(1j * torch.from_numpy(rng.uniform(-np.pi, np.pi, len(pos)).astype(np.float32)))[:, None, None]
    pred = torch.stack([zn.abs(), torch.angle(zn)], 1)
    cov = _covered(pos, obj.shape)
    got = ws.stitch(pred, pos, obj.shape, align=True).numpy()
    assert _rel_up_to_phase(got[cov], obj[cov]) < 0.12


def test_stitch_without_phase_offsets_is_the_plain_average():
    rng, obj, pos = _scene(3)
    t = ws.target_from_object(ws.footprints(torch.from_numpy(obj.astype(np.complex64)), pos))
    a = ws.stitch(t, pos, obj.shape, align=True).numpy()
    b = ws.stitch(t, pos, obj.shape, align=False).numpy()
    cov = _covered(pos, obj.shape)
    # the same average, turned as a whole to the common phase reference
    assert _rel_up_to_phase(a[cov], b[cov]) < 1e-5
    assert np.allclose(b[cov], obj[cov], rtol=0, atol=1e-5)


def test_fit_metrics_ignore_the_gauge_and_the_sign_convention():
    """fit_of: a prediction equal to the target up to a phase factor per
    patch, or written with negative amplitudes and phases moved by pi, fits
    perfectly; the flat patch does not."""
    from paper_1808_10375_gb300 import warmstart
    rng, obj, pos = _scene(6)
    t = ws.target_from_object(ws.footprints(torch.from_numpy(obj.astype(np.complex64)), pos)).double()
    turned = t.clone()
    turned[:, 1] += torch.from_numpy(rng.uniform(-3, 3, len(pos)))[:, None, None]
    signed = turned.clone()
    signed[:, 0] = -signed[:, 0]
    signed[:, 1] += np.pi
    for pred in (t, turned, signed):
        f = warmstart.fit_of(pred, t)
        assert f["amplitude_r2"] > 1 - 1e-9 and f["phase_r2_gauge_aligned"] > 1 - 1e-9
        assert f["complex_rel_err_gauge_aligned"] < 1e-7
    flat = torch.zeros_like(t)
    flat[:, 0] = 1.0
    f = warmstart.fit_of(flat, t)
    assert f["amplitude_r2"] < 0.0 and f["complex_rel_err_gauge_aligned"] > 0.1
