"""Seeded synthetic scans: object, probe modes, positions, intensities.

Everything here is an *input* to a reconstruction.  The recipe follows the
workloads the paper reconstructs (Sec. IV): a complex object with bounded
amplitude and phase, one or several orthogonal probe modes (the mixed-state
description of fly-scan blur, Sec. I and Eq. 1), a raster of integer scan
positions whose footprints overlap, and far-field intensities recorded as the
incoherent sum over modes (Eq. 1 with the field product of Eq. 2), optionally
with Poisson counting noise.

Workload names describe what they are:

* ``sm64``  -- single mode, 64x64 frames, 10x10 raster (100 views) at 8 px
  with +-1 px jitter, 160x160 object, Gaussian-apertured probe of 32 px FWHM
  with quadratic phase, 1e6 photons per frame.
* ``mm128`` -- 4 Hermite-Gauss modes (power 0.6/0.25/0.1/0.05), 128x128
  frames, 50x50 fly scan (2500 views) at 10 px, 640x640 object array,
  1e7 photons per frame.
* ``mm256`` -- 8 Hermite-Gauss modes, 256x256 frames, 100x100 scan (10,000
  views) at 18 px, 2100x2100 object, 1e7 photons per frame.

Random numbers come from ``numpy.random.Generator(PCG64(seed))`` for the host
backend and from a seeded ``torch.Generator`` for the device backend; the two
backends are distinct datasets, and every consumer is handed one of them.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Sixteen scans of uneven size for the batched form: frames 64/128/256,
# 400 to 6400 views, 1 to 8 probe modes, objects 454 to 1442 px.  Each entry
# is (n, modes, grid side, step); the object is sized to hold the raster.
BATCH16 = [
    (256, 8, 40, 30), (256, 4, 30, 40), (256, 2, 50, 24), (256, 6, 20, 60),
    (128, 4, 80, 16), (128, 8, 60, 20), (128, 1, 50, 24), (128, 3, 40, 30),
    (128, 5, 30, 40), (128, 2, 70, 18),
    (64, 8, 80, 8), (64, 1, 70, 10), (64, 2, 60, 12), (64, 6, 50, 14),
    (64, 4, 40, 16), (64, 3, 20, 20),
]


def batch16_configs():
    """Workload dicts of the sixteen-scan batch (seeds 2001..2016)."""
    out = []
    for i, (n, modes, g, step) in enumerate(BATCH16):
        side = (g - 1) * step + n + 10
        out.append(dict(n=n, modes=modes, grid=(g, g), step=step, jitter=1, obj=(side, side),
                        probe="gauss" if modes == 1 else "hg", fwhm=n / 2.0,
                        photons=1e6 if n == 64 else 1e7, seed=2001 + i))
    return out


WORKLOADS = {
    "sm64": dict(n=64, modes=1, grid=(10, 10), step=8, jitter=1,
                 obj=(160, 160), probe="gauss", fwhm=32.0, photons=1e6,
                 seed=1001),
    "mm128": dict(n=128, modes=4, grid=(50, 50), step=10, jitter=1,
                  obj=(640, 640), probe="hg", fwhm=64.0, photons=1e7,
                  seed=1002),
    "mm256": dict(n=256, modes=8, grid=(100, 100), step=18, jitter=1,
                  obj=(2100, 2100), probe="hg", fwhm=64.0, photons=1e7,
                  seed=1003),
}

HG4_WEIGHTS = (0.6, 0.25, 0.1, 0.05)


@dataclass
class Scan:
    """One synthetic ptychographic scan (all arrays are host numpy arrays
    unless a device backend produced ``intensities``)."""
    n: int
    modes: int
    pos: np.ndarray            # int32 [J, 2]: top-left (row, col) of each footprint
    probe: np.ndarray          # complex128 [M, N, N]: true probe modes
    obj: np.ndarray            # complex128 [H, W]: true object
    intensities: object        # float32 [J, N, N] (numpy, or a torch tensor on a device)
    meta: dict = field(default_factory=dict)

    @property
    def views(self) -> int:
        return int(self.pos.shape[0])

    @property
    def obj_shape(self):
        return tuple(self.obj.shape)


def _gaussian_smooth_periodic(a: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic convolution of a real 2-D field with a unit-sum Gaussian."""
    h, w = a.shape
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (fy ** 2 + fx ** 2))
    return np.fft.irfft2(np.fft.rfft2(a) * g, s=a.shape)


def grf_object(shape, rng: np.random.Generator, corr_px: float = 4.0,
               amp_range=(0.5, 1.0), phase_range=(-math.pi / 2, math.pi / 2)):
    """Complex object from two Gaussian random fields (correlation length
    ``corr_px``), min-max mapped to the amplitude and phase ranges."""
    def field01():
        f = _gaussian_smooth_periodic(rng.standard_normal(shape), corr_px)
        f -= f.min()
        return f / max(f.max(), 1e-300)
    amp = amp_range[0] + (amp_range[1] - amp_range[0]) * field01()
    ph = phase_range[0] + (phase_range[1] - phase_range[0]) * field01()
    return amp * np.exp(1j * ph)


def _centered_grid(n: int):
    c = (n - 1) / 2.0
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    return y - c, x - c


def gaussian_probe(n: int, fwhm: float, photons: float):
    """Single probe mode: Gaussian amplitude of the given FWHM (in px) times a
    quadratic phase that reaches pi at radius fwhm/2; scaled so that the
    total power sum |P|^2 equals ``photons``.  Shape [1, n, n]."""
    y, x = _centered_grid(n)
    r2 = x * x + y * y
    amp = np.exp(-4.0 * math.log(2.0) * r2 / fwhm ** 2 / 2.0)
    p = amp * np.exp(1j * math.pi * r2 / (fwhm / 2.0) ** 2)
    p *= math.sqrt(photons / np.sum(np.abs(p) ** 2))
    return p[None].astype(np.complex128)


def _hermite(order: int, t: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomial H_order(t) by the three-term recurrence."""
    h0 = np.ones_like(t)
    if order == 0:
        return h0
    h1 = 2.0 * t
    for m in range(1, order):
        h0, h1 = h1, 2.0 * t * h1 - 2.0 * m * h0
    return h1


def hg_orders(modes: int):
    """Mode orders (m along x, n along y): the first four are elongated along
    x (fly-scan motion), then the same four with one node along y, etc."""
    out = []
    ny = 0
    while len(out) < modes:
        for mx in range(4):
            if len(out) < modes:
                out.append((mx, ny))
        ny += 1
    return out


def hg_weights(modes: int):
    if modes == 4:
        return np.array(HG4_WEIGHTS)
    w = 0.45 ** np.arange(modes)
    return w / w.sum()


def hg_probe_modes(n: int, modes: int, fwhm: float, photons: float):
    """Orthonormal Hermite-Gauss probe modes with a common quadratic phase,
    Gram-Schmidt orthonormalised in FP64, mode k carrying power
    ``photons * weight_k``.  Shape [modes, n, n]."""
    y, x = _centered_grid(n)
    w0 = fwhm / math.sqrt(2.0 * math.log(2.0))
    r2 = x * x + y * y
    env = np.exp(-r2 / w0 ** 2) * np.exp(1j * math.pi * r2 / (fwhm / 2.0) ** 2)
    basis = []
    for (mx, my) in hg_orders(modes):
        b = _hermite(mx, math.sqrt(2.0) * x / w0) * _hermite(my, math.sqrt(2.0) * y / w0) * env
        for q in basis:
            b = b - np.vdot(q, b) * q
        b = b / math.sqrt(np.vdot(b, b).real)
        basis.append(b)
    wts = hg_weights(modes)
    return np.stack([math.sqrt(photons * wk) * bk for wk, bk in zip(wts, basis)]).astype(np.complex128)


def raster_positions(grid, step: int, jitter: int, n: int, obj_shape,
                     rng: np.random.Generator):
    """Integer top-left corners of a ny x nx raster, centred in the object,
    each jittered by a uniform integer in [-jitter, jitter]."""
    ny, nx = grid
    h, w = obj_shape
    span_y = (ny - 1) * step + n
    span_x = (nx - 1) * step + n
    oy = (h - span_y) // 2
    ox = (w - span_x) // 2
    if oy < jitter or ox < jitter:
        raise ValueError("object too small for the scan")
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r = oy + iy.ravel() * step
    c = ox + ix.ravel() * step
    if jitter:
        r = r + rng.integers(-jitter, jitter + 1, size=r.shape)
        c = c + rng.integers(-jitter, jitter + 1, size=c.shape)
    pos = np.stack([r, c], axis=1).astype(np.int32)
    assert pos.min() >= 0 and pos[:, 0].max() + n <= h and pos[:, 1].max() + n <= w
    return pos


def simulate_intensities(probe, obj, pos, rng=None, noise=True, backend="numpy",
                         device=None, seed=0, chunk=64):
    """Recorded intensities sum_k |F[P_k * O_patch_j]|^2 (ortho 2-D DFT,
    DC at [0, 0]) with optional Poisson noise.

    backend="numpy": FP64 on the host, Poisson from ``rng``; returns float64.
    backend="torch": complex64 on ``device`` in chunks of views, Poisson from a
    torch.Generator seeded with ``seed``; returns a float32 torch tensor."""
    n = probe.shape[-1]
    j_total = pos.shape[0]
    if backend == "numpy":
        out = np.empty((j_total, n, n), dtype=np.float64)
        for j in range(j_total):
            r, c = int(pos[j, 0]), int(pos[j, 1])
            ex = probe * obj[None, r:r + n, c:c + n]
            out[j] = np.sum(np.abs(np.fft.fft2(ex, norm="ortho")) ** 2, axis=0)
        if noise:
            out = rng.poisson(out).astype(np.float64)
        return out
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    p_t = torch.from_numpy(probe.astype(np.complex64)).to(dev)
    o_t = torch.from_numpy(obj.astype(np.complex64)).to(dev)
    out = torch.empty((j_total, n, n), dtype=torch.float32, device=dev)
    ar = torch.arange(n, device=dev)
    pos_t = torch.from_numpy(pos.astype(np.int64)).to(dev)
    for j0 in range(0, j_total, chunk):
        j1 = min(j_total, j0 + chunk)
        rr = pos_t[j0:j1, 0][:, None, None] + ar[None, :, None]
        cc = pos_t[j0:j1, 1][:, None, None] + ar[None, None, :]
        patch = o_t[rr, cc]                                   # [b, n, n]
        ex = p_t[None] * patch[:, None]                       # [b, M, n, n]
        inten = (torch.fft.fft2(ex, norm="ortho").abs() ** 2).sum(dim=1)
        if noise:
            inten = torch.poisson(inten, generator=gen)
        out[j0:j1] = inten
    return out


def make_scan(name_or_cfg, noise=True, backend="numpy", device=None, seed=None,
              views=None):
    """Build a named workload (or a dict with the same keys).  ``views``
    keeps only the first ``views`` positions (a subset of the same scan)."""
    cfg = dict(WORKLOADS[name_or_cfg]) if isinstance(name_or_cfg, str) else dict(name_or_cfg)
    if seed is None:
        seed = cfg.get("seed", 0)
    rng = np.random.Generator(np.random.PCG64(seed))
    n, modes = cfg["n"], cfg["modes"]
    obj = grf_object(cfg["obj"], rng)
    if cfg["probe"] == "gauss":
        if modes != 1:
            raise ValueError("gauss probe is single-mode")
        probe = gaussian_probe(n, cfg["fwhm"], cfg["photons"])
    else:
        probe = hg_probe_modes(n, modes, cfg["fwhm"], cfg["photons"])
    pos = raster_positions(cfg["grid"], cfg["step"], cfg["jitter"], n, cfg["obj"], rng)
    if views is not None:
        pos = pos[:views].copy()
    inten = simulate_intensities(probe, obj, pos, rng=rng, noise=noise, backend=backend,
                                 device=device, seed=seed)
    if backend == "numpy":
        inten = inten.astype(np.float32)
    return Scan(n=n, modes=modes, pos=pos, probe=probe, obj=obj, intensities=inten,
                meta=dict(cfg, seed=seed, noise=noise, backend=backend))


def initial_guess(scan: Scan, rng: np.random.Generator, kind="perturbed"):
    """Starting (P0, O0).  ``known_probe``: true probe, flat object.
    ``perturbed``: flat object with a weak random phase, probe modes with
    random multiplicative amplitude/phase noise (so that every mode is
    updated from a non-trivial state)."""
    h, w = scan.obj_shape
    if kind == "known_probe":
        return scan.probe.copy(), np.ones((h, w), dtype=np.complex128)
    obj0 = np.exp(1j * 0.1 * rng.standard_normal((h, w)))
    noise = 1.0 + 0.2 * (rng.standard_normal(scan.probe.shape) + 1j * rng.standard_normal(scan.probe.shape))
    return scan.probe * noise, obj0


def random_exit_waves(probe, obj, pos, rng: np.random.Generator, rel=0.3):
    """Exit waves near the field products P_k * O_patch_j, with complex
    Gaussian noise of relative size ``rel`` (a generic DM state)."""
    n = probe.shape[-1]
    j_total = pos.shape[0]
    out = np.empty((j_total,) + probe.shape, dtype=np.complex128)
    for j in range(j_total):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        prod = probe * obj[None, r:r + n, c:c + n]
        noise = rng.standard_normal(prod.shape) + 1j * rng.standard_normal(prod.shape)
        out[j] = prod + rel * np.abs(prod).mean() * noise
    return out


def random_exit_waves_device(probe, obj, pos, seed, rel=0.3, device="cuda", chunk=256):
    """Device counterpart of ``random_exit_waves`` for scans too large for
    the host: psi_j = P_k O_patch_j + rel * mean|P O_patch_j| * (a + i b) with
    a, b standard normal from a torch.Generator seeded with ``seed``.
    ``probe`` and ``obj`` are complex64 arrays; returns a complex64 tensor
    [J, M, N, N] on ``device``."""
    import torch
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    p_t = torch.as_tensor(np.ascontiguousarray(probe, np.complex64)).to(dev)
    o_t = torch.as_tensor(np.ascontiguousarray(obj, np.complex64)).to(dev)
    n = p_t.shape[-1]
    j_total = pos.shape[0]
    out = torch.empty((j_total,) + tuple(p_t.shape), dtype=torch.complex64, device=dev)
    ar = torch.arange(n, device=dev)
    pos_t = torch.from_numpy(pos.astype(np.int64)).to(dev)
    for j0 in range(0, j_total, chunk):
        j1 = min(j_total, j0 + chunk)
        rr = pos_t[j0:j1, 0][:, None, None] + ar[None, :, None]
        cc = pos_t[j0:j1, 1][:, None, None] + ar[None, None, :]
        prod = p_t[None] * o_t[rr, cc][:, None]                      # [b, M, n, n]
        scale = rel * prod.abs().mean(dim=(1, 2, 3), keepdim=True)
        re = torch.randn(prod.shape, generator=gen, device=dev, dtype=torch.float32)
        im = torch.randn(prod.shape, generator=gen, device=dev, dtype=torch.float32)
        out[j0:j1] = prod + scale * torch.complex(re, im)
    return out
