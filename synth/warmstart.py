"""Training pairs for the learned warm start, and the scan it is judged on.

A pair is one recorded diffraction amplitude of a 128 x 128 footprint under
the 4-mode probe (the fly-scan probe of the 4-mode workload) and the object's
amplitude and phase over the central 64 x 64 pixels of that footprint.  The
footprints are random crops of large seeded objects drawn with the same
Gaussian-random-field recipe as the scans (so the network sees the objects'
own distribution), and the intensities are the exact mixed-state model of
Eq. 1 with Poisson counting noise.  Like the rest of this package it holds
none of the difference-map iteration.
"""
from __future__ import annotations

import math

import numpy as np

from .scan import grf_object, hg_probe_modes

N = 128          # frame and footprint side
PATCH = 64       # predicted central patch side
MODES = 4
FWHM = 64.0
PHOTONS = 1e7


def probe():
    """The 4-mode Hermite-Gauss probe of the 4-mode workload (FWHM 64 px)."""
    return hg_probe_modes(N, MODES, FWHM, PHOTONS)


def input_from_intensity(inten):
    """Network input from recorded intensities [..., N, N]: log(1 + sqrt(I)),
    scaled to order one."""
    import torch
    return torch.log1p(torch.sqrt(torch.clamp(inten, min=0.0))) / 4.0


def target_from_object(patch):
    """[..., 2, 64, 64] target (amplitude, phase) of the central 64 x 64 pixels
    of complex footprints [..., N, N]."""
    import torch
    c = (N - PATCH) // 2
    centre = patch[..., c:c + PATCH, c:c + PATCH]
    return torch.stack([centre.abs(), torch.angle(centre)], dim=-3).float()


def pairs(count, seed, device="cuda", objects=8, object_side=768, noise=True):
    """``count`` (input [count, 1, N, N], target [count, 2, 64, 64]) pairs on
    ``device``: crops of ``objects`` seeded objects, intensities of Eq. 1."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    objs = torch.from_numpy(np.stack([grf_object((object_side, object_side), rng) for _ in range(objects)])
                            .astype(np.complex64)).to(device)
    p = torch.from_numpy(probe().astype(np.complex64)).to(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    which = torch.from_numpy(rng.integers(0, objects, count)).to(device)
    ys = torch.from_numpy(rng.integers(0, object_side - N, count)).to(device)
    xs = torch.from_numpy(rng.integers(0, object_side - N, count)).to(device)
    ar = torch.arange(N, device=device)
    x_out = torch.empty((count, 1, N, N), dtype=torch.float32, device=device)
    t_out = torch.empty((count, 2, PATCH, PATCH), dtype=torch.float32, device=device)
    for i0 in range(0, count, 256):
        i1 = min(count, i0 + 256)
        rr = ys[i0:i1, None, None] + ar[None, :, None]
        cc = xs[i0:i1, None, None] + ar[None, None, :]
        patch = objs[which[i0:i1, None, None], rr, cc]                     # [b, N, N]
        inten = (torch.fft.fft2(p[None] * patch[:, None], norm="ortho").abs() ** 2).sum(dim=1)
        if noise:
            inten = torch.poisson(inten, generator=gen)
        x_out[i0:i1, 0] = input_from_intensity(inten)
        t_out[i0:i1] = target_from_object(patch)
    return x_out, t_out


def footprints(obj, pos):
    """The N x N footprints [J, N, N] of a complex object (torch tensor) at
    top-left corners ``pos`` [J, 2]."""
    import torch
    dev = obj.device
    p = torch.as_tensor(np.asarray(pos), device=dev).long()
    ar = torch.arange(N, device=dev)
    return obj[p[:, 0, None, None] + ar[None, :, None], p[:, 1, None, None] + ar[None, None, :]]


def _unit(s):
    """s / |s|, and 1 where s = 0."""
    import torch
    mag = torch.abs(s)
    return torch.where(mag > 0, s / torch.clamp(mag, min=1e-30), torch.ones_like(s))


def stitch(pred, pos, obj_shape, align=False, sweeps=20):
    """Object start from per-view predictions [J, 2, 64, 64] (amplitude, phase)
    at footprints with top-left corners ``pos`` [J, 2]: overlapping
    predictions are averaged as complex values; pixels no prediction covers
    are 1.

    One view's intensities fix its patch z_j only up to a constant phase
    factor w_j, so with ``align`` the factors are chosen to make the
    overlapping patches agree: maximise sum_{j != k} Re(conj(w_j z_j) w_k z_k)
    summed over the overlaps, the angular synchronisation problem.  Start:
    each prediction in the order of ``pos`` takes the phase that best fits
    what the views before it laid down (w_j = S_j/|S_j|, S_j = sum conj(z_j)
    acc over its patch).  Then ``sweeps`` steps of the projected power method
    (every w_j at once from the sum of all other aligned patches over its
    patch), which removes the drift the one-pass start accumulates along the
    scan.  Last, all patches are turned together so that their sum is real and
    positive: the pixels no prediction covers keep the value 1, and the
    predictions must share its phase reference (the objects have mean phase
    about 0)."""
    import torch
    h, w = obj_shape
    dev = pred.device
    c = (N - PATCH) // 2
    z = pred[:, 0] * torch.exp(1j * pred[:, 1])
    if align:
        acc2 = torch.zeros((h, w), dtype=torch.complex64, device=dev)
        u = torch.empty_like(z)
        for j in range(pos.shape[0]):
            r, q = int(pos[j, 0]) + c, int(pos[j, 1]) + c
            u[j] = z[j] * _unit(torch.sum(torch.conj(z[j]) * acc2[r:r + PATCH, q:q + PATCH]))
            acc2[r:r + PATCH, q:q + PATCH] += u[j]
        p = torch.as_tensor(np.asarray(pos), device=dev).long() + c
        ar = torch.arange(PATCH, device=dev)
        idx = ((p[:, 0, None, None] + ar[None, :, None]) * w + p[:, 1, None, None] + ar[None, None, :]).reshape(-1)
        for _ in range(sweeps):
            acc = torch.zeros(h * w, dtype=torch.complex64, device=dev).index_add_(0, idx, u.reshape(-1))
            others = acc[idx].reshape(z.shape) - u
            u = z * _unit(torch.sum(torch.conj(z) * others, dim=(1, 2)))[:, None, None]
        z = u * torch.conj(_unit(torch.sum(u)))
    acc = torch.zeros((h, w), dtype=torch.complex64, device=dev)
    cnt = torch.zeros((h, w), dtype=torch.float32, device=dev)
    for j in range(pos.shape[0]):
        r, q = int(pos[j, 0]) + c, int(pos[j, 1]) + c
        acc[r:r + PATCH, q:q + PATCH] += z[j]
        cnt[r:r + PATCH, q:q + PATCH] += 1
    out = torch.ones((h, w), dtype=torch.complex64, device=dev)
    m = cnt > 0
    out[m] = acc[m] / cnt[m]
    return out


def object_error(obj, truth, covered):
    """Relative L2 error of ``obj`` against ``truth`` on the ``covered`` pixels
    after the best complex scalar (the object is fixed only up to one)."""
    a = np.asarray(obj)[covered].astype(np.complex128)
    b = np.asarray(truth)[covered].astype(np.complex128)
    c = np.vdot(a, b) / max(np.vdot(a, a).real, 1e-300)
    return float(np.linalg.norm(c * a - b) / np.linalg.norm(b))
