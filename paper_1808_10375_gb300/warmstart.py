"""Learned warm start for the difference map: train the encoder-decoder of
the C ABI (dm_net_*) on simulated pairs, stitch its per-view predictions into
a starting object, and compare DM from that start with DM from a flat start.

Every network step runs in the library's kernels (forward, backward, Adam);
this module only draws the data from the simulator, calls the C ABI and keeps
the records.  DM decides: the comparison reports the object error of both
runs against the true object at every iteration.
"""
from __future__ import annotations

import time

import numpy as np

from . import dm


def train(net, steps, batch=64, lr=1e-3, seed=0, data_count=50000, device="cuda"):
    """``steps`` Adam steps on ``data_count`` simulated pairs (drawn once,
    visited in seeded random order); returns the loss of every 50th step."""
    import torch
    from synth import warmstart as ws
    x, t = ws.pairs(data_count, seed, device)
    g = torch.Generator(device=device)
    g.manual_seed(seed + 1)
    losses = []
    order = torch.randperm(data_count, generator=g, device=device)
    k = 0
    for s in range(steps):
        if k + batch > data_count:
            order = torch.randperm(data_count, generator=g, device=device)
            k = 0
        idx = order[k:k + batch]
        k += batch
        want = s % 50 == 0 or s == steps - 1
        loss = dm.dm_net_train_step(net, x[idx].contiguous(), t[idx].contiguous(), lr, want_loss=want)
        if want:
            losses.append((s, loss))
    return losses


def predict_start(net, intensities, pos, obj_shape):
    """Starting object [H, W] complex64 (CUDA) stitched from the network's
    predictions for every view of a scan (intensities [J, 128, 128])."""
    import torch
    from synth import warmstart as ws
    inten = intensities if isinstance(intensities, torch.Tensor) else torch.from_numpy(np.asarray(intensities))
    inten = inten.float().cuda()
    preds = []
    for j0 in range(0, inten.shape[0], net.max_batch):
        xb = ws.input_from_intensity(inten[j0:j0 + net.max_batch])[:, None].contiguous()
        preds.append(dm.dm_net_forward(net, xb))
    return ws.stitch(torch.cat(preds), pos, obj_shape)


def compare(scan, probe0, obj_warm, iters, record_every=5, flat=None):
    """DM from a flat object and from ``obj_warm`` (same probe ``probe0``):
    object error against the scan's true object on covered pixels after the
    best complex scalar, recorded every ``record_every`` iterations, and the
    wall time of each run."""
    from synth import warmstart as ws
    h, w = scan.obj_shape
    n = scan.n
    den = np.zeros((h, w))
    p2 = np.sum(np.abs(scan.probe) ** 2, axis=0)
    for r, c in scan.pos:
        den[r:r + n, c:c + n] += p2
    covered = den >= 0.1 * den.max()
    starts = {"flat": np.ones((h, w), np.complex64) if flat is None else flat,
              "warm": obj_warm.detach().cpu().numpy().astype(np.complex64) if hasattr(obj_warm, "detach")
              else np.asarray(obj_warm, np.complex64)}
    out = {}
    for name, o0 in starts.items():
        params = dm.dm_params_default(n=n, modes=scan.modes, views=scan.views, obj_h=h, obj_w=w)
        ctx = dm.dm_init(params, scan.pos, scan.intensities, probe0.astype(np.complex64), o0)
        errs = [(0, ws.object_error(o0, scan.obj, covered))]
        t0 = time.perf_counter()
        for it in range(record_every, iters + 1, record_every):
            dm.dm_iterate(ctx, record_every)
            errs.append((it, ws.object_error(dm.dm_get_object(ctx), scan.obj, covered)))
        wall = time.perf_counter() - t0
        dm.dm_free(ctx)
        out[name] = {"errors": errs, "wall_s": wall}
    return out


def judged_start(scan, probe0, obj_warm, trial_iters=10):
    """Plain DM as the judge and the fallback: run ``trial_iters`` iterations
    from the flat start and from ``obj_warm`` and keep the start whose Fourier
    error (the library's E_F, which needs no ground truth) is lower.  Returns
    (chosen start as a host array, "warm" or "flat", {start: E_F})."""
    h, w = scan.obj_shape
    warm = obj_warm.detach().cpu().numpy().astype(np.complex64) if hasattr(obj_warm, "detach") \
        else np.asarray(obj_warm, np.complex64)
    starts = {"flat": np.ones((h, w), np.complex64), "warm": warm}
    ef = {}
    for name, o0 in starts.items():
        params = dm.dm_params_default(n=scan.n, modes=scan.modes, views=scan.views, obj_h=h, obj_w=w)
        ctx = dm.dm_init(params, scan.pos, scan.intensities, probe0.astype(np.complex64), o0)
        dm.dm_iterate(ctx, trial_iters)
        ef[name] = dm.dm_get_error(ctx)[2]
        dm.dm_free(ctx)
    pick = "warm" if ef["warm"] < ef["flat"] else "flat"
    return starts[pick], pick, ef


def iterations_to(errors, level):
    """First recorded iteration whose error is at or below ``level``."""
    for it, e in errors:
        if e <= level:
            return it
    return None
