"""Learned warm start for the difference map: train the encoder-decoder of
the C ABI (dm_net_*) on simulated pairs, stitch its per-view predictions into
a starting object, and compare DM from that start with DM from a flat start.

Training pairs come in two kinds.  Crops (``synth.warmstart.pairs``): random
footprints of seeded objects, with the true object patch as the target.
DM-refined (``refined_pairs``): every view of simulated 4-mode scans, with
the target taken from the object that DM itself reconstructs from that scan
in a few iterations from the flat start with the probe held; the network
then learns what DM produces, in the gauge DM settles in.

Every network step runs in the library's kernels (forward, backward, Adam),
and every DM iteration in the library's DM kernels; this module only draws
the data from the simulator, calls the C ABI and keeps the records.  DM
decides: the comparison reports the object error of both runs against the
true object at every iteration.
"""
from __future__ import annotations

import time

import numpy as np

from . import dm


def refined_scan_cfg(seed):
    """A 4-mode scan shaped like the 4-mode workload (128 x 128 frames, 50 x 50
    views at 10 px, 640 x 640 object, 1e7 photons) with its own seed."""
    from synth import warmstart as ws
    return dict(n=ws.N, modes=ws.MODES, grid=(50, 50), step=10, jitter=1, obj=(640, 640), probe="hg",
                fwhm=ws.FWHM, photons=ws.PHOTONS, seed=int(seed))


def refined_pairs(scans, seed, dm_iters=20, device="cuda"):
    """DM-refined pairs from ``scans`` simulated scans (2,500 views each, seeds
    seed, seed + 1, ...): input [J, 1, 128, 128] from each view's recorded
    intensities; target [J, 2, 64, 64], the amplitude and phase of the
    central patch of the object DM reconstructs from that scan in
    ``dm_iters`` iterations (flat start, true probe held fixed); and
    ``truth``, the same patch of the true object.  Returns (x, target, truth)
    on ``device``."""
    import torch
    from synth import make_scan
    from synth import warmstart as ws
    xs, ts, gs = [], [], []
    for k in range(scans):
        scan = make_scan(refined_scan_cfg(seed + k), backend="torch", device=device)
        h, w = scan.obj_shape
        params = dm.dm_params_default(n=scan.n, modes=scan.modes, views=scan.views, obj_h=h, obj_w=w, beta=0.8,
                                      probe_update_start=1 << 30)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        ctx = dm.dm_init(params, dev(scan.pos), scan.intensities, dev(scan.probe.astype(np.complex64)),
                         dev(np.ones((h, w), np.complex64)))
        dm.dm_iterate(ctx, dm_iters)
        obj = dm.dm_get_object(ctx, device=True)
        dm.dm_free(ctx)
        xs.append(ws.input_from_intensity(scan.intensities.float())[:, None])
        ts.append(ws.target_from_object(ws.footprints(obj, scan.pos)))
        truth = torch.from_numpy(scan.obj.astype(np.complex64)).to(device)
        gs.append(ws.target_from_object(ws.footprints(truth, scan.pos)))
        del scan
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous(), torch.cat(gs).contiguous()


def fit(net, x, target):
    """How well the network's predictions for inputs x fit ``target`` (both
    [B, 2, 64, 64], amplitude and phase); see ``fit_of``."""
    import torch
    ys = torch.cat([dm.dm_net_forward(net, x[i:i + net.max_batch].contiguous())
                    for i in range(0, x.shape[0], net.max_batch)])
    return fit_of(ys, target)


def fit_of(pred, target):
    """R^2 of the amplitude |z|; R^2 of the phase after each predicted patch
    is turned by the global phase that fits its target best (one view fixes
    its patch only up to such a phase), against the target's spread about
    its own circular mean per patch; and the relative L2 distance of the
    turned complex patches.  pred and target are [B, 2, 64, 64] (a, phi) with
    z = a exp(i phi); a predicted a < 0 is the value |a| at phase phi + pi."""
    import torch
    ys = pred.double()
    t = target.double()
    zp = ys[:, 0] * torch.exp(1j * ys[:, 1])
    zt = t[:, 0] * torch.exp(1j * t[:, 1])
    ap, at = torch.abs(zp), torch.abs(zt)
    s = torch.sum(torch.conj(zp) * zt, dim=(1, 2))
    rot = torch.where(torch.abs(s) > 0, s / torch.clamp(torch.abs(s), min=1e-300), torch.ones_like(s))
    zp = zp * rot[:, None, None]
    dphi = torch.angle(zp * torch.conj(zt))
    ut = torch.exp(1j * torch.angle(zt))
    mean_t = torch.angle(torch.sum(ut, dim=(1, 2)))
    spread = torch.angle(ut * torch.exp(-1j * mean_t)[:, None, None])
    return {"amplitude_r2": float(1.0 - torch.sum((ap - at) ** 2) / torch.sum((at - at.mean()) ** 2)),
            "phase_r2_gauge_aligned": float(1.0 - torch.sum(dphi ** 2) / torch.sum(spread ** 2)),
            "complex_rel_err_gauge_aligned": float(torch.linalg.norm((zp - zt).flatten()) /
                                                   torch.linalg.norm(zt.flatten())),
            "samples": int(pred.shape[0])}


def train(net, steps, batch=64, lr=1e-3, seed=0, data_count=50000, device="cuda", data=None):
    """``steps`` Adam steps on ``data`` (inputs, targets) or, if None, on
    ``data_count`` simulated crop pairs (drawn once); the pairs are visited
    in seeded random order.  Returns the loss of every 50th step."""
    import torch
    from synth import warmstart as ws
    x, t = data if data is not None else ws.pairs(data_count, seed, device)
    data_count = x.shape[0]
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


def predict_start(net, intensities, pos, obj_shape, align=True):
    """Starting object [H, W] complex64 (CUDA) stitched from the network's
    predictions for every view of a scan (intensities [J, 128, 128]); with
    ``align`` each prediction's global phase is fitted to its neighbours
    before it is laid down."""
    import torch
    from synth import warmstart as ws
    inten = intensities if isinstance(intensities, torch.Tensor) else torch.from_numpy(np.asarray(intensities))
    inten = inten.float().cuda()
    preds = []
    for j0 in range(0, inten.shape[0], net.max_batch):
        xb = ws.input_from_intensity(inten[j0:j0 + net.max_batch])[:, None].contiguous()
        preds.append(dm.dm_net_forward(net, xb))
    return ws.stitch(torch.cat(preds), pos, obj_shape, align=align)


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
