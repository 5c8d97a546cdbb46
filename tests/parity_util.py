"""Helpers shared by the GPU parity tests: build a seeded case, run one (or
more) iterations through the C ABI and through the FP64 oracle from the same
complex64-rounded state, and compare."""
from __future__ import annotations

import numpy as np

from oracle import dm as odm
from synth import make_scan, initial_guess, random_exit_waves

# One-iteration parity bound for the FP32 path (relative L2 against the
# FP64 oracle), as the target states.
REL_L2 = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / den) if den > 0 else float(np.linalg.norm(a.ravel()))


def case(n, modes, grid, step, obj, seed, jitter=1, probe="hg", fwhm=None, photons=1e6, noise=True):
    cfg = dict(n=n, modes=modes, grid=grid, step=step, jitter=jitter, obj=obj,
               probe=("gauss" if modes == 1 and probe == "gauss" else "hg"),
               fwhm=fwhm or n / 2.0, photons=photons, seed=seed)
    s = make_scan(cfg, noise=noise)
    rng = np.random.default_rng(seed + 7)
    p0, o0 = initial_guess(s, rng, kind="perturbed")
    p0 = p0.astype(np.complex64)
    o0 = o0.astype(np.complex64)
    psi0 = random_exit_waves(p0.astype(np.complex128), o0.astype(np.complex128), s.pos, rng).astype(np.complex64)
    return s, p0, o0, psi0


def run_gpu(s, p0, o0, psi0, n_iter=1, beta=0.8, delta_rel=1e-6, n_inner=1, probe_update_start=0,
            scratch_bytes=0, use_torch_allocator=None, order="gauss-seidel", form=None):
    from paper_1808_10375_gb300 import dm
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w, beta=beta,
                                  denom_floor_rel=delta_rel, n_inner=n_inner,
                                  probe_update_start=probe_update_start, scratch_bytes=scratch_bytes,
                                  update_order=dm.DM_ORDER_JACOBI if order == "jacobi" else dm.DM_ORDER_GAUSS_SEIDEL)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0, use_torch_allocator=use_torch_allocator)
    if psi0 is not None:
        dm.dm_set_exit_waves(ctx, psi0)
    if form is not None:
        dm.dm_set_fourier_form(ctx, form)
        assert dm.dm_get_fourier_form(ctx) == form
    dm.dm_iterate(ctx, n_iter)
    out = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
               metrics=[dm.dm_get_error(ctx, i) for i in range(n_iter)])
    dm.dm_free(ctx)
    return out


def run_oracle(s, p0, o0, psi0, n_iter=1, beta=0.8, delta_rel=1e-6, n_inner=1, probe_update_start=0,
               order="gauss-seidel"):
    psi = psi0.astype(np.complex128) if psi0 is not None else odm.init_exit_waves(
        p0.astype(np.complex128), o0.astype(np.complex128), s.pos)
    probe = p0.astype(np.complex128)
    obj = o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float64)
    hist = []
    for t in range(n_iter):
        psi, probe, obj, m = odm.dm_iteration(psi, probe, obj, s.pos, inten, beta, delta_rel, n_inner,
                                              update_probe=(t >= probe_update_start), order=order)
        hist.append(m)
    return dict(psi=psi, probe=probe, obj=obj, metrics=hist)


def compare(g, o, tol=REL_L2, metric_rtol=1e-4):
    errs = {"psi": rel_l2(g["psi"], o["psi"]), "obj": rel_l2(g["obj"], o["obj"])}
    for k in range(o["probe"].shape[0]):
        errs[f"probe{k}"] = rel_l2(g["probe"][k], o["probe"][k])
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"relative L2 above {tol}: {bad} (all: {errs})"
    for (eo, ep, ef), m in zip(g["metrics"], o["metrics"]):
        assert abs(eo - m["eps_obj"]) <= metric_rtol * max(m["eps_obj"], 1e-12) + 1e-9, (eo, m["eps_obj"])
        assert abs(ef - m["fourier_err"]) <= metric_rtol * max(m["fourier_err"], 1e-12) + 1e-9, (ef, m["fourier_err"])
        for a, b in zip(ep, m["eps_probe"]):
            assert abs(a - b) <= metric_rtol * max(b, 1e-12) + 1e-9, (a, b)
    return errs
