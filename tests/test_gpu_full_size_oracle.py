"""Whole-iteration parity at full size against the FP64 oracle: the 8-mode
256x256-frame workload with 10,000 views and a 2100x2100 object, launched as
bench.py times it, one iteration from the exit waves dm_init builds
(psi_j^k = P_k O on every footprint).

The oracle runs that whole iteration here, split over host processes (a
spawn pool, each worker single-threaded): every worker takes a contiguous
range of views, applies Eq. 3 to them in FP64 and returns its share of the
Eq. 5 numerator (a band of object rows), its Fourier-error sums and the new
exit waves at a few sampled probe pixels.  From those the test forms, in
FP64 and with nothing taken from the CUDA path:

* the object of Eq. 5 over the whole array, compared element by element;
* the probe of Eq. 4 with that object, at the sampled probe pixels of every
  mode (delta from the maximum of the Eq. 4 denominator over all pixels);
* the Fourier error and the Eq. 6 object monitor.

This takes about a minute of host time on 16 cores.
"""
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np
import pytest

from parity_util import REL_L2, rel_l2

BETA = 0.8
DELTA_REL = 1e-6


def _attach(spec):
    name, shape, dtype = spec
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=dtype, buffer=shm.buf)


def _worker(args):
    """Eq. 3 in FP64 for views [a, b); returns the Eq. 5 numerator over the
    band of object rows those views cover, the Fourier-error sums and the new
    exit waves at the sampled probe pixels."""
    (a, b, specs, uy, ux) = args
    from oracle import dm as odm
    handles = [_attach(s) for s in specs]
    (_, inten), (_, pos), (_, probe), (_, obj) = handles
    n = probe.shape[-1]
    r0 = int(pos[a:b, 0].min())
    r1 = int(pos[a:b, 0].max()) + n
    num = np.zeros((r1 - r0, obj.shape[1]), np.complex128)
    pc = np.conj(probe)
    ef = isum = 0.0
    at_u = np.empty((b - a, probe.shape[0], len(uy)), np.complex128)
    for j in range(a, b):
        psi0 = odm.field_products(probe, obj, pos[j])
        psi1, e, s = odm.fourier_update_view(psi0, probe, obj, pos[j], inten[j].astype(np.float64), BETA)
        ef += e
        isum += s
        r, c = int(pos[j, 0]), int(pos[j, 1])
        num[r - r0:r - r0 + n, c:c + n] += np.sum(pc * psi1, axis=0)
        at_u[j - a] = psi1[:, uy, ux]
    for shm, _ in handles:
        shm.close()
    return a, r0, num, ef, isum, at_u


def oracle_iteration_parallel(inten, pos, probe, obj, uy, ux, workers=None):
    """One oracle iteration (Eq. 3, Eq. 5, then Eq. 4 at the probe pixels
    (uy, ux)) from psi = P O, with Eq. 3 spread over a spawn pool.  Returns
    the new object over the whole array, the probe at the sampled pixels
    [M, U], the Fourier error and the Eq. 6 object monitor."""
    from oracle import dm as odm
    jn, n, m = inten.shape[0], probe.shape[-1], probe.shape[0]
    h, w = obj.shape
    pos = np.ascontiguousarray(np.asarray(pos).astype(np.int64))
    shms, specs = [], []
    try:
        for arr in (inten, pos, probe, obj):
            shm = shared_memory.SharedMemory(create=True, size=arr.nbytes)
            np.ndarray(arr.shape, arr.dtype, buffer=shm.buf)[...] = arr
            shms.append(shm)
            specs.append((shm.name, arr.shape, arr.dtype))
        workers = workers or max(1, min(32, os.cpu_count() or 1))
        bounds = np.linspace(0, jn, 4 * workers + 1).astype(int)
        tasks = [(int(a), int(b), specs, uy, ux) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in env:
            os.environ[k] = "1"
        try:
            with mp.get_context("spawn").Pool(min(workers, len(tasks))) as pool:
                results = pool.map(_worker, tasks)
        finally:
            for k, v in env.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    finally:
        for shm in shms:
            shm.close()
            shm.unlink()

    # Eq. 5 over the whole object, from the summed numerator bands
    num_o = np.zeros((h, w), np.complex128)
    ef = isum = 0.0
    psi1_u = np.empty((jn, m, len(uy)), np.complex128)
    for a, r0, num, e, si, at_u in results:
        num_o[r0:r0 + num.shape[0]] += num
        ef += e
        isum += si
        psi1_u[a:a + at_u.shape[0]] = at_u
    den_o = odm.object_denominator(probe, pos, (h, w))
    o_want = obj.copy()
    cov = den_o > 0
    o_want[cov] = num_o[cov] / (den_o[cov] + DELTA_REL * den_o.max())
    # Eq. 4 with the new object at the sampled probe pixels
    a2 = np.abs(o_want) ** 2
    den_p = np.zeros((n, n))
    for rr, cc in pos:
        den_p += a2[rr:rr + n, cc:cc + n]
    o_at = o_want[pos[:, 0:1] + uy[None], pos[:, 1:2] + ux[None]]          # [J, U]
    num_p = np.einsum("ju,jmu->mu", np.conj(o_at), psi1_u)
    p_want = num_p / (den_p[uy, ux] + DELTA_REL * den_p.max())[None]
    return dict(o_want=o_want, p_want=p_want, ef_want=float(np.sqrt(ef / isum)),
                eps_obj_want=odm.rel_change(o_want, obj))


def test_parallel_oracle_equals_the_oracle_iteration():
    """The split over processes reproduces oracle.dm.dm_iteration (CPU)."""
    from oracle import dm as odm
    from synth import make_scan, initial_guess
    s = make_scan(dict(n=32, modes=3, grid=(5, 6), step=7, jitter=1, obj=(80, 80), probe="hg", fwhm=14.0,
                       photons=1e6, seed=9))
    p0, o0 = initial_guess(s, np.random.default_rng(9), kind="perturbed")
    probe, obj = p0.astype(np.complex128), o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float32)
    uy, ux = np.array([0, 5, 31, 17]), np.array([0, 9, 31, 3])
    got = oracle_iteration_parallel(inten, s.pos, probe, obj, uy, ux, workers=2)
    psi0 = odm.init_exit_waves(probe, obj, s.pos)
    _, p1, o1, met = odm.dm_iteration(psi0, probe, obj, s.pos, inten.astype(np.float64), BETA, DELTA_REL)
    assert rel_l2(got["o_want"], o1) <= 1e-13
    assert rel_l2(got["p_want"], p1[:, uy, ux]) <= 1e-13
    assert got["ef_want"] == pytest.approx(met["fourier_err"], rel=1e-12)
    assert got["eps_obj_want"] == pytest.approx(met["eps_obj"], rel=1e-12)


@pytest.fixture(scope="module")
def full_oracle_run():
    import torch
    import bench
    from paper_1808_10375_gb300 import build, dm
    build.build()

    s, p0, o0 = bench.make_inputs(None, "cuda")
    n, m, jn = s.n, s.modes, s.views
    h, w = s.obj_shape
    params = dm.dm_params_default(n=n, modes=m, views=jn, obj_h=h, obj_w=w, beta=BETA,
                                  denom_floor_rel=DELTA_REL)
    prev = torch.cuda.current_stream()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ctx = dm.dm_init(params, dev(s.pos), s.intensities, dev(p0), dev(o0), stream=stream.cuda_stream)
    dm.dm_iterate(ctx, 1)
    o1 = dm.dm_get_object(ctx).astype(np.complex128)
    p1 = dm.dm_get_probe(ctx).astype(np.complex128)
    eps_obj, eps_probe, ferr = dm.dm_get_error(ctx)
    dm.dm_free(ctx)
    torch.cuda.set_stream(prev)
    inten = s.intensities.cpu().numpy()
    s.intensities = None
    torch.cuda.empty_cache()

    rng = np.random.default_rng(77)
    up = [(n // 2, n // 2), (0, 0), (n - 1, n - 1)] + [tuple(int(x) for x in rng.integers(0, n, 2))
                                                       for _ in range(29)]
    uy = np.array([u[0] for u in up])
    ux = np.array([u[1] for u in up])

    probe = p0.astype(np.complex128)
    obj = o0.astype(np.complex128)
    want = oracle_iteration_parallel(inten, s.pos, probe, obj, uy, ux)
    return dict(o1=o1, p1=p1, uy=uy, ux=ux, ferr=ferr, eps_obj=eps_obj, m=m, **want)


@pytest.mark.gpu
def test_full_size_object_matches_oracle_everywhere(full_oracle_run):
    r = full_oracle_run
    assert rel_l2(r["o1"], r["o_want"]) <= REL_L2


@pytest.mark.gpu
def test_full_size_probe_matches_oracle_at_sampled_pixels(full_oracle_run):
    r = full_oracle_run
    got = r["p1"][:, r["uy"], r["ux"]]
    for k in range(r["m"]):
        assert rel_l2(got[k], r["p_want"][k]) <= REL_L2, (k, rel_l2(got[k], r["p_want"][k]))


@pytest.mark.gpu
def test_full_size_fourier_error_and_object_monitor(full_oracle_run):
    r = full_oracle_run
    assert r["ferr"] == pytest.approx(r["ef_want"], rel=1e-4)
    assert r["eps_obj"] == pytest.approx(r["eps_obj_want"], rel=1e-4)
