"""Whole-iteration parity at full size against the FP64 oracle: the 8-mode
256x256-frame workload with 10,000 views and a 2100x2100 object, launched as
bench.py times it, one iteration from the exit waves dm_init builds
(psi_j^k = P_k O on every footprint).

The oracle runs that whole iteration on the host with its views split over
processes (``oracle.parallel.ProcessDM``, each worker single-threaded; the
FP64 exit waves of 10,000 views do not fit in host memory, so each worker
recomputes its views' new exit waves for Eq. 4 instead of storing them).
Nothing is taken from the CUDA path.  Compared element by element:

* the object after Eq. 5 over the whole array;
* every probe mode after Eq. 4 over the whole frame;
* the Fourier error and the Eq. 6 monitors.

About a minute of host time on 16 cores.
"""
import numpy as np
import pytest

from parity_util import REL_L2, rel_l2

pytestmark = pytest.mark.gpu

BETA = 0.8
DELTA_REL = 1e-6


@pytest.fixture(scope="module")
def full_run():
    import torch
    import bench
    from paper_1808_10375_gb300 import build, dm
    from oracle.parallel import ProcessDM
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
    got = dict(obj=dm.dm_get_object(ctx).astype(np.complex128), probe=dm.dm_get_probe(ctx).astype(np.complex128),
               metrics=dm.dm_get_error(ctx))
    dm.dm_free(ctx)
    torch.cuda.set_stream(prev)
    inten = s.intensities.cpu().numpy()
    s.intensities = None
    torch.cuda.empty_cache()

    with ProcessDM(inten, s.pos, p0.astype(np.complex128), o0.astype(np.complex128), beta=BETA,
                   delta_rel=DELTA_REL, keep_psi=False) as pdm:
        want_metrics = pdm.iterate()
    return dict(got=got, obj=pdm.obj, probe=pdm.probe, metrics=want_metrics, m=m)


def test_full_size_object_matches_oracle_everywhere(full_run):
    assert rel_l2(full_run["got"]["obj"], full_run["obj"]) <= REL_L2


def test_full_size_probe_matches_oracle_everywhere(full_run):
    for k in range(full_run["m"]):
        err = rel_l2(full_run["got"]["probe"][k], full_run["probe"][k])
        assert err <= REL_L2, (k, err)


def test_full_size_monitors_match_oracle(full_run):
    eps_obj, eps_probe, ferr = full_run["got"]["metrics"]
    want = full_run["metrics"]
    assert ferr == pytest.approx(want["fourier_err"], rel=1e-4)
    assert eps_obj == pytest.approx(want["eps_obj"], rel=1e-4)
    assert np.allclose(eps_probe, want["eps_probe"], rtol=1e-4, atol=0)
