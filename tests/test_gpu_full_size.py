"""Parity at full size: the 8-mode 256x256-frame workload with 10,000 views
and a 2100x2100 object, built and launched exactly as bench.py times it
(same seeded inputs, default parameters and scratch budget, a dedicated
stream), one iteration from seeded random exit waves.

The oracle cannot run a whole iteration at this size in seconds, so the
checks are on outputs it can compute one by one:

* psi after Eq. 3 for sampled views (first, last, middle, random ones):
  element by element, relative L2 <= 1e-5 per view;
* the object after Eq. 5 at sampled pixels (an interior block, the corners
  of the first and last footprints, pixels no footprint covers): the oracle
  computes the new exit waves of every view covering those pixels itself;
* the Eq. 6 monitors against the returned object and probe.

The probe after Eq. 4 at full size, and the object over the whole array, are
compared with a complete oracle iteration in test_gpu_full_size_oracle.py.
"""
import numpy as np
import pytest

from oracle import dm as odm
from parity_util import REL_L2, rel_l2

pytestmark = pytest.mark.gpu

BETA = 0.8
DELTA_REL = 1e-6


@pytest.fixture(scope="module")
def full_run():
    import torch
    import bench
    from paper_1808_10375_gb300 import build, dm
    from synth import random_exit_waves_device
    build.build()

    s, p0, o0 = bench.make_inputs(None, "cuda")
    n, m, j_total = s.n, s.modes, s.views
    h, w = s.obj_shape
    params = dm.dm_params_default(n=n, modes=m, views=j_total, obj_h=h, obj_w=w, beta=BETA,
                                  denom_floor_rel=DELTA_REL)
    prev_stream = torch.cuda.current_stream()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = dm.dm_init(params, dev(s.pos), s.intensities, dev(p0), dev(o0), stream=stream.cuda_stream)
    psi0 = random_exit_waves_device(p0, o0, s.pos, seed=s.meta["seed"] + 11, device="cuda")
    dm.dm_set_exit_waves(ctx, psi0)
    dm.dm_sync(ctx)

    rng = np.random.default_rng(2024)
    views = sorted(set([0, 1, j_total // 2, j_total - 2, j_total - 1] +
                       rng.choice(j_total, 5, replace=False).tolist()))
    # object pixels: an interior block, the first and last footprint corners,
    # and (chosen below) pixels outside every footprint
    block = [(1040 + a, 1013 + b) for a in range(4) for b in range(4)]
    last = s.pos[j_total - 1]
    corners = [(int(s.pos[0, 0]), int(s.pos[0, 1])), (int(last[0]) + n - 1, int(last[1]) + n - 1)]
    den_o = odm.object_denominator(p0.astype(np.complex128), s.pos, (h, w))
    uncovered = np.argwhere(den_o == 0)
    assert len(uncovered) > 0
    outside = [tuple(int(x) for x in uncovered[0]), tuple(int(x) for x in uncovered[-1])]
    pixels = block + corners + outside
    need = set(views)
    for px in pixels:
        need.update(odm.views_covering(s.pos, n, px).tolist())
    need = sorted(need)
    idx = torch.tensor(need, device="cuda")
    psi0_h = dict(zip(need, psi0.index_select(0, idx).cpu().numpy()))
    inten_h = dict(zip(need, s.intensities.index_select(0, idx).cpu().numpy()))
    del psi0
    torch.cuda.empty_cache()

    dm.dm_iterate(ctx, 1)
    psi1 = dm.dm_get_exit_waves(ctx, device=True)
    o1 = dm.dm_get_object(ctx).astype(np.complex128)
    p1 = dm.dm_get_probe(ctx).astype(np.complex128)
    eps_obj, eps_probe, _ = dm.dm_get_error(ctx)
    dm.dm_free(ctx)
    psi1_views = dict(zip(views, psi1.index_select(0, torch.tensor(views, device="cuda")).cpu().numpy()))
    del psi1
    torch.cuda.empty_cache()
    torch.cuda.set_stream(prev_stream)
    return dict(s=s, p0=p0, o0=o0, n=n, m=m, views=views, pixels=pixels, den_o=den_o,
                psi0=psi0_h, inten=inten_h, o1=o1, p1=p1, eps_obj=eps_obj, eps_probe=eps_probe,
                psi1_views=psi1_views)


@pytest.fixture(scope="module")
def oracle_waves(full_run):
    """psi after Eq. 3, computed by the oracle for every view it needs."""
    r = full_run
    probe = r["p0"].astype(np.complex128)
    obj = r["o0"].astype(np.complex128)
    out = {}
    for j, psi0 in r["psi0"].items():
        out[j], _, _ = odm.fourier_update_view(psi0.astype(np.complex128), probe, obj, r["s"].pos[j],
                                               r["inten"][j].astype(np.float64), BETA)
    return out


def test_full_size_exit_waves_of_sampled_views(full_run, oracle_waves):
    for j in full_run["views"]:
        err = rel_l2(full_run["psi1_views"][j], oracle_waves[j])
        assert err <= REL_L2, (j, err)


def test_full_size_object_at_sampled_pixels(full_run, oracle_waves):
    r = full_run
    probe = r["p0"].astype(np.complex128)
    obj = r["o0"].astype(np.complex128)
    want = odm.object_update_at(r["pixels"], lambda j: oracle_waves[j], probe, obj, r["s"].pos,
                                DELTA_REL, r["den_o"].max())
    got = np.array([r["o1"][px] for px in r["pixels"]])
    assert rel_l2(got, want) <= REL_L2
    # pixels outside every footprint are returned unchanged
    for px in r["pixels"][-2:]:
        assert r["o1"][px] == r["o0"][px]


def test_full_size_monitors(full_run):
    r = full_run
    o0 = r["o0"].astype(np.complex128)
    p0 = r["p0"].astype(np.complex128)
    eo = np.sqrt(np.sum(np.abs(r["o1"] - o0) ** 2) / np.sum(np.abs(r["o1"]) ** 2))
    assert r["eps_obj"] == pytest.approx(eo, rel=1e-4)
    for k in range(r["m"]):
        ep = np.sqrt(np.sum(np.abs(r["p1"][k] - p0[k]) ** 2) / np.sum(np.abs(r["p1"][k]) ** 2))
        assert r["eps_probe"][k] == pytest.approx(ep, rel=1e-4)
