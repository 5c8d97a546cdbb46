"""GPU parity of the cluster form of the Fourier step (64 x 64 and 128 x 128
frames, 1 to 8 modes), through the C ABI against the FP64 oracle: one and three
iterations, more views than resident clusters (several views per cluster),
footprints at the object edges, one mode and eight, and agreement with the
strip form to FP32 rounding.  Both forms compute Eq. 3 with the constrained
transform F_c of Sec. II and the object source of Eq. 5; the cluster form
keeps each mode's frame in one CTA's shared memory and sums over the modes
through distributed shared memory."""

import numpy as np
import pytest

from parity_util import case, compare, rel_l2, run_gpu, run_oracle, REL_L2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def _dm():
    from paper_1808_10375_gb300 import dm
    return dm


@pytest.mark.parametrize("n,modes,grid,step,obj,seed", [
    (128, 4, (3, 3), 18, (170, 175), 41),
    (128, 1, (3, 2), 18, (170, 155), 42),
    (128, 3, (2, 3), 18, (160, 170), 43),
    (128, 8, (3, 3), 18, (170, 175), 44),
    (64, 4, (4, 4), 10, (100, 100), 52),
    (64, 1, (3, 4), 9, (86, 95), 53),
    (64, 8, (3, 3), 12, (92, 92), 54),
])
def test_cluster_form_matches_oracle(n, modes, grid, step, obj, seed):
    dm = _dm()
    s, p0, o0, psi0 = case(n, modes, grid, step, obj, seed, probe="hg")
    g = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_CLUSTER)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_cluster_form_more_views_than_clusters_and_edges():
    # 8 modes: at most 152 / 8 clusters fit at once, so 42 views put two or
    # three views on each cluster; footprints touch all four object edges
    dm = _dm()
    n, m = 128, 8
    s, p0, o0, psi0 = case(n, m, (7, 6), 12, (200, 188), 45, jitter=0, probe="hg")
    h, w = s.obj_shape
    assert s.views == 42
    assert s.pos[:, 0].min() == 0 and s.pos[:, 0].max() == h - n
    assert s.pos[:, 1].min() == 0 and s.pos[:, 1].max() == w - n
    g = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_CLUSTER)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_cluster_form_64_more_views_than_clusters_and_edges():
    # 64 x 64 frames, 8 modes: 400 views are several per resident cluster;
    # footprints touch all four object edges
    dm = _dm()
    n, m = 64, 8
    s, p0, o0, psi0 = case(n, m, (20, 20), 4, (140, 140), 55, jitter=0, probe="hg")
    h, w = s.obj_shape
    assert s.views == 400
    assert s.pos[:, 0].min() == 0 and s.pos[:, 0].max() == h - n
    assert s.pos[:, 1].min() == 0 and s.pos[:, 1].max() == w - n
    g = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_CLUSTER)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_cluster_form_three_iterations_beta_one():
    dm = _dm()
    s, p0, o0, psi0 = case(128, 4, (3, 4), 14, (165, 180), 46, probe="hg")
    kw = dict(n_iter=3, beta=1.0)
    g = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_CLUSTER, **kw)
    o = run_oracle(s, p0, o0, psi0, **kw)
    compare(g, o, tol=5 * REL_L2, metric_rtol=1e-3)


def test_cluster_and_strip_agree_to_fp32_rounding():
    dm = _dm()
    s, p0, o0, psi0 = case(128, 4, (4, 4), 16, (190, 190), 47, probe="hg")
    a = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_STRIP)
    b = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_CLUSTER)
    for key in ("psi", "obj", "probe"):
        assert rel_l2(b[key], a[key]) <= 2e-6, key
    ea, eb = a["metrics"][0], b["metrics"][0]
    assert abs(ea[2] - eb[2]) <= 1e-5 * ea[2]


def test_cluster_form_selection_rules():
    dm = _dm()
    # other shapes have no cluster form
    for n, m, obj in ((256, 8, (290, 290)), (32, 2, (60, 60)), (128, 9, (170, 170)), (64, 9, (95, 95))):
        s, p0, o0, psi0 = case(n, m, (2, 2), 24, obj, 48, probe="hg")
        h, w = s.obj_shape
        params = dm.dm_params_default(n=n, modes=m, views=s.views, obj_h=h, obj_w=w)
        ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
        with pytest.raises(dm.DMError):
            dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_CLUSTER)
        assert dm.dm_get_fourier_form(ctx) != dm.DM_FOURIER_CLUSTER
        dm.dm_free(ctx)
    # 128 x 128 with 4 modes: the form can be chosen and left; tracking the
    # exit-wave change runs the strip form; the plan reports no scratch ring
    s, p0, o0, psi0 = case(128, 4, (2, 2), 24, (170, 170), 49, probe="hg")
    h, w = s.obj_shape
    params = dm.dm_params_default(n=128, modes=4, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_CLUSTER   # a short scan starts in it
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_STRIP)
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_CLUSTER)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_CLUSTER
    plan = dm.dm_get_plan(ctx)
    assert plan["scratch_bytes"] == 0 and plan["views_per_chunk"] == 1 and plan["ctas"] == 4 * s.views
    dm.dm_set_psi_error(ctx, 1)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_STRIP
    dm.dm_set_psi_error(ctx, 0)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_CLUSTER
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_STRIP)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_STRIP
    dm.dm_free(ctx)
    # a long scan (400 views: more than three per resident cluster) starts in
    # the strip form with 4 modes, in the cluster form with 1 or 2
    for m, want in ((4, dm.DM_FOURIER_STRIP), (2, dm.DM_FOURIER_CLUSTER), (1, dm.DM_FOURIER_CLUSTER)):
        s, p0, o0, psi0 = case(128, m, (20, 20), 8, (285, 285), 51, probe="hg", noise=False)
        h, w = s.obj_shape
        params = dm.dm_params_default(n=128, modes=m, views=s.views, obj_h=h, obj_w=w)
        ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
        assert dm.dm_get_fourier_form(ctx) == want, m
        dm.dm_free(ctx)


def test_cluster_form_complex_half_within_the_mixed_bounds():
    # the cluster form's complex-half instance against the oracle run from
    # the same half-rounded exit waves (the mixed-precision form's stated
    # bounds: psi 5e-4 from the final rounding, object 1e-5, each probe mode
    # 2e-4)
    from oracle import dm as odm
    dm = _dm()
    s, p0, o0, psi0 = case(128, 4, (3, 3), 18, (170, 175), 50, probe="hg")
    h, w = s.obj_shape
    psi_h = psi0.astype(np.complex64)
    psi_h = (psi_h.real.astype(np.float16).astype(np.float64)
             + 1j * psi_h.imag.astype(np.float16).astype(np.float64))
    params = dm.dm_params_default(n=128, modes=4, views=s.views, obj_h=h, obj_w=w,
                                  psi_precision=dm.DM_PSI_FP16)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi_h.astype(np.complex64))
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_CLUSTER)
    dm.dm_iterate(ctx, 1)
    g = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx))
    dm.dm_free(ctx)
    psi, probe, obj, _ = odm.dm_iteration(psi_h, p0.astype(np.complex128), o0.astype(np.complex128), s.pos,
                                          np.asarray(s.intensities, np.float64), 0.8, 1e-6, 1)
    assert rel_l2(g["psi"], psi) <= 5e-4
    assert rel_l2(g["obj"], obj) <= 1e-5
    for k in range(4):
        assert rel_l2(g["probe"][k], probe[k]) <= 2e-4
