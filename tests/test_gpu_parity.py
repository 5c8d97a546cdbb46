"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, one
iteration (or a few) from identical seeded complex64 states, element by
element (relative L2 <= 1e-5 for psi, the object and every probe mode; the
Eq. 6 and Fourier-error metrics to 1e-4 relative).

Sizes are chosen so that the oracle finishes in seconds while the kernels
see several object tiles, several Fourier chunks (with a ragged last one),
odd mode counts, views touching the object edges, and every frame size the
library supports."""
import numpy as np
import pytest

from parity_util import case, compare, rel_l2, run_gpu, run_oracle, REL_L2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


CASES = {
    #        n  M  grid    step  object       seed
    "n16_m2": (16, 2, (3, 4), 4, (26, 30), 11),     # footprints reach the object edges
    "n32_m3": (32, 3, (5, 5), 5, (60, 64), 12),
    "n64_m1": (64, 1, (6, 7), 8, (120, 130), 13),
    "n128_m4": (128, 4, (5, 6), 12, (200, 210), 14),
    # 256 x 256 frames: 8 modes fill the column task's slots, 5 and 7 leave some idle
    "n256_m8": (256, 8, (3, 3), 18, (320, 330), 15),
    "n256_m5": (256, 5, (3, 2), 20, (310, 300), 19),
    "n256_m7": (256, 7, (2, 2), 24, (290, 290), 20),
    "n256_m3": (256, 3, (2, 3), 30, (300, 330), 16),
    # fewer modes than column slots: several strips transformed together
    "n256_m1": (256, 1, (2, 2), 40, (300, 300), 17),
    "n128_m2": (128, 2, (3, 3), 20, (170, 180), 18),
}


@pytest.mark.parametrize("name", list(CASES))
def test_one_iteration_matches_oracle(name):
    n, m, grid, step, obj, seed = CASES[name]
    s, p0, o0, psi0 = case(n, m, grid, step, obj, seed, probe="gauss" if m == 1 else "hg")
    g = run_gpu(s, p0, o0, psi0)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_many_chunks_and_slot_reuse():
    # A small scratch budget forces 3 views per chunk: 14 chunks, slot reuse
    # across the pipeline and a ragged last chunk (41 = 13*3 + 2).
    n, m = 64, 2
    s, p0, o0, psi0 = case(n, m, (6, 7), 9, (130, 140), 21)
    s.pos = s.pos[:41].copy()
    s.intensities = s.intensities[:41].copy()
    psi0 = psi0[:41].copy()
    budget = 4 * 3 * m * n * n * 8
    g = run_gpu(s, p0, o0, psi0, scratch_bytes=budget)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_beta_one_zero_floor_inner_passes_and_frozen_probe():
    s, p0, o0, psi0 = case(32, 2, (4, 5), 6, (60, 70), 22)
    kw = dict(n_iter=3, beta=1.0, delta_rel=0.0, n_inner=2, probe_update_start=1)
    g = run_gpu(s, p0, o0, psi0, **kw)
    o = run_oracle(s, p0, o0, psi0, **kw)
    # three iterations: the bound grows with the iteration count
    compare(g, o, tol=5 * REL_L2, metric_rtol=1e-3)
    assert g["metrics"][0][1] == [0.0, 0.0]        # probe frozen in iteration 0


def test_default_initial_waves_and_several_iterations():
    s, p0, o0, _ = case(64, 1, (5, 5), 8, (110, 110), 23, probe="gauss")
    g = run_gpu(s, p0, o0, None, n_iter=4)
    o = run_oracle(s, p0, o0, None, n_iter=4)
    compare(g, o, tol=1e-4, metric_rtol=1e-3)


def test_bitwise_deterministic():
    s, p0, o0, psi0 = case(128, 4, (4, 4), 16, (190, 190), 24)
    a = run_gpu(s, p0, o0, psi0, n_iter=2)
    b = run_gpu(s, p0, o0, psi0, n_iter=2)
    for k in ("psi", "probe", "obj"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), k
    assert a["metrics"] == b["metrics"]


def test_steps_match_oracle_steps():
    from oracle import dm as odm
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(64, 3, (4, 5), 10, (110, 120), 25)
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    psi = psi0.astype(np.complex128)
    probe = p0.astype(np.complex128)
    obj = o0.astype(np.complex128)
    dm.dm_run_step(ctx, dm.DM_STEP_FOURIER)
    psi, _ = odm.fourier_update(psi, probe, obj, s.pos, s.intensities.astype(np.float64), 0.8)
    assert rel_l2(dm.dm_get_exit_waves(ctx), psi) <= REL_L2
    dm.dm_run_step(ctx, dm.DM_STEP_OBJECT)
    obj = odm.object_update(psi, probe, obj, s.pos, 1e-6)
    assert rel_l2(dm.dm_get_object(ctx), obj) <= REL_L2
    dm.dm_run_step(ctx, dm.DM_STEP_PROBE)
    probe = odm.probe_update(psi, probe, obj, s.pos, 1e-6)
    assert rel_l2(dm.dm_get_probe(ctx), probe) <= REL_L2
    assert dm.dm_iterations_done(ctx) == 0
    pw = dm.dm_get_mode_power(ctx)
    np.testing.assert_allclose(pw, odm.mode_power(probe), rtol=1e-5)
    dm.dm_free(ctx)


def test_host_and_device_inputs_agree():
    import torch
    from paper_1808_10375_gb300 import dm
    s, p0, o0, _ = case(32, 2, (3, 3), 6, (50, 50), 26)
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    a = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    b = dm.dm_init(params, dev(s.pos), dev(s.intensities), dev(p0), dev(o0))
    for c in (a, b):
        dm.dm_iterate(c, 2)
    assert np.array_equal(dm.dm_get_object(a), dm.dm_get_object(b))
    od = dm.dm_get_object(b, device=True)
    assert od.is_cuda and np.array_equal(od.cpu().numpy(), dm.dm_get_object(a))
    dm.dm_free(a)
    dm.dm_free(b)


def test_library_allocator_path():
    s, p0, o0, psi0 = case(32, 1, (3, 3), 6, (50, 50), 27, probe="gauss")
    g = run_gpu(s, p0, o0, psi0, use_torch_allocator=False)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


@pytest.mark.parametrize("bad", [-1.0, float("nan"), float("inf")])
def test_bad_intensity_rejected(bad):
    from paper_1808_10375_gb300 import dm
    s, p0, o0, _ = case(16, 1, (2, 2), 4, (24, 24), 28, probe="gauss")
    inten = s.intensities.copy()
    inten[1, 3, 5] = bad
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    with pytest.raises(dm.DMError) as e:
        dm.dm_init(params, s.pos, inten, p0, o0)
    assert e.value.code == dm.DM_EINVAL


def test_error_queries():
    from paper_1808_10375_gb300 import dm
    s, p0, o0, _ = case(16, 2, (2, 2), 4, (24, 24), 29)
    h, w = s.obj_shape
    ctx = dm.dm_init(dm.dm_params_default(n=16, modes=2, views=s.views, obj_h=h, obj_w=w), s.pos,
                     s.intensities, p0, o0)
    with pytest.raises(dm.DMError):
        dm.dm_get_error(ctx)                        # nothing has run yet
    dm.dm_iterate(ctx, 3)
    assert dm.dm_iterations_done(ctx) == 3
    last = dm.dm_get_error(ctx, -1)
    assert last == dm.dm_get_error(ctx, 2)
    with pytest.raises(dm.DMError):
        dm.dm_get_error(ctx, 3)
    dm.dm_sync(ctx)
    assert dm.dm_device_bytes(ctx) > 0
    dm.dm_free(ctx)


@pytest.mark.parametrize("n,m,seed", [(64, 2, 51), (256, 3, 52)])
def test_jacobi_order_matches_oracle(n, m, seed):
    # Eqs. 4 and 5 as simultaneous updates: the probe divides by the object
    # the iteration started with.
    grid, step, obj = ((5, 5), 9, (110, 110)) if n == 64 else ((2, 2), 30, (290, 290))
    s, p0, o0, psi0 = case(n, m, grid, step, obj, seed)
    g = run_gpu(s, p0, o0, psi0, n_iter=2, order="jacobi")
    o = run_oracle(s, p0, o0, psi0, n_iter=2, order="jacobi")
    compare(g, o)
    gs = run_oracle(s, p0, o0, psi0, n_iter=1)
    assert rel_l2(o["probe"], gs["probe"]) > 10 * REL_L2   # the order shows in the result
