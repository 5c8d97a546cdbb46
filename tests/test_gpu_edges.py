"""GPU parity on the degenerate and extreme cases of the method: the largest
mode count at the largest frame, a scan of one view, a view whose projected
field is zero (mode sum S = 0: the projection returns zero), a view that
recorded no photons (I = 0), and the exit-wave bound held view by view."""
import numpy as np
import pytest

from parity_util import case, compare, rel_l2, run_gpu, run_oracle, REL_L2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def test_sixteen_modes_at_256():
    # the mode maximum: the column tasks fall back to one strip buffer
    s, p0, o0, psi0 = case(256, 16, (2, 2), 30, (300, 300), 31)
    compare(run_gpu(s, p0, o0, psi0), run_oracle(s, p0, o0, psi0))


def test_single_view():
    s, p0, o0, psi0 = case(64, 2, (1, 1), 8, (70, 72), 32)
    assert s.views == 1
    compare(run_gpu(s, p0, o0, psi0), run_oracle(s, p0, o0, psi0))


def test_zero_field_view_and_dark_view():
    n, m = 32, 3
    s, p0, o0, psi0 = case(n, m, (4, 4), 6, (60, 60), 33)
    # view 5: object zero on its footprint and psi zero, so 2 P O - psi = 0
    # exactly and the mode sum S vanishes at every frequency
    r, c = s.pos[5]
    o0 = o0.copy()
    o0[r:r + n, c:c + n] = 0
    psi0 = psi0.copy()
    psi0[5] = 0
    # view 9: no photons recorded
    s.intensities = s.intensities.copy()
    s.intensities[9] = 0
    g = run_gpu(s, p0, o0, psi0)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)
    assert np.all(g["psi"][5] == 0)
    assert rel_l2(g["psi"][9], o["psi"][9]) <= REL_L2


def test_every_view_within_bound():
    # the bound holds view by view, not only over the whole exit-wave array
    s, p0, o0, psi0 = case(128, 4, (3, 4), 16, (190, 200), 34)
    g = run_gpu(s, p0, o0, psi0)
    o = run_oracle(s, p0, o0, psi0)
    for j in range(s.views):
        assert rel_l2(g["psi"][j], o["psi"][j]) <= REL_L2, j


def test_contexts_of_one_frame_size_with_different_plans():
    """Kernel launch limits are shared by all contexts: a context created
    after another one with a smaller plan must not stop the first from
    running (the first needs more shared memory per CTA)."""
    from paper_1808_10375_gb300 import dm
    from parity_util import case, compare, run_oracle
    big = case(128, 4, (3, 3), 14, (170, 170), 81)
    small = case(128, 1, (3, 3), 14, (170, 170), 82, probe="gauss")
    ctxs = []
    for s, p0, o0, psi0 in (big, small):
        h, w = s.obj_shape
        params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
        c = dm.dm_init(params, s.pos, s.intensities, p0, o0)
        dm.dm_set_exit_waves(c, psi0)
        dm.dm_set_fourier_form(c, dm.DM_FOURIER_STRIP)   # the form whose plans differ in shared memory
        ctxs.append(c)
    dm.dm_autotune(ctxs[1], sample_views=9)
    dm.dm_set_fourier_form(ctxs[1], dm.DM_FOURIER_STRIP)
    for c in ctxs:
        dm.dm_iterate(c, 1)
    for c, (s, p0, o0, psi0) in zip(ctxs, (big, small)):
        g = dict(psi=dm.dm_get_exit_waves(c), probe=dm.dm_get_probe(c), obj=dm.dm_get_object(c),
                 metrics=[dm.dm_get_error(c, 0)])
        dm.dm_free(c)
        compare(g, run_oracle(s, p0, o0, psi0))


def test_bounded_waits_give_up_and_the_device_stays_usable():
    """The failure path without a fault: a counter wait on a flag that nothing
    raises and an mbarrier wait on a phase that nothing completes each give
    up after their 1 s limit and set the timeout status (what turns a stalled
    Fourier step into DM_ETIMEOUT); afterwards a whole iteration still runs
    and matches the oracle."""
    from paper_1808_10375_gb300 import dm
    ms = dm.dm_selftest_bounded_waits()
    assert 1900.0 <= ms <= 20000.0, ms
    s, p0, o0, psi0 = case(32, 2, (3, 3), 6, (50, 50), 61)
    compare(run_gpu(s, p0, o0, psi0), run_oracle(s, p0, o0, psi0))
