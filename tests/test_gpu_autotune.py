"""The Fourier-step autotuner (dm_autotune): it leaves the state unchanged
(the sample's exit waves are restored), picks one of its candidate plans,
and the iteration that follows still matches the FP64 oracle."""
import numpy as np
import pytest

from parity_util import case, compare, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def test_autotune_keeps_state_and_parity():
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(128, 4, (6, 7), 12, (210, 220), 61)
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    before = dm.dm_get_plan(ctx)
    best = dm.dm_autotune(ctx, sample_views=30)
    after = dm.dm_get_plan(ctx)
    print("plan before", before, "after", after, f"best {best:.3f} ms on 30 views")
    assert best > 0
    view_bytes = s.modes * s.n * s.n * 8
    if dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_CLUSTER:   # no knobs, no ring
        assert after["scratch_bytes"] == 0 and after["views_per_chunk"] == 1
    else:
        assert after["strip_buffers"] in (1, 2, 3)
        assert after["scratch_bytes"] <= (128 << 20) + 4 * view_bytes
    assert np.array_equal(dm.dm_get_exit_waves(ctx), psi0)
    dm.dm_iterate(ctx, 1)
    g = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
             metrics=[dm.dm_get_error(ctx, 0)])
    dm.dm_free(ctx)
    compare(g, run_oracle(s, p0, o0, psi0))


def test_autotune_chooses_between_the_fourier_forms():
    # a 256 x 256, 8-mode scan has both forms: the autotuner times both and
    # keeps one; whichever it keeps, state is unchanged and parity holds
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(256, 8, (3, 3), 18, (320, 330), 62)
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    best = dm.dm_autotune(ctx, sample_views=s.views)
    form = dm.dm_get_fourier_form(ctx)
    plan = dm.dm_get_plan(ctx)
    print("form", form, "plan", plan, f"best {best:.3f} ms")
    assert best > 0 and form in (dm.DM_FOURIER_STRIP, dm.DM_FOURIER_SPLIT)
    if form == dm.DM_FOURIER_SPLIT:
        assert plan["strips_per_column_task"] == 0 and plan["strip_buffers"] == 3
    assert np.array_equal(dm.dm_get_exit_waves(ctx), psi0)
    dm.dm_iterate(ctx, 1)
    g = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
             metrics=[dm.dm_get_error(ctx, 0)])
    dm.dm_free(ctx)
    compare(g, run_oracle(s, p0, o0, psi0))
