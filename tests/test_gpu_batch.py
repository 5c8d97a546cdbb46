"""The batched form: scans of uneven frame size, mode count and view count
advanced together (one persistent Fourier launch per frame size, then each
scan's overlap projection) give, scan by scan, the same results bit for bit
as iterating each scan alone, with and without CUDA-graph replay, and the
first scan still matches the FP64 oracle."""
import numpy as np
import pytest

from parity_util import case, compare, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


SCANS = [
    #  n   M  grid    step  object      seed
    (64, 3, (5, 6), 9, (120, 130), 71),
    (64, 1, (4, 4), 10, (110, 100), 72),
    (128, 4, (4, 5), 14, (200, 190), 73),
    (32, 2, (6, 5), 5, (64, 60), 74),
    (64, 2, (3, 7), 8, (90, 130), 75),
]


def _contexts(cases):
    from paper_1808_10375_gb300 import dm
    ctxs = []
    for s, p0, o0, psi0 in cases:
        h, w = s.obj_shape
        params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
        c = dm.dm_init(params, s.pos, s.intensities, p0, o0)
        dm.dm_set_exit_waves(c, psi0)
        ctxs.append(c)
    return ctxs


def _state(ctx):
    from paper_1808_10375_gb300 import dm
    return dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
                metrics=[dm.dm_get_error(ctx, i) for i in range(dm.dm_iterations_done(ctx))])


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_scans_alone(graph):
    from paper_1808_10375_gb300 import dm
    cases = [case(*spec[:5], spec[5]) for spec in SCANS]
    alone = _contexts(cases)
    assert dm.dm_get_fourier_form(alone[2]) == dm.DM_FOURIER_CLUSTER
    for c in alone:
        # each scan's own form (the 20-view 128 x 128 scan starts in the
        # cluster form, which the batch keeps)
        dm.dm_iterate(c, 3)
    ref = [_state(c) for c in alone]
    for c in alone:
        dm.dm_free(c)
    ctxs = _contexts(cases)
    b = dm.dm_batch_create(ctxs)
    dm.dm_batch_set_graph(b, graph)
    dm.dm_batch_iterate(b, 1)
    dm.dm_batch_iterate(b, 2)
    got = [_state(c) for c in ctxs]
    dm.dm_batch_free(b)
    for i, (g, r) in enumerate(zip(got, ref)):
        for k in ("psi", "probe", "obj"):
            assert np.array_equal(g[k], r[k]), (i, k)
        assert g["metrics"] == r["metrics"], i
    s, p0, o0, psi0 = cases[0]
    first = dict(got[0])
    for c in ctxs:
        dm.dm_free(c)
    compare(first, run_oracle(s, p0, o0, psi0, n_iter=3))
