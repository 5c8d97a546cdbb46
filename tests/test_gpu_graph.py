"""Iterations replayed as CUDA graphs (dm_set_graph) give the same results
as kernel-by-kernel launches, bit for bit, including the switch from eager
iterations with a frozen probe to captured ones, and record the same
metrics; the replay is timed against the eager path on a small scan where
launches dominate."""
import numpy as np
import pytest

from parity_util import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def _run(s, p0, o0, psi0, graph, n_iter, probe_update_start=0, n_inner=1):
    from paper_1808_10375_gb300 import dm
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w,
                                  probe_update_start=probe_update_start, n_inner=n_inner)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    dm.dm_set_graph(ctx, graph)
    dm.dm_iterate(ctx, n_iter)
    out = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
               metrics=[dm.dm_get_error(ctx, i) for i in range(n_iter)])
    dm.dm_free(ctx)
    return out


@pytest.mark.parametrize("start,n_inner", [(0, 1), (2, 1), (0, 2)])
def test_graph_replay_is_bitwise_equal(start, n_inner):
    s, p0, o0, psi0 = case(64, 3, (5, 6), 9, (120, 130), 51)
    a = _run(s, p0, o0, psi0, False, 5, start, n_inner)
    b = _run(s, p0, o0, psi0, True, 5, start, n_inner)
    for k in ("psi", "probe", "obj"):
        assert np.array_equal(a[k], b[k]), k
    assert a["metrics"] == b["metrics"]


def test_graph_replay_time_on_a_small_scan():
    import torch
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(64, 1, (10, 10), 8, (160, 160), 52, probe="gauss")
    h, w = s.obj_shape
    times = {}
    for graph in (False, True):
        params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
        ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
        dm.dm_set_graph(ctx, graph)
        dm.dm_iterate(ctx, 4)
        dm.dm_sync(ctx)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record()
        dm.dm_iterate(ctx, 100)
        dm.dm_sync(ctx)
        t1.record()
        torch.cuda.synchronize()
        times[graph] = t0.elapsed_time(t1) / 100 * 1e3
        dm.dm_free(ctx)
    print(f"64x64, 100 views, 1 mode: {times[False]:.1f} us per iteration launched, "
          f"{times[True]:.1f} us replayed as a graph")
    assert times[True] < 1.5 * times[False]
