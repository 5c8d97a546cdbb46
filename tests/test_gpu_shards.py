"""View-sharded iteration (the data-parallel split of Sec. III) emulated on
one GPU: the scan's views are divided among shard contexts, each runs the
Fourier step on its views, and the partial sums of Eq. 5 and Eq. 4 are added
over the shards before every shard applies them.  The result must match the
unsharded iteration of the C ABI and the FP64 oracle on the whole scan."""
import numpy as np
import pytest

from parity_util import case, compare, rel_l2, run_gpu, run_oracle, REL_L2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def run_sharded(s, p0, o0, psi0, shards, n_iter=1, order="gauss-seidel"):
    from paper_1808_10375_gb300 import dm
    from paper_1808_10375_gb300.shard import sharded_iteration, split_views
    h, w = s.obj_shape
    ctxs, ranges = [], split_views(s.views, shards)
    for r in ranges:
        idx = np.arange(r.start, r.stop)
        params = dm.dm_params_default(n=s.n, modes=s.modes, views=len(idx), obj_h=h, obj_w=w,
                                      update_order=dm.DM_ORDER_JACOBI if order == "jacobi"
                                      else dm.DM_ORDER_GAUSS_SEIDEL)
        c = dm.dm_init(params, s.pos[idx], s.intensities[idx], p0, o0)
        dm.dm_set_exit_waves(c, psi0[idx])
        ctxs.append(c)
    metrics = []
    for _ in range(n_iter):
        sharded_iteration(ctxs)
        metrics.append([dm.dm_get_error(c, -1) for c in ctxs])
    out = dict(psi=np.concatenate([dm.dm_get_exit_waves(c) for c in ctxs]),
               probes=[dm.dm_get_probe(c) for c in ctxs], objs=[dm.dm_get_object(c) for c in ctxs],
               metrics=metrics, done=[dm.dm_iterations_done(c) for c in ctxs])
    for c in ctxs:
        dm.dm_free(c)
    return out


@pytest.mark.parametrize("shards", [2, 3])
def test_sharded_iteration_matches_unsharded_and_oracle(shards):
    s, p0, o0, psi0 = case(64, 3, (5, 6), 9, (120, 130), 41)
    sh = run_sharded(s, p0, o0, psi0, shards, n_iter=2)
    g = run_gpu(s, p0, o0, psi0, n_iter=2)
    o = run_oracle(s, p0, o0, psi0, n_iter=2)
    # every shard ends with the same object and probe
    for k in range(1, shards):
        assert np.array_equal(sh["objs"][k], sh["objs"][0])
        assert np.array_equal(sh["probes"][k], sh["probes"][0])
    assert sh["done"] == [2] * shards
    # against the unsharded library (only the order of the sums differs)
    for key, a, b in (("psi", sh["psi"], g["psi"]), ("obj", sh["objs"][0], g["obj"]),
                      ("probe", sh["probes"][0], g["probe"])):
        assert rel_l2(a, b) <= 1e-6, (key, rel_l2(a, b))
    # against the FP64 oracle on the whole scan
    compare(dict(psi=sh["psi"], obj=sh["objs"][0], probe=sh["probes"][0],
                 metrics=[m[0] for m in sh["metrics"]]), o, tol=REL_L2)
    # every shard records the same metrics (the summed Fourier error included)
    for it in range(2):
        for m in sh["metrics"][it][1:]:
            assert np.allclose(m[0], sh["metrics"][it][0][0], rtol=1e-12)
            assert np.allclose(m[2], sh["metrics"][it][0][2], rtol=1e-12)


def test_partials_sum_to_the_unsharded_partials():
    """The object and probe partial sums of two shards add up to those of the
    whole scan (before any update is applied)."""
    from paper_1808_10375_gb300 import dm
    from paper_1808_10375_gb300.shard import split_views
    s, p0, o0, psi0 = case(32, 2, (5, 5), 5, (60, 64), 42)
    h, w = s.obj_shape

    def partials(idx):
        params = dm.dm_params_default(n=s.n, modes=s.modes, views=len(idx), obj_h=h, obj_w=w)
        c = dm.dm_init(params, s.pos[idx], s.intensities[idx], p0, o0)
        dm.dm_set_exit_waves(c, psi0[idx])
        dm.dm_run_step(c, dm.DM_STEP_FOURIER)
        on, od = dm.dm_object_partials(c)
        pn, pd = dm.dm_probe_partials(c)
        ef = dm.dm_fourier_error_partials(c)
        dm.dm_free(c)
        return on.astype(np.complex128), od.astype(np.float64), pn, pd, np.asarray(ef)

    whole = partials(np.arange(s.views))
    parts = [partials(np.arange(r.start, r.stop)) for r in split_views(s.views, 2)]
    for i in range(5):
        tot = parts[0][i] + parts[1][i]
        assert rel_l2(tot, whole[i]) <= 1e-6, (i, rel_l2(tot, whole[i]))


def test_sharded_jacobi_order_matches_oracle():
    s, p0, o0, psi0 = case(64, 3, (5, 6), 9, (120, 130), 43)
    sh = run_sharded(s, p0, o0, psi0, 2, n_iter=2, order="jacobi")
    o = run_oracle(s, p0, o0, psi0, n_iter=2, order="jacobi")
    compare(dict(psi=sh["psi"], obj=sh["objs"][0], probe=sh["probes"][0],
                 metrics=[m[0] for m in sh["metrics"]]), o, tol=REL_L2)
