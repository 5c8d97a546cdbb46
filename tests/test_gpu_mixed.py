"""The mixed-precision form of the iteration (complex-half exit waves, FP32
arithmetic) against the FP64 oracle, through the C ABI.

What the form computes.  One iteration reads psi from its complex-half
storage, runs Eq. 3 in FP32 and stores psi' rounded to complex half; the
object (Eq. 5) is built from psi' before that rounding (the object source
c_j is summed in registers), the probe (Eq. 4) from the stored, rounded psi'.
The oracle is given the same starting exit waves, rounded to half, and runs
in FP64.  Stated bounds, relative L2 per result:

* psi: the rounding of the stored psi' to 11 significant bits, unit roundoff
  u = 2^-11 = 4.9e-4 per component; bound 5e-4 (the L2 error of rounding a
  large set of values is about u / sqrt(3));
* object: FP32 level, as the FP32 form (1e-5), since psi' is summed before
  rounding;
* each probe mode: the psi' roundings of the views covering a pixel average
  out in the Eq. 4 sum; bound 2e-4;
* monitors (Eq. 6, Fourier error): 1e-4 relative, as the FP32 form.

Over several iterations the oracle rounds its own psi to half after every
iteration (the form's own definition).  The FP32 and FP64 psi' differ by
FP32 rounding, so where a value lies that close to a boundary between two
halves the two sides round it to neighbouring halves; from the second
iteration on every result carries those one-ulp differences of psi, and the
object is held to the probe's bound (2e-4) instead of the FP32 one.
"""
import numpy as np
import pytest

from oracle import dm as odm
from parity_util import REL_L2, case, rel_l2

pytestmark = pytest.mark.gpu

PSI_BOUND = 5e-4
PROBE_BOUND = 2e-4


def to_half(x):
    x = np.asarray(x)
    return (x.real.astype(np.float16).astype(np.float64) + 1j * x.imag.astype(np.float16).astype(np.float64))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def run_half(s, p0, o0, psi0, n_iter=1, psi_switch=0.0):
    from paper_1808_10375_gb300 import dm
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w,
                                  psi_precision=dm.DM_PSI_FP16, psi_switch=psi_switch)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    dm.dm_iterate(ctx, n_iter)
    out = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx),
               metrics=[dm.dm_get_error(ctx, i) for i in range(n_iter)], precision=dm.dm_get_psi_precision(ctx))
    dm.dm_free(ctx)
    return out


def oracle_half(s, p0, o0, psi0, n_iter=1):
    psi = to_half(psi0)
    probe = p0.astype(np.complex128)
    obj = o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float64)
    hist = []
    for _ in range(n_iter):
        psi, probe, obj, m = odm.dm_iteration(psi, probe, obj, s.pos, inten)
        hist.append(m)
        psi_store = to_half(psi)
        psi = psi_store
    return dict(psi=psi, probe=probe, obj=obj, metrics=hist)


CASES = {
    "n64_m2": (64, 2, (5, 6), 9, (120, 130), 61),
    "n128_m4": (128, 4, (4, 4), 14, (190, 190), 62),
    "n256_m8": (256, 8, (3, 3), 18, (320, 330), 63),
    "n256_m3": (256, 3, (2, 3), 30, (300, 330), 64),
}


def check(g, o, psi_bound=PSI_BOUND, obj_bound=REL_L2):
    errs = {"psi": rel_l2(g["psi"], o["psi"]), "obj": rel_l2(g["obj"], o["obj"])}
    for k in range(o["probe"].shape[0]):
        errs[f"probe{k}"] = rel_l2(g["probe"][k], o["probe"][k])
    assert errs["psi"] <= psi_bound, errs
    assert errs["obj"] <= obj_bound, errs
    assert all(errs[f"probe{k}"] <= PROBE_BOUND for k in range(o["probe"].shape[0])), errs
    for (eo, ep, ef), m in zip(g["metrics"], o["metrics"]):
        assert eo == pytest.approx(m["eps_obj"], rel=1e-4)
        assert ef == pytest.approx(m["fourier_err"], rel=1e-4)
    return errs


@pytest.mark.parametrize("name", list(CASES))
def test_one_mixed_iteration_within_the_stated_bounds(name):
    n, m, grid, step, obj, seed = CASES[name]
    s, p0, o0, psi0 = case(n, m, grid, step, obj, seed)
    g = run_half(s, p0, o0, psi0)
    o = oracle_half(s, p0, o0, psi0)
    check(g, o)
    # the stored exit waves are complex-half values
    assert np.array_equal(g["psi"], to_half(g["psi"]).astype(np.complex64))


def test_three_mixed_iterations_follow_the_rounded_oracle():
    s, p0, o0, psi0 = case(128, 4, (4, 4), 14, (190, 190), 65)
    g = run_half(s, p0, o0, psi0, n_iter=3)
    o = oracle_half(s, p0, o0, psi0, n_iter=3)
    check(g, o, psi_bound=2 * PSI_BOUND, obj_bound=PROBE_BOUND)


def test_switch_to_complex64_after_the_threshold():
    """psi_switch above the first iteration's Eq. 6 change: the context is back
    in complex64 storage after one iteration, and the next iteration is the
    FP32 form (the oracle without rounding from there)."""
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(64, 2, (5, 6), 9, (120, 130), 66)
    g = run_half(s, p0, o0, psi0, n_iter=2, psi_switch=10.0)
    assert g["precision"] == (dm.DM_PSI_FP32, 1)
    psi = to_half(psi0)
    probe, obj = p0.astype(np.complex128), o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float64)
    psi, probe, obj, _ = odm.dm_iteration(psi, probe, obj, s.pos, inten)
    psi = to_half(psi)                       # stored in half by the first iteration
    psi, probe, obj, _ = odm.dm_iteration(psi, probe, obj, s.pos, inten)   # FP32 form
    # the FP32 iteration starts from the stored halves of the first one
    assert rel_l2(g["obj"], obj) <= PROBE_BOUND
    assert rel_l2(g["psi"], psi) <= PSI_BOUND
    for k in range(s.modes):
        assert rel_l2(g["probe"][k], probe[k]) <= PROBE_BOUND


def test_explicit_conversions_round_and_widen():
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(64, 2, (3, 3), 9, (90, 90), 67)
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    assert dm.dm_get_psi_precision(ctx) == (dm.DM_PSI_FP32, -1)
    dm.dm_set_psi_precision(ctx, dm.DM_PSI_FP16)
    got = dm.dm_get_exit_waves(ctx)
    assert np.array_equal(got, to_half(psi0).astype(np.complex64))
    dm.dm_set_psi_precision(ctx, dm.DM_PSI_FP32)
    assert np.array_equal(dm.dm_get_exit_waves(ctx), got)
    # the exit-wave change is tracked with complex64 storage only
    dm.dm_set_psi_precision(ctx, dm.DM_PSI_FP16)
    with pytest.raises(dm.DMError):
        dm.dm_set_psi_error(ctx, True)
    dm.dm_free(ctx)


def test_mixed_form_on_the_first_1000_views_of_the_256x256x8_scan():
    """The per-result bound on the precision-form workload: one mixed-precision
    iteration over the first 1,000 views of the 8-mode 256 x 256 scan (2100 x
    2100 object), from the exit waves dm_init builds (P O, stored as complex
    half), against a complete FP64 oracle iteration from the same rounded
    start (views split over host processes).  Object over the whole array,
    every probe mode over the whole frame, Eq. 6 and the Fourier error."""
    import torch
    import bench
    from paper_1808_10375_gb300 import dm
    from oracle.parallel import ProcessDM
    s, p0, o0 = bench.make_inputs(1000, "cuda")
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w,
                                  psi_precision=dm.DM_PSI_FP16)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ctx = dm.dm_init(params, dev(s.pos), s.intensities, dev(p0), dev(o0))
    dm.dm_iterate(ctx, 1)
    o1, p1 = dm.dm_get_object(ctx), dm.dm_get_probe(ctx)
    eps_obj, eps_probe, ferr = dm.dm_get_error(ctx)
    dm.dm_free(ctx)
    inten = s.intensities.cpu().numpy()
    with ProcessDM(inten, s.pos, p0.astype(np.complex128), o0.astype(np.complex128), keep_psi=False,
                   round_start=True) as pdm:
        want = pdm.iterate()
    assert rel_l2(o1, pdm.obj) <= REL_L2
    for k in range(s.modes):
        assert rel_l2(p1[k], pdm.probe[k]) <= PROBE_BOUND, (k, rel_l2(p1[k], pdm.probe[k]))
    assert ferr == pytest.approx(want["fourier_err"], rel=1e-4)
    assert eps_obj == pytest.approx(want["eps_obj"], rel=1e-4)
