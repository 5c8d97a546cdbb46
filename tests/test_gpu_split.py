"""GPU parity of the split-column form of the Fourier step (256 x 256 frames,
8 modes), through the C ABI against the FP64 oracle: one and three
iterations, several Fourier chunks with slot reuse and a ragged last chunk,
footprints at the object edges, and agreement with the strip form to FP32
rounding.  Both forms compute Eq. 3 with the constrained transform F_c of
Sec. II; only the split of the column DFT into stages differs."""
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


@pytest.mark.parametrize("form", ["strip", "split"])
def test_both_forms_match_oracle(form):
    # (the complex-half instance: test_split_form_complex_half_within_the_mixed_bounds)
    dm = _dm()
    f = dm.DM_FOURIER_SPLIT if form == "split" else dm.DM_FOURIER_STRIP
    s, p0, o0, psi0 = case(256, 8, (3, 3), 18, (320, 330), 15, probe="hg")
    g = run_gpu(s, p0, o0, psi0, form=f)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_split_form_many_chunks_ragged_and_edges():
    # one view per chunk (scratch of 4 slots x 1 view): 11 chunks, every slot
    # reused; footprints touch all four object edges
    dm = _dm()
    n, m = 256, 8
    s, p0, o0, psi0 = case(n, m, (3, 4), 21, (298, 319), 31, jitter=0, probe="hg")
    s.pos = s.pos[:11].copy()
    s.intensities = s.intensities[:11].copy()
    psi0 = psi0[:11].copy()
    h, w = s.obj_shape
    assert s.pos[:, 0].min() == 0 and s.pos[:, 0].max() == h - n
    assert s.pos[:, 1].min() == 0 and s.pos[:, 1].max() == w - n
    budget = 4 * 1 * m * n * n * 8
    g = run_gpu(s, p0, o0, psi0, scratch_bytes=budget, form=dm.DM_FOURIER_SPLIT)
    o = run_oracle(s, p0, o0, psi0)
    compare(g, o)


def test_split_form_three_iterations_beta_one():
    dm = _dm()
    s, p0, o0, psi0 = case(256, 8, (2, 3), 24, (290, 320), 32, probe="hg")
    kw = dict(n_iter=3, beta=1.0)
    g = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_SPLIT, **kw)
    o = run_oracle(s, p0, o0, psi0, **kw)
    compare(g, o, tol=5 * REL_L2, metric_rtol=1e-3)


def test_split_and_strip_agree_to_fp32_rounding():
    dm = _dm()
    s, p0, o0, psi0 = case(256, 8, (3, 3), 18, (320, 330), 33, probe="hg")
    a = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_STRIP)
    b = run_gpu(s, p0, o0, psi0, form=dm.DM_FOURIER_SPLIT)
    for key in ("psi", "obj", "probe"):
        assert rel_l2(b[key], a[key]) <= 2e-6, key
    ea, eb = a["metrics"][0], b["metrics"][0]
    assert abs(ea[2] - eb[2]) <= 1e-5 * ea[2]


def test_form_selection_rules():
    dm = _dm()
    # other shapes have the strip form only
    s, p0, o0, psi0 = case(256, 7, (2, 2), 24, (290, 290), 20, probe="hg")
    h, w = s.obj_shape
    params = dm.dm_params_default(n=256, modes=7, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_STRIP
    with pytest.raises(dm.DMError):
        dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_SPLIT)
    dm.dm_free(ctx)
    # 256 x 256 with 8 modes starts in the split form and can switch; tracking
    # the exit-wave change runs the strip form
    s, p0, o0, psi0 = case(256, 8, (2, 2), 24, (290, 290), 34, probe="hg")
    h, w = s.obj_shape
    params = dm.dm_params_default(n=256, modes=8, views=s.views, obj_h=h, obj_w=w)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_SPLIT
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_STRIP)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_STRIP
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_SPLIT)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_SPLIT
    dm.dm_set_psi_error(ctx, 1)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_STRIP
    dm.dm_set_psi_error(ctx, 0)
    assert dm.dm_get_fourier_form(ctx) == dm.DM_FOURIER_SPLIT
    with pytest.raises(dm.DMError):
        dm.dm_set_fourier_form(ctx, 7)
    dm.dm_free(ctx)


def test_split_form_complex_half_within_the_mixed_bounds():
    # the split form's complex-half instance against the oracle run from the
    # same half-rounded exit waves (the mixed-precision form's stated bounds:
    # psi 5e-4 from the final rounding, object 1e-5, each probe mode 2e-4)
    import numpy as np
    from oracle import dm as odm
    dm = _dm()
    s, p0, o0, psi0 = case(256, 8, (3, 3), 18, (320, 330), 35, probe="hg")
    h, w = s.obj_shape
    psi_h = psi0.astype(np.complex64)
    psi_h = (psi_h.real.astype(np.float16).astype(np.float64)
             + 1j * psi_h.imag.astype(np.float16).astype(np.float64))
    params = dm.dm_params_default(n=256, modes=8, views=s.views, obj_h=h, obj_w=w,
                                  psi_precision=dm.DM_PSI_FP16)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi_h.astype(np.complex64))
    dm.dm_set_fourier_form(ctx, dm.DM_FOURIER_SPLIT)
    dm.dm_iterate(ctx, 1)
    g = dict(psi=dm.dm_get_exit_waves(ctx), probe=dm.dm_get_probe(ctx), obj=dm.dm_get_object(ctx))
    dm.dm_free(ctx)
    psi, probe, obj, _ = odm.dm_iteration(psi_h, p0.astype(np.complex128), o0.astype(np.complex128), s.pos,
                                          np.asarray(s.intensities, np.float64), 0.8, 1e-6, 1)
    assert rel_l2(g["psi"], psi) <= 5e-4
    assert rel_l2(g["obj"], obj) <= 1e-5
    for k in range(8):
        assert rel_l2(g["probe"][k], probe[k]) <= 2e-4
