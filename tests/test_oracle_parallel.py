"""The process-parallel oracle driver (views split over worker processes, as
Sec. III splits them over ranks) reproduces oracle.dm.dm_iteration: exit
waves, object, probe and the Eq. 6 / Fourier-error monitors over two
iterations, up to the order of the floating-point sums."""
import numpy as np

from oracle import dm as odm
from oracle.parallel import ProcessDM
from synth import make_scan, initial_guess


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_process_driver_equals_the_oracle_iteration():
    s = make_scan(dict(n=32, modes=3, grid=(5, 6), step=7, jitter=1, obj=(80, 80), probe="hg", fwhm=14.0,
                       photons=1e6, seed=9))
    p0, o0 = initial_guess(s, np.random.default_rng(9), kind="perturbed")
    probe, obj = p0.astype(np.complex128), o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float32)
    psi = odm.init_exit_waves(probe, obj, s.pos)
    p_ref, o_ref = probe, obj
    uy, ux = np.array([0, 5, 31, 17]), np.array([0, 9, 31, 3])
    with ProcessDM(inten, s.pos, probe, obj, workers=3) as pdm:
        for _ in range(2):
            got = pdm.iterate()
            psi, p_ref, o_ref, want = odm.dm_iteration(psi, p_ref, o_ref, s.pos, inten.astype(np.float64))
            assert rel(pdm.obj, o_ref) <= 1e-13
            assert rel(pdm.probe, p_ref) <= 1e-13
            for key in ("eps_obj", "fourier_err", "eps_psi"):
                assert abs(got[key] - want[key]) <= 1e-12 * want[key], key
            assert np.allclose(got["eps_probe"], want["eps_probe"], rtol=1e-12, atol=0)
        assert rel(pdm.psi_at(uy, ux), psi[:, :, uy, ux]) <= 1e-13
    assert rel(pdm.obj, o_ref) <= 1e-13     # readable after close


def test_process_driver_without_stored_exit_waves():
    """keep_psi=False (the new exit waves recomputed for Eq. 4) gives the same
    single iteration."""
    s = make_scan(dict(n=32, modes=2, grid=(4, 5), step=7, jitter=1, obj=(70, 80), probe="hg", fwhm=14.0,
                       photons=1e6, seed=10))
    p0, o0 = initial_guess(s, np.random.default_rng(10), kind="perturbed")
    probe, obj = p0.astype(np.complex128), o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float32)
    psi = odm.init_exit_waves(probe, obj, s.pos)
    _, p1, o1, want = odm.dm_iteration(psi, probe, obj, s.pos, inten.astype(np.float64))
    with ProcessDM(inten, s.pos, probe, obj, workers=2, keep_psi=False) as pdm:
        got = pdm.iterate()
    assert rel(pdm.obj, o1) <= 1e-13 and rel(pdm.probe, p1) <= 1e-13
    assert abs(got["fourier_err"] - want["fourier_err"]) <= 1e-12 * want["fourier_err"]


def test_process_driver_rounded_start():
    """round_start=True equals the oracle iteration from exit waves rounded to
    complex half (the start of the mixed-precision form)."""
    s = make_scan(dict(n=32, modes=2, grid=(4, 5), step=7, jitter=1, obj=(70, 80), probe="hg", fwhm=14.0,
                       photons=1e6, seed=11))
    p0, o0 = initial_guess(s, np.random.default_rng(11), kind="perturbed")
    probe, obj = p0.astype(np.complex128), o0.astype(np.complex128)
    inten = np.asarray(s.intensities, np.float32)
    psi = odm.init_exit_waves(probe, obj, s.pos)
    psi = psi.real.astype(np.float16).astype(np.float64) + 1j * psi.imag.astype(np.float16).astype(np.float64)
    _, p1, o1, _ = odm.dm_iteration(psi, probe, obj, s.pos, inten.astype(np.float64))
    with ProcessDM(inten, s.pos, probe, obj, workers=2, keep_psi=False, round_start=True) as pdm:
        pdm.iterate()
    assert rel(pdm.obj, o1) <= 1e-13 and rel(pdm.probe, p1) <= 1e-13
