"""Pins for one whole oracle DM iteration (Eq. 3, Eq. 5, Eq. 4, Eq. 6).

* fixed point: noise-free intensities of (P*, O*) with psi = P* O* are left
  unchanged by one iteration, in either update order;
* gauges: a global phase on (O, psi) and the scalar ambiguity (cP, O/c);
* modes: a unitary mixing of the probe modes commutes with the iteration,
  and an extra all-zero mode stays zero and changes nothing;
* brute force: an independent loop-by-loop implementation written from the
  equations (explicit DFT sums) on tiny inputs, single- and multi-mode, in
  both update orders (the probe from the new object or from the old one);
* metrics: Eq. 6 on a known perturbation, the Fourier error on data that is
  exactly four times the model intensity, and the exit-wave change (with the
  exit-wave update itself) on data equal to one or four times the model
  intensity, where Eq. 3 has a closed form;
* convergence: a noise-free scan reconstructs the true object (up to a
  complex scalar) to 1e-3 on well-covered pixels.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import dm
from synth import make_scan


def rand_c(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def small_state(rng, m=2, n=8, grid=3, step=3, jitter=True):
    h = w = (grid - 1) * step + n + 3
    probe = rand_c(rng, (m, n, n))
    obj = rand_c(rng, (h, w))
    pos = []
    for a in range(grid):
        for b in range(grid):
            ja, jb = (rng.integers(-1, 2), rng.integers(-1, 2)) if jitter else (0, 0)
            pos.append([1 + a * step + ja, 1 + b * step + jb])
    return probe, obj, np.array(pos, np.int32)


def model_intensities(probe, obj, pos):
    n = probe.shape[-1]
    out = []
    for r, c in pos:
        ex = probe * obj[None, r:r + n, c:c + n]
        out.append(np.sum(np.abs(np.fft.fft2(ex, norm="ortho")) ** 2, axis=0))
    return np.array(out)


def test_exact_solution_is_a_fixed_point():
    rng = np.random.default_rng(11)
    probe, obj, pos = small_state(rng, m=3)
    inten = model_intensities(probe, obj, pos)
    psi = dm.init_exit_waves(probe, obj, pos)
    for beta, order in ((0.8, "gauss-seidel"), (1.0, "gauss-seidel"), (0.8, "jacobi")):
        psi1, p1, o1, m = dm.dm_iteration(psi, probe, obj, pos, inten, beta=beta, delta_rel=0.0, order=order)
        np.testing.assert_allclose(psi1, psi, rtol=0, atol=1e-12 * np.abs(psi).max())
        np.testing.assert_allclose(o1, obj, rtol=0, atol=1e-12 * np.abs(obj).max())
        np.testing.assert_allclose(p1, probe, rtol=0, atol=1e-12 * np.abs(probe).max())
        assert m["fourier_err"] < 1e-12 and m["eps_obj"] < 1e-12 and max(m["eps_probe"]) < 1e-12


def generic_inputs(rng, m=2):
    probe, obj, pos = small_state(rng, m=m)
    inten = model_intensities(probe * 1.3, obj * np.exp(0.4j), pos) + rng.uniform(0, 0.5, (len(pos), 8, 8))
    psi = dm.init_exit_waves(probe, obj, pos) + 0.4 * rand_c(rng, (len(pos), m, 8, 8))
    return psi, probe, obj, pos, inten


def test_global_phase_gauge():
    rng = np.random.default_rng(12)
    psi, probe, obj, pos, inten = generic_inputs(rng)
    a = dm.dm_iteration(psi, probe, obj, pos, inten)
    ph = np.exp(0.7j)
    b = dm.dm_iteration(psi * ph, probe, obj * ph, pos, inten)
    np.testing.assert_allclose(b[0], a[0] * ph, atol=1e-12)
    np.testing.assert_allclose(b[1], a[1], atol=1e-12)
    np.testing.assert_allclose(b[2], a[2] * ph, atol=1e-12)


def test_probe_object_scalar_gauge():
    rng = np.random.default_rng(13)
    psi, probe, obj, pos, inten = generic_inputs(rng, m=3)
    c = 1.7 - 0.6j
    a = dm.dm_iteration(psi, probe, obj, pos, inten, delta_rel=1e-3)
    b = dm.dm_iteration(psi, probe * c, obj / c, pos, inten, delta_rel=1e-3)
    np.testing.assert_allclose(b[0], a[0], atol=1e-12)
    np.testing.assert_allclose(b[1], a[1] * c, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(b[2], a[2] / c, rtol=1e-11, atol=1e-12)


def test_unitary_mode_mixing_commutes():
    rng = np.random.default_rng(14)
    m = 3
    psi, probe, obj, pos, inten = generic_inputs(rng, m=m)
    q, _ = np.linalg.qr(rand_c(rng, (m, m)))
    mix = lambda x: np.einsum("kl,...lyx->...kyx", q, x)
    a = dm.dm_iteration(psi, probe, obj, pos, inten, delta_rel=1e-4)
    b = dm.dm_iteration(mix(psi), mix(probe), obj, pos, inten, delta_rel=1e-4)
    np.testing.assert_allclose(b[0], mix(a[0]), atol=1e-11)
    np.testing.assert_allclose(b[1], mix(a[1]), atol=1e-11)
    np.testing.assert_allclose(b[2], a[2], atol=1e-11)


def test_extra_zero_mode_is_inert():
    rng = np.random.default_rng(15)
    psi, probe, obj, pos, inten = generic_inputs(rng, m=2)
    a = dm.dm_iteration(psi, probe, obj, pos, inten)
    pz = np.concatenate([probe, np.zeros_like(probe[:1])])
    psz = np.concatenate([psi, np.zeros_like(psi[:, :1])], axis=1)
    b = dm.dm_iteration(psz, pz, obj, pos, inten)
    np.testing.assert_allclose(b[0][:, :2], a[0], atol=1e-12)
    assert np.all(b[0][:, 2] == 0) and np.all(b[1][2] == 0)
    np.testing.assert_allclose(b[1][:2], a[1], atol=1e-12)
    np.testing.assert_allclose(b[2], a[2], atol=1e-12)


# ---------------------------------------------------------------------------
# An independent implementation, written from the equations with explicit
# loops and DFT sums, for tiny inputs only.
# ---------------------------------------------------------------------------
def _dft(frame, sign):
    n = len(frame)
    out = [[0j] * n for _ in range(n)]
    for qy in range(n):
        for qx in range(n):
            acc = 0j
            for uy in range(n):
                for ux in range(n):
                    acc += frame[uy][ux] * cmath.exp(sign * 2j * math.pi * (qy * uy + qx * ux) / n)
            out[qy][qx] = acc / n
    return out


def loop_dm_iteration(psi, probe, obj, pos, inten, beta, delta_rel, jacobi=False):
    J, M, N = len(psi), len(probe), len(probe[0])
    H, W = len(obj), len(obj[0])
    psi = [[[list(row) for row in psi[j][k]] for k in range(M)] for j in range(J)]
    new_psi = []
    for j in range(J):
        r0, c0 = int(pos[j][0]), int(pos[j][1])
        po = [[[probe[k][y][x] * obj[r0 + y][c0 + x] for x in range(N)] for y in range(N)] for k in range(M)]
        spec = [_dft([[2 * po[k][y][x] - psi[j][k][y][x] for x in range(N)] for y in range(N)], -1) for k in range(M)]
        for qy in range(N):
            for qx in range(N):
                s = sum(abs(spec[k][qy][qx]) ** 2 for k in range(M))
                f = math.sqrt(max(inten[j][qy][qx], 0.0)) / math.sqrt(s) if s > 0 else 0.0
                for k in range(M):
                    spec[k][qy][qx] *= f
        back = [_dft(spec[k], +1) for k in range(M)]
        new_psi.append([[[psi[j][k][y][x] + beta * (back[k][y][x] - po[k][y][x]) for x in range(N)]
                         for y in range(N)] for k in range(M)])
    num = [[0j] * W for _ in range(H)]
    den = [[0.0] * W for _ in range(H)]
    for j in range(J):
        r0, c0 = int(pos[j][0]), int(pos[j][1])
        for k in range(M):
            for y in range(N):
                for x in range(N):
                    num[r0 + y][c0 + x] += probe[k][y][x].conjugate() * new_psi[j][k][y][x]
                    den[r0 + y][c0 + x] += abs(probe[k][y][x]) ** 2
    dmax = max(max(row) for row in den)
    new_obj = [[num[y][x] / (den[y][x] + delta_rel * dmax) if den[y][x] > 0 else obj[y][x]
                for x in range(W)] for y in range(H)]
    pnum = [[[0j] * N for _ in range(N)] for _ in range(M)]
    pden = [[0.0] * N for _ in range(N)]
    for j in range(J):
        r0, c0 = int(pos[j][0]), int(pos[j][1])
        for y in range(N):
            for x in range(N):
                o = (obj if jacobi else new_obj)[r0 + y][c0 + x]
                pden[y][x] += abs(o) ** 2
                for k in range(M):
                    pnum[k][y][x] += o.conjugate() * new_psi[j][k][y][x]
    pmax = max(max(row) for row in pden)
    new_probe = [[[pnum[k][y][x] / (pden[y][x] + delta_rel * pmax) for x in range(N)] for y in range(N)]
                 for k in range(M)]
    return np.array(new_psi), np.array(new_probe), np.array(new_obj)


@pytest.mark.parametrize("m,n", [(1, 4), (2, 4), (3, 2)])
def test_matches_independent_loop_implementation(m, n):
    rng = np.random.default_rng(20 + m)
    h = w = n + 3
    probe = rand_c(rng, (m, n, n))
    obj = rand_c(rng, (h, w))
    pos = np.array([[0, 0], [2, 1], [3, 3], [1, 2]], np.int32)
    psi = dm.init_exit_waves(probe, obj, pos) + 0.5 * rand_c(rng, (len(pos), m, n, n))
    inten = rng.uniform(0, 4, (len(pos), n, n))
    inten[1, 0, 0] = -1.0
    for beta, dr, order in ((0.8, 1e-3, "gauss-seidel"), (1.0, 0.0, "gauss-seidel"), (0.8, 1e-3, "jacobi")):
        a = dm.dm_iteration(psi, probe, obj, pos, inten, beta=beta, delta_rel=dr, order=order)
        b = loop_dm_iteration(psi.tolist(), probe.tolist(), obj.tolist(), pos.tolist(), inten.tolist(), beta, dr,
                              jacobi=(order == "jacobi"))
        np.testing.assert_allclose(a[0], b[0], atol=1e-12)
        np.testing.assert_allclose(a[1], b[1], atol=1e-11)
        np.testing.assert_allclose(a[2], b[2], atol=1e-12)


def test_eq6_on_known_perturbation():
    rng = np.random.default_rng(30)
    x = rand_c(rng, (6, 6))
    a = 0.3 - 0.2j
    assert dm.rel_change(x * (1 + a), x) == pytest.approx(abs(a) / abs(1 + a), rel=1e-13)


def test_fourier_error_closed_form():
    # Data exactly 4x the mode sum S of 2PO - psi gives
    # E_F = sqrt(sum (sqrt S - 2 sqrt S)^2 / sum 4 S) = 1/2.
    rng = np.random.default_rng(31)
    psi, probe, obj, pos, _ = generic_inputs(rng, m=2)
    n = probe.shape[-1]
    inten = []
    for j, (r, c) in enumerate(pos):
        phi = 2 * probe * obj[None, r:r + n, c:c + n] - psi[j]
        s = sum(np.abs(np.array(_dft(phi[k].tolist(), -1))) ** 2 for k in range(phi.shape[0]))
        inten.append(4.0 * s)
    _, _, _, m = dm.dm_iteration(psi, probe, obj, pos, np.array(inten))
    assert m["fourier_err"] == pytest.approx(0.5, rel=1e-12)


def test_noise_free_scan_converges_to_true_object():
    cfg = dict(n=32, modes=1, grid=(6, 6), step=6, jitter=1, obj=(70, 70), probe="gauss",
               fwhm=16.0, photons=1e6, seed=7)
    s = make_scan(cfg, noise=False)
    n = s.n
    den = np.zeros(s.obj_shape)
    for r, c in s.pos:
        den[r:r + n, c:c + n] += np.abs(s.probe[0]) ** 2
    cov = den >= 0.5 * den.max()
    probe, obj = s.probe.copy(), np.ones(s.obj_shape, complex)
    psi = dm.init_exit_waves(probe, obj, s.pos)
    inten = s.intensities.astype(np.float64)
    errs = []
    for it in range(700):
        psi, probe, obj, _ = dm.dm_iteration(psi, probe, obj, s.pos, inten, beta=0.8, update_probe=False)
        a, b = obj[cov], s.obj[cov]
        c = np.vdot(a, b) / np.vdot(a, a)
        errs.append(np.linalg.norm(c * a - b) / np.linalg.norm(b))
        if errs[-1] < 1e-3:
            break
    assert errs[-1] < 1e-3, (len(errs), errs[-1])
    assert errs[-1] < 0.01 * errs[0]


@pytest.mark.parametrize("scale", [1.0, 4.0])
def test_exit_wave_change_closed_form(scale):
    # Data equal to `scale` times the mode sum S of Phi = 2PO - psi makes the
    # modulus projection a plain factor sqrt(scale) on every mode, so Eq. 3
    # gives psi' = psi + beta (sqrt(scale) Phi - PO) in closed form, and the
    # exit-wave change is |psi' - psi| / |psi'| over the whole scan.
    rng = np.random.default_rng(37)
    psi, probe, obj, pos, _ = generic_inputs(rng, m=2)
    n = probe.shape[-1]
    beta = 0.7
    inten, want = [], []
    for j, (r, c) in enumerate(pos):
        po = probe * obj[None, r:r + n, c:c + n]
        phi = 2 * po - psi[j]
        s = sum(np.abs(np.array(_dft(phi[k].tolist(), -1))) ** 2 for k in range(phi.shape[0]))
        inten.append(scale * s)
        want.append(psi[j] + beta * (math.sqrt(scale) * phi - po))
    want = np.array(want)
    psi_new, _, _, m = dm.dm_iteration(psi, probe, obj, pos, np.array(inten), beta=beta)
    assert np.abs(psi_new - want).max() <= 1e-12 * np.abs(want).max()
    d = np.sqrt(np.sum(np.abs(want - psi) ** 2) / np.sum(np.abs(want) ** 2))
    assert m["eps_psi"] == pytest.approx(d, rel=1e-12)


def test_update_orders_differ_only_in_the_probe():
    # The two orders share Eq. 3 and Eq. 5; only the object Eq. 4 divides by
    # differs, and a Jacobi order needs a single inner pass.
    rng = np.random.default_rng(41)
    psi, probe, obj, pos, inten = generic_inputs(rng, m=2)
    gs = dm.dm_iteration(psi, probe, obj, pos, inten, order="gauss-seidel")
    ja = dm.dm_iteration(psi, probe, obj, pos, inten, order="jacobi")
    np.testing.assert_array_equal(gs[0], ja[0])
    np.testing.assert_array_equal(gs[2], ja[2])
    assert np.abs(gs[1] - ja[1]).max() > 1e-3 * np.abs(gs[1]).max()
    with pytest.raises(ValueError):
        dm.dm_iteration(psi, probe, obj, pos, inten, order="jacobi", n_inner=2)
