"""The pins are strong enough: plant plausible mistakes in the oracle (on the
CPU, via monkeypatching) and check that the hand-derived examples or the
independent loop implementation catch every one of them."""
import json
import os

import numpy as np
import pytest

from oracle import dm

import test_oracle_iteration as it

HERE = os.path.dirname(os.path.abspath(__file__))


def _mut_fft_sign(a):             # forward transform with the inverse's sign
    return np.fft.ifft2(a, norm="ortho")


def _mut_fft_norm(a):             # unnormalised forward transform
    return np.fft.fft2(a)


def _mut_fft_axes(a):             # transform over the wrong axes
    return np.fft.fftn(a, axes=(0, 1), norm="ortho")


def _mut_modulus_per_mode(phi_hat, intensity):   # each mode projected alone
    s = np.abs(phi_hat) ** 2
    scale = np.where(s > 0, np.sqrt(np.maximum(intensity, 0)) / np.sqrt(np.where(s > 0, s, 1)), 0)
    return phi_hat * scale, np.sum(s, axis=0)


def _object_noconj(psi, probe, obj, pos, delta_rel):
    n = probe.shape[-1]
    num = np.zeros(obj.shape, complex)
    den = np.zeros(obj.shape)
    for j in range(psi.shape[0]):
        r, c = pos[j]
        num[r:r + n, c:c + n] += np.sum(probe * psi[j], axis=0)
        den[r:r + n, c:c + n] += np.sum(np.abs(probe) ** 2, axis=0)
    new = obj.copy()
    cov = den > 0
    new[cov] = num[cov] / (den[cov] + delta_rel * den.max())
    return new


def _probe_transposed(psi, probe, obj, pos, delta_rel):
    n = probe.shape[-1]
    num = np.zeros(probe.shape, complex)
    den = np.zeros((n, n))
    for j in range(psi.shape[0]):
        r, c = pos[j]
        op = obj[c:c + n, r:r + n] if obj.shape[0] >= c + n and obj.shape[1] >= r + n else obj[r:r + n, c:c + n].T
        num += np.conj(op)[None] * psi[j]
        den += np.abs(op) ** 2
    new = probe.copy()
    cov = den > 0
    new[:, cov] = num[:, cov] / (den[cov] + delta_rel * den.max())
    return new


_orig_fourier_view = dm.fourier_update_view


def _fourier_beta_sign(psi_j, probe, obj, pos_j, intensity_j, beta):
    return _orig_fourier_view(psi_j, probe, obj, pos_j, intensity_j, -beta)


def _fourier_drop_2(psi_j, probe, obj, pos_j, intensity_j, beta):
    po = dm.field_products(probe, obj, pos_j)
    phi = po - psi_j                       # "2 P O - psi" written as "P O - psi"
    proj, s = dm.modulus_projection(dm.fft2(phi), intensity_j)
    out = psi_j + beta * (dm.ifft2(proj) - po)
    i_pos = np.maximum(intensity_j, 0.0)
    return out, float(np.sum((np.sqrt(s) - np.sqrt(i_pos)) ** 2)), float(np.sum(i_pos))


MUTANTS = {
    "fft sign": ("fft2", _mut_fft_sign),
    "fft normalisation": ("fft2", _mut_fft_norm),
    "fft axes": ("fft2", _mut_fft_axes),
    "F_c per mode": ("modulus_projection", _mut_modulus_per_mode),
    "object update without conj": ("object_update", _object_noconj),
    "probe update transposed patch": ("probe_update", _probe_transposed),
    "beta sign": ("fourier_update_view", _fourier_beta_sign),
    "dropped factor 2": ("fourier_update_view", _fourier_drop_2),
}


def _pins_pass():
    with open(os.path.join(HERE, "golden", "n2_worked_examples.json")) as f:
        cases = json.load(f)["cases"]
    try:
        import test_oracle_golden as g
        for c in cases:
            g.test_hand_derived_example(c)
        for m, n in [(1, 4), (2, 4), (3, 2)]:
            it.test_matches_independent_loop_implementation(m, n)
        it.test_exact_solution_is_a_fixed_point()
    except AssertionError:
        return False
    return True


def test_unmutated_oracle_passes_the_pins():
    assert _pins_pass()


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(dm, attr, fn)
    assert not _pins_pass(), f"mutant '{name}' survived the pins"
