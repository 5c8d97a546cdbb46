"""FP64 CPU oracle of one multi-mode difference-map (DM) iteration.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code, tables or helpers
with the CUDA library; the seeded generators in ``synth`` are the only thing
both sides see.

It is deliberately plain: NumPy in float64/complex128, one view at a time, the
steps in the order of the paper (Sec. II), with ``numpy.fft`` as the only
library primitive.  Notation: J views j, M probe modes k (one object mode,
M_O = 1, which the paper reports is the only useful case), N x N frames, an
H x W object O, probe modes P_k, exit waves psi_j^k, integer top-left scan
positions r_j = (row, col).

Readings of points the paper leaves open:

* F is the orthonormal 2-D DFT, F[x](q) = (1/N) sum_u x(u) exp(-2 pi i q.u/N),
  with the zero frequency at index [0, 0] (no shift).
* The constrained transform F_c (Sec. II, after Eq. 3) is applied jointly to
  all modes of its argument 2 P O - psi; its denominator sums that argument's
  modes.  Where the mode sum S(q) is zero the projected field is zero;
  negative intensities are clamped to zero.
* Eq. 4 and Eq. 5 are applied Gauss-Seidel: the object first (with the probe
  the Fourier step used), then each probe mode with the new object.  The pair
  is repeated ``n_inner`` times (default once).
* Zero denominators: delta = delta_rel * max(denominator) is added to each
  denominator; object pixels outside every footprint keep their value.
* The convergence monitor is Eq. 6 with sums in place of the integrals, for
  the object and for each probe mode.  The Fourier error (the "error
  estimation for psi" of Sec. III, which the paper does not define) is
  E_F = sqrt( sum_j sum_q (sqrt(S_j(q)) - sqrt(I_j(q)))^2 / sum_j sum_q I_j(q) )
  on the S of the Fourier step.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Transforms (Eq. 1 / Eq. 3): orthonormal 2-D DFT over the last two axes.
# --------------------------------------------------------------------------
def fft2(a):
    """F: orthonormal forward 2-D DFT over the last two axes, DC at [0, 0]."""
    return np.fft.fft2(a, norm="ortho")


def ifft2(a):
    """F^-1: orthonormal inverse 2-D DFT over the last two axes."""
    return np.fft.ifft2(a, norm="ortho")


# --------------------------------------------------------------------------
# Field product (Eq. 2) and the initial exit waves (Sec. II, first step).
# --------------------------------------------------------------------------
def object_patch(obj, pos_j, n):
    """O(r) on the footprint of view j, as an N x N array indexed by the
    probe coordinate u = r - r_j."""
    r, c = int(pos_j[0]), int(pos_j[1])
    return obj[r:r + n, c:c + n]


def field_products(probe, obj, pos_j):
    """P_k(u) O(r_j + u) for every mode k: shape [M, N, N] (Eq. 2)."""
    n = probe.shape[-1]
    return probe * object_patch(obj, pos_j, n)[None]


def init_exit_waves(probe, obj, pos):
    """psi_j^k = P_k O on every footprint: the initial fields built from the
    initial guesses (Sec. II)."""
    return np.stack([field_products(probe, obj, p) for p in pos])


# --------------------------------------------------------------------------
# Constrained Fourier transform F_c (Sec. II).
# --------------------------------------------------------------------------
def modulus_projection(phi_hat, intensity):
    """Rescale every mode of phi_hat [M, N, N] by sqrt(I / sum_k |phi_hat_k|^2),
    keeping each mode's phase.  Returns (projected, S) with S the mode sum."""
    s = np.sum(np.abs(phi_hat) ** 2, axis=0)
    i_pos = np.maximum(intensity, 0.0)
    scale = np.zeros_like(s)
    nz = s > 0
    scale[nz] = np.sqrt(i_pos[nz]) / np.sqrt(s[nz])
    return phi_hat * scale[None], s


# --------------------------------------------------------------------------
# Exit-wave update (Eq. 3).
# --------------------------------------------------------------------------
def fourier_update_view(psi_j, probe, obj, pos_j, intensity_j, beta):
    """One view of Eq. 3:
        psi <- psi + beta * ( F^-1 F_c[2 P O - psi] - P O ).
    Returns (psi_new [M, N, N], fourier-error numerator, sum of I)."""
    po = field_products(probe, obj, pos_j)
    phi = 2.0 * po - psi_j
    phi_hat = fft2(phi)
    proj, s = modulus_projection(phi_hat, intensity_j)
    psi_new = psi_j + beta * (ifft2(proj) - po)
    i_pos = np.maximum(intensity_j, 0.0)
    err_num = float(np.sum((np.sqrt(s) - np.sqrt(i_pos)) ** 2))
    return psi_new, err_num, float(np.sum(i_pos))


def fourier_update(psi, probe, obj, pos, intensities, beta):
    """Eq. 3 over all views.  Returns (psi_new, E_F)."""
    out = np.empty_like(psi)
    num = 0.0
    den = 0.0
    for j in range(psi.shape[0]):
        out[j], e, s = fourier_update_view(psi[j], probe, obj, pos[j], intensities[j], beta)
        num += e
        den += s
    ef = float(np.sqrt(num / den)) if den > 0 else 0.0
    return out, ef


# --------------------------------------------------------------------------
# Overlap projection: object (Eq. 5) and probe (Eq. 4).
# --------------------------------------------------------------------------
def object_update(psi, probe, obj, pos, delta_rel):
    """Eq. 5 with one object mode:
        O(r) = sum_j sum_k conj(P_k(r - r_j)) psi_j^k(r - r_j)
               / (sum_j sum_k |P_k(r - r_j)|^2 + delta),
    delta = delta_rel * max_r(denominator); pixels no footprint covers keep
    their value.  The per-view accumulation is the embedding loop of Sec. III
    (a slice add per scan point)."""
    n = probe.shape[-1]
    num = np.zeros(obj.shape, dtype=np.complex128)
    den = np.zeros(obj.shape, dtype=np.float64)
    pc = np.conj(probe)
    p2 = np.sum(np.abs(probe) ** 2, axis=0)
    for j in range(psi.shape[0]):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        num[r:r + n, c:c + n] += np.sum(pc * psi[j], axis=0)
        den[r:r + n, c:c + n] += p2
    delta = delta_rel * den.max()
    new = obj.copy()
    cov = den > 0
    new[cov] = num[cov] / (den[cov] + delta)
    return new


def object_denominator(probe, pos, shape):
    """The denominator of Eq. 5 over the whole object array,
    sum_j sum_k |P_k(r - r_j)|^2, accumulated one footprint at a time."""
    n = probe.shape[-1]
    den = np.zeros(shape, dtype=np.float64)
    p2 = np.sum(np.abs(probe) ** 2, axis=0)
    for j in range(pos.shape[0]):
        r, c = int(pos[j, 0]), int(pos[j, 1])
        den[r:r + n, c:c + n] += p2
    return den


def views_covering(pos, n, pixel):
    """Indices j of the footprints that contain the object pixel (row, col)."""
    r, c = pixel
    inside = (pos[:, 0] <= r) & (r < pos[:, 0] + n) & (pos[:, 1] <= c) & (c < pos[:, 1] + n)
    return np.nonzero(inside)[0]


def object_update_at(pixels, psi_of_view, probe, obj, pos, delta_rel, den_max):
    """Eq. 5 evaluated at a few object pixels only, for scans too large for
    ``object_update``.  ``psi_of_view(j)`` returns the [M, N, N] exit waves of
    view j; ``den_max`` is the maximum of ``object_denominator`` over the
    whole array (it fixes delta).  Pixels no footprint covers keep their
    value.  Returns the new object values at ``pixels``."""
    n = probe.shape[-1]
    delta = delta_rel * den_max
    out = np.empty(len(pixels), dtype=np.complex128)
    for i, (r, c) in enumerate(pixels):
        num = 0.0 + 0.0j
        den = 0.0
        for j in views_covering(pos, n, (r, c)):
            u, v = r - int(pos[j, 0]), c - int(pos[j, 1])
            pk = probe[:, u, v]
            num += np.sum(np.conj(pk) * psi_of_view(j)[:, u, v])
            den += float(np.sum(np.abs(pk) ** 2))
        out[i] = num / (den + delta) if den > 0 else obj[r, c]
    return out


def probe_update(psi, probe, obj, pos, delta_rel):
    """Eq. 4 with one object mode, for every probe mode k:
        P_k(u) = sum_j conj(O(r_j + u)) psi_j^k(u)
                 / (sum_j |O(r_j + u)|^2 + delta),
    delta = delta_rel * max_u(denominator)."""
    n = probe.shape[-1]
    num = np.zeros(probe.shape, dtype=np.complex128)
    den = np.zeros((n, n), dtype=np.float64)
    for j in range(psi.shape[0]):
        op = object_patch(obj, pos[j], n)
        num += np.conj(op)[None] * psi[j]
        den += np.abs(op) ** 2
    delta = delta_rel * den.max()
    new = probe.copy()
    cov = den > 0
    new[:, cov] = num[:, cov] / (den[cov] + delta)
    return new


# --------------------------------------------------------------------------
# Convergence monitor (Eq. 6).
# --------------------------------------------------------------------------
def rel_change(new, old):
    """sqrt( sum |new - old|^2 / sum |new|^2 ) (Eq. 6, sums for integrals)."""
    d = float(np.sum(np.abs(new - old) ** 2))
    s = float(np.sum(np.abs(new) ** 2))
    return float(np.sqrt(d / s)) if s > 0 else 0.0


# --------------------------------------------------------------------------
# One DM iteration.
# --------------------------------------------------------------------------
def dm_iteration(psi, probe, obj, pos, intensities, beta=0.8, delta_rel=1e-6,
                 n_inner=1, update_probe=True, order="gauss-seidel"):
    """Eq. 3, then (Eq. 5, Eq. 4) x n_inner, then Eq. 6.

    Eqs. 4 and 5 are written as simultaneous updates.  ``order`` picks how
    they are taken:
    - "gauss-seidel" (the default): the object from the current probe, then
      the probe from the new object, n_inner times;
    - "jacobi": both from the values the iteration started with, so the
      probe uses the old object (n_inner must be 1).

    All inputs are left untouched.  Returns (psi, probe, obj, metrics) with
    metrics = {"eps_obj", "eps_probe" (list over modes), "fourier_err",
    "eps_psi"}.  eps_psi is the relative change of the exit waves over the
    whole scan, sqrt(sum |psi_new - psi|^2 / sum |psi_new|^2), the reading
    taken here of the "psi error" whose estimation Sec. III counts among the
    costly CPU steps without defining it."""
    psi = np.asarray(psi, dtype=np.complex128)
    probe = np.asarray(probe, dtype=np.complex128)
    obj = np.asarray(obj, dtype=np.complex128)
    intensities = np.asarray(intensities, dtype=np.float64)
    if order not in ("gauss-seidel", "jacobi"):
        raise ValueError(f"unknown order {order!r}")
    if order == "jacobi" and n_inner != 1:
        raise ValueError("the Jacobi order takes one inner pass")
    psi_new, ef = fourier_update(psi, probe, obj, pos, intensities, beta)
    o_new, p_new = obj, probe
    for _ in range(max(1, n_inner)):
        o_prev = o_new
        o_new = object_update(psi_new, p_new, o_new, pos, delta_rel)
        if update_probe:
            p_new = probe_update(psi_new, p_new, o_prev if order == "jacobi" else o_new, pos, delta_rel)
    metrics = {
        "eps_obj": rel_change(o_new, obj),
        "eps_probe": [rel_change(p_new[k], probe[k]) for k in range(probe.shape[0])],
        "fourier_err": ef,
        "eps_psi": rel_change(psi_new, psi),
    }
    return psi_new, p_new, o_new, metrics


def mode_power(probe):
    """sum_u |P_k(u)|^2 for every mode (the per-mode contribution used to
    choose the number of modes, Sec. II)."""
    return np.sum(np.abs(probe) ** 2, axis=(-2, -1))
