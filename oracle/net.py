"""FP64 NumPy reference of the warm-start encoder-decoder (test
infrastructure only: it checks the CUDA training kernels and is never on the
product path).

The network is fixed by the library's C ABI description: 3 x 3 convolutions
with zero padding 1; an encoder of six stride-2 layers
1->16->32->64->128->256->256 channels (128 -> 2 pixels) with ReLU; a decoder
of five layers that upsample by 2 (nearest) then convolve with stride 1,
256->256->128->64->32->16 channels (2 -> 64 pixels) with ReLU; a linear 16->2
head at 64 x 64 (amplitude, phase).  Parameters are one flat array, per layer
the weights [co][ci][3][3] then the biases [co].  The kernels multiply with
weights rounded to BF16 (round to nearest even on the float32 value), so the
forward pass here does the same when ``bf16_weights`` is set; gradients are
taken with respect to the unrounded parameters (the rounding is treated as
the identity, as in the straight-through update the kernels perform).

Two losses: the mean squared error over both output channels, and the
phase-gauge-invariant loss.  One view's intensities do not change when its
object patch is multiplied by a constant phase factor, so the second loss
compares each predicted complex patch z = a exp(i phi) with its target t
after the global phase that fits best:
    L = (1 / (B P)) sum_b min_theta sum_p |exp(i theta) z_bp - t_bp|^2
      = (1 / (B P)) sum_b (sum_p |z_bp|^2 + sum_p |t_bp|^2 - 2 |S_b|),
    S_b = sum_p conj(z_bp) t_bp,
over B samples of P pixels each.
"""
from __future__ import annotations

import numpy as np


def layers():
    """(ci, co, hin, hout, stride, up, relu) per layer, in order."""
    ch = [1, 16, 32, 64, 128, 256, 256]
    out, h = [], 128
    for i in range(6):
        out.append((ch[i], ch[i + 1], h, h // 2, 2, False, True))
        h //= 2
    for i in range(6, 1, -1):
        out.append((ch[i], ch[i - 1], h, 2 * h, 1, True, True))
        h *= 2
    out.append((16, 2, 64, 64, 1, False, False))
    return out


def param_count():
    return sum(co * ci * 9 + co for ci, co, *_ in layers())


def unpack(params):
    """[(w [co][ci][3][3], b [co])] views of the flat parameter array."""
    out, off = [], 0
    for ci, co, *_ in layers():
        w = params[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        out.append((w, params[off:off + co]))
        off += co
    return out


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as
    float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _conv_input(a, up):
    """Zero-padded (by 1) convolution input, upsampled by 2 if ``up``."""
    if up:
        a = a.repeat(2, axis=2).repeat(2, axis=3)
    return np.pad(a, ((0, 0), (0, 0), (1, 1), (1, 1)))


def forward(params, x, bf16_weights=True):
    """Activations [x, out_1, ..., out_L] for input x [B, 1, 128, 128]."""
    acts = [np.asarray(x, np.float64)]
    for (ci, co, hin, hout, s, up, relu), (w, b) in zip(layers(), unpack(np.asarray(params, np.float64))):
        we = bf16_round(w) if bf16_weights else w
        xp = _conv_input(acts[-1], up)
        out = np.broadcast_to(b[None, :, None, None], (x.shape[0], co, hout, hout)).copy()
        for ky in range(3):
            for kx in range(3):
                patch = xp[:, :, ky:ky + s * hout:s, kx:kx + s * hout:s]
                out += np.einsum("oc,bcyx->boyx", we[:, :, ky, kx], patch)
        acts.append(np.maximum(out, 0.0) if relu else out)
    return acts


def mse_loss(y, target):
    """Mean squared error over every output value, and its gradient."""
    return float(np.mean((y - target) ** 2)), 2.0 * (y - target) / y.size


def gauge_loss(y, target):
    """The phase-gauge-invariant loss of outputs y [B, 2, P, P] (amplitude,
    phase) against target (the same layout), and its gradient dL/dy.

    With z = a exp(i phi), w = t conj(S)/|S| (the target turned by the
    fitted phase; w = 0 where S = 0) and u = exp(i phi), differentiating
    L = (sum |z|^2 + sum |t|^2 - 2|S|) / (B P) gives
        dL/da   = 2 (a - Re(conj(w) u)) / (B P),
        dL/dphi = 2 a Im(conj(w) u) / (B P)."""
    y = np.asarray(y, np.float64)
    target = np.asarray(target, np.float64)
    b = y.shape[0]
    npix = b * y.shape[2] * y.shape[3]
    a, phi = y[:, 0], y[:, 1]
    u = np.exp(1j * phi)
    z = a * u
    t = target[:, 0] * np.exp(1j * target[:, 1])
    s = np.sum(np.conj(z) * t, axis=(1, 2))
    mag = np.abs(s)
    loss = float(np.sum(np.sum(np.abs(z) ** 2, axis=(1, 2)) + np.sum(np.abs(t) ** 2, axis=(1, 2)) - 2 * mag) / npix)
    c = np.where(mag > 0, np.conj(s) / np.where(mag > 0, mag, 1.0), 0.0)
    w = t * c[:, None, None]
    cw = np.conj(w) * u
    g = np.empty_like(y)
    g[:, 0] = 2.0 * (a - cw.real) / npix
    g[:, 1] = 2.0 * a * cw.imag / npix
    return loss, g


def loss_and_gradients(params, x, target, bf16_weights=True, loss="mse"):
    """The loss (``"mse"`` or ``"gauge"``) of the output against ``target``
    [B, 2, 64, 64] and its gradient with respect to the flat parameters."""
    params = np.asarray(params, np.float64)
    acts = forward(params, x, bf16_weights)
    y = acts[-1]
    loss, g = (gauge_loss if loss == "gauge" else mse_loss)(y, target)
    grads = []
    ls = layers()
    wb = unpack(params)
    for li in range(len(ls) - 1, -1, -1):
        ci, co, hin, hout, s, up, relu = ls[li]
        w, _ = wb[li]
        we = bf16_round(w) if bf16_weights else w
        if relu:
            g = g * (acts[li + 1] > 0)
        xp = _conv_input(acts[li], up)
        gw = np.zeros_like(w)
        gxp = np.zeros_like(xp)
        for ky in range(3):
            for kx in range(3):
                patch = xp[:, :, ky:ky + s * hout:s, kx:kx + s * hout:s]
                gw[:, :, ky, kx] = np.einsum("boyx,bcyx->oc", g, patch)
                gxp[:, :, ky:ky + s * hout:s, kx:kx + s * hout:s] += np.einsum("oc,boyx->bcyx", we[:, :, ky, kx], g)
        grads.append((gw, g.sum(axis=(0, 2, 3))))
        gx = gxp[:, :, 1:-1, 1:-1]
        if up:
            gx = gx.reshape(gx.shape[0], gx.shape[1], hin, 2, hin, 2).sum(axis=(3, 5))
        g = gx
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in reversed(grads)])
    return loss, flat


def he_params(rng):
    """He-normal weights and zero biases (for the host-side pins)."""
    parts = []
    for ci, co, *_ in layers():
        parts.append(rng.standard_normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci)))
        parts.append(np.zeros(co))
    return np.concatenate(parts)
