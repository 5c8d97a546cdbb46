"""Batched 2-D DFT of 256 x 256 frames (dm_dft2) in both precision forms
against numpy's FP64 FFT: random frames and exit waves of the 8-mode
workload (probe modes times object patches), forward and inverse.

Bounds (relative L2 over the batch): the FP32 register FFT 1e-6; the split
BF16 tensor-core form 2e-5 (measured 6.3e-6; operands carry 16 significant bits after the
hi/lo split, and the dropped lo*lo term is of the same order)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = {0: 1e-6, 1: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _frames_random(count, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((count, 256, 256)) + 1j * rng.standard_normal((count, 256, 256))).astype(np.complex64)


def _frames_exit_waves():
    from synth import make_scan
    s = make_scan("mm256", views=2, noise=False)
    out = []
    for j in range(2):
        r, c = s.pos[j]
        out.extend(s.probe * s.obj[None, r:r + 256, c:c + 256])
    return np.asarray(out, np.complex64)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("inverse", [False, True])
@pytest.mark.parametrize("kind", ["random", "exit_waves"])
def test_dft2_against_fp64(precision, inverse, kind):
    import torch
    from paper_1808_10375_gb300 import dm
    x = _frames_random(5, 91) if kind == "random" else _frames_exit_waves()
    xd = torch.from_numpy(x).cuda()
    y = dm.dm_dft2(xd, inverse=inverse, precision=precision)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    x64 = x.astype(np.complex128)
    ref = np.fft.ifft2(x64) * (256 * 256) if inverse else np.fft.fft2(x64)
    err = _rel(got, ref)
    print(f"precision {precision} inverse {inverse} {kind}: relative L2 {err:.2e}")
    assert err <= BOUND[precision], err


def test_dft2_output_may_equal_input_and_rejects_bad_calls():
    import torch
    from paper_1808_10375_gb300 import dm
    x = _frames_random(2, 92)
    xd = torch.from_numpy(x).cuda()
    ref = np.fft.fft2(x.astype(np.complex128))
    dm.dm_dft2(xd, out=xd, precision=1)
    torch.cuda.synchronize()
    assert _rel(xd.cpu().numpy(), ref) <= BOUND[1]
    lib = dm.load()
    w = torch.empty_like(xd)
    assert lib.dm_dft2(xd.data_ptr(), w.data_ptr(), xd.data_ptr(), 128, 2, 0, 0, None) == dm.DM_EINVAL
    assert lib.dm_dft2(xd.data_ptr(), xd.data_ptr(), w.data_ptr(), 256, 2, 0, 0, None) == dm.DM_EINVAL
    assert lib.dm_dft2(xd.data_ptr(), w.data_ptr(), xd.data_ptr(), 256, 2, 0, 7, None) == dm.DM_EINVAL
