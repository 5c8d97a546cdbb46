"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/dm.h declares, and rejects bad arguments before it
touches a GPU.  Also runs the host-side check of the FFT building blocks the
CUDA kernels are made of (tests/native/fft_host_check.cpp)."""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1808_10375_gb300 import build, dm
    build.build()
    return dm.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(dm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ["dm_init", "dm_iterate", "dm_get_object", "dm_get_probe", "dm_get_error", "dm_free",
                 "dm_last_error", "dm_get_exit_waves", "dm_get_mode_power"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1808_10375_gb300 import dm
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(dm.EXPORTS) == declared_functions()
    nm = shutil.which("nm")
    if nm:
        out = subprocess.run([nm, "-D", "--defined-only", dm.LIB_PATH], capture_output=True, text=True).stdout
        exported = set(re.findall(r"\b(dm_[a-z0-9_]+)\b", out))
        assert set(declared_functions()) <= exported


def test_params_default(lib):
    from paper_1808_10375_gb300 import dm
    p = dm.dm_params_default()
    assert abs(p.beta - 0.8) < 1e-7 and p.n_inner == 1 and p.probe_update_start == 0
    assert p.denom_floor_rel == 1e-6 and p.mem_kind == dm.DM_HOST and p.scratch_bytes == 0
    assert dm.dm_kernel_name(dm.DM_KERNEL_FOURIER) == "fourier"
    assert dm.dm_kernel_name(99) == "unknown"


def _init_rc(lib, dm, **kw):
    p = dm.dm_params_default(n=16, modes=1, views=2, obj_h=20, obj_w=20)
    for k, v in kw.items():
        setattr(p, k, v)
    pos = np.array([[0, 0], [4, 4]], np.int32)
    inten = np.zeros((2, 16, 16), np.float32)
    probe = np.zeros((1, 16, 16), np.complex64)
    obj = np.zeros((20, 20), np.complex64)
    h = ctypes.c_void_p()
    return lib.dm_init(ctypes.byref(h), ctypes.byref(p), pos.ctypes.data, inten.ctypes.data,
                       probe.ctypes.data, obj.ctypes.data), h


@pytest.mark.parametrize("kw", [dict(n=48), dict(n=512), dict(modes=0), dict(modes=17), dict(views=0),
                                dict(obj_h=8), dict(beta=1.5), dict(beta=float("nan")), dict(n_inner=0),
                                dict(probe_update_start=-1), dict(denom_floor_rel=-1.0),
                                dict(denom_floor_rel=float("inf")), dict(mem_kind=7), dict(scratch_bytes=-1),
                                dict(update_order=2), dict(update_order=1, n_inner=2)])
def test_invalid_params_rejected_without_gpu(lib, kw):
    from paper_1808_10375_gb300 import dm
    rc, h = _init_rc(lib, dm, **kw)
    assert rc == dm.DM_EINVAL
    assert not h.value
    assert dm.dm_last_error(None) != ""


def test_footprint_outside_object_rejected(lib):
    from paper_1808_10375_gb300 import dm
    p = dm.dm_params_default(n=16, modes=1, views=2, obj_h=20, obj_w=20)
    pos = np.array([[0, 0], [5, 4]], np.int32)            # 5 + 16 > 20
    buf = np.zeros(4096, np.complex64)
    h = ctypes.c_void_p()
    rc = lib.dm_init(ctypes.byref(h), ctypes.byref(p), pos.ctypes.data, buf.ctypes.data, buf.ctypes.data,
                     buf.ctypes.data)
    assert rc == dm.DM_EINVAL and "outside" in dm.dm_last_error(None)
    rc = lib.dm_init(ctypes.byref(h), ctypes.byref(p), None, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data)
    assert rc == dm.DM_EINVAL


def test_null_context_calls(lib):
    from paper_1808_10375_gb300 import dm
    assert lib.dm_iterate(None, 1) == dm.DM_EINVAL
    assert lib.dm_sync(None) == dm.DM_EINVAL
    assert lib.dm_iterations_done(None) == -1
    assert lib.dm_device_bytes(None) == 0
    lib.dm_free(None)


def test_host_fft_building_blocks(tmp_path):
    gxx = shutil.which("g++") or shutil.which("c++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cuda_inc = "/usr/local/cuda/include"
    exe = str(tmp_path / "fft_host_check")
    src = os.path.join(ROOT, "tests", "native", "fft_host_check.cpp")
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", cuda_inc, src, "-o", exe], check=True)
    r = subprocess.run([exe, "5e-7"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]


def test_binding_rejects_handles_of_another_kind():
    """Each release call takes only its own kind of handle (a network or a
    batch handed to dm_free would be released as a context)."""
    from paper_1808_10375_gb300 import dm
    for fn in (dm.dm_free, dm.dm_net_free, dm.dm_batch_free):
        with pytest.raises(TypeError):
            fn(object())
    with pytest.raises(TypeError):
        dm.dm_free(dm.Net(None, 1))


def test_static_probe_update_binding_rejects_bad_tensors():
    """The binding of dm_probe_update_static checks dtypes, shapes and the
    device before the C call (a too-small probe_out would be written past its
    end; int64 positions would be read as wrong pairs)."""
    import torch
    from paper_1808_10375_gb300 import dm
    j, m, n, h, w = 3, 2, 16, 40, 40
    good = dict(psi=torch.zeros(j, m, n, n, dtype=torch.complex64), obj=torch.zeros(h, w, dtype=torch.complex64),
                positions=torch.zeros(j, 2, dtype=torch.int32), probe_in=torch.zeros(m, n, n, dtype=torch.complex64),
                probe_out=torch.zeros(m, n, n, dtype=torch.complex64))
    bad_cases = [
        ("positions", torch.zeros(j, 2, dtype=torch.int64), "int32"),
        ("psi", torch.zeros(j, m, n, n, dtype=torch.complex128), "complex64"),
        ("probe_out", torch.zeros(m - 1, n, n, dtype=torch.complex64), "probe_out must be"),
        ("probe_in", torch.zeros(m, n, n + 1, dtype=torch.complex64), "probe_in must be"),
        ("positions", torch.zeros(j + 1, 2, dtype=torch.int32), "positions must be"),
        ("obj", torch.zeros(n - 1, w, dtype=torch.complex64), "at least"),
        ("psi", torch.zeros(j, m, n, n, dtype=torch.complex64).transpose(2, 3), "contiguous"),
    ]
    for name, t, msg in bad_cases:
        args = dict(good, **{name: t})
        with pytest.raises(ValueError, match=msg):
            dm._static_probe_args(**args)
    with pytest.raises(ValueError, match="CUDA"):
        dm._static_probe_args(**good)


def test_psi_precision_parameters_are_checked():
    """dm_init rejects an unknown exit-wave storage, the half form for frame
    sizes without one, and a negative switch threshold (no GPU needed: the
    checks come before any CUDA call)."""
    from paper_1808_10375_gb300 import dm
    lib = dm.load()
    pos = np.zeros((1, 2), np.int32)
    inten = np.zeros((1, 16, 16), np.float32)
    pr = np.zeros((1, 16, 16), np.complex64)
    ob = np.zeros((16, 16), np.complex64)
    for kw, msg in [(dict(psi_precision=7), "psi_precision"), (dict(psi_precision=dm.DM_PSI_FP16), "complex-half"),
                    (dict(psi_switch=-1.0), "psi_switch")]:
        params = dm.dm_params_default(n=16, modes=1, views=1, obj_h=16, obj_w=16, **kw)
        h = ctypes.c_void_p()
        rc = lib.dm_init(ctypes.byref(h), ctypes.byref(params), pos.ctypes.data, inten.ctypes.data, pr.ctypes.data,
                         ob.ctypes.data)
        assert rc == dm.DM_EINVAL and msg in dm.dm_last_error(None), (kw, dm.dm_last_error(None))
    p = dm.dm_params_default()
    assert p.psi_precision == dm.DM_PSI_FP32 and p.psi_switch == 0.0
