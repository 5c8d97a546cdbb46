"""ctypes binding of the C ABI in include/dm.h (argument marshalling only).

Every function keeps the C name.  Arrays may be NumPy arrays (host memory) or
torch tensors (host or CUDA); complex arrays are complex64, intensities
float32, positions int32.  Device memory for a context comes from torch's
caching allocator when torch has CUDA (passed through the ``alloc``/``free``
hooks of ``dm_params``), and all work runs on the stream given at dm_init
(torch's current stream by default).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptycho_dm.so")

DM_OK, DM_EINVAL, DM_ENOMEM, DM_ECUDA, DM_ENONFINITE, DM_ETIMEOUT = 0, -1, -2, -3, -4, -5
DM_HOST, DM_DEVICE = 0, 1
DM_STEP_FOURIER, DM_STEP_OBJECT, DM_STEP_PROBE = 0, 1, 2
DM_DFT_FP32, DM_DFT_BF16X3, DM_DFT_BF16X3_TC05 = 0, 1, 2
DM_ORDER_GAUSS_SEIDEL, DM_ORDER_JACOBI = 0, 1
DM_PSI_FP32, DM_PSI_FP16 = 0, 1
DM_FOURIER_STRIP, DM_FOURIER_SPLIT, DM_FOURIER_CLUSTER = 0, 1, 2
DM_NET_LOSS_MSE, DM_NET_LOSS_GAUGE = 0, 1
(DM_KERNEL_FOURIER, DM_KERNEL_OBJECT_GATHER, DM_KERNEL_OBJECT_FINAL, DM_KERNEL_PROBE_PARTIAL,
 DM_KERNEL_PROBE_FINAL, DM_KERNEL_METRICS, DM_KERNEL_OTHER, DM_KERNEL_COUNT) = range(8)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class dm_params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("modes", ctypes.c_int32), ("views", ctypes.c_int32),
        ("obj_h", ctypes.c_int32), ("obj_w", ctypes.c_int32),
        ("beta", ctypes.c_float), ("n_inner", ctypes.c_int32),
        ("probe_update_start", ctypes.c_int32), ("denom_floor_rel", ctypes.c_double),
        ("mem_kind", ctypes.c_int32),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("scratch_bytes", ctypes.c_int64),
        ("update_order", ctypes.c_int32),
        ("psi_precision", ctypes.c_int32),
        ("psi_switch", ctypes.c_double),
    ]


class DMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"DM error {code}: {msg}")
        self.code = code


EXPORTS = ["dm_params_default", "dm_init", "dm_iterate", "dm_run_step", "dm_get_object", "dm_get_probe",
           "dm_get_exit_waves", "dm_set_exit_waves", "dm_set_object", "dm_set_probe", "dm_get_error",
           "dm_set_psi_error", "dm_get_psi_error", "dm_selftest_bounded_waits", "dm_iterations_done", "dm_get_mode_power", "dm_sync", "dm_set_timing", "dm_get_timing",
           "dm_kernel_name", "dm_device_bytes", "dm_free", "dm_last_error", "dm_probe_update_static",
           "dm_object_partials", "dm_object_apply", "dm_probe_partials", "dm_probe_apply",
           "dm_fourier_error_partials", "dm_finish_iteration", "dm_set_graph", "dm_autotune",
           "dm_get_plan", "dm_batch_create", "dm_batch_iterate", "dm_batch_set_graph", "dm_batch_free",
           "dm_batch_last_error", "dm_dft2", "dm_dft2_check", "dm_fp32_peak", "dm_set_psi_precision", "dm_get_psi_precision", "dm_set_fourier_form", "dm_get_fourier_form", "dm_net_create", "dm_net_param_count", "dm_net_get_params",
           "dm_net_set_params", "dm_net_forward", "dm_net_gradients", "dm_net_train_step", "dm_net_set_loss",
           "dm_net_free"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1808_10375_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, f32p, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, P(ctypes.c_float), P(ctypes.c_double)
    sig = {
        "dm_params_default": (None, [P(dm_params)]),
        "dm_init": (ctypes.c_int, [P(vp), P(dm_params), vp, vp, vp, vp]),
        "dm_iterate": (ctypes.c_int, [vp, i32]),
        "dm_run_step": (ctypes.c_int, [vp, i32]),
        "dm_get_object": (ctypes.c_int, [vp, vp, i32]),
        "dm_get_probe": (ctypes.c_int, [vp, vp, i32]),
        "dm_get_exit_waves": (ctypes.c_int, [vp, vp, i32]),
        "dm_set_exit_waves": (ctypes.c_int, [vp, vp, i32]),
        "dm_set_object": (ctypes.c_int, [vp, vp, i32]),
        "dm_set_probe": (ctypes.c_int, [vp, vp, i32]),
        "dm_get_error": (ctypes.c_int, [vp, i32, dp, dp, dp]),
        "dm_set_psi_error": (ctypes.c_int, [vp, i32]),
        "dm_selftest_bounded_waits": (ctypes.c_int, [dp]),
        "dm_fp32_peak": (ctypes.c_int, [dp]),
        "dm_set_psi_precision": (ctypes.c_int, [vp, i32]),
        "dm_get_psi_precision": (ctypes.c_int, [vp, P(ctypes.c_int32), P(ctypes.c_int64)]),
        "dm_get_psi_error": (ctypes.c_int, [vp, i32, dp]),
        "dm_iterations_done": (i64, [vp]),
        "dm_get_mode_power": (ctypes.c_int, [vp, dp]),
        "dm_sync": (ctypes.c_int, [vp]),
        "dm_set_timing": (ctypes.c_int, [vp, i32]),
        "dm_get_timing": (ctypes.c_int, [vp, i32, dp, P(i64)]),
        "dm_kernel_name": (ctypes.c_char_p, [i32]),
        "dm_device_bytes": (ctypes.c_size_t, [vp]),
        "dm_free": (None, [vp]),
        "dm_last_error": (ctypes.c_char_p, [vp]),
        "dm_probe_update_static": (ctypes.c_int, [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32,
                                                  ctypes.c_double, vp]),
        "dm_object_partials": (ctypes.c_int, [vp, vp, vp, i32]),
        "dm_object_apply": (ctypes.c_int, [vp, vp, vp, i32]),
        "dm_probe_partials": (ctypes.c_int, [vp, vp, vp, i32]),
        "dm_probe_apply": (ctypes.c_int, [vp, vp, vp, i32]),
        "dm_fourier_error_partials": (ctypes.c_int, [vp, dp]),
        "dm_finish_iteration": (ctypes.c_int, [vp, dp]),
        "dm_set_graph": (ctypes.c_int, [vp, i32]),
        "dm_autotune": (ctypes.c_int, [vp, i32, dp]),
        "dm_get_plan": (ctypes.c_int, [vp, P(i64)]),
        "dm_set_fourier_form": (ctypes.c_int, [vp, i32]),
        "dm_get_fourier_form": (ctypes.c_int, [vp, P(i32)]),
        "dm_batch_create": (ctypes.c_int, [P(vp), P(vp), i32]),
        "dm_batch_iterate": (ctypes.c_int, [vp, i32]),
        "dm_batch_set_graph": (ctypes.c_int, [vp, i32]),
        "dm_batch_free": (None, [vp]),
        "dm_batch_last_error": (ctypes.c_char_p, [vp]),
        "dm_dft2": (ctypes.c_int, [vp, vp, vp, i32, i32, i32, i32, vp]),
        "dm_dft2_check": (ctypes.c_int, []),
        "dm_net_create": (ctypes.c_int, [P(vp), i32, ctypes.c_uint64]),
        "dm_net_param_count": (i64, [vp]),
        "dm_net_get_params": (ctypes.c_int, [vp, f32p]),
        "dm_net_set_params": (ctypes.c_int, [vp, f32p]),
        "dm_net_forward": (ctypes.c_int, [vp, vp, i32, vp]),
        "dm_net_gradients": (ctypes.c_int, [vp, vp, vp, i32, f32p, dp]),
        "dm_net_train_step": (ctypes.c_int, [vp, vp, vp, i32, ctypes.c_float, dp]),
        "dm_net_set_loss": (ctypes.c_int, [vp, i32]),
        "dm_net_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _ptr(x, dtype):
    """(pointer, mem_kind, keepalive) for a contiguous array of `dtype`."""
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.complex64: torch.complex64}[dtype]
        if x.dtype != tdt or not x.is_contiguous():
            x = x.to(tdt).contiguous()
        return x.data_ptr(), (DM_DEVICE if x.is_cuda else DM_HOST), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, DM_HOST, a


class Context:
    """Handle of one dm_ctx plus what must outlive it (allocator hooks)."""

    def __init__(self, handle, params, keep):
        self.handle = handle
        self.params = params
        self._keep = keep

    @property
    def shape(self):
        p = self.params
        return dict(n=p.n, modes=p.modes, views=p.views, obj_h=p.obj_h, obj_w=p.obj_w)

    def __del__(self):
        try:
            if self.handle:
                dm_free(self)
        except Exception:
            pass


def _check(rc, ctx=None):
    if rc != DM_OK:
        lib = load()
        msg = lib.dm_last_error(ctx.handle if ctx is not None else None)
        raise DMError(rc, (msg or b"").decode())
    return rc


def _torch_allocator():
    import torch
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ALLOC_FN(_alloc), FREE_FN(_free), stream


# ---------------------------------------------------------------------------
# the ABI, one function each
# ---------------------------------------------------------------------------
def dm_params_default(**kw) -> dm_params:
    p = dm_params()
    load().dm_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def dm_init(params: dm_params, positions, intensities, probe0, object0, use_torch_allocator=None,
            stream=None) -> Context:
    """Create a context (copies the inputs).  Inputs on a CUDA device are
    passed as device pointers, otherwise as host pointers; mixing is an
    error.  With torch CUDA available the context allocates through torch's
    caching allocator and runs on torch's current stream unless told
    otherwise."""
    lib = load()
    pp, mk0, k0 = _ptr(positions, np.int32)
    ip, mk1, k1 = _ptr(intensities, np.float32)
    bp, mk2, k2 = _ptr(probe0, np.complex64)
    op, mk3, k3 = _ptr(object0, np.complex64)
    kinds = {mk0, mk1, mk2, mk3}
    if len(kinds) != 1:
        raise ValueError("all dm_init inputs must be on the host or all on the device")
    p = dm_params()
    ctypes.pointer(p)[0] = params
    p.mem_kind = kinds.pop()
    keep = [k0, k1, k2, k3]
    if use_torch_allocator is None:
        try:
            import torch
            use_torch_allocator = torch.cuda.is_available()
        except ImportError:  # pragma: no cover
            use_torch_allocator = False
    if use_torch_allocator:
        a, f, tstream = _torch_allocator()
        p.alloc, p.free = a, f
        keep += [a, f]
        if stream is None:
            stream = tstream.cuda_stream
    if stream is not None:
        # handle 0 is the legacy default stream; NULL would ask the library
        # for a stream of its own, so pass cudaStreamLegacy instead
        p.stream = ctypes.c_void_p(int(stream) if int(stream) != 0 else 1)
    h = ctypes.c_void_p()
    rc = lib.dm_init(ctypes.byref(h), ctypes.byref(p), pp, ip, bp, op)
    _check(rc)
    return Context(h, p, keep[4:])


def dm_iterate(ctx: Context, n_iter: int = 1):
    return _check(load().dm_iterate(ctx.handle, int(n_iter)), ctx)


def dm_set_graph(ctx: Context, enable: bool = True):
    return _check(load().dm_set_graph(ctx.handle, 1 if enable else 0), ctx)


def dm_autotune(ctx: Context, sample_views: int = 500) -> float:
    """Time the candidate Fourier-step plans on the first views; keeps the
    fastest.  Returns its time per run (ms) on the sample."""
    best = ctypes.c_double()
    _check(load().dm_autotune(ctx.handle, int(sample_views), ctypes.byref(best)), ctx)
    return best.value


def dm_get_plan(ctx: Context) -> dict:
    out = (ctypes.c_int64 * 5)()
    _check(load().dm_get_plan(ctx.handle, out), ctx)
    return dict(scratch_bytes=out[0], views_per_chunk=out[1], strips_per_column_task=out[2],
                strip_buffers=out[3], ctas=out[4])


class Batch:
    """Handle of one dm_batch and the contexts it advances."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)

    def __del__(self):
        try:
            if self.handle:
                load().dm_batch_free(self.handle)
                self.handle = None
        except Exception:
            pass


def _bcheck(rc, batch=None):
    if rc != DM_OK:
        msg = load().dm_batch_last_error(batch.handle if batch is not None else None)
        raise DMError(rc, (msg or b"").decode())
    return rc


def dm_batch_create(ctxs) -> Batch:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle for c in ctxs])
    h = ctypes.c_void_p()
    _bcheck(load().dm_batch_create(ctypes.byref(h), arr, len(ctxs)))
    return Batch(h.value, ctxs)


def dm_batch_iterate(batch: Batch, n_iter: int = 1):
    return _bcheck(load().dm_batch_iterate(batch.handle, int(n_iter)), batch)


def dm_batch_set_graph(batch: Batch, enable: bool = True):
    return _bcheck(load().dm_batch_set_graph(batch.handle, 1 if enable else 0), batch)


def dm_batch_free(batch: Batch):
    if not isinstance(batch, Batch):
        raise TypeError("dm_batch_free takes a batch from dm_batch_create")
    if batch.handle:
        load().dm_batch_free(batch.handle)
        batch.handle = None


def dm_dft2(x, work=None, out=None, inverse=False, precision=DM_DFT_FP32, stream=None):
    """Batched unnormalised 2-D DFT of complex64 CUDA frames [F, 256, 256]."""
    import torch
    if not (_is_torch(x) and x.is_cuda and x.dtype == torch.complex64 and x.is_contiguous() and x.dim() == 3):
        raise ValueError("x must be a contiguous complex64 CUDA tensor [frames, N, N]")
    work = torch.empty_like(x) if work is None else work
    out = torch.empty_like(x) if out is None else out
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = load().dm_dft2(x.data_ptr(), work.data_ptr(), out.data_ptr(), x.shape[-1], x.shape[0],
                        1 if inverse else 0, int(precision), s)
    if rc != DM_OK:
        raise DMError(rc, (load().dm_last_error(None) or b"").decode())
    return out


def dm_dft2_check():
    """Synchronise the device and raise DMError(DM_ETIMEOUT) if a bounded wait
    of the tcgen05 DFT form gave up since the last check (see dm.h)."""
    rc = load().dm_dft2_check()
    if rc != DM_OK:
        raise DMError(rc, (load().dm_last_error(None) or b"").decode())


class Net:
    """Handle of one dm_net (the warm-start encoder-decoder)."""

    def __init__(self, handle, max_batch):
        self.handle = handle
        self.max_batch = max_batch

    def __del__(self):
        try:
            if self.handle:
                load().dm_net_free(self.handle)
                self.handle = None
        except Exception:
            pass


def _ncheck(rc):
    if rc != DM_OK:
        raise DMError(rc, (load().dm_last_error(None) or b"").decode())
    return rc


def _cuda_f32(t, shape):
    """Device pointer of a network input; the tensor's producers on torch's
    current stream are waited for, because the network runs on its own
    stream."""
    import torch
    if not (_is_torch(t) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and tuple(t.shape) == shape):
        raise ValueError(f"expected a contiguous float32 CUDA tensor of shape {shape}")
    torch.cuda.current_stream(t.device).synchronize()
    return t.data_ptr()


def dm_net_create(max_batch: int = 64, seed: int = 0) -> Net:
    h = ctypes.c_void_p()
    _ncheck(load().dm_net_create(ctypes.byref(h), int(max_batch), int(seed)))
    return Net(h.value, max_batch)


def dm_net_param_count(net: Net) -> int:
    return int(load().dm_net_param_count(net.handle))


def dm_net_get_params(net: Net):
    out = np.empty(dm_net_param_count(net), np.float32)
    _ncheck(load().dm_net_get_params(net.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def dm_net_set_params(net: Net, params):
    a = np.ascontiguousarray(params, np.float32)
    if a.size != dm_net_param_count(net):
        raise ValueError("wrong parameter count")
    _ncheck(load().dm_net_set_params(net.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def dm_net_forward(net: Net, x):
    """x: float32 CUDA [B, 1, 128, 128] -> float32 CUDA [B, 2, 64, 64]."""
    import torch
    b = x.shape[0]
    y = torch.empty((b, 2, 64, 64), dtype=torch.float32, device=x.device)
    _ncheck(load().dm_net_forward(net.handle, _cuda_f32(x, (b, 1, 128, 128)), b, y.data_ptr()))
    return y


def dm_net_gradients(net: Net, x, target):
    b = x.shape[0]
    g = np.empty(dm_net_param_count(net), np.float32)
    loss = ctypes.c_double()
    _ncheck(load().dm_net_gradients(net.handle, _cuda_f32(x, (b, 1, 128, 128)), _cuda_f32(target, (b, 2, 64, 64)), b,
                                    g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
    return g, loss.value


def dm_net_train_step(net: Net, x, target, lr: float = 1e-3, want_loss: bool = False):
    b = x.shape[0]
    loss = ctypes.c_double()
    _ncheck(load().dm_net_train_step(net.handle, _cuda_f32(x, (b, 1, 128, 128)), _cuda_f32(target, (b, 2, 64, 64)), b,
                                     float(lr), ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def dm_net_set_loss(net: Net, kind: int):
    """The training loss: DM_NET_LOSS_MSE or DM_NET_LOSS_GAUGE (the
    phase-gauge-invariant loss)."""
    _ncheck(load().dm_net_set_loss(net.handle, int(kind)))


def dm_net_free(net: Net):
    if not isinstance(net, Net):
        raise TypeError("dm_net_free takes a network from dm_net_create")
    if net.handle:
        load().dm_net_free(net.handle)
        net.handle = None


def dm_run_step(ctx: Context, step: int):
    return _check(load().dm_run_step(ctx.handle, int(step)), ctx)


def _out(ctx, shape, out, device):
    if out is None:
        if device:
            import torch
            out = torch.empty(shape, dtype=torch.complex64, device="cuda")
        else:
            out = np.empty(shape, dtype=np.complex64)
    if _is_torch(out):
        if out.dtype.__str__() != "torch.complex64" or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor")
        return out, out.data_ptr(), (DM_DEVICE if out.is_cuda else DM_HOST)
    if out.dtype != np.complex64 or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous complex64 array")
    return out, out.ctypes.data, DM_HOST


def dm_get_object(ctx: Context, out=None, device=False):
    p = ctx.params
    out, ptr, mk = _out(ctx, (p.obj_h, p.obj_w), out, device)
    _check(load().dm_get_object(ctx.handle, ptr, mk), ctx)
    return out


def dm_get_probe(ctx: Context, out=None, device=False):
    p = ctx.params
    out, ptr, mk = _out(ctx, (p.modes, p.n, p.n), out, device)
    _check(load().dm_get_probe(ctx.handle, ptr, mk), ctx)
    return out


def dm_get_exit_waves(ctx: Context, out=None, device=False):
    p = ctx.params
    out, ptr, mk = _out(ctx, (p.views, p.modes, p.n, p.n), out, device)
    _check(load().dm_get_exit_waves(ctx.handle, ptr, mk), ctx)
    return out


def _set(fn, ctx, arr):
    ptr, mk, keep = _ptr(arr, np.complex64)
    _check(fn(ctx.handle, ptr, mk), ctx)
    del keep


def dm_set_exit_waves(ctx: Context, psi):
    _set(load().dm_set_exit_waves, ctx, psi)


def dm_set_object(ctx: Context, obj):
    _set(load().dm_set_object, ctx, obj)


def dm_set_probe(ctx: Context, probe):
    _set(load().dm_set_probe, ctx, probe)


def _buf(x, shape, np_dtype, device):
    """(array, pointer, mem_kind) of a contiguous buffer of `np_dtype`: `x`
    itself (NumPy array or torch tensor, host or CUDA) or a new one."""
    if x is None:
        if device:
            import torch
            tdt = {np.float32: torch.float32, np.float64: torch.float64, np.complex64: torch.complex64,
                   np.complex128: torch.complex128}[np_dtype]
            x = torch.empty(shape, dtype=tdt, device="cuda")
        else:
            x = np.empty(shape, dtype=np_dtype)
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.complex64: torch.complex64,
                   np.complex128: torch.complex128}[np_dtype]
        if x.dtype != tdt or not x.is_contiguous() or tuple(x.shape) != tuple(shape):
            raise ValueError(f"expected a contiguous {tdt} tensor of shape {shape}")
        return x, x.data_ptr(), (DM_DEVICE if x.is_cuda else DM_HOST)
    if x.dtype != np_dtype or not x.flags.c_contiguous or x.shape != tuple(shape):
        raise ValueError(f"expected a contiguous {np_dtype.__name__} array of shape {shape}")
    return x, x.ctypes.data, DM_HOST


def dm_object_partials(ctx: Context, num=None, den=None, device=False):
    """(num [H][W] complex64, den [H][W] float64) of Eq. 5 over the context's views."""
    p = ctx.params
    num, pn, mk = _buf(num, (p.obj_h, p.obj_w), np.complex64, device)
    den, pd, mk2 = _buf(den, (p.obj_h, p.obj_w), np.float64, device)
    if mk != mk2:
        raise ValueError("num and den must both be host or both be device buffers")
    _check(load().dm_object_partials(ctx.handle, pn, pd, mk), ctx)
    return num, den


def dm_object_apply(ctx: Context, num, den):
    """Eq. 5 from numerator and denominator sums over all shards, in FP64:
    num [H][W] complex128, den [H][W] float64."""
    p = ctx.params
    num, pn, mk = _buf(num, (p.obj_h, p.obj_w), np.complex128, False)
    den, pd, mk2 = _buf(den, (p.obj_h, p.obj_w), np.float64, False)
    if mk != mk2:
        raise ValueError("num and den must both be host or both be device buffers")
    _check(load().dm_object_apply(ctx.handle, pn, pd, mk), ctx)


def dm_probe_partials(ctx: Context, num=None, den=None, device=False):
    """(num [M][N][N][2] float64, den [N][N] float64) of Eq. 4 over the context's views."""
    p = ctx.params
    num, pn, mk = _buf(num, (p.modes, p.n, p.n, 2), np.float64, device)
    den, pd, mk2 = _buf(den, (p.n, p.n), np.float64, device)
    if mk != mk2:
        raise ValueError("num and den must both be host or both be device buffers")
    _check(load().dm_probe_partials(ctx.handle, pn, pd, mk), ctx)
    return num, den


def dm_probe_apply(ctx: Context, num, den):
    p = ctx.params
    num, pn, mk = _buf(num, (p.modes, p.n, p.n, 2), np.float64, False)
    den, pd, mk2 = _buf(den, (p.n, p.n), np.float64, False)
    if mk != mk2:
        raise ValueError("num and den must both be host or both be device buffers")
    _check(load().dm_probe_apply(ctx.handle, pn, pd, mk), ctx)


def dm_fourier_error_partials(ctx: Context):
    """[sum (sqrt S - sqrt I)^2, sum I] over the context's views (host)."""
    out = (ctypes.c_double * 2)()
    _check(load().dm_fourier_error_partials(ctx.handle, out), ctx)
    return [out[0], out[1]]


def dm_finish_iteration(ctx: Context, sums):
    arr = (ctypes.c_double * 2)(float(sums[0]), float(sums[1]))
    _check(load().dm_finish_iteration(ctx.handle, arr), ctx)


def dm_get_error(ctx: Context, iteration: int = -1):
    """(eps_obj, eps_probe[M], fourier_err) of one iteration."""
    eo = ctypes.c_double()
    ef = ctypes.c_double()
    ep = (ctypes.c_double * ctx.params.modes)()
    _check(load().dm_get_error(ctx.handle, int(iteration), ctypes.byref(eo), ep, ctypes.byref(ef)), ctx)
    return eo.value, list(ep), ef.value


def dm_set_psi_error(ctx: Context, enable: bool = True):
    """Track the exit-wave change eps_psi in the following iterations (the
    Fourier step then reads the old exit waves back)."""
    _check(load().dm_set_psi_error(ctx.handle, 1 if enable else 0), ctx)


def dm_get_psi_error(ctx: Context, iteration: int = -1) -> float:
    """eps_psi of one iteration (NaN where it was not tracked)."""
    out = ctypes.c_double()
    _check(load().dm_get_psi_error(ctx.handle, int(iteration), ctypes.byref(out)), ctx)
    return out.value


def dm_set_psi_precision(ctx: Context, precision: int):
    """Convert the exit waves to DM_PSI_FP32 or DM_PSI_FP16 storage (see dm.h)."""
    return _check(load().dm_set_psi_precision(ctx.handle, int(precision)), ctx)


def dm_get_psi_precision(ctx: Context):
    """(current exit-wave storage, iteration count of the automatic switch to
    complex64 or -1)."""
    prec = ctypes.c_int32()
    at = ctypes.c_int64()
    _check(load().dm_get_psi_precision(ctx.handle, ctypes.byref(prec), ctypes.byref(at)), ctx)
    return prec.value, at.value


def dm_set_fourier_form(ctx: Context, form: int):
    """Run the Fourier step in DM_FOURIER_STRIP, DM_FOURIER_SPLIT or DM_FOURIER_CLUSTER form (see dm.h)."""
    return _check(load().dm_set_fourier_form(ctx.handle, int(form)), ctx)


def dm_get_fourier_form(ctx: Context) -> int:
    """The form the next Fourier step runs (DM_FOURIER_STRIP, DM_FOURIER_SPLIT or DM_FOURIER_CLUSTER)."""
    form = ctypes.c_int32()
    _check(load().dm_get_fourier_form(ctx.handle, ctypes.byref(form)), ctx)
    return form.value


def dm_fp32_peak() -> float:
    """FP32-pipe peak of the current device in TFLOP/s (see dm.h)."""
    v = ctypes.c_double()
    rc = load().dm_fp32_peak(ctypes.byref(v))
    if rc != DM_OK:
        raise DMError(rc, (load().dm_last_error(None) or b"").decode())
    return v.value


def dm_selftest_bounded_waits() -> float:
    """Make the library's bounded device waits run out (see dm.h); returns
    the test kernel's device time in ms, raises if a wait did not give up."""
    ms = ctypes.c_double()
    rc = load().dm_selftest_bounded_waits(ctypes.byref(ms))
    if rc != DM_OK:
        raise DMError(rc, (load().dm_last_error(None) or b"").decode())
    return ms.value


def dm_iterations_done(ctx: Context) -> int:
    return int(load().dm_iterations_done(ctx.handle))


def dm_get_mode_power(ctx: Context):
    out = (ctypes.c_double * ctx.params.modes)()
    _check(load().dm_get_mode_power(ctx.handle, out), ctx)
    return list(out)


def dm_sync(ctx: Context):
    return _check(load().dm_sync(ctx.handle), ctx)


def dm_set_timing(ctx: Context, enable: bool = True):
    return _check(load().dm_set_timing(ctx.handle, 1 if enable else 0), ctx)


def dm_get_timing(ctx: Context, kernel: int):
    """(total device ms, launches) of one kernel class."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().dm_get_timing(ctx.handle, int(kernel), ctypes.byref(ms), ctypes.byref(n)), ctx)
    return ms.value, n.value


def dm_kernel_name(kernel: int) -> str:
    return load().dm_kernel_name(int(kernel)).decode()


def dm_device_bytes(ctx: Context) -> int:
    return int(load().dm_device_bytes(ctx.handle))


def dm_free(ctx: Context):
    if not isinstance(ctx, Context):
        raise TypeError("dm_free takes a context from dm_init")
    if ctx.handle:
        load().dm_free(ctx.handle)
        ctx.handle = None


def dm_last_error(ctx: Context | None = None) -> str:
    return (load().dm_last_error(ctx.handle if ctx is not None else None) or b"").decode()


def _static_probe_args(psi, obj, positions, probe_in, probe_out):
    """Shapes (J, M, N, H, W) of dm_probe_update_static's tensors after
    checking their types, layouts and shapes (ValueError on a mismatch)."""
    import torch
    names = ("psi", "obj", "positions", "probe_in", "probe_out")
    want = (torch.complex64, torch.complex64, torch.int32, torch.complex64, torch.complex64)
    dims = (4, 2, 2, 3, 3)
    for name, t, dt, nd in zip(names, (psi, obj, positions, probe_in, probe_out), want, dims):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, not {t.dtype}")
        if t.dim() != nd:
            raise ValueError(f"{name} must have {nd} dimensions, not {t.dim()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    j, m, n, n2 = psi.shape
    h, w = obj.shape
    if n2 != n:
        raise ValueError("psi frames must be square")
    if tuple(positions.shape) != (j, 2):
        raise ValueError(f"positions must be [{j}, 2]")
    for name, t in (("probe_in", probe_in), ("probe_out", probe_out)):
        if tuple(t.shape) != (m, n, n):
            raise ValueError(f"{name} must be [{m}, {n}, {n}]")
    if h < n or w < n:
        raise ValueError("the object must be at least N x N")
    for name, t in zip(names, (psi, obj, positions, probe_in, probe_out)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    dev = psi.device
    if any(t.device != dev for t in (obj, positions, probe_in, probe_out)):
        raise ValueError("all tensors must be on the same device")
    return j, m, n, h, w


def dm_probe_update_static(psi, obj, positions, probe_in, probe_out, denom_floor_rel=1e-6, stream=None):
    """Probe update (Eq. 4) that allocates no device memory: for callers that
    cannot call cudaMalloc (the C call's comment in include/dm.h has the
    details and the size limit).  All arguments are contiguous CUDA tensors
    on one device: psi [J, M, N, N] complex64, obj [H, W] complex64,
    positions [J, 2] int32, probe_in / probe_out [M, N, N] complex64.  The
    call returns once probe_out holds the result."""
    import torch
    j, m, n, h, w = _static_probe_args(psi, obj, positions, probe_in, probe_out)
    if stream is None:
        stream = torch.cuda.current_stream(psi.device).cuda_stream
    with torch.cuda.device(psi.device):
        rc = load().dm_probe_update_static(psi.data_ptr(), obj.data_ptr(), positions.data_ptr(),
                                           probe_in.data_ptr(), probe_out.data_ptr(), n, m, j, h, w,
                                           float(denom_floor_rel), ctypes.c_void_p(int(stream)))
    return _check(rc)
