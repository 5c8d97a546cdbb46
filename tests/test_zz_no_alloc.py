"""The allocation-free probe update, dm_probe_update_static, through the C ABI.

Some callers of this library cannot allocate device memory: a host
application that owns all of it and hands the library no allocator, or code
that must not call cudaMalloc/cudaFree.  dm_probe_update_static gives them the
probe update (Eq. 4) with its reduction scratch in a fixed array inside the
library.  This file checks it, on two calls in a row of different sizes,
against the FP64 oracle's probe update on the same inputs and against the
probe update of a normal context (dm_run_step with DM_STEP_PROBE), within the
parity tolerance of the other GPU tests; that the call changes the device's
free memory by nothing; and that it refuses sizes beyond its array, bad
positions and a capturing stream.  It is collected last and passes both alone
and after the other tests."""
import ctypes

import numpy as np
import pytest

from oracle import dm as odm
from parity_util import REL_L2, case, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_10375_gb300 import build
    build.build()


def reference_probe_update(s, p0, o0, psi0, delta_rel):
    from paper_1808_10375_gb300 import dm
    h, w = s.obj_shape
    params = dm.dm_params_default(n=s.n, modes=s.modes, views=s.views, obj_h=h, obj_w=w,
                                  denom_floor_rel=delta_rel)
    ctx = dm.dm_init(params, s.pos, s.intensities, p0, o0)
    dm.dm_set_exit_waves(ctx, psi0)
    dm.dm_run_step(ctx, dm.DM_STEP_PROBE)
    out = dm.dm_get_probe(ctx)
    dm.dm_free(ctx)
    return out


def device_args(s, p0, o0, psi0, pos=None):
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    pin = dev(p0)
    return dict(psi=dev(psi0), obj=dev(o0), pos=dev(s.pos if pos is None else pos), pin=pin,
                pout=torch.empty_like(pin))


def call_static(t, s, delta_rel, stream=None):
    import torch
    from paper_1808_10375_gb300 import dm
    lib = dm.load()
    h, w = s.obj_shape
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return lib.dm_probe_update_static(t["psi"].data_ptr(), t["obj"].data_ptr(), t["pos"].data_ptr(),
                                      t["pin"].data_ptr(), t["pout"].data_ptr(), s.n, s.modes, s.views, h, w,
                                      delta_rel, ctypes.c_void_p(stream))


def test_static_probe_update_matches_oracle_and_context_on_consecutive_calls():
    import torch
    from paper_1808_10375_gb300 import dm
    cases = [case(64, 3, (4, 5), 10, (110, 120), 41), case(128, 4, (4, 4), 14, (190, 190), 42)]
    for delta_rel, (s, p0, o0, psi0) in zip((1e-6, 1e-3), cases):
        want = odm.probe_update(psi0.astype(np.complex128), p0.astype(np.complex128), o0.astype(np.complex128),
                                s.pos, delta_rel)
        ref = reference_probe_update(s, p0, o0, psi0, delta_rel)
        t = device_args(s, p0, o0, psi0)
        torch.cuda.synchronize()
        rc = call_static(t, s, delta_rel)
        assert rc == dm.DM_OK, dm.dm_last_error(None)
        got = t["pout"].cpu().numpy()
        for k in range(s.modes):
            assert rel_l2(got[k], want[k]) <= REL_L2, (s.n, k, rel_l2(got[k], want[k]))
            assert rel_l2(got[k], ref[k]) <= REL_L2, (s.n, k, rel_l2(got[k], ref[k]))


def test_static_probe_update_allocates_no_device_memory():
    import torch
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(64, 2, (3, 3), 10, (90, 90), 44)
    t = device_args(s, p0, o0, psi0)
    assert call_static(t, s, 1e-6) == dm.DM_OK, dm.dm_last_error(None)   # warmed up: module loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call_static(t, s, 1e-6) == dm.DM_OK, dm.dm_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_probe_update_rejects_what_does_not_fit():
    import torch
    from paper_1808_10375_gb300 import dm
    lib = dm.load()
    z = torch.zeros(4, dtype=torch.complex64, device="cuda")
    # 16 modes of 256 x 256 need more than the fixed scratch
    rc = lib.dm_probe_update_static(z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                    256, 16, 1, 256, 256, 1e-6, None)
    assert rc == dm.DM_EINVAL and "static scratch" in dm.dm_last_error(None)
    # a footprint outside the object is caught on the device before any work
    s, p0, o0, psi0 = case(32, 2, (2, 2), 6, (50, 50), 43)
    bad = s.pos.copy()
    bad[1, 0] = 50 - 32 + 1
    t = device_args(s, p0, o0, psi0, pos=bad)
    rc = call_static(t, s, 1e-6, stream=0)
    assert rc == dm.DM_EINVAL and "outside" in dm.dm_last_error(None)


def test_static_probe_update_refuses_a_capturing_stream():
    import torch
    from paper_1808_10375_gb300 import dm
    s, p0, o0, psi0 = case(32, 2, (2, 2), 6, (50, 50), 45)
    t = device_args(s, p0, o0, psi0)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.graph(g, stream=side):
        rcs.append(call_static(t, s, 1e-6, stream=side.cuda_stream))
    assert rcs == [dm.DM_EINVAL] and "captured" in dm.dm_last_error(None)
    # the stream is usable afterwards and the call works there
    assert call_static(t, s, 1e-6) == dm.DM_OK, dm.dm_last_error(None)
