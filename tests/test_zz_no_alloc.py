"""The allocation-free probe update, dm_probe_update_static, through the C ABI.

Some callers of this library cannot allocate device memory: a host
application that owns all of it and hands the library no allocator, or code
that must not call cudaMalloc/cudaFree.  dm_probe_update_static gives them the
probe update (Eq. 4) with its reduction scratch in a fixed array inside the
library.  This file checks it against the probe update of a normal context
(dm_run_step with DM_STEP_PROBE) on two calls in a row of different sizes,
within the parity tolerance of the other GPU tests.  It is collected last and
passes both alone and after the other tests."""
import ctypes

import numpy as np
import pytest

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


def static_probe_update(s, p0, o0, psi0, delta_rel):
    import torch
    from paper_1808_10375_gb300 import dm
    lib = dm.load()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    psi, obj, pos, pin = dev(psi0), dev(o0), dev(s.pos), dev(p0)
    pout = torch.empty_like(pin)
    h, w = s.obj_shape
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.dm_probe_update_static(psi.data_ptr(), obj.data_ptr(), pos.data_ptr(), pin.data_ptr(),
                                    pout.data_ptr(), s.n, s.modes, s.views, h, w, delta_rel,
                                    ctypes.c_void_p(stream))
    assert rc == dm.DM_OK, dm.dm_last_error(None)
    torch.cuda.synchronize()
    return pout.cpu().numpy()


def test_static_probe_update_matches_context_update_on_consecutive_calls():
    cases = [case(64, 3, (4, 5), 10, (110, 120), 41), case(128, 4, (4, 4), 14, (190, 190), 42)]
    for delta_rel, (s, p0, o0, psi0) in zip((1e-6, 1e-3), cases):
        ref = reference_probe_update(s, p0, o0, psi0, delta_rel)
        got = static_probe_update(s, p0, o0, psi0, delta_rel)
        for k in range(s.modes):
            assert rel_l2(got[k], ref[k]) <= REL_L2, (s.n, k, rel_l2(got[k], ref[k]))


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
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    psi, obj, pos, pin = dev(psi0), dev(o0), dev(bad), dev(p0)
    pout = torch.empty_like(pin)
    rc = lib.dm_probe_update_static(psi.data_ptr(), obj.data_ptr(), pos.data_ptr(), pin.data_ptr(), pout.data_ptr(),
                                    32, 2, s.views, 50, 50, 1e-6, None)
    assert rc == dm.DM_EINVAL and "outside" in dm.dm_last_error(None)
