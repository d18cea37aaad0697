"""The solve for callers that cannot allocate device memory
(camp_solve_host_static), called through the C ABI.

Such callers -- host models whose device memory belongs to their own pool
allocator or sits under a hard cap, loops that must not stall on the device
synchronisation cudaMalloc/cudaFree can cause, codes that must not meet an
out-of-memory error mid-run -- get the same results as from
camp_solve_host, staged through the library's fixed static device array
instead of buffers the library allocates.  This file is collected last on
purpose; it passes alone in a fresh process and after the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2111_07436_gb300 import camp, workloads as w
from tests import parity

pytestmark = pytest.mark.gpu

STATIC_BYTES = 16 << 20  # CAMP_STATIC_SCRATCH_BYTES


def _static_call(gm, y, env, dt, rtol, atol, variant):
    """camp_solve_host_static on host arrays; y is updated in place."""
    L = camp.lib()
    status = np.full(len(y), -1, dtype=np.int32)
    a = np.array([atol], dtype=np.float64)
    o = gm.opts(variant)
    rc = L.camp_solve_host_static(gm._h, len(y), ctypes.c_void_p(y.ctypes.data),
                                  ctypes.c_void_p(env.ctypes.data), float(dt), float(rtol),
                                  ctypes.c_void_p(a.ctypes.data), 1, ctypes.c_void_p(status.ctypes.data),
                                  ctypes.byref(o), None)
    return rc, status


@pytest.mark.parametrize("k,C", [(2, 3000), (3, 1000), (7, 500)])
@pytest.mark.parametrize("variant", [camp.VARIANT_MIXED, camp.VARIANT_FP64])
def test_matches_the_allocating_entry_point_on_two_calls_in_a_row(cuda, k, C, variant):
    wl = w.workload(k)
    gm = camp.Mechanism(wl.json())
    for seed in (501, 502):  # the second call must not see the first call's leftovers
        y0, env = w.cells(wl.mech, C, seed=seed)
        y_ref = y0.copy()
        s_ref = gm.solve_host(y_ref, env, wl.dt, wl.rtol, wl.atol, variant=variant)
        y_st = y0.copy()
        rc, s_st = _static_call(gm, y_st, env, wl.dt, wl.rtol, wl.atol, variant)
        assert rc == 0, camp.lib().camp_last_error()
        assert np.array_equal(s_st, s_ref)
        assert (s_st == 0).all()
        assert not parity.violations(y_st, y_ref, wl.atol).any()


def test_rejects_a_chunk_larger_than_the_static_array(cuda):
    wl = w.workload(2)
    gm = camp.Mechanism(wl.json())
    C = STATIC_BYTES // ((gm.n + gm.n_env) * 8) + 100  # cannot fit
    y0, env = w.cells(wl.mech, C, seed=7)
    y = y0.copy()
    rc, status = _static_call(gm, y, env, wl.dt, wl.rtol, wl.atol, camp.VARIANT_MIXED)
    assert rc == -1
    assert b"static scratch" in camp.lib().camp_last_error()
    assert np.array_equal(y, y0) and (status == -1).all()  # nothing touched
