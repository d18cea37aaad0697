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


class _DeviceMemory:
    """Device-wide free memory and the default stream-ordered pool's
    high-water mark, read through the CUDA driver API (the pool is a driver
    object shared by every runtime in the process)."""
    USED_MEM_HIGH = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def free_bytes(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return free.value

    def pool_high(self):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value

    def reset_pool_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


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


@pytest.mark.parametrize("variant", [camp.VARIANT_MIXED, camp.VARIANT_FP64])
def test_calls_allocate_no_device_memory(cuda, variant):
    """After the first call on a device (which may load kernels and look up
    the array's address), further calls change neither the device's free
    memory nor the default memory pool's high-water mark."""
    import torch
    wl = w.workload(3)
    gm = camp.Mechanism(wl.json())
    y0, env = w.cells(wl.mech, 800, seed=503)
    y = y0.copy()
    rc, _ = _static_call(gm, y, env, wl.dt, wl.rtol, wl.atol, variant)
    assert rc == 0, camp.lib().camp_last_error()
    torch.cuda.synchronize()
    mem = _DeviceMemory(torch.cuda.current_device())
    free0 = mem.free_bytes()
    torch_reserved0 = torch.cuda.memory_reserved()
    mem.reset_pool_high()
    high0 = mem.pool_high()
    for _ in range(3):
        y = y0.copy()
        rc, status = _static_call(gm, y, env, wl.dt, wl.rtol, wl.atol, variant)
        assert rc == 0 and (status == 0).all()
        assert mem.free_bytes() == free0
        assert mem.pool_high() == high0
        assert torch.cuda.memory_reserved() == torch_reserved0


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
