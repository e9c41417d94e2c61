"""fwi_misfit_noalloc, the misfit for callers that cannot allocate device memory.

Such callers (a framework that owns all device memory through its own pool, or a
latency-critical loop that must not call the allocator) get the same reduction with its
partial sums kept in a fixed array inside the library.  This file is collected last so a
failure here leaves every other test already run; it passes alone in a fresh process and
after the other tests (the array's address is looked up on the first call per device).
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# CUmemPool_attribute values (cuda.h)
_RESERVED_MEM_CURRENT = 5
_USED_MEM_CURRENT = 7
_USED_MEM_HIGH = 8


def _entry():
    from paper_1912_08063_gb300 import fwi
    f = fwi.lib().fwi_misfit_noalloc          # the C ABI symbol, called directly
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return fwi, f


def test_noalloc_misfit_matches_misfit_on_two_calls_in_a_row():
    fwi, f = _entry()
    rng = np.random.default_rng(77)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on different sizes: the second must not see the first's partials
    for n in (5_000_003, 70_001):
        a_h = rng.standard_normal(n).astype(np.float32)
        b_h = (rng.standard_normal(n) * 0.3).astype(np.float32)
        a, b = torch.from_numpy(a_h).cuda(), torch.from_numpy(b_h).cuda()
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        fwi.fwi_misfit(a, b, n, ref)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = f(a.data_ptr(), b.data_ptr(), n, out.data_ptr(), stream)
        assert rc == 0, fwi.fwi_last_error()
        torch.cuda.synchronize()
        r, o = ref.item(), out.item()
        # same terms, different FP64 summation order: |error| <= n eps sum|terms|
        assert abs(o - r) <= n * 2.0 ** -52 * r, (o, r)
        # and against the FP64 oracle on the FP32 residual the kernel forms (Eq. 1)
        res = (a_h - b_h).astype(np.float64)
        phi = oracle.misfit(res, np.zeros_like(res))
        assert abs(o - phi) <= n * 2.0 ** -52 * phi, (o, phi)


def test_noalloc_misfit_rejects_sizes_beyond_its_array():
    fwi, f = _entry()
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = 4096 * 65536 + 1
    rc = f(a.data_ptr(), a.data_ptr(), too_many, out.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == fwi.FWI_ERR_ARG
    assert "exceeds the maximum" in fwi.fwi_last_error()


class _Pool:
    """The device's default memory pool (the one stream-ordered allocation draws from),
    read through the driver API."""

    def __init__(self, ordinal):
        cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert cu.cuDeviceGet(ctypes.byref(dev), ctypes.c_int(ordinal)) == 0
        self.pool = ctypes.c_void_p(0)
        assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0
        self.cu = cu

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)   # resets the high watermark to the current value
        assert self.cu.cuMemPoolSetAttribute(self.pool, ctypes.c_int(_USED_MEM_HIGH),
                                             ctypes.byref(zero)) == 0


def test_noalloc_misfit_allocates_nothing():
    fwi, f = _entry()
    n = 3_000_017
    rng = np.random.default_rng(78)
    a = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert f(a.data_ptr(), b.data_ptr(), n, out.data_ptr(), stream) == 0   # set-up call
    torch.cuda.synchronize()
    pool = _Pool(torch.cuda.current_device())

    def watch(call):
        torch.cuda.synchronize()
        pool.reset_high()
        used0, res0 = pool.get(_USED_MEM_CURRENT), pool.get(_RESERVED_MEM_CURRENT)
        free0 = torch.cuda.mem_get_info()[0]
        call()
        torch.cuda.synchronize()
        return (pool.get(_USED_MEM_HIGH) - used0, pool.get(_RESERVED_MEM_CURRENT) - res0,
                free0 - torch.cuda.mem_get_info()[0])

    # control: the allocating entry point does raise the pool's high watermark
    ctl = watch(lambda: fwi.fwi_misfit(a, b, n, out))
    assert ctl[0] > 0, ctl
    for _ in range(2):
        d_high, d_res, d_free = watch(
            lambda: f(a.data_ptr(), b.data_ptr(), n, out.data_ptr(), stream))
        assert (d_high, d_res, d_free) == (0, 0, 0)
