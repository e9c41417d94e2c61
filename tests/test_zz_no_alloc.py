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

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
        a = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        b = torch.from_numpy((rng.standard_normal(n) * 0.3).astype(np.float32)).cuda()
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        fwi.fwi_misfit(a, b, n, ref)
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = f(a.data_ptr(), b.data_ptr(), n, out.data_ptr(), stream)
        assert rc == 0, fwi.fwi_last_error()
        torch.cuda.synchronize()
        r, o = ref.item(), out.item()
        # same terms, different FP64 summation order: |error| <= n eps sum|terms|
        assert abs(o - r) <= n * 2.0 ** -52 * r, (o, r)


def test_noalloc_misfit_rejects_sizes_beyond_its_array():
    fwi, f = _entry()
    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = 4096 * 65536 + 1
    rc = f(a.data_ptr(), a.data_ptr(), too_many, out.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == fwi.FWI_ERR_ARG
    assert "exceeds the maximum" in fwi.fwi_last_error()
