"""Pins of the oracle's checkpoint codec: IEEE half conversion against numpy's (a library
RNE conversion), bfloat16 against brute-force nearest-even search, and the scale against
its defining property (the largest power of two with max * s <= T)."""
import numpy as np
import pytest

import oracle


def _edge_floats():
    vals = [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 7e4, 2.0 ** -14, 2.0 ** -24,
            2.0 ** -25, 2.0 ** -25 * 1.0000001, 3 * 2.0 ** -26, 2.0 ** -14 * (1 - 2 ** -11),
            1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 3.0e38,
            np.inf, -np.inf, 1e-40, 6.1e-5, 5.96e-8]
    return np.array(vals, dtype=np.float32)


def test_f16_conversion_matches_numpy():
    rng = np.random.default_rng(0)
    x = np.concatenate([
        _edge_floats(),
        (rng.standard_normal(20000) * 10.0 ** rng.uniform(-9, 5, 20000)).astype(np.float32),
        rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32).view(np.float32),
    ])
    x = x[np.isfinite(x) | np.isinf(x)]
    got = oracle.f32_to_f16(x)
    want = x.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, want)


def _bf16_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_bf16_conversion_is_nearest_even():
    rng = np.random.default_rng(1)
    x = np.concatenate([
        _edge_floats()[np.isfinite(_edge_floats())],
        (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32),
        ((rng.integers(0, 2 ** 16, 5000, dtype=np.uint32) << 16) | 0x8000).view(np.float32),
    ])
    x = x[np.isfinite(x) & (np.abs(x) < 3.3e38)]
    b = oracle.f32_to_bf16(x)
    xd = x.astype(np.float64)
    r = _bf16_to_f64(b)
    # neighbouring codes (bit patterns +-1); a neighbour that is a NaN pattern is no
    # candidate
    eu = np.nan_to_num(np.abs(_bf16_to_f64(b + np.uint16(1)) - xd), nan=np.inf)
    ed = np.nan_to_num(np.abs(_bf16_to_f64(b - np.uint16(1)) - xd), nan=np.inf)
    err = np.abs(r - xd)
    assert np.all(err <= eu) and np.all(err <= ed)
    ties = (err == eu) | (err == ed)
    ties &= err > 0
    assert np.all((b[ties] & 1) == 0)


@pytest.mark.parametrize("dtype,T", [("fp16", 2.0 ** 14), ("bf16", 1.0)])
def test_snapshot_scale_is_largest_power_of_two(dtype, T):
    rng = np.random.default_rng(2)
    for m in np.concatenate([10.0 ** rng.uniform(-12, 6, 500), [1.0, 2.0 ** -20, 2.0 ** 14]]):
        m = float(np.float32(m))
        s = oracle.snap_scale(m, dtype)
        assert np.log2(s) == np.round(np.log2(s))
        assert m * s <= T < 2.0 * m * s
    assert oracle.snap_scale(0.0, dtype) == 1.0
    assert np.isnan(oracle.snap_scale(np.inf, dtype))


@pytest.mark.parametrize("dtype,rel", [("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_snapshot_roundtrip_error_bound(dtype, rel):
    """a comes back to the format's relative precision; the difference a - b (the part of
    the state that drives the time stepping) comes back to its own relative precision,
    although it is ten times smaller than a."""
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(5000) * 3e-5).astype(np.float32)
    b = (a - rng.standard_normal(5000) * 3e-6).astype(np.float32)
    code, s = oracle.snap_encode(a, b, dtype)
    ra, rb = oracle.snap_decode(code, s, dtype)
    d, rd = (a - b).astype(np.float64), (ra - rb).astype(np.float64)
    T = 2.0 ** 14 if dtype == "fp16" else 1.0
    # relative error of a normal number, plus the absolute floor of the format's subnormals
    fa = (2.0 ** -24 if dtype == "fp16" else 0.0) / s[0]
    fd = (2.0 ** -24 if dtype == "fp16" else 0.0) / s[1]
    assert np.all(np.abs(ra - a) <= rel * np.abs(a) + fa)
    # the decoded difference is (a' - (a' - d')) in FP32: one extra rounding of size |a| eps
    assert np.all(np.abs(rd - d) <= rel * np.abs(d) + fd + 2.0 ** -23 * np.abs(a) * 2)
    assert np.abs(a).max() * s[0] <= T and np.abs(d).max() * s[1] <= T
    assert s[1] >= 8 * s[0]   # the difference gets a finer scale
