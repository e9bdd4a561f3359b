"""The floating-point facts the panel-block inverses rest on, checked on the
CPU from their definitions (no kernel code is imported):

- the complex reciprocal (x - iy) / (x^2 + y^2), with x and y first scaled by
  the power of two 2^-e (e the exponent of max(|x|, |y|), capped at 1022) and
  one correctly rounded reciprocal of the sum of squares, is within a few
  ulp of 1 / z over the whole double range where 1 / z is finite and normal;
- the pivot search's magnitude |Re| + |Im| (compared in FP32) picks an entry
  whose modulus is at least 1 / sqrt(2) of the largest, up to FP32 rounding,
  so the partial pivoting keeps its growth bound up to that factor.
"""
import struct

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")


def _hi(x):
    return struct.unpack("<q", struct.pack("<d", x))[0] >> 32


def _from_hi(h):
    return struct.unpack("<d", struct.pack("<q", (h & 0xFFFFFFFF) << 32))[0]


def _scaled_reciprocal(x, y):
    m = max(abs(x), abs(y))
    e = min(((_hi(m) >> 20) & 0x7FF) - 1023, 1022)
    sc = _from_hi((1023 - e) << 20)
    xs, ys = x * sc, y * sc
    # [1, 2) after the exact scaling ([2, 4) when the cap applies; a subnormal m lands below 1)
    assert 1.0 <= max(abs(xs), abs(ys)) < (4.0 if e == 1022 else 2.0) or m < 2.0 ** -1022
    r = 1.0 / (xs * xs + ys * ys)  # one correctly rounded reciprocal
    return xs * r * sc, -(ys * r) * sc


def test_scaled_complex_reciprocal_accuracy():
    mpmath.mp.prec = 200
    rng = np.random.default_rng(5)
    cases = [(3.0, 4.0), (-7.25, 1e-3), (1e154, 1e-154), (1e-300, -3e-300), (8.9e307, -1e307), (1.0, 0.0),
             (0.0, -2.0), (1.7e308, 1.7e308)]
    for _ in range(20000):
        ex = int(rng.integers(-300, 300))
        cases.append((rng.standard_normal() * 10.0 ** ex, rng.standard_normal() * 10.0 ** (ex + int(rng.integers(-8, 9)))))
    worst = 0.0
    for x, y in cases:
        ref = 1 / mpmath.mpc(x, y)
        if not (1e-300 < abs(ref) < 1e300):
            continue
        gx, gy = _scaled_reciprocal(x, y)
        worst = max(worst, float(abs(mpmath.mpc(gx, gy) - ref) / abs(ref)))
    assert worst < 4 * 2.0 ** -52, worst


def test_l1_pivot_choice_is_within_sqrt2_of_the_largest_modulus():
    rng = np.random.default_rng(6)
    for _ in range(2000):
        n = int(rng.integers(1, 65))
        scale = 10.0 ** rng.uniform(-30, 30, n)
        col = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * scale
        mag = np.abs(col.real).astype(np.float32) + np.abs(col.imag).astype(np.float32)
        best = int(np.argmax(mag))  # ties: the lowest index, as in the kernels
        assert np.abs(col[best]) >= np.max(np.abs(col)) / np.sqrt(2.0) * (1 - 1e-6)
