"""The integer facts the split-precision (Ozaki-scheme) kernels rest on,
checked from their definitions on the CPU (no kernel code is imported):

- balanced base-128 digits of a 7S-bit integer taken without a carry chain
  (through X + 64 (1 + 128 + ... + 128^(S-2))) equal the sequential ones and
  reconstruct X, with |d_1| <= 128 and |d_s| <= 64;
- a masked digit under the exponent field of 2^(23 - p) becomes u - 64 with one
  float32 subtraction;
- x 2^(7S - e) + 1.5 2^52 in one FP64 rounding is the integer nearest to
  x 2^(7S - e) (ties to even) in the low mantissa bits;
- with digits so bounded, every diagonal accumulator of a 256-deep K chunk
  stays within 2^24 (exact in FP32), and the int64 combination of eight chunks
  stays below 2^61.1;
- float32 integers below 2^22 convert exactly by adding and subtracting
  1.5 2^23, and two adjacent diagonals then combine in 32 bits.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest


def _seq_digits(X, S):
    d = [0] * S
    for s in range(S - 1, 0, -1):
        dd = ((X + 64) & 127) - 64
        d[s] = dd
        X = (X - dd) >> 7
    d[0] = X
    return d


def _carry_free_digits(X, S):
    C = sum(64 * 128 ** k for k in range(S - 1))
    Y = X + C
    return [Y >> (7 * (S - 1))] + [((Y >> (7 * (S - 1 - s))) & 127) - 64 for s in range(1, S)]


@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_carry_free_digits(S):
    rng = np.random.default_rng(S)
    lim = 1 << (7 * S)
    xs = [0, 1, -1, lim, -lim, lim - 1, -lim + 1, 64, -64, 63, -65] + [int(v) for v in rng.integers(-lim, lim + 1, 20000)]
    for X in xs:
        d = _carry_free_digits(X, S)
        assert d == _seq_digits(X, S)
        assert sum(v * 128 ** (S - 1 - s) for s, v in enumerate(d)) == X
        assert abs(d[0]) <= 128 and all(-64 <= v <= 63 for v in d[1:])


def test_float_add_digit():
    for p in (0, 7, 14):
        for u in range(128):
            for noise in (0, 0x5A5A5A5A):
                w = (u << p) | (noise & ~(127 << p) & 0xFFFFFFFF)
                bits = ((150 - p) << 23) | (w & (127 << p))
                f = np.frombuffer(np.uint32(bits).tobytes(), dtype=np.float32)[0]
                assert f - np.float32(2.0 ** (23 - p) + 64) == np.float32(u - 64)


@pytest.mark.parametrize("S", [2, 4, 6])
def test_fma_fixed_point_rounds_to_nearest_even(S):
    rng = np.random.default_rng(10 + S)
    magic = 1.5 * 2.0 ** 52
    mbits = struct.unpack("<q", struct.pack("<d", magic))[0]
    for _ in range(5000):
        e = int(rng.integers(-40, 40))
        # values on a grid fine enough to hit exact ties now and then
        x = float(rng.integers(-(1 << 50), 1 << 50)) * 2.0 ** (e - 50)
        if abs(x) >= 2.0 ** e:
            continue
        t = x * 2.0 ** (7 * S - e) + magic  # exact product, one rounding
        X = struct.unpack("<q", struct.pack("<d", t))[0] - mbits
        q = Fraction(x) * Fraction(2) ** (7 * S - e)
        fl = q.numerator // q.denominator
        r = q - fl
        want = fl + (1 if r > Fraction(1, 2) or (r == Fraction(1, 2) and fl % 2) else 0)
        assert X == want and abs(X) <= 2 ** (7 * S)


@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_accumulator_bounds(S):
    """Diagonal D = s + t <= S + 1 sums, per k, two real products per slice
    pair (complex: Ar Br - Ai Bi); with |a_1|, |b_1| <= 128 and the other
    digits <= 64 in magnitude, 256 values of k stay within 2^24."""
    bound = [128] + [64] * (S - 1)
    chunk = 0
    for D in range(2, S + 2):
        per_k = sum(2 * bound[s - 1] * bound[D - s - 1] for s in range(1, D) if 1 <= D - s <= S)
        assert 256 * per_k <= 2 ** 24
        chunk += 256 * per_k * 2 ** (7 * (S + 1 - D))
    # int64 combination sum_D acc_D 2^(7 (S + 1 - D)): below 2^58.1 per chunk
    # for S = 6, and eight chunks (one int64 partial sum) below 2^61.1 < 2^63
    assert chunk < 2 ** (7 * S + 16.1)  # 2^58.1 for S = 6
    assert 8 * chunk < 2 ** (7 * S + 19.1) <= 2 ** 61.1 < 2 ** 63


def test_fast_conversion_and_pairing():
    rng = np.random.default_rng(7)
    v = np.concatenate([rng.integers(-(1 << 22) + 1, 1 << 22, 100000), [-(1 << 22) + 1, (1 << 22) - 1, 0]])
    f = v.astype(np.float32)
    assert np.array_equal(f.astype(np.int64), v)  # exact in float32
    t = (f + np.float32(12582912.0)).view(np.int32).astype(np.int64) - 0x4B400000
    assert np.array_equal(t, v)
    a, b = v[:50000], v[50000:100000]
    assert np.max(np.abs(a * 128 + b)) < 2 ** 30
