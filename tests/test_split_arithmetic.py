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


@pytest.mark.parametrize("S", [2, 3, 4, 5, 6])
def test_biased_word_pairing_and_drain_sum(S):
    """The drain's 32-bit pairing on the biased words: h = bits(a + 1.5 2^23),
    l = bits(b + 1.5 2^23) give a 2^7 + b = 128 h + l - 129 * 0x4B400000
    modulo 2^32 (exact, as |a 2^7 + b| < 2^30); summed with the pairs' powers
    of two (diagonals D and D + 1 at 2^(7 (S - D)), a last odd diagonal alone)
    it equals sum_D acc_D 2^(7 (S + 1 - D)) in int64."""
    rng = np.random.default_rng(20 + S)
    n = 20000
    acc = rng.integers(-(1 << 22) + 1, 1 << 22, size=(S, n))  # acc[D - 2], |v| < 2^22
    acc[:, 0], acc[:, 1], acc[:, 2] = -(1 << 22) + 1, (1 << 22) - 1, 0  # extremes
    acc[::2, 3], acc[1::2, 3] = (1 << 22) - 1, -(1 << 22) + 1
    f = acc.astype(np.float32)
    words = (f + np.float32(12582912.0)).view(np.uint32).astype(np.uint64)
    total = np.zeros(n, dtype=np.int64)
    for D in range(2, S + 2, 2):
        h = words[D - 2]
        if D + 1 <= S + 1:
            l = words[D - 1]
            pr = ((h * 128 + l - 0x4B400000 * 129) % (1 << 32)).astype(np.int64)
            pr = np.where(pr >= 1 << 31, pr - (1 << 32), pr)
            assert np.array_equal(pr, acc[D - 2] * 128 + acc[D - 1])
            total += pr * (1 << (7 * (S - D)))
        else:
            total += (h.astype(np.int64) - 0x4B400000) * (1 << (7 * (S + 1 - D)))
    want = sum(acc[D - 2].astype(object) * (1 << (7 * (S + 1 - D))) for D in range(2, S + 2))
    assert all(int(t) == int(w) for t, w in zip(total, want))
