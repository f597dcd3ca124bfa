"""The tile deposit's fixed-point arithmetic, checked on the host with exact rationals.

The deposit sums each node in two int32 words (hi 2^sb + lo, units of 2^-s).  Its
per-tile choice of the split bits sb and the scale s, made from the tile's record
count n and largest |w| with float logarithms, must keep every sum from overflowing:

* n 2^(sb-1) < 2^31 (each |lo| <= 2^(sb-1));
* one stencil weight |V| = |w| W 2^s < 2^(22+sb) (the rounding below needs it);
* sum |V| / 2^sb + n/2 < 2^31 (the hi sums, each hi rounded to nearest).

One weight is split without conversion instructions: t = fma(wxy, wz, K) with
K = 1.5 2^(23+sb) rounds V + K to float (a multiple of 2^sb in K's binade), hi is the
difference of the bit patterns of t and K, lf = fma(wxy, wz, -(t - K)) is the remainder
to one float rounding, and lo = lf rounded to an integer by adding 1.5 2^23.  Here every
float operation is emulated as one correct rounding of the exact rational result, and
hi 2^sb + lo must be V to within 0.5 + 2^(sb-24) units.
"""
import math
import random
import struct
from fractions import Fraction

import numpy as np


def fl32(x: Fraction) -> Fraction:
    """Round an exact rational to the nearest float32 (ties to even); no overflow here."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)
    ulp = Fraction(2) ** (e - 23)
    q = a / ulp
    n = q.numerator // q.denominator
    r = q - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * n * ulp


def bits(x: Fraction) -> int:
    return struct.unpack("<i", struct.pack("<f", float(x)))[0]


def choose(nrec: int, wm: float):
    """The kernel's choice of (sb, s), with float32 logarithms as on the device."""
    ln = float(np.log2(np.float32(nrec)))
    lw = float(np.log2(np.float32(wm)))
    sb = min(22, math.floor(np.float32(31.0) - np.float32(ln)))
    sf = math.floor(min(np.float32(30.0 + sb) - np.float32(ln) - np.float32(lw), np.float32(21.0 + sb) - np.float32(lw)))
    return sb, min(100, sf), sf >= -100


def test_scale_keeps_every_sum_in_range():
    rng = random.Random(5)
    ns = sorted({1, 2, 3, 7, 8, 255, 256, 257, 2999, 3000, 65535, 65536, 65537, 1 << 20, (1 << 20) + 1,
                 1_250_000, (1 << 29) - 1, 1 << 29, (1 << 30) - 1} | {rng.randrange(1, 1 << 30) for _ in range(300)})
    wms = [2.0 ** k for k in range(-60, 61, 7)] + [float(np.nextafter(np.float32(2.0 ** k), np.float32(0)))
                                                  for k in range(-40, 41, 9)] + [rng.uniform(1e-6, 1e6) for _ in range(40)]
    for n in ns:
        for wm in wms:
            wm = float(np.float32(wm))
            sb, s, ok = choose(n, wm)
            assert ok and 0 <= sb <= 22
            two_s = Fraction(2) ** s
            assert n * Fraction(2) ** (sb - 1) < 2 ** 31
            assert Fraction(wm) * two_s < Fraction(2) ** (22 + sb)
            assert n * Fraction(wm) * two_s / Fraction(2) ** sb + Fraction(n, 2) < 2 ** 31


def split(wxy: Fraction, wz: Fraction, sb: int):
    K = Fraction(3, 2) * Fraction(2) ** (23 + sb)
    t = fl32(wxy * wz + K)
    hi = bits(t) - bits(K)
    hf = fl32(t - K)
    lf = fl32(wxy * wz - hf)
    magic = Fraction(3, 2) * Fraction(2) ** 23
    lo = bits(fl32(lf + magic)) - bits(magic)
    return hi, lo


def test_split_reconstructs_each_weight():
    rng = random.Random(11)
    for sb in (1, 5, 10, 16, 19, 22):
        top = 2.0 ** (21 + sb)  # |V| bound the scale guarantees
        cases = [top * 0.999999, -top * 0.999999, 1.0, -1.0, 0.5, 0.49, 2.0 ** -30, 0.0, 2.0 ** sb - 0.5,
                 2.0 ** (sb - 1), 3 * 2.0 ** (sb - 1)]
        cases += [rng.choice((-1, 1)) * top * rng.random() ** 8 for _ in range(300)]
        for v in cases:
            wz = Fraction(float(np.float32(rng.uniform(0.01, 0.75))))   # one stencil weight
            wxy = fl32(Fraction(v) / wz)                                # the float wxy of a product near v
            V = wxy * wz                                                # exact product, as the fma sees it
            if abs(V) >= Fraction(2) ** (22 + sb):
                continue
            hi, lo = split(wxy, wz, sb)
            assert abs(lo) <= 2 ** (sb - 1)
            assert abs(hi * Fraction(2) ** sb + lo - V) <= Fraction(1, 2) + Fraction(2) ** (sb - 24)
