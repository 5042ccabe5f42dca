"""The integer and table arithmetic the kernels rely on, restated in Python
word for word and checked against exact rational arithmetic (CPU): the
balanced base-64 slice digits in offset form (slice_write_kernel), the FP32
level sums read by bit extraction, four levels and three level groups summed
exactly on 32-bit words and converted once with round-to-nearest-even
(f32_exact_int, add96, i96_ldexp of ozaki_tc.cu), the all-levels kernel's
FP32 fast readout of small level sums and its stacked-B MMA schedule, the
Cholesky trailing update's closed-form tile row (chol.cu), and the
table-driven tanh of the feature kernels (tanh_half of features.cu: Tang's
exponential with a Cody-Waite split of ln2/256), whose absolute error must
stay below 2e-16."""
import math
import random
import struct
from fractions import Fraction

import numpy as np
import pytest


def _digits_offset(v, S):
    """a_p of X = v: the base-64 digits of X + 32 (1 + 64 + ... + 64^(S-1)), less 32."""
    off = sum(32 * 64 ** p for p in range(S))
    w = v + off
    out = []
    for p in range(S):
        k = 6 * (S - 1 - p)
        out.append((w >> k) - 32 if p == 0 else ((w >> k) & 63) - 32)
    return out


def test_slice_digits_reproduce_the_fixed_point_value():
    rng = random.Random(1)
    for S in range(1, 11):
        lim = 64 ** S
        cases = [0, 1, -1, lim, -lim, lim - 1, 1 - lim] + [rng.randint(-lim, lim) for _ in range(3000)]
        for v in cases:
            d = _digits_offset(v, S)
            assert sum(a * 64 ** (S - 1 - i) for i, a in enumerate(d)) == v
            assert abs(d[0]) <= 64 and all(-32 <= a <= 31 for a in d[1:])


def _f32_exact_int(f):
    """The FP32 level sum's integer value from its bits (|f| < 2^24)."""
    u = struct.unpack("<I", struct.pack("<f", f))[0]
    e = (u >> 23) & 0xFF
    m = (u & 0x7FFFFF) | 0x800000
    v = m >> min(150 - e, 31)
    return -v if u >> 31 else v


M32 = 0xFFFFFFFF


def _s32(v):
    v &= M32
    return v - (1 << 32) if v >> 31 else v


def _add96(w, x01, x23, q):
    """The epilogue's w += (x01 + 4096 x23) 2^(24 q) on three 32-bit words."""
    w0, w1, w2 = w
    t = (x01 & M32) + (((x23 & M32) << 12) & M32)
    yl, c = t & M32, t >> 32
    yh = (((x01 >> 31) & M32) + ((x23 >> 20) & M32) + c) & M32
    if q == 0:
        u = (yl, yh, (_s32(yh) >> 31) & M32)
    elif q == 1:
        u = ((yl << 24) & M32, ((yl >> 8) | (yh << 24)) & M32, (_s32(yh) >> 8) & M32)
    else:
        u = (0, (yl << 16) & M32, ((yl >> 16) | (yh << 16)) & M32)
    t = w0 + u[0]
    w0, c = t & M32, t >> 32
    t = w1 + u[1] + c
    w1, c = t & M32, t >> 32
    return (w0, w1, (w2 + u[2] + c) & M32)


def _i96_ldexp(w, eoff):
    """The epilogue's correctly rounded X 2^eoff of the 96-bit integer X."""
    w0, w1, w2 = w
    sg = M32 if w2 >> 31 else 0
    t = (w0 ^ sg) + (sg & 1)
    a0, c = t & M32, t >> 32
    t = (w1 ^ sg) + c
    a1, c = t & M32, t >> 32
    a2 = ((w2 ^ sg) + c) & M32
    if a0 | a1 | a2 == 0:
        return 0.0
    clz = lambda v: 32 - v.bit_length()
    n = clz(a2) if a2 else (32 + clz(a1) if a1 else 64 + clz(a0))
    fl = lambda lo, hi, k: ((hi << k) | (lo >> (32 - k))) & M32 if k else hi
    if n >= 64:
        b2, b1, b0 = (a0 << (n - 64)) & M32, 0, 0
    elif n >= 32:
        b2, b1, b0 = fl(a0, a1, n - 32), (a0 << (n - 32)) & M32, 0
    else:
        b2, b1, b0 = fl(a1, a2, n), fl(a0, a1, n), (a0 << n) & M32
    E = 1023 + 95 - n + eoff
    assert 1 <= E <= 2046
    hi = (((E - 1) << 20) + (b2 >> 11)) & M32
    lo = ((b2 << 21) | (b1 >> 11)) & M32
    up = ((b1 >> 10) & 1) and (((b1 & 0x3FF) | b0) or (lo & 1))
    t = lo + (1 if up else 0)
    lo, hi = t & M32, (hi + (t >> 32)) & M32
    return struct.unpack("<d", struct.pack("<Q", ((hi | (sg & 0x80000000)) << 32) | lo))[0]


def test_level_sums_combine_exactly():
    rng = random.Random(2)
    for _ in range(3000):
        S = rng.choice([4, 5, 6, 9, 10])
        nchunk = rng.choice([1, 2, 5])
        w, X = (0, 0, 0), 0
        for q in range((S + 3) // 4):
            for _c in range(nchunk):
                L = [rng.randint(-(2 ** 23) + 1, 2 ** 23 - 1) if rng.random() < 0.9 else 0 for _ in range(4)]
                assert [_f32_exact_int(float(np.float32(x))) for x in L] == L
                x01, x23 = L[0] + 64 * L[1], L[2] + 64 * L[3]
                w = _add96(w, x01, x23, q)
                X += (x01 + 4096 * x23) * 2 ** (24 * q)
        e = rng.randint(-300, 100)
        want = float(Fraction(X) * Fraction(2) ** e) if X else 0.0  # correctly rounded
        assert _i96_ldexp(w, e) == want


def _tanh_half(u, tab):
    """tanh(u / 2) as the feature kernels compute it (FMAs emulated exactly)."""
    def fma(a, b, c):
        return float(Fraction(a) * Fraction(b) + Fraction(c))

    inv_l = float.fromhex("0x1.71547652b82fep+8")
    l_hi = float.fromhex("0x1.62e42fefa4000p-9")
    l_lo = float.fromhex("-0x1.8432a1b0e2634p-51")
    shifter = float.fromhex("0x1.8p52")
    a = min(abs(u), 40.0)
    kt = fma(a, inv_l, shifter)
    k = struct.unpack("<Q", struct.pack("<d", kt))[0] & 0xFFFFFFFF
    kd = kt - shifter
    r = fma(-kd, l_hi, a)
    r = fma(-kd, l_lo, r)
    q = fma(r, 1.0 / 24.0, -1.0 / 6.0)
    q = fma(r, q, 0.5)
    q = fma(r, q, -1.0)
    e = fma(tab[k & 255], r * q, tab[k & 255])
    e = math.ldexp(e, -(k >> 8))
    num, den = 1.0 - e, 1.0 + e
    y = float(np.float32(1.0) / np.float32(den))  # FP32 reciprocal of den
    y = fma(y, fma(-den, y, 1.0), y)
    q0 = num * y
    t = fma(fma(-den, q0, num), y, q0)
    return -t if u < 0 else t


def test_table_driven_tanh_absolute_error():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    tab = [float(mpmath.mpf(2) ** (-mpmath.mpf(j) / 256)) for j in range(256)]
    # the Cody-Waite high part is exact in 39 bits: k * l_hi is exact for k < 2^14
    l_hi = float.fromhex("0x1.62e42fefa4000p-9")
    assert (Fraction(l_hi) * 2 ** 47).denominator == 1
    rng = random.Random(3)
    us = [0.0, 1e-20, 1e-8, 1e-3, 0.5, 1.0, 2.0, 10.0, 37.0, 40.0, 41.0, 1e300]
    us += [rng.uniform(-45, 45) for _ in range(1500)] + [rng.uniform(-1, 1) for _ in range(1500)]
    worst = 0.0
    for u in us:
        ref = mpmath.tanh(mpmath.mpf(u) / 2)
        worst = max(worst, float(abs(mpmath.mpf(_tanh_half(u, tab)) - ref)))
    assert worst < 2e-16, worst


def _f32_magic_int(x):
    """The all-levels epilogue's fast readout of an integer-valued FP32 sum:
    the bits of x + 1.5 2^23 less those of 1.5 2^23."""
    y = np.float32(x) + np.float32(12582912.0)
    return int(np.array(y, dtype=np.float32).view(np.int32)) - 0x4B400000


def test_fp32_fast_integer_readout():
    # exact for every integer below 2^22 in magnitude (the kernel takes this
    # path only when the warp's sums all are); sampled plus the edges
    rng = random.Random(7)
    vals = [0, 1, -1, 2 ** 22 - 1, -(2 ** 22 - 1), 2 ** 21, -(2 ** 21), 12345, -54321]
    vals += [rng.randrange(-(2 ** 22) + 1, 2 ** 22) for _ in range(20000)]
    for v in vals:
        assert float(np.float32(v)) == v
        assert _f32_magic_int(v) == v, v
    # the guard is needed: beyond 2^22 the readout is wrong for some sums
    bad = [v for v in (2 ** 22 + 1, 2 ** 23 - 3, -(2 ** 22) - 5) if _f32_magic_int(v) != v]
    assert bad
    # the guard's threshold: |x| < 2^22 exactly when the FP32 bits of |x| are below those of 2^22
    two22 = int(np.array(np.float32(2.0 ** 22)).view(np.int32))
    assert two22 == 0x4A800000


def test_syrk_tile_row_closed_form():
    """The Cholesky trailing update's tile row from the inverse of the
    triangular count S(b) = b nbt - b (b - 1) / 2 (FP32 root, corrected to
    the integer) equals the linear search for every tile, up to M = 1024."""
    for nbt in list(range(1, 64)) + [100, 128, 200, 250, 256]:
        ntiles = nbt * (nbt + 1) // 2
        for q in range(ntiles):
            bi, rem = 0, q
            while rem >= nbt - bi:
                rem -= nbt - bi
                bi += 1
            tw = 2 * nbt + 1
            root = np.float32(math.sqrt(np.float32(tw * tw - 8 * q)))
            b = int(np.float32(0.5) * (np.float32(tw) - root))
            b = max(0, min(b, nbt - 1))
            while b > 0 and b * nbt - b * (b - 1) // 2 > q:
                b -= 1
            while b + 1 < nbt and (b + 1) * nbt - (b + 1) * b // 2 <= q:
                b += 1
            assert (b, q - (b * nbt - b * (b - 1) // 2)) == (bi, rem), (nbt, q)


@pytest.mark.parametrize("S", range(1, 11))
def test_stacked_b_mma_schedule(S):
    """The all-levels kernel's MMA schedule: per A level p, B levels q0 ..
    q0 + n - 1 (n <= 5) stacked into one MMA of N = 48 n columns written at
    TMEM column 48 (p + q0).  Every pair p + q < S lands once in the
    accumulator of level p + q, N is a valid kind::f16 width for M = 128 (a
    multiple of 16, at most 256) and the S accumulators fit 512 columns; the
    first MMA into each level of a chunk (the one that starts it) is issued
    before any other MMA into that level."""
    BN = 48
    hits = {}
    first_seen = {}
    order = 0
    for kk in range(2):
        for p in range(S):
            q0 = 0
            while q0 < S - p:
                n = min(5, S - p - q0)
                N = BN * n
                assert N % 16 == 0 and 16 <= N <= 256
                col0 = BN * (p + q0)
                assert col0 + N <= BN * S <= 512
                starts = not (kk > 0 or p > 0)  # accumulate flag 0 only for kk = 0, p = 0
                for j in range(n):
                    lvl = (col0 + BN * j) // BN
                    assert lvl == p + q0 + j
                    hits[(kk, p, q0 + j)] = hits.get((kk, p, q0 + j), 0) + 1
                    if lvl not in first_seen:
                        first_seen[lvl] = (order, starts)
                order += 1
                q0 += 5
    for kk in range(2):
        for p in range(S):
            for q in range(S - p):
                assert hits[(kk, p, q)] == 1
    assert len(hits) == 2 * S * (S + 1) // 2
    assert sorted(first_seen) == list(range(S)) and all(st for _, st in first_seen.values())
