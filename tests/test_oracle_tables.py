"""Pins of the table-driven log1p and expm1 (the oracle's, and the constant
tables the FP64 kernels carry), from outside both:

* every table entry equals the correctly rounded value of its definition,
  evaluated here with mpmath at 300 bits (the oracle's generator uses exact
  integer arithmetic, the device generator Python's decimal module);
* the logarithm's reduction r = m R - 1 is exactly representable in every
  bucket (so one fma gives it exactly) and stays below the bound the series
  is sized for; e ln2_hi + Lh is exact for every exponent;
* the exponential's reduction, with k rounded in FP32 from the truncated
  argument, keeps |r| below the bound its series is sized for;
* the oracle's log1p and expm1 stay within 1 and 2 ulp of the correctly
  rounded result (mpmath) for arguments in every bucket and every j;
* the mirror quotient's reciprocal is correctly rounded on a sample and
  the quotient within one ulp of the IEEE one.
"""
import math
import os
import re
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

mpmath = pytest.importorskip("mpmath")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEY0 = (1022 << 8) + 106
LN2_HI = 6.93147180369123816490e-01
LN2_LO = 1.90821492927058770002e-10


def _d(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


N_EXP = 256                  # entries 2^(j/256) of the exponential table


N_E = 6                      # device log rows, e = -2 .. 3
E0 = -2
N_M = 4                      # reconstruction rows (A, B), m = -2 .. 1 (k = -512 .. 511)
M0 = -2
DEV_EXTRA = 4 * N_E * 257 + 2 * N_M * N_EXP
ORC_EXTRA = 2 * N_M * N_EXP


def _words(path):
    return [int(x, 16) for x in re.findall(r"0x([0-9a-f]{16})ULL", open(path).read())]


def _read(path, per_log, extra=0):
    words = _words(path)
    n_log = 257 * per_log
    log = [tuple(_d(w) for w in words[i:i + 3]) for i in range(0, n_log, per_log)]
    exp = [(_d(words[n_log + 2 * j]), _d(words[n_log + 2 * j + 1])) for j in range(N_EXP)]
    assert len(words) == n_log + 2 * N_EXP + extra
    return log, exp


def _tables():
    oracle = _read(os.path.join(ROOT, "oracle", "orc_tables.h"), 3, extra=ORC_EXTRA)
    # the device header pads each bucket with a literal 0x0ULL (not matched)
    device = _read(os.path.join(ROOT, "paper_2302_13590_gb300", "csrc", "mp_f64_tables.h"), 3, extra=DEV_EXTRA)
    return {"oracle": oracle, "device": device}


def _bucket_c(i):
    key = KEY0 + i
    e, k = key >> 8, key & 255
    return Fraction(2) ** (e - 1023) * Fraction(512 + 2 * k + 1, 512)


def _rn8(x):
    e = math.floor(math.log2(x))
    unit = Fraction(2) ** (e - 7)
    q = x / unit
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2):
        n += 1
    return n * unit


def _expected():
    mpmath.mp.prec = 300
    log = []
    for i in range(257):
        R = _rn8(1 / _bucket_c(i))
        L = -mpmath.log(mpmath.mpf(R.numerator) / R.denominator)
        Lh = mpmath.nint(L * 2 ** 32) / 2 ** 32
        log.append((float(R), float(Lh), float(L - Lh)))
    exp = []
    for j in range(N_EXP):
        T = mpmath.power(2, mpmath.mpf(j) / N_EXP)
        Th = float(T)
        exp.append((Th, float(T - Th)))
    return log, exp


@pytest.fixture(scope="module")
def expected():
    return _expected()


@pytest.mark.parametrize("which", ["oracle", "device"])
def test_tables_are_correctly_rounded(which, expected):
    log, exp = _tables()[which]
    assert log == expected[0]
    assert exp == expected[1]
    # the bucket of 1 (from either side) needs no table correction
    assert log[150][0] == 1.0 and log[149][0] == 1.0 and log[150][1] == 0.0


def test_log_reduction_exact_in_every_bucket():
    log, _ = _tables()["oracle"]
    rng = np.random.default_rng(3)
    for i, (R, Lh, _) in enumerate(log):
        key = KEY0 + i
        lo = _d(key << 44)
        hi = _d(((key + 1) << 44) - 1)
        lo, hi = max(lo, 1 / math.sqrt(2)), min(hi, math.nextafter(math.sqrt(2), 0))
        ms = [lo, hi] + list(rng.uniform(lo, hi, 20))
        for m in ms:
            r = Fraction(m) * Fraction(R) - 1
            assert Fraction(float(r)) == r, (i, m)            # one fma is exact
            assert abs(r) < Fraction(3, 500), (i, m)          # |r| < 0.006
        assert (Fraction(Lh) * 2 ** 32).denominator == 1
    assert (Fraction(LN2_HI) * 2 ** 32).denominator == 1
    for e in (-1075, -1022, -1, 1, 1023, 1024):
        s = Fraction(e) * Fraction(LN2_HI) + Fraction(log[0][1])
        assert Fraction(float(s)) == s


def _f32_trunc(x):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    s = (b >> 63) << 31
    e = ((b >> 52) & 0x7ff) - 1023
    if e < -126:
        f = s
    elif e > 127:
        f = s | 0x7f800000
    else:
        f = s | ((e + 127) << 23) | ((b >> 29) & 0x7fffff)
    return np.frombuffer(struct.pack("<I", f), np.float32)[0]


def test_exp_reduction_bound():
    mpmath.mp.prec = 200
    ln2_n = mpmath.log(2) / N_EXP
    rng = np.random.default_rng(4)
    edges = [(k + 0.5) * math.log(2) / N_EXP for k in range(-295464, 295464, 7817)]
    ws = list(rng.uniform(-800, 800, 3000)) + edges + [math.nextafter(x, 0) for x in edges] + [800.0, -800.0]
    worst = 0.0
    c32 = np.float32(float.fromhex("0x1.715476p+8"))     # 256/ln2 rounded to FP32
    assert c32 == np.float32(N_EXP / math.log(2))
    for w in ws:
        y = np.float32(_f32_trunc(w)) * c32
        sh = np.float32(y) + np.float32(12582912.0)
        k = int(np.frombuffer(np.float32(sh).tobytes(), np.uint32)[0]) - 0x4B400000
        worst = max(worst, abs(float(mpmath.mpf(w) - k * ln2_n)))
    assert worst < 0.0016


def _ulps(a, ref):
    return abs(a - ref) / np.spacing(abs(ref)) if ref != 0 else abs(a)


def test_log1p_within_one_ulp_in_every_bucket():
    mpmath.mp.prec = 200
    rng = np.random.default_rng(5)
    worst = 0.0
    for i in range(257):
        key = KEY0 + i
        lo = max(_d(key << 44), 1 / math.sqrt(2))
        hi = min(_d(((key + 1) << 44) - 1), math.nextafter(math.sqrt(2), 0))
        for m in (lo, hi, float(rng.uniform(lo, hi))):
            for e in (-40, -2, 0, 1, 30):
                x = math.ldexp(m, e) - 1.0
                if x <= -1.0 or x == 0.0:
                    continue
                ref = float(mpmath.log1p(mpmath.mpf(x)))
                worst = max(worst, _ulps(O.log1p(x), ref))
    for x in list(rng.uniform(-1e-6, 1e-6, 200)) + list(-np.exp(-rng.uniform(30, 36, 50))):
        worst = max(worst, _ulps(O.log1p(x), float(mpmath.log1p(mpmath.mpf(x)))))
    # arguments whose 1 + x is inexact (the rounding of the sum must not
    # enter), in every bucket and every exponent row of the table and
    # either side of it
    for i in range(257):
        key = KEY0 + i
        lo = max(_d(key << 44), 1 / math.sqrt(2))
        hi = min(_d(((key + 1) << 44) - 1), math.nextafter(math.sqrt(2), 0))
        for e in (-2, -1, 0, 1, 2, 3):
            u = math.ldexp(float(rng.uniform(lo, hi)), e)
            x = (u - 1.0) + float(rng.uniform(-0.5, 0.5)) * math.ulp(u)
            if x > -1.0:
                worst = max(worst, _ulps(O.log1p(x), float(mpmath.log1p(mpmath.mpf(x)))))
    # around -1/2, near -1, large arguments and the edges of the table rows
    for x in (-0.5, math.nextafter(-0.5, -1.0), math.nextafter(-0.5, 0.0), math.nextafter(-1.0, 0.0),
              -1.0 + 2.0 ** -40, 2.0 ** 24, 2.0 ** 24 + 1.0, 2.0 ** 128, 1e300, 5e-324, -5e-324,
              4 * math.sqrt(2) - 1, math.nextafter(4 * math.sqrt(2) - 1, 0.0), 1 / (2 * math.sqrt(2)) - 1):
        worst = max(worst, _ulps(O.log1p(x), float(mpmath.log1p(mpmath.mpf(x)))))
    assert worst <= 1.0
    assert O.log1p(math.inf) == math.inf and O.log1p(-1.0) == -math.inf and math.isnan(O.log1p(-2.0))


def test_expm1_within_two_ulp_for_every_j():
    mpmath.mp.prec = 200
    rng = np.random.default_rng(6)
    worst = 0.0
    h = math.log(2) / N_EXP
    for m in (-1100, -40, -2, -1, 0, 1, 3, 20, 1000, 1022):
        for j in range(N_EXP):
            c = (N_EXP * m + j) * h
            for d in (0.0, 0.49 * h, -0.49 * h, float(rng.uniform(-0.5, 0.5)) * h):
                w = c + d
                if w == 0.0 or w > 709.7:
                    continue
                worst = max(worst, _ulps(O.expm1(w), float(mpmath.expm1(mpmath.mpf(w)))))
    assert worst <= 2.0
    # 2^m beyond the double range: the product is formed in two steps
    for w in (709.5, 709.78, 709.782):
        assert O.expm1(w) == float(mpmath.expm1(mpmath.mpf(w)))
    assert O.expm1(709.8) == math.inf and O.expm1(1e300) == math.inf and O.expm1(-1e300) == -1.0


def test_reciprocal_correctly_rounded():
    """With d = 1 the mirror quotient is its refined reciprocal alone:
    y0 + y0 (e + e^2) rounded once, within 2^-67 of 1 / v before that
    rounding, so it is the correctly rounded 1 / v except within 2^-15 ulp
    of a rounding midpoint (none in this sample); a step without the e^2
    term (2^-46 off) or with a wrong sign fails at once."""
    rng = np.random.default_rng(4)
    n = 20000
    v = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-120, 121, n)) * rng.choice([-1.0, 1.0], n)
    y = np.array([O.div(1.0, float(b)) for b in v])
    assert np.array_equal(y, 1.0 / v)


def test_quotient_within_one_ulp():
    """The mirror quotient d / v (the single-precision IEEE reciprocal of the
    truncated v, one third-order step, one product) is within one ulp of the
    correctly rounded quotient over the range of v it serves, exact where
    1 / v is a power of two, and outside that range (|v| < 2^-120 or
    >= 2^121, zero, infinity, NaN) it is the IEEE division."""
    rng = np.random.default_rng(3)
    n = 20000
    v = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-120, 121, n)) * rng.choice([-1.0, 1.0], n)
    d = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-60, 60, n)) * rng.choice([-1.0, 1.0], n)
    v[:200] = np.ldexp(1.0, rng.integers(-120, 121, 200)) * rng.choice([-1.0, 1.0], 200)
    worst = 0.0
    exact = 0
    for a, b in zip(d, v):
        q, ref = O.div(a, b), a / b
        worst = max(worst, abs(q - ref) / np.spacing(abs(ref)))
        exact += q == ref
    assert worst <= 1.0
    assert exact >= 0.7 * n          # measured: 73 %
    assert all(O.div(a, b) == a / b for a, b in zip(d[:200], v[:200]))
    with np.errstate(all="ignore"):
        for b in [2.0 ** -121, -(2.0 ** -121) * 1.5, 2.0 ** 121, -(2.0 ** 125), 5e-324, 0.0, -0.0, math.inf,
                  -math.inf, math.nan]:
            for a in [1.7, -3.25, 0.0]:
                q, ref = O.div(a, b), float(np.float64(a) / np.float64(b))
                assert (q == ref and math.copysign(1, q) == math.copysign(1, ref)) or (math.isnan(q) and math.isnan(ref))
    # signed zeros as the division gives them
    assert math.copysign(1, O.div(0.0, -3.0)) == -1 and math.copysign(1, O.div(-0.0, -3.0)) == 1


def test_log_e_terms_table():
    """The device's rows of the logarithm for e = -2 .. 3: e ln2_hi + Lh
    exactly and e ln2_lo + Ll rounded to the nearest double (which is what
    fma(e, ln2_lo, Ll) gives, so the table and the fmas are interchangeable
    bit for bit), and R' = R 2^-e and R' - 1 exactly, so that
    fma(x, R', R' - 1) is (1 + x) R' - 1 to one rounding."""
    path = os.path.join(ROOT, "paper_2302_13590_gb300", "csrc", "mp_f64_tables.h")
    words = _words(path)
    log, _ = _read(path, 3, extra=DEV_EXTRA)
    base = 257 * 3 + 2 * N_EXP
    for r in range(N_E):
        e = r + E0
        for i, (R, Lh, Ll) in enumerate(log):
            hi, lo, Rp, Rm = (_d(w) for w in words[base + 4 * (r * 257 + i):base + 4 * (r * 257 + i) + 4])
            assert Fraction(hi) == e * Fraction(LN2_HI) + Fraction(Lh)
            assert lo == float(e * Fraction(LN2_LO) + Fraction(Ll))
            assert lo == math.fma(float(e), LN2_LO, Ll) if hasattr(math, "fma") else True
            assert Fraction(Rp) == Fraction(R) / 2 ** e and Fraction(Rm) == Fraction(R) / 2 ** e - 1


def test_exp_reconstruction_table():
    """The exponential's fused reconstruction for m = -2 .. 1 (k = 256 m + j):
    A = e^(k c) and B = e^(k c) - 1 correctly rounded (mpmath at 300 bits),
    c the double ln2_hi / 256, the same words in the oracle's table and the
    device's; A is 2^(k/256) up to the low part of k ln2/256 (below 4e-10
    relative)."""
    mpmath.mp.prec = 300
    dev = _words(os.path.join(ROOT, "paper_2302_13590_gb300", "csrc", "mp_f64_tables.h"))
    orc = _words(os.path.join(ROOT, "oracle", "orc_tables.h"))
    _, exp = _read(os.path.join(ROOT, "oracle", "orc_tables.h"), 3, extra=ORC_EXTRA)
    dbase = 257 * 3 + 2 * N_EXP + 4 * N_E * 257
    obase = 257 * 3 + 2 * N_EXP
    for r in range(N_M):
        m = r + M0
        for j, (Th, Tl) in enumerate(exp):
            n = 2 * (r * N_EXP + j)
            A, B = _d(dev[dbase + n]), _d(dev[dbase + n + 1])
            assert (dev[dbase + n], dev[dbase + n + 1]) == (orc[obase + n], orc[obase + n + 1])
            x = (N_EXP * m + j) * mpmath.mpf(LN2_HI) / 256
            assert A == float(mpmath.exp(x)) and B == float(mpmath.exp(x) - 1)
            # e^(-k ln2_lo/256) - 1 for |k| <= 512
            assert abs(A / math.ldexp(Th, m) - 1) < 512 * LN2_LO / 256 * 1.01
