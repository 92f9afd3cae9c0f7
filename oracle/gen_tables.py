"""Write ``oracle/orc_tables.h``: the constant tables of the oracle's
table-driven log1p and expm1 (test infrastructure, like the rest of
``oracle/``).

Every entry is a correctly rounded value of a plain mathematical quantity,
computed here in exact integer fixed-point arithmetic (2^-256 units):

* logarithm table, 257 buckets of the reduced argument m in [1/sqrt2, sqrt2):
  the bucket of m is the top 8 fraction bits of its double representation
  together with its exponent; c is the bucket's midpoint;
  R = 1/c rounded to 8 significant bits (nearest, ties to even);
  Lh = -ln R rounded to the nearest multiple of 2^-32; Ll = -ln R - Lh
  rounded to the nearest double.
* exponential table, j = 0..255: Th = 2^(j/256) rounded to the nearest
  double, Tl = 2^(j/256) - Th rounded to the nearest double.
* for k = 256 m + j with m = -2 .. 1 (k = -512 .. 511): A = e^(k c) and
  B = e^(k c) - 1, each rounded to the nearest double, where c is the
  double ln2_hi / 256 (ln2_hi = 0x3fe62e42fee00000, a multiple of 2^-32).
  With r = w - k c (exact) and em = e^r - 1, e^w - 1 = e^(k c) (1 + em) - 1
  = A em + B to one rounding: the low part of k ln2/256 is in the table,
  not in the reduction.

ln is evaluated as 2 atanh((a - b) / (a + b)) for R = a / b by its odd
series; 2^(j/256) as the integer 256th root of 2^(j + 256 P); e^(k c) by
its Taylor series (|k c| < 0.7), with a bound on the truncation that the
rounding to a double is checked against.

Run: python oracle/gen_tables.py   (rewrites the header next to this file)
"""
import math
import os
import struct
from fractions import Fraction

P = 256                      # fixed-point fraction bits
KEY0 = (1022 << 8) + 106     # first bucket: exponent of 0.5, fraction bits 106/256
N_LOG = 257
N_EXP = 256
M0, N_M = -2, 4             # exponent rows of the reconstruction table


def rn53(num: int, scale: int) -> float:
    """num * 2^-scale rounded to the nearest double (ties to even)."""
    if num == 0:
        return 0.0
    neg = num < 0
    a = -num if neg else num
    shift = a.bit_length() - 53
    if shift > 0:
        q, r = divmod(a, 1 << shift)
        half = 1 << (shift - 1)
        if r > half or (r == half and q & 1):
            q += 1
        a, e = q, shift - scale
    else:
        a, e = a, -scale
    v = math.ldexp(a, e)
    return -v if neg else v


def rn_bits(x: Fraction, bits: int) -> Fraction:
    """x > 0 rounded to `bits` significant bits (nearest, ties to even)."""
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    unit = Fraction(2) ** (e - bits + 1)
    q = x / unit
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n & 1):
        n += 1
    return n * unit


def ln_fixed(x: Fraction) -> int:
    """ln(x) * 2^P for a positive rational x near 1 (|x - 1| < 1/2)."""
    a, b = x.numerator, x.denominator
    neg = a < b
    y = (abs(a - b) << P) // (a + b)          # |(x - 1) / (x + 1)|, truncated
    y2 = (y * y) >> P
    term, s, n = y, 0, 0
    while term:
        s += term // (2 * n + 1)
        term = (term * y2) >> P
        n += 1
    return -2 * s if neg else 2 * s


def iroot(v: int, n: int) -> int:
    """floor(v^(1/n)) for v > 0."""
    x = 1 << ((v.bit_length() + n - 1) // n)
    while True:
        y = ((n - 1) * x + v // x ** (n - 1)) // n
        if y >= x:
            break
        x = y
    while x ** n > v:
        x -= 1
    while (x + 1) ** n <= v:
        x += 1
    return x


def bits_of(v: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", v))[0]


def log_table():
    rows = []
    for i in range(N_LOG):
        key = KEY0 + i
        ex, k = key >> 8, key & 255
        c = Fraction(2) ** (ex - 1023) * (1 + Fraction(2 * k + 1, 512))
        R = rn_bits(1 / c, 8)
        L = -ln_fixed(R)                          # -ln R in 2^-P units
        unit = 1 << (P - 32)
        q, r = divmod(L, unit)
        if 2 * r > unit or (2 * r == unit and q & 1):
            q += 1
        Lh = q * unit
        rows.append((float(R), rn53(Lh, P), rn53(L - Lh, P)))
    return rows


def exp_table():
    rows = []
    for j in range(N_EXP):
        T = iroot(1 << (j + N_EXP * P), N_EXP)    # floor(2^(j/256) 2^P)
        Th = rn53(T, P)
        Tl = rn53(T - int(Fraction(Th) * (1 << P)), P)
        rows.append((Th, Tl))
    return rows


LN2_HI = 0x3fe62e42fee00000      # bit pattern of the double ln2_hi


def exp_fixed(x: Fraction):
    """Bounds (lo, hi) on e^x 2^P for |x| < 1, lo <= e^x 2^P <= hi."""
    X = x * (1 << P)
    assert X.denominator == 1                  # x is a multiple of 2^-P
    X = X.numerator
    if X == 0:
        return 1 << P, 1 << P
    s, term, n = 1 << P, 1 << P, 0
    while term:
        n += 1
        term = (term * X >> P) // n if X >= 0 else -((term * -X >> P) // n)
        s += term
    return s - 2 * n - 2, s + 2 * n + 2        # each term truncated by < 1 + its carry


def rn53_checked(lo: int, hi: int, scale: int) -> float:
    a, b = rn53(lo, scale), rn53(hi, scale)
    assert a == b, "bounds round apart"
    return a


def exp_ab_table():
    lh = struct.unpack("<d", struct.pack("<Q", LN2_HI))[0]
    c = Fraction(lh) / 256                     # a multiple of 2^-40
    rows = []
    for k in range(N_EXP * M0, N_EXP * (M0 + N_M)):
        lo, hi = exp_fixed(k * c)
        one = 1 << P
        rows.append((rn53_checked(lo, hi, P), rn53_checked(lo - one, hi - one, P)))
    return rows


def render() -> str:
    out = ["/* orc_tables.h - constant tables of the oracle's log1p and expm1, written by",
           " * oracle/gen_tables.py (exact integer arithmetic; see there for the",
           " * definitions).  Bit patterns of IEEE doubles. */",
           "#pragma once", "#include <stdint.h>", "",
           f"#define ORC_LOG_KEY0 {KEY0}", f"#define ORC_LOG_N {N_LOG}", f"#define ORC_EXP_N {N_EXP}",
           f"#define ORC_EXP_M0 ({M0})", f"#define ORC_EXP_NM {N_M}", "",
           "/* per bucket: R, Lh, Ll */",
           "static const uint64_t orc_log_tab[ORC_LOG_N][3] = {"]
    for R, Lh, Ll in log_table():
        out.append(f"    {{0x{bits_of(R):016x}ULL, 0x{bits_of(Lh):016x}ULL, 0x{bits_of(Ll):016x}ULL}},")
    out += ["};", "", "/* per j: Th, Tl */", "static const uint64_t orc_exp_tab[ORC_EXP_N][2] = {"]
    for Th, Tl in exp_table():
        out.append(f"    {{0x{bits_of(Th):016x}ULL, 0x{bits_of(Tl):016x}ULL}},")
    out += ["};", "", "/* per m = -2 .. 1 and j (k = 256 m + j): A = RN(e^(k c)), B = RN(e^(k c) - 1),",
            " * c = ln2_hi / 256 */",
            "static const uint64_t orc_exp_ab[ORC_EXP_NM][ORC_EXP_N][2] = {"]
    for r, (A, B) in enumerate(exp_ab_table()):
        if r % N_EXP == 0:
            out.append("  {")
        out.append(f"    {{0x{bits_of(A):016x}ULL, 0x{bits_of(B):016x}ULL}},")
        if r % N_EXP == N_EXP - 1:
            out.append("  },")
    out += ["};", ""]
    return "\n".join(out)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "orc_tables.h")
    with open(path, "w") as f:
        f.write(render())
    print(path)
