"""Write ``mp_f64_tables.h``: the constant tables of the FP64 kernels'
table-driven log1p and expm1.

Each entry is a correctly rounded value of a mathematical constant,
evaluated here with Python's ``decimal`` module at 90 significant digits
(its ln, exp and power are correctly rounded at that precision) and then
rounded exactly to the binary format:

* logarithm table, 257 buckets of the reduced argument m in [1/sqrt2, sqrt2);
  a bucket is one value of (exponent, top 8 fraction bits) of the double m,
  c its midpoint; R = 1/c rounded to 8 significant bits (nearest, ties to
  even), Lh = -ln R rounded to the nearest multiple of 2^-32, Ll = -ln R - Lh
  rounded to the nearest double.  With 8-bit R, m * R - 1 is a multiple of
  2^-60 below 2^-7 in magnitude, so one fused multiply-add gives it exactly;
  with Lh and e * ln2_hi both multiples of 2^-32, their sum is exact.
* exponential table, j = 0..255: Th = 2^(j/256) and Tl = 2^(j/256) - Th,
  each rounded to the nearest double.
* the logarithm's rows for e = -2..3, per bucket: e ln2_hi + Lh (exact:
  both are multiples of 2^-32), e ln2_lo + Ll rounded to the nearest
  double (what fma(e, ln2_lo, Ll) gives), with ln2_hi and ln2_lo the two
  doubles the kernels use, and R' = R 2^-e and R' - 1 (both exact: R has 8
  significant bits), so that r = (1 + x) R' - 1 = x R' + (R' - 1) is one
  fma on x itself.
* for k = 256 m + j with m = -2..1: A = e^(k c) and B = e^(k c) - 1,
  each rounded to the nearest double, c the double ln2_hi / 256; with
  r = w - k c (exact) and em = e^r - 1, e^w - 1 = A em + B to one
  rounding (the low part of k ln2/256 is in the table).

Run: python gen_f64_tables.py   (rewrites the header next to this file)
"""
import decimal
import os
import struct
from decimal import Decimal
from fractions import Fraction

KEY0 = (1022 << 8) + 106
N_LOG = 257
N_EXP = 256
E0, N_E = -2, 6                       # exponent rows of the log table's e terms
M0, N_M = -2, 4                       # exponent rows of the exp table's 2^m Th - 1
LN2_HI = 6.93147180369123816490e-01   # the kernels' split of ln 2
LN2_LO = 1.90821492927058770002e-10


def _round_to(x: Fraction, unit: Fraction) -> Fraction:
    q = x / unit
    n = q.numerator // q.denominator
    rem = q - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return n * unit


def _sig8(x: Fraction) -> Fraction:
    e = 0
    while Fraction(2) ** (e + 1) <= x:
        e += 1
    while Fraction(2) ** e > x:
        e -= 1
    return _round_to(x, Fraction(2) ** (e - 7))


def _hex(v: float) -> str:
    return "0x%016xULL" % struct.unpack("<Q", struct.pack("<d", v))[0]


def tables():
    ctx = decimal.Context(prec=90)
    logs = []
    for i in range(N_LOG):
        key = KEY0 + i
        e, k = key >> 8, key & 255
        c = Fraction(2) ** (e - 1023) * Fraction(512 + 2 * k + 1, 512)
        R = _sig8(1 / c)
        lnR = ctx.ln(ctx.divide(Decimal(R.numerator), Decimal(R.denominator)))
        L = -Fraction(lnR)
        Lh = _round_to(L, Fraction(1, 2 ** 32))
        logs.append((float(R), float(Lh), float(L - Lh)))
    exps = []
    for j in range(N_EXP):
        T = Fraction(ctx.power(Decimal(2), ctx.divide(Decimal(j), Decimal(N_EXP))))
        Th = float(T)
        exps.append((Th, float(T - Fraction(Th))))
    return logs, exps


def e_terms(logs):
    """(e ln2_hi + Lh, e ln2_lo + Ll rounded, R 2^-e, R 2^-e - 1) for
    e = E0 .. E0 + N_E - 1, per bucket."""
    rows = []
    for e in range(E0, E0 + N_E):
        for R, Lh, Ll in logs:
            hi = e * Fraction(LN2_HI) + Fraction(Lh)
            Rp = Fraction(R) / Fraction(2) ** e
            for v in (hi, Rp, Rp - 1):
                assert Fraction(float(v)) == v
            rows.append((float(hi), float(e * Fraction(LN2_LO) + Fraction(Ll)), float(Rp), float(Rp - 1)))
    return rows


def ab_terms():
    """(RN(e^(k c)), RN(e^(k c) - 1)) for k = 256 M0 .. 256 (M0 + N_M) - 1,
    c = ln2_hi / 256."""
    ctx = decimal.Context(prec=90)
    c = ctx.divide(Decimal(LN2_HI), Decimal(256))    # exact: Decimal(float) is the binary value
    rows = []
    for k in range(N_EXP * M0, N_EXP * (M0 + N_M)):
        T = Fraction(ctx.exp(ctx.multiply(Decimal(k), c)))
        rows.append((float(T), float(T - 1)))
    return rows


def render() -> str:
    logs, exps = tables()
    out = ["// mp_f64_tables.h - constant tables of the FP64 log1p and expm1 (bit",
           "// patterns of IEEE doubles), written by gen_f64_tables.py; the definitions",
           "// are in that script's docstring.",
           "#pragma once", "",
           "namespace mp {", "",
           f"constexpr int F64_LOG_KEY0 = {KEY0};", f"constexpr int F64_LOG_N = {N_LOG};",
           f"constexpr int F64_EXP_N = {N_EXP};", "",
           "// per bucket: R, Lh, Ll, 0 (32 bytes)",
           "static __device__ __align__(16) const unsigned long long f64_log_tab[F64_LOG_N * 4] = {"]
    for R, Lh, Ll in logs:
        out.append(f"    {_hex(R)}, {_hex(Lh)}, {_hex(Ll)}, 0x0ULL,")
    out += ["};", "", "// per j: Th, Tl (16 bytes)",
            "static __device__ __align__(16) const unsigned long long f64_exp_tab[F64_EXP_N * 2] = {"]
    for Th, Tl in exps:
        out.append(f"    {_hex(Th)}, {_hex(Tl)},")
    out += ["};", "", f"constexpr int F64_LOG_E0 = {E0};", f"constexpr int F64_LOG_NE = {N_E};",
            "// per exponent e (rows E0 ..) and bucket: e ln2_hi + Lh, RN(e ln2_lo + Ll), R 2^-e,",
            "// R 2^-e - 1 (32 bytes)",
            "static __device__ __align__(16) const unsigned long long f64_log_e_tab[F64_LOG_NE * F64_LOG_N * 4] = {"]
    for hi, lo, Rp, Rm in e_terms(logs):
        out.append(f"    {_hex(hi)}, {_hex(lo)}, {_hex(Rp)}, {_hex(Rm)},")
    out += ["};", "", f"constexpr int F64_EXP_M0 = {M0};", f"constexpr int F64_EXP_NM = {N_M};",
            "// per exponent m (rows M0 ..) and j, k = 256 m + j: RN(e^(k c)), RN(e^(k c) - 1),",
            "// c = ln2_hi / 256 (16 bytes)",
            "static __device__ __align__(16) const unsigned long long f64_exp_ab_tab[F64_EXP_NM * F64_EXP_N * 2] = {"]
    for A, B in ab_terms():
        out.append(f"    {_hex(A)}, {_hex(B)},")
    out += ["};", "", "}  // namespace mp", ""]
    return "\n".join(out)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mp_f64_tables.h")
    with open(path, "w") as f:
        f.write(render())
    print(path)
