"""Build step: write the Payne-Hanek tables of the CUDA library.

Section 5.8 and Appendix A (the Payne-Hanek table-generation figure) define the
FP64 table: for E = 0..1023 and M = (E > 700 ? -128 : 0),
    m = frac(2/pi * 2^(E-53)) * 2^-(E-53+M),
and four times t = RN_double(m) with the lowest bit cleared, tab[4E+i] = t,
m -= t.  Alongside it goes the parity bit of I(E) = floor(2/pi * 2^(E-53)):
the table drops M*I(E)/2 turns, a half turn when the mantissa M and I(E)
are odd, which a full-turn (sin/cos) reduction has to put back.

The FP32 table has the same definition with 24-bit words over E = 0..127:
M = (E > 64 ? -64 : 0), m = frac(2/pi * 2^(E-24)) * 2^-(E-24+M), four
RN-float words with the lowest bit cleared (the 2^64 scaling keeps the last
word a normal float).

pi comes from the Chudnovsky series in Python integers; every rounding is
done by Python's correctly rounded Fraction -> float conversion.
"""
import math
import struct
import sys
from fractions import Fraction

BITS = 1900


def pi_fixed(bits):
    """floor(pi * 2^bits) by the Chudnovsky series (binary splitting)."""
    guard = bits + 64
    C = 640320
    C3_24 = C ** 3 // 24

    def bs(a, b):
        if b - a == 1:
            if a == 0:
                Pab = Qab = 1
            else:
                Pab = (6 * a - 5) * (2 * a - 1) * (6 * a - 1)
                Qab = a * a * a * C3_24
            Tab = Pab * (13591409 + 545140134 * a)
            if a & 1:
                Tab = -Tab
            return Pab, Qab, Tab
        m = (a + b) // 2
        P1, Q1, T1 = bs(a, m)
        P2, Q2, T2 = bs(m, b)
        return P1 * P2, Q1 * Q2, Q2 * T1 + P1 * T2

    terms = guard // 47 + 2
    _, Q, T = bs(0, terms)
    sqrt_c = math.isqrt(10005 << (2 * guard))
    pi = (Q * 426880 * sqrt_c) // T
    return pi >> 64


def two_over_pi_fixed(bits):
    """floor(2/pi * 2^bits)"""
    p = pi_fixed(bits + 8)
    return (1 << (2 * bits + 9)) // p


def _clear_lsb_d(t):
    b = struct.unpack("<Q", struct.pack("<d", t))[0] & ~1
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _round_f(fr):
    """correctly rounded float32 of a Fraction (via exact double first only
    when that is exact; otherwise by integer rounding)."""
    if fr == 0:
        return 0.0
    neg = fr < 0
    a = -fr if neg else fr
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulpe = max(e - 23, -149)
    scaled = a / Fraction(2) ** ulpe
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and (m & 1)):
        m += 1
    v = math.ldexp(m, ulpe)
    return -v if neg else v


def _clear_lsb_f(t):
    b = struct.unpack("<I", struct.pack("<f", t))[0] & ~1
    return struct.unpack("<f", struct.pack("<I", b))[0]


def tables():
    y = two_over_pi_fixed(BITS)              # 2/pi = y / 2^BITS
    tab64, ib64 = [], []
    for E in range(1024):
        sh = E - 53
        M = -128 if E > 700 else 0
        v = Fraction(y * 2 ** sh, 2 ** BITS) if sh >= 0 else Fraction(y, 2 ** (BITS - sh))
        ip = v.numerator // v.denominator
        ib64.append(ip & 1)
        m = (v - ip) * Fraction(2) ** (-(E - 53 + M))
        for _ in range(4):
            t = _clear_lsb_d(float(m))
            tab64.append(t)
            m -= Fraction(t)
    tab32, ib32 = [], []
    for E in range(128):
        sh = E - 24
        M = -64 if E > 64 else 0
        v = Fraction(y * 2 ** sh, 2 ** BITS) if sh >= 0 else Fraction(y, 2 ** (BITS - sh))
        ip = v.numerator // v.denominator
        ib32.append(ip & 1)
        m = (v - ip) * Fraction(2) ** (-(E - 24 + M))
        for _ in range(4):
            t = _clear_lsb_f(_round_f(m))
            tab32.append(t)
            m -= Fraction(t)
    return tab64, ib64, tab32, ib32


def words(bits):
    return [sum(bits[32 * w + k] << k for k in range(32)) for w in range(len(bits) // 32)]


def main(out):
    tab64, ib64, tab32, ib32 = tables()
    with open(out, "w") as f:
        f.write("// generated by gen_phtab.py: Payne-Hanek tables (Section 5.8)\n#pragma once\n")
        f.write("static __device__ __align__(32) const double k_phtab64[4096] = {\n")
        for i in range(0, 4096, 4):
            f.write("  " + ", ".join(float(t).hex() for t in tab64[i:i + 4]) + ",\n")
        f.write("};\nstatic __device__ const unsigned k_phbit64[32] = {\n")
        f.write("  " + ", ".join(f"0x{w:08x}u" for w in words(ib64)) + "};\n")
        f.write("static __device__ __align__(16) const float k_phtab32[512] = {\n")
        for i in range(0, 512, 4):
            f.write("  " + ", ".join(float(t).hex() + "f" for t in tab32[i:i + 4]) + ",\n")
        f.write("};\nstatic __device__ const unsigned k_phbit32[4] = {\n")
        f.write("  " + ", ".join(f"0x{w:08x}u" for w in words(ib32)) + "};\n")


if __name__ == "__main__":
    main(sys.argv[1])
