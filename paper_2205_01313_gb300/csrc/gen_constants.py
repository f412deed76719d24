"""Print the float32 constants that cupso_device.cuh hard-codes.

Run by hand when the polynomial degrees change; the output is pasted into
cupso_device.cuh. Everything is computed with exact rationals (pi from
Machin's formula to 80 digits) and rounded once to the nearest float32:
  cos(2 pi a) = sum_j (-1)^j (2 pi)^(2j) / (2j)!  a^(2j),  j = 0..7
  exp(r)      = sum_k r^k / k!,                           k = 0..8
  log2(e); ln 2 = LN2_HI + LN2_LO with LN2_HI cut to 16 significant bits.
"""
from decimal import Decimal, getcontext
from fractions import Fraction
import math
import struct

getcontext().prec = 90


def _arctan_inv(n):
    x = Decimal(1) / n
    x2 = x * x
    term, total, k = x, x, 1
    while True:
        term *= -x2
        k += 2
        d = term / k
        if abs(d) < Decimal(10) ** -88:
            return total
        total += d


PI = Fraction(16 * _arctan_inv(5) - 4 * _arctan_inv(239))


def _ln2():
    # ln 2 = sum_{k>=1} 1 / (k 2^k)
    total, k = Fraction(0), 1
    while k < 300:
        total += Fraction(1, k * 2 ** k)
        k += 1
    return total


def round_f32(q: Fraction) -> float:
    """Nearest float32 (ties to even) of a rational in the normal range."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = math.floor(math.log2(q.numerator) - math.log2(q.denominator))
    while Fraction(2) ** e > q:
        e -= 1
    while Fraction(2) ** (e + 1) <= q:
        e += 1
    scaled = q / Fraction(2) ** (e - 23)          # in [2^23, 2^24)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return sign * m * 2.0 ** (e - 23)


def hexf(x: float) -> str:
    return float(struct.unpack("f", struct.pack("f", x))[0]).hex()


def main():
    two_pi_sq = (2 * PI) ** 2
    for j in range(8):
        c = Fraction((-1) ** j) * two_pi_sq ** j / math.factorial(2 * j)
        print("cos c%d = %sf" % (j, hexf(round_f32(c))))
    for k in range(9):
        print("exp c%d = %sf" % (k, hexf(round_f32(Fraction(1, math.factorial(k))))))
    ln2 = _ln2()
    print("log2e  = %sf" % hexf(round_f32(1 / ln2)))
    hi = Fraction(math.floor(ln2 * 2 ** 16), 2 ** 16)
    print("ln2_hi = %sf" % hexf(round_f32(hi)))
    print("ln2_lo = %sf" % hexf(round_f32(ln2 - hi)))


if __name__ == "__main__":
    main()
