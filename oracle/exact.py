"""Exact dyadic arithmetic on multi-component numbers (test infrastructure).

A multi-component number is the exact sum of its components (Sec. 1: DD,
TD, QD are 2, 3, 4 binary64 words; TS is 3 binary32 words).  Every finite
binary floating-point number is a dyadic rational N * 2^e, so every value
here is kept exactly as a pair (N, e) of Python integers.

Nothing in this module rounds except the functions whose name says so
(``round_f64``, ``round_f32``, ``to_components``) and the float conversions
used for error *metrics*.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

#: exponent recorded for an all-zero row/column (no digit is non-zero)
EXP_ZERO = -(2 ** 31)


# ---------------------------------------------------------------------------
# dyadic helpers
# ---------------------------------------------------------------------------
def decode(x: float):
    """x = N * 2^e exactly (N signed, at most 53 bits); (0, 0) for zero."""
    x = float(x)
    if x == 0.0:
        return 0, 0
    if not math.isfinite(x):
        raise ValueError("non-finite component")
    m, e = math.frexp(x)          # x = m * 2^e, 0.5 <= |m| < 1
    return int(m * (1 << 53)), e - 53


def add(a, b):
    """Exact sum of two dyadics."""
    (na, ea), (nb, eb) = a, b
    if na == 0:
        return b
    if nb == 0:
        return a
    e = min(ea, eb)
    return (na << (ea - e)) + (nb << (eb - e)), e


def neg(a):
    return -a[0], a[1]


def mul(a, b):
    return a[0] * b[0], a[1] + b[1]


def to_fraction(a) -> Fraction:
    n, e = a
    return Fraction(n) * (Fraction(2) ** e)


def from_fraction(f: Fraction):
    """Exact dyadic of a Fraction whose denominator is a power of two."""
    if f == 0:
        return 0, 0
    d = f.denominator
    assert d & (d - 1) == 0, "not dyadic"
    return f.numerator, -(d.bit_length() - 1)


def elem_value(comps):
    """Exact value of one multi-component number (sum of its components)."""
    acc = (0, 0)
    for c in comps:
        acc = add(acc, decode(c))
    return acc


def cmp_abs(a, b):
    """Sign of |a| - |b| (exact)."""
    d = add((abs(a[0]), a[1]), (-abs(b[0]), b[1]))
    return (d[0] > 0) - (d[0] < 0)


def exponent(a):
    """E(x) = floor(log2|x|) + 1: the unique integer with 2^(E-1) <= |x| < 2^E.

    This is the per-element form of the shift constant of Algorithm 1 (the
    tau vectors, Sec. 3): a power of two bounding the magnitude.  Zero gives
    EXP_ZERO.
    """
    n, e = a
    if n == 0:
        return EXP_ZERO
    return abs(n).bit_length() + e


def to_float(a) -> float:
    """Nearest double (for error metrics only)."""
    n, e = a
    if n == 0:
        return 0.0
    return float(Fraction(n) * (Fraction(2) ** e))


# ---------------------------------------------------------------------------
# rounding to binary64 / binary32 and to canonical components
# ---------------------------------------------------------------------------
def round_f64(a) -> float:
    """RN64 (ties to even) of an exact dyadic; CPython's int/int division is
    correctly rounded, including the subnormal range."""
    return to_float(a)


def round_f32(a) -> float:
    """RN32 (ties to even) of an exact dyadic, returned as a Python float."""
    n, e = a
    if n == 0:
        return 0.0
    s = -1 if n < 0 else 1
    m = abs(n)
    top = m.bit_length() - 1 + e            # 2^top <= |x| < 2^(top+1)
    lsb = max(top - 23, -149)               # binary32: 24 bits, subnormal LSB 2^-149
    sh = lsb - e
    if sh <= 0:
        q = m << (-sh)
    else:
        q = m >> sh
        rem = m - (q << sh)
        half = 1 << (sh - 1)
        if rem > half or (rem == half and (q & 1)):
            q += 1
    if q * 2.0 ** lsb >= 2.0 ** 128:
        raise OverflowError("binary32 overflow")
    return s * math.ldexp(float(q), lsb)


def to_components(a, q: int, kind: str = "f64"):
    """Canonical q-component expansion: c_0 = RN(x), c_t = RN(x - c_0 - ... - c_{t-1})."""
    rnd = round_f64 if kind == "f64" else round_f32
    out = []
    r = a
    for _ in range(q):
        c = rnd(r)
        out.append(c)
        r = add(r, neg(decode(c)))
    return out


# ---------------------------------------------------------------------------
# exact products (tiny brute force) and error metrics
# ---------------------------------------------------------------------------
def matrix_values(comps):
    """Exact values of a multi-component matrix given as component arrays."""
    r, c = comps[0].shape
    return [[elem_value([x[i, j] for x in comps]) for j in range(c)] for i in range(r)]


def exact_product_fraction(A, B, i, j) -> Fraction:
    """Brute force C*_ij = sum_p (sum_c a^(c)_ip)(sum_c b^(c)_pj) in Fractions."""
    k = A[0].shape[1]
    s = Fraction(0)
    for p in range(k):
        a = sum((Fraction(float(x[i, p])) for x in A), Fraction(0))
        b = sum((Fraction(float(y[p, j])) for y in B), Fraction(0))
        s += a * b
    return s


def comps_value(cs):
    acc = (0, 0)
    for c in cs:
        acc = add(acc, decode(c))
    return acc


def _dyadic_sqrt_ratio(num, den) -> float:
    """sqrt(num / den) of two non-negative dyadics, as a double, without
    overflow or underflow on the way (only the result is rounded)."""
    (nn, en), (nd, ed) = num, den
    if nn == 0:
        return 0.0
    # num / den = mm * 2^ee with mm in (1/2, 2)
    t = nn.bit_length() - nd.bit_length()
    mm = Fraction(nn, nd << t) if t >= 0 else Fraction(nn << -t, nd)
    ee = en - ed + t
    if ee % 2:
        mm *= 2
        ee -= 1
    return math.ldexp(math.sqrt(float(mm)), ee // 2)


def _dyadic_ratio(num, den) -> float:
    """|num| / |den| of two dyadics (den non-zero) as a double."""
    (nn, en), (nd, ed) = num, den
    if nn == 0:
        return 0.0
    nn, nd = abs(nn), abs(nd)
    t = nn.bit_length() - nd.bit_length()
    mm = Fraction(nn, nd << t) if t >= 0 else Fraction(nn << -t, nd)
    return math.ldexp(float(mm), en - ed + t)


def error_metrics(chat, cstar):
    """Errors of computed multi-component entries against exact ones.

    chat: nested list [i][j] -> list of components; cstar: nested list of
    exact dyadics.  Returns dict with
      err_nw   = ||Chat - C*||_F / ||C*||_F        (normwise relative)
      err_max  = max_ij |Chat_ij - C*_ij| / |C*_ij|  (the paper's metric,
                 Sec. 1: the largest relative error over all elements; an
                 error on an exact zero counts as infinite)
    Both sums of squares are exact dyadics; only the final ratios are
    rounded, so errors far below the binary64 range of a square (relative
    2^-600 and less, as with 12 or more components) are still measured.
    """
    num = (0, 0)
    den = (0, 0)
    emax = 0.0
    for row_h, row_s in zip(chat, cstar):
        for ch, cs in zip(row_h, row_s):
            d = add(comps_value(ch), neg(cs))
            num = add(num, mul(d, d))
            den = add(den, mul(cs, cs))
            if cs[0] != 0:
                emax = max(emax, _dyadic_ratio(d, cs))
            elif d[0] != 0:
                emax = math.inf
    if den[0] == 0:
        err_nw = 0.0 if num[0] == 0 else math.inf
    else:
        err_nw = _dyadic_sqrt_ratio(num, den)
    return {"err_nw": err_nw, "err_max": emax}


def nonoverlapping(cs, kind: str = "f64") -> bool:
    """|c_{t+1}| <= ulp(c_t)/2 for consecutive non-zero components (zeros
    allowed only at the tail)."""
    p = 52 if kind == "f64" else 23
    seen_zero = False
    for a, b in zip(cs, cs[1:]):
        if a == 0.0:
            seen_zero = True
        if seen_zero and b != 0.0:
            return False
        if a == 0.0:
            continue
        _, e = math.frexp(a)                 # |a| in [2^(e-1), 2^e)
        half_ulp = 2.0 ** (e - 1 - p - 1)
        if abs(b) > half_ulp:
            return False
    return True


def as_array(vals, dtype=object):
    return np.array(vals, dtype=dtype)
