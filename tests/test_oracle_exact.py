"""Pins for oracle/exact.py, oracle/_clib (mp512.c) and oracle/eft.py.

Everything is checked against exact rational arithmetic (fractions), closed
forms of floating-point rounding, or constructed tie cases -- never against
a retyped copy of the code under test.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import _clib, eft
from oracle import exact as X
from ozmp_inputs import gen_problem


def _rand_double(rng, lo=-60, hi=60):
    return math.ldexp(rng.uniform(0.5, 1.0) * rng.choice([-1, 1]), rng.randint(lo, hi))


ADVERSARIAL = [0.0, 1.0, -1.0, 2.0 ** -1074, -(2.0 ** -1074), 2.0 ** -1022, 1.7976931348623157e308,
               2.0 ** -300, -(2.0 ** -300), 1.0 - 2.0 ** -53, 3.0, 0.1, -0.1, 2.0 ** 600]


def test_decode_and_value_exact():
    rng = random.Random(1)
    vals = ADVERSARIAL + [_rand_double(rng, -1070, 1000) for _ in range(300)]
    for x in vals:
        n, e = X.decode(x)
        assert X.to_fraction((n, e)) == Fraction(x)
        assert abs(n) < 2 ** 53
    for _ in range(300):
        cs = [rng.choice(vals) for _ in range(rng.randint(1, 4))]
        assert X.to_fraction(X.elem_value(cs)) == sum((Fraction(c) for c in cs), Fraction(0))


def test_exponent_definition():
    rng = random.Random(2)
    cases = [[1.0], [2.0], [0.75], [1.0, -(2.0 ** -300)], [1.0, 2.0 ** -300], [-4.0, 1.0],
             [2.0 ** -1074], [1.0, -1.0, 2.0 ** -200], [3.0, -1.0]]
    cases += [[_rand_double(rng, -100, 100) for _ in range(rng.randint(1, 4))] for _ in range(500)]
    for cs in cases:
        v = X.elem_value(cs)
        f = abs(X.to_fraction(v))
        E = X.exponent(v)
        if f == 0:
            assert E == X.EXP_ZERO
            continue
        assert Fraction(2) ** (E - 1) <= f < Fraction(2) ** E
    # closed forms
    assert X.exponent(X.elem_value([1.0])) == 1
    assert X.exponent(X.elem_value([1.0, -(2.0 ** -300)])) == 0
    assert X.exponent(X.elem_value([0.0, 0.0])) == X.EXP_ZERO


def test_round_f64_f32_against_numpy_and_ties():
    rng = random.Random(3)
    for _ in range(2000):
        x = _rand_double(rng, -160, 120)
        # a double input is rounded once by numpy's float32 conversion
        assert X.round_f32(X.decode(x)) == float(np.float32(x))
        assert X.round_f64(X.decode(x)) == x
    # ties to even in binary32: 1 + 2^-24 is a tie between 1 and 1 + 2^-23
    assert X.round_f32((2 ** 24 + 1, -24)) == 1.0
    assert X.round_f32((2 ** 24 + 3, -24)) == 1.0 + 2.0 ** -22
    # binary64 tie and subnormal rounding
    assert X.round_f64((2 ** 53 + 1, -53)) == 1.0
    assert X.round_f64((3, -1076)) == 2.0 ** -1074          # 0.75 ulp -> 1 ulp
    assert X.round_f64((1, -1075)) == 0.0                   # half of the least subnormal, tie to 0


def test_to_components_canonical():
    rng = random.Random(4)
    for _ in range(300):
        cs = [_rand_double(rng, -20, 20) for _ in range(4)]
        v = X.elem_value(cs)
        for q, kind in [(2, "f64"), (3, "f64"), (4, "f64"), (3, "f32")]:
            out = X.to_components(v, q, kind)
            assert X.nonoverlapping(out, kind)
            resid = abs(X.to_fraction(v) - sum(Fraction(c) for c in out))
            if out[-1] != 0:
                _, e = math.frexp(out[-1])
                p = 53 if kind == "f64" else 24
                assert resid <= Fraction(2) ** (e - p - 1)
    # an exactly representable DD is reproduced
    assert X.to_components(X.elem_value([1.0, 2.0 ** -60]), 2) == [1.0, 2.0 ** -60]


@pytest.mark.parametrize("prec", ["dd", "td", "qd", "ts"])
def test_exact_block_matches_fraction_bruteforce(prec):
    A, B = gen_problem(prec, 5, 4, 7, phi=1.0, seed=11)
    got = _clib.exact_block(A, B, range(5), range(4))
    for i in range(5):
        for j in range(4):
            ex = X.exact_product_fraction(A, B, i, j)
            g = X.to_fraction(got[i][j])
            # exact when it fits 512 bits; always within half an ulp of 512 bits
            assert abs(g - ex) <= abs(ex) * Fraction(1, 2 ** 511)


def test_exact_block_adversarial_ranges():
    # subnormal x subnormal, huge x huge, total cancellation, sign mixing
    A = [np.array([[2.0 ** -1074, 1e300, 1.0, -1.0]]), np.array([[0.0, 1e284, -(2.0 ** -60), 2.0 ** -60]])]
    B = [np.array([[2.0 ** -1074], [1e-300], [1.0], [1.0]]), np.array([[0.0], [0.0], [0.0], [2.0 ** -80]])]
    got = _clib.exact_block(A, B, [0], [0])[0][0]
    ex = X.exact_product_fraction(A, B, 0, 0)
    assert abs(X.to_fraction(got) - ex) <= abs(ex) * Fraction(1, 2 ** 511)


def test_512bit_rounding_ties_to_even():
    # exact sums 2^600 + 2^88 (tie, even -> down) and 2^600 + 2^89 + 2^88
    # (tie, odd -> up): the 512-bit significand of 2^600 has its LSB at 2^89.
    A = [np.array([[2.0 ** 300, 2.0 ** 44, 0.0]])]
    B = [np.array([[2.0 ** 300], [2.0 ** 44], [0.0]])]
    r = _clib.exact_block(A, B, [0], [0])[0][0]
    assert X.to_fraction(r) == Fraction(2) ** 600
    A = [np.array([[2.0 ** 300, 2.0 ** 44, 2.0 ** 45]])]
    B = [np.array([[2.0 ** 300], [2.0 ** 44], [2.0 ** 44]])]
    r = _clib.exact_block(A, B, [0], [0])[0][0]
    assert X.to_fraction(r) == Fraction(2) ** 600 + Fraction(2) ** 90
    # just above the tie rounds up regardless of parity
    A = [np.array([[2.0 ** 300, 2.0 ** 44, 2.0 ** -300]])]
    B = [np.array([[2.0 ** 300], [2.0 ** 44], [1.0]])]
    r = _clib.exact_block(A, B, [0], [0])[0][0]
    assert X.to_fraction(r) == Fraction(2) ** 600 + Fraction(2) ** 89


def test_mp512_add_mul_against_fractions():
    rng = random.Random(5)
    xs, ys = [], []
    for _ in range(400):
        xs.append((rng.getrandbits(rng.randint(1, 512)) * rng.choice([-1, 1]), rng.randint(-800, 800)))
        ys.append((rng.getrandbits(rng.randint(1, 512)) * rng.choice([-1, 1]), rng.randint(-800, 800)))
    xs.append((2 ** 511, 0)); ys.append((-(2 ** 511 - 1), 0))        # cancellation
    xs.append((1, 0)); ys.append((2 ** 511, 2000))                    # far apart
    for op, f in [("add", lambda a, b: a + b), ("mul", lambda a, b: a * b)]:
        rs = _clib.mp_binop(op, xs, ys)
        for x, y, r in zip(xs, ys, rs):
            ex = f(X.to_fraction(x), X.to_fraction(y))
            got = X.to_fraction(r)
            assert abs(got - ex) <= abs(ex) * Fraction(1, 2 ** 512)
            assert abs(r[0]) < 2 ** 512


def test_naive512_close_to_exact():
    A, B = gen_problem("qd", 3, 3, 40, phi=1.0, seed=2)
    ex = _clib.exact_block(A, B, range(3), range(3))
    nv = _clib.naive512_block(A, B, range(3), range(3))
    k = 40
    for i in range(3):
        for j in range(3):
            bound = sum(abs(X.to_fraction(X.elem_value([a[i, p] for a in A])) *
                            X.to_fraction(X.elem_value([b[p, j] for b in B]))) for p in range(k))
            d = abs(X.to_fraction(ex[i][j]) - X.to_fraction(nv[i][j]))
            assert d <= 3 * k * bound * Fraction(1, 2 ** 511)


def test_eft_closed_forms():
    rng = random.Random(6)
    pairs = [(1.0, 2.0 ** -53), (1.0, -(2.0 ** -53)), (2.0 ** 100, 1.0), (0.1, 0.2), (1e308, 1e308 * 0.5),
             (3.0, -3.0), (2.0 ** -1074, 2.0 ** -1074)]
    pairs += [(_rand_double(rng), _rand_double(rng)) for _ in range(2000)]
    for a, b in pairs:
        if not math.isfinite(a + b):
            continue
        s, e = eft.two_sum(a, b)
        assert s == a + b and Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)
        if abs(a) >= abs(b):
            s2, e2 = eft.fast_two_sum(a, b)
            assert (s2, e2) == (s, e)
        if abs(a) < 1e150 and abs(b) < 1e150 and (a == 0 or abs(a) > 1e-140) and (b == 0 or abs(b) > 1e-140):
            p, e = eft.two_prod(a, b)
            assert p == a * b and Fraction(p) + Fraction(e) == Fraction(a) * Fraction(b)
