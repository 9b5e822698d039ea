"""Pins of the exact block LU (oracle/lu_exact.py), the Sec. 4.6 iteration in
rational arithmetic.

* L is unit lower triangular, U upper triangular and L U = A exactly, for
  random dyadic matrices and every iteration width K;
* the factors do not depend on K (LU without pivoting is unique);
* the 2 x 2 closed form: l21 = c / a, u22 = d - b c / a;
* integer factors with unit L are recovered exactly;
* a zero leading pivot, and a singular leading 2 x 2 block, raise.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import lu_exact as LE


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n)) + np.eye(n) * rng.uniform(0.0, 2.0)
    tail = A * 2.0 ** -53 * rng.uniform(-1, 1, size=(n, n))
    return LE.values([np.asfortranarray(A), np.asfortranarray(tail)])


def _matmul(L, U):
    n = len(L)
    return [[sum((L[i][p] * U[p][j] for p in range(n)), Fraction(0)) for j in range(n)] for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_factors_reproduce_A_for_every_width(n):
    A = _rand(n, 10 + n)
    first = None
    for K in sorted({1, 2, 4, n}):
        L, U = LE.lu_blocked(A, K)
        for i in range(n):
            assert L[i][i] == 1
            for j in range(n):
                if j > i:
                    assert L[i][j] == 0
                if j < i:
                    assert U[i][j] == 0
        assert _matmul(L, U) == A
        if first is None:
            first = (L, U)
        else:
            assert (L, U) == first


def test_two_by_two_closed_form():
    a, b, c, d = Fraction(3, 4), Fraction(-5), Fraction(7, 2), Fraction(1, 8)
    L, U = LE.lu_blocked([[a, b], [c, d]], 1)
    assert L == [[1, 0], [c / a, 1]]
    assert U == [[a, b], [0, d - b * c / a]]


def test_integer_factors_recovered():
    n = 12
    rng = np.random.default_rng(4)
    L0 = np.tril(rng.integers(-3, 4, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U0 = np.triu(rng.integers(-3, 4, size=(n, n)), 1) + np.diag(rng.choice([-2, -1, 1, 3], size=n))
    A = [[Fraction(int(v)) for v in row] for row in (L0 @ U0)]
    L, U = LE.lu_blocked(A, 5)
    assert L == [[Fraction(int(v)) for v in row] for row in L0]
    assert U == [[Fraction(int(v)) for v in row] for row in U0]


def test_zero_pivots_raise():
    with pytest.raises(LE.ZeroPivot):
        LE.lu_blocked([[Fraction(0), Fraction(1)], [Fraction(1), Fraction(1)]], 2)
    # a11 != 0 but the leading 2 x 2 block is singular
    A = [[Fraction(v) for v in row] for row in ([1, 2, 0], [2, 4, 1], [0, 1, 1])]
    with pytest.raises(LE.ZeroPivot):
        LE.lu_blocked(A, 3)
