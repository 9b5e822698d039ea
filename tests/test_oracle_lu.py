"""Pins of the LU oracle (oracle/lu.py) against closed forms and bounds.

* A = L U with a unit lower integer L and an upper integer U whose diagonal
  holds powers of two: every operation of the factorisation is exact (the
  pivots' reciprocals are exact, the Ozaki products of small integers keep
  every bit), so the oracle must return L and U themselves;
* the solve of such a system with an integer right-hand side returns the
  integer solution;
* the Newton reciprocal is within 2^(2 - 53 q) relative of 1 / d;
* for random matrices the factors reproduce A to the precision: the exact
  product L U differs from A by at most n 2^(-50 q) relative to |L||U|.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X
from oracle import lu as LU


def _exact_lu_problem(n, q, seed):
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-3, 4, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, size=(n, n)).astype(np.float64), 1)
    U += np.diag(2.0 ** rng.integers(0, 3, size=n) * rng.choice([-1.0, 1.0], size=n))
    A = L @ U            # integers below 2^53: exact in binary64
    comps = [np.asfortranarray(A)] + [np.zeros((n, n), order="F") for _ in range(q - 1)]
    return L, U, comps


def _packed(L, U):
    return np.tril(L, -1) + U


@pytest.mark.parametrize("q,n", [(2, 70), (3, 40)])
def test_exact_factors_are_recovered(q, n):
    L, U, comps = _exact_lu_problem(n, q, seed=n)
    F = LU.lu(comps)
    np.testing.assert_array_equal(F[0], _packed(L, U))
    for c in F[1:]:
        assert not c.any()


def test_exact_solve():
    q, n = 2, 40
    L, U, comps = _exact_lu_problem(n, q, seed=7)
    F = LU.lu(comps)
    x = np.arange(1, n + 1, dtype=np.float64)[:, None] - 20.0
    b = (L @ U) @ x
    bc = [np.asfortranarray(b), np.zeros_like(b, order="F")]
    sol = LU.lu_solve(F, bc)
    np.testing.assert_array_equal(sol[0], x)
    assert not sol[1].any()


@pytest.mark.parametrize("q", [2, 3, 4])
def test_reciprocal_bound(q):
    rng = np.random.default_rng(q)
    for _ in range(50):
        d = [float(rng.uniform(0.1, 10.0) * rng.choice([-1, 1]))]
        for t in range(1, q):
            d.append(float(np.float64(d[-1]) * 2.0 ** -53 * rng.uniform(-1, 1)))
        r = LU.recip(d, q)
        dv = X.to_fraction(X.elem_value(d))
        rv = X.to_fraction(X.elem_value(r))
        assert abs(rv * dv - 1) <= Fraction(4, 2 ** (53 * q))


@pytest.mark.parametrize("q,n", [(2, 48), (3, 40)])
def test_random_backward_error(q, n):
    rng = np.random.default_rng(100 + n)
    A = rng.random((n, n))           # the paper's a_ij = ru
    comps = [np.asfortranarray(A)] + [np.zeros((n, n), order="F") for _ in range(q - 1)]
    F = LU.lu(comps)
    val = [[X.to_fraction(X.elem_value([c[i, j] for c in F])) for j in range(n)] for i in range(n)]
    for i in range(0, n, 5):
        for j in range(0, n, 7):
            s = Fraction(0)
            mag = Fraction(0)
            for k in range(min(i, j) + 1):
                lik = Fraction(1) if k == i else val[i][k]
                ukj = val[k][j]
                s += lik * ukj
                mag += abs(lik * ukj)
            assert abs(s - Fraction(float(A[i, j]))) <= mag * n * Fraction(1, 2 ** (50 * q))
