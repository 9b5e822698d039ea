"""GPU parity of the LU application (Sec. 4.6) against the CPU oracle.

* factors and solutions bit-exact against oracle.lu (the same operations,
  each an exact value rounded canonically, the Ozaki products the exact
  Ozaki sums rounded the same way);
* an exactly representable factorisation (integer L, power-of-two pivots) is
  returned exactly, and its integer system is solved exactly;
* at sizes the oracle cannot follow step by step, the factors reproduce A:
  on sampled entries the exact product L U differs from A by at most
  n 2^(-50 q) |L||U|;
* against the exact rational factors of the Sec. 4.6 block iteration
  (oracle.lu_exact, independent of the library's recursion, block size
  and reciprocal iteration): the normwise errors of L and U lie within the
  first-order perturbation bound of a backward error n 2^(-50 q) |L||U|;
* a zero pivot is reported as a range error.

The bit-exact comparison with oracle.lu is an agreement check between two
statements of the same operations; the exact-rational and backward-error
checks tie the factors to the factorisation itself.
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import exact as X
from oracle import lu as LU
from oracle import lu_exact as LE

from _util import from_dev, to_dev

pytestmark = pytest.mark.gpu


def _random(n, q, seed):
    rng = np.random.default_rng(seed)
    A = rng.random((n, n))                     # the paper's a_ij = ru
    comps = [np.asfortranarray(A)]
    for t in range(1, q):                      # tails below the head, as the multi-component inputs
        comps.append(np.asfortranarray(comps[-1] * 2.0 ** -53 * rng.uniform(-1, 1, size=(n, n))))
    return comps


@pytest.mark.parametrize("q,n", [(2, 70), (3, 40), (4, 36)])
def test_factors_bit_exact(q, n):
    comps = _random(n, q, seed=q * 100 + n)
    Ad = to_dev(comps)
    assert oz.ozmp_lu(Ad) == oz.Status.OK
    got = from_dev(Ad)
    want = LU.lu(comps)
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)


def test_solve_bit_exact():
    q, n, w = 2, 70, 3
    comps = _random(n, q, seed=5)
    rng = np.random.default_rng(6)
    b = [np.asfortranarray(rng.random((n, w)))] + [np.zeros((n, w), order="F")]
    F = LU.lu(comps)
    Fd = to_dev(F)
    bd = to_dev(b)
    assert oz.ozmp_lu_solve(Fd, bd) == oz.Status.OK
    for g, ww in zip(from_dev(bd), LU.lu_solve(F, b)):
        np.testing.assert_array_equal(g, ww)


def test_exact_factorisation_and_solve():
    n, q = 100, 2
    rng = np.random.default_rng(9)
    L = np.tril(rng.integers(-3, 4, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    U = np.triu(rng.integers(-3, 4, size=(n, n)).astype(np.float64), 1)
    U += np.diag(2.0 ** rng.integers(0, 3, size=n) * rng.choice([-1.0, 1.0], size=n))
    A = L @ U
    Ad = to_dev([np.asfortranarray(A), np.zeros((n, n), order="F")])
    assert oz.ozmp_lu(Ad) == oz.Status.OK
    got = from_dev(Ad)
    np.testing.assert_array_equal(got[0], np.tril(L, -1) + U)
    assert not got[1].any()
    x = (np.arange(n, dtype=np.float64) - 50.0)[:, None]
    bd = to_dev([np.asfortranarray(A @ x), np.zeros((n, 1), order="F")])
    assert oz.ozmp_lu_solve(Ad, bd) == oz.Status.OK
    sol = from_dev(bd)
    np.testing.assert_array_equal(sol[0], x)


@pytest.mark.parametrize("q,n", [(2, 512), (3, 300)])
def test_backward_error_sampled(q, n):
    comps = _random(n, q, seed=11 + n)
    Ad = to_dev(comps)
    assert oz.ozmp_lu(Ad) == oz.Status.OK
    F = from_dev(Ad)

    def val(i, j):
        return X.to_fraction(X.elem_value([c[i, j] for c in F]))

    def aval(i, j):
        return X.to_fraction(X.elem_value([c[i, j] for c in comps]))

    for i in [0, 1, n // 2, n - 1]:
        for j in [0, n // 3, n - 1]:
            s, mag = Fraction(0), Fraction(0)
            for k in range(min(i, j) + 1):
                lik = Fraction(1) if k == i else val(i, k)
                term = lik * val(k, j)
                s += term
                mag += abs(term)
            assert abs(s - aval(i, j)) <= mag * n * Fraction(1, 2 ** (50 * q)), (i, j)


def test_zero_pivot_is_a_range_error():
    n = 40
    comps = _random(n, 2, seed=3)
    comps[0][0, 0] = 0.0
    comps[1][0, 0] = 0.0
    Ad = to_dev(comps)
    assert oz.ozmp_lu(Ad) == oz.Status.ERR_RANGE


@pytest.mark.parametrize("q,n,dominant", [(2, 48, False), (3, 40, False), (4, 36, False), (2, 48, True),
                                          (3, 40, True)])
def test_factors_near_the_exact_rational_lu(q, n, dominant):
    # The exact factors L, U of A (Fractions).  A backward error
    # L^ U^ = A + dA with ||dA||_F <= eps ||(|L||U|)||_F, eps = n 2^(-50 q),
    # moves the factors by at most (first order)
    #   ||dL||_F <= eps ||L||_2 ||L^-1||_2 ||U^-1||_2 ||(|L||U|)||_F,
    #   ||dU||_F <= eps ||L^-1||_2 ||U^-1||_2 ||U||_2 ||(|L||U|)||_F;
    # the test allows twice that.  A wrong entry anywhere is off by O(1).
    comps = _random(n, q, seed=700 + 10 * q + n)
    if dominant:
        # the paper's matrix plus n/2 on the diagonal: a well-conditioned LU
        comps[0] = np.asfortranarray(comps[0] + np.eye(n) * (n / 2))
    L, U = LE.lu_blocked(LE.values(comps), n)
    Ad = to_dev(comps)
    assert oz.ozmp_lu(Ad) == oz.Status.OK
    F = from_dev(Ad)
    Lf = np.array([[float(x) for x in row] for row in L])
    Uf = np.array([[float(x) for x in row] for row in U])
    nrm2 = lambda M: float(np.linalg.norm(M, 2))
    Li, Ui = np.linalg.inv(Lf), np.linalg.inv(Uf)
    base = float(np.linalg.norm(np.abs(Lf) @ np.abs(Uf)))
    eps = n * 2.0 ** (-50 * q)
    bound_L = 2 * eps * nrm2(Lf) * nrm2(Li) * nrm2(Ui) * base
    bound_U = 2 * eps * nrm2(Li) * nrm2(Ui) * nrm2(Uf) * base
    dL2 = dU2 = 0.0
    for i in range(n):
        for j in range(n):
            got = X.to_fraction(X.elem_value([c[i, j] for c in F]))
            if i > j:
                dL2 += float(got - L[i][j]) ** 2
            else:
                dU2 += float(got - U[i][j]) ** 2
    assert dL2 ** 0.5 <= bound_L, (dL2 ** 0.5, bound_L)
    assert dU2 ** 0.5 <= bound_U, (dU2 ** 0.5, bound_U)
    # and the bound is not vacuous: it is below what binary64 arithmetic can
    # reach (2^-60 relative), and for the well-conditioned matrices within a
    # factor 2^20 of the target
    rel = 2.0 ** (20 - 50 * q) if dominant else 2.0 ** -60
    assert bound_L < rel * nrm2(Lf) and bound_U < rel * nrm2(Uf)
