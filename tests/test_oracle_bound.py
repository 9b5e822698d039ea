"""Pin of the truncation error bound that chooses the slice count.

With exact truncating digits (weights 2^(E_i + eo - beta t), |d_t| <= D) the
sum S of the slice pairs t + u <= s + 1 satisfies, for every element,
  |S_ij - C*_ij| <= k c(s) 2^(E_i + F_j - W(s)),  W(s) = beta s - eo,
  c(s) = 2 + 2^(eo - beta s) + (s - 1) D^2 2^(eo - 2 beta) / (1 - 2^-beta)
(the cross terms with the remainders, their product and the dropped pairs).
Checked here in exact arithmetic with the oracle's split and Ozaki sum, for
the balanced radix-32 digits (beta 5, eo 1, D 16), the 4-bit e4m3 digits
(beta 4, D 15), int8 (beta 7, D 127) and binary64 digits (beta 20,
D 2^20 - 1), over slice counts from far too few to plenty, on operands with
exponent spreads phi = 1 and 4.  The bound must hold everywhere and be
reached within a factor 2^12 somewhere (so a bound that is too loose fails
as well as one that is too tight).
"""
import math

import numpy as np
import pytest

from oracle import exact as X
from oracle import ozaki as O
from ozmp_inputs import gen_problem

FORMS = {"bal": (5, 1, 16), "fp8": (4, 0, 15), "int8": (7, 0, 127), "fp64": (20, 0, 2 ** 20 - 1)}


def _c(beta, eo, D, s):
    return 2.0 + 2.0 ** (eo - beta * s) + (s - 1) * D * D * 2.0 ** (eo - 2 * beta) / (1.0 - 2.0 ** -beta)


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("phi", [1.0, 4.0])
def test_truncation_bound_holds_and_is_tight(form, phi):
    beta, eo, D = FORMS[form]
    m, n, k = 6, 5, 40
    A, B = gen_problem("dd", m, n, k, phi=phi, seed=int(phi * 10) + beta)
    Bt = [np.asfortranarray(b.T) for b in B]
    exact = [[None] * n for _ in range(m)]
    Av, Bv = X.matrix_values(A), X.matrix_values(Bt)
    for i in range(m):
        for j in range(n):
            acc = (0, 0)
            for p in range(k):
                acc = X.add(acc, X.mul(Av[i][p], Bv[j][p]))
            exact[i][j] = acc
    worst = 0.0
    for s in (1, 2, 3, 5, 8, 13, 21):
        if form == "fp64" and s > 8:
            continue
        if form == "bal":
            E, Ad = O.split_balanced(A, s)
            F, Bd = O.split_balanced(Bt, s)
        else:
            E, Ad = O.split(A, beta, s)
            F, Bd = O.split(Bt, beta, s)
        assert np.abs(Ad).max() <= D and np.abs(Bd).max() <= D
        S = O.ozaki_sum(E, F, O.slice_products(Ad, Bd), beta, s, 2 * eo)
        c = _c(beta, eo, D, s)
        for i in range(m):
            for j in range(n):
                err = abs(X.to_fraction(X.add(S[i][j], X.neg(exact[i][j]))))
                bound = k * c * 2.0 ** (E[i] + F[j] - (beta * s - eo))
                assert err <= bound, (form, s, i, j)
                worst = max(worst, float(err) / bound)
    assert worst > 2.0 ** -12, worst
