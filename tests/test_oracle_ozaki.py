"""Pins for oracle/ozaki.py: the digit split, slice products, the exact
Ozaki sum and the paper-literal Algorithm 1.

Pins come from the paper (the 3x3 worked example's pair set, Sec. 3; the
error-free slice products claimed for Algorithm 1), from invariants of the
split (slices plus remainder sum back exactly), from a third, iterative
digit computation in Fractions, and from exact special cases whose product
is known in closed form (TwoProd, small integers).
"""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import _clib, eft
from oracle import exact as X
from oracle import ozaki as O
from ozmp_inputs import gen_problem, gen_operand

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_pairs_match_paper_3x3_example():
    toks = [l for l in open(os.path.join(GOLD, "pairs_D3.txt")) if not l.startswith("#")][0].split()
    want = [(int(t[0]), int(t[1])) for t in toks]
    assert O.pairs(3) == want


@pytest.mark.parametrize("D", [1, 2, 5, 12, 40])
def test_pair_count_triangle(D):
    ps = O.pairs(D)
    assert len(ps) == D * (D + 1) // 2
    assert all(a + b <= D + 1 for a, b in ps) and len(set(ps)) == len(ps)


def test_beta_rules():
    # exactness of one slice product in the S-bit accumulator, and maximality
    for k in [1, 7, 128, 1000, 1024, 4096, 8192, 16384, 100000]:
        b = O.beta_fp64(k)
        assert k * (2 ** b - 1) ** 2 <= 2 ** 53 < k * (2 ** (b + 1) - 1) ** 2
        b = O.beta_fp32(k)
        assert k * (2 ** b - 1) ** 2 <= 2 ** 24 < k * (2 ** (b + 1) - 1) ** 2


def _iterative_digits(x: Fraction, E: int, beta: int, s: int):
    """Third computation: repeated scaling and flooring in Fractions."""
    sg = 1 if x > 0 else -1
    y = abs(x) / Fraction(2) ** E
    ds = []
    for _ in range(s):
        y *= 2 ** beta
        d = math.floor(y)
        ds.append(sg * d)
        y -= d
    return ds


@pytest.mark.parametrize("prec,beta,s", [("dd", 7, 17), ("td", 4, 40), ("qd", 20, 12), ("ts", 7, 11), ("dd", 23, 6)])
def test_split_invariants_and_digits(prec, beta, s):
    rng = np.random.default_rng(3)
    A = gen_operand(rng, prec, 6, 9, phi=2.0)
    E, dig = O.split(A, beta, s)
    rem = O.split_remainder(A, E, dig, beta)
    vals = X.matrix_values(A)
    for i in range(6):
        mx = max(abs(X.to_fraction(v)) for v in vals[i])
        assert Fraction(2) ** (E[i] - 1) <= mx < Fraction(2) ** E[i]
        for p in range(9):
            x = X.to_fraction(vals[i][p])
            ds = [int(dig[t, i, p]) for t in range(s)]
            assert all(abs(d) <= 2 ** beta - 1 for d in ds)
            assert all(d == 0 or (d > 0) == (x > 0) for d in ds)
            back = sum(Fraction(d) * Fraction(2) ** (E[i] - beta * (t + 1)) for t, d in enumerate(ds))
            r = X.to_fraction(rem[i][p])
            assert back + r == x
            assert abs(r) < Fraction(2) ** (E[i] - beta * s)
            assert x == 0 or r == 0 or (r > 0) == (x > 0)      # truncation toward zero
            assert ds == _iterative_digits(x, E[i], beta, s)


def test_split_unnormalised_and_zero_rows():
    A = [np.array([[1.0, 0.0, 3.0], [0.0, 0.0, 0.0], [2.0 ** 60, 0.25, 0.5]]),
         np.array([[-(2.0 ** -300), 0.0, -1.0], [0.0, 0.0, 0.0], [-(2.0 ** 60), 0.0, 2.0 ** -70]]),
         np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])]
    E, dig = O.split(A, 7, 10)
    assert E[0] == 2 and E[1] == O.EXP_ZERO and E[2] == 1
    assert not dig[:, 1, :].any()
    # 1 - 2^-300 truncates to all-ones digits below 2^E = 4: first digit 0b0011111
    assert [int(d) for d in dig[:, 0, 0]] == _iterative_digits(Fraction(1) - Fraction(2) ** -300, 2, 7, 10)
    assert int(dig[0, 0, 0]) == 0b0011111 and all(int(d) == 127 for d in dig[1:, 0, 0])
    # 2^60 - 2^60 + 1 = 1 (complete cancellation of the leading pair)
    assert E[2] == 1
    assert [int(d) for d in dig[:, 2, 0]] == _iterative_digits(Fraction(1), 1, 7, 10)


def test_split_single_slice_case():
    # x = 2^(E - beta) * d with |d| < 2^beta has exactly one non-zero digit
    beta = 7
    for d in [1, 5, 64, 127, -3, -127]:
        A = [np.array([[d * 2.0 ** -20, 127 * 2.0 ** -20]])]
        E, dig = O.split(A, beta, 5)
        assert E[0] == -13
        assert [int(v) for v in dig[:, 0, 0]] == [d, 0, 0, 0, 0]


def test_slice_products_bruteforce():
    rng = np.random.default_rng(4)
    s, m, n, k = 4, 3, 5, 6
    Ad = rng.integers(-127, 128, (s, m, k))
    Bd = rng.integers(-127, 128, (s, n, k))
    T = O.slice_products(Ad, Bd)
    assert sorted(T) == list(range(2, s + 2))
    for d in T:
        for i in range(m):
            for j in range(n):
                want = sum(int(Ad[t - 1, i, p]) * int(Bd[d - t - 1, j, p])
                           for t in range(1, d) if 1 <= d - t <= s for p in range(k))
                assert int(T[d][i, j]) == want


def test_ozaki_sum_error_bound():
    # |S_ij - C*_ij| <= 2 k s 2^(E_i + F_j - beta s)  (bound derived from the
    # truncated split: remainders below 2^(E - beta s), dropped pairs t+u > s+1)
    for prec, beta, s in [("dd", 7, 9), ("td", 4, 12), ("qd", 20, 4)]:
        A, B = gen_problem(prec, 4, 5, 16, phi=1.0, seed=5)
        r = O.ozaki_product(A, B, beta, s)
        ex = _clib.exact_block(A, B, range(4), range(5))
        k = 16
        for i in range(4):
            for j in range(5):
                d = abs(X.to_fraction(r["S"][i][j]) - X.to_fraction(ex[i][j]))
                assert d <= 2 * k * s * Fraction(2) ** (r["E"][i] + r["F"][j] - beta * s)


def test_ozaki_exact_special_case_twoprod():
    # k = 1, one component: with all 53 bits in 8 slices of 7 bits and
    # s = 15, no non-zero pair is dropped, so S = a*b exactly and its
    # canonical DD is TwoProd(a, b).
    rng = random.Random(9)
    for _ in range(50):
        a = math.ldexp(rng.uniform(0.5, 1) * rng.choice([-1, 1]), rng.randint(-30, 30))
        b = math.ldexp(rng.uniform(0.5, 1) * rng.choice([-1, 1]), rng.randint(-30, 30))
        A = [np.array([[a]]), np.array([[0.0]])]
        B = [np.array([[b]]), np.array([[0.0]])]
        r = O.ozaki_product(A, B, 7, 15)
        assert X.to_fraction(r["S"][0][0]) == Fraction(a) * Fraction(b)
        assert X.to_components(r["S"][0][0], 2) == list(eft.two_prod(a, b))


def test_ozaki_exact_small_integers():
    rng = np.random.default_rng(6)
    Ai = rng.integers(-1000, 1001, (5, 8)).astype(np.float64)
    Bi = rng.integers(-1000, 1001, (8, 4)).astype(np.float64)
    A = [np.asfortranarray(Ai), np.zeros((5, 8), order="F")]
    B = [np.asfortranarray(Bi), np.zeros((8, 4), order="F")]
    r = O.ozaki_product(A, B, 4, 5)     # 20 bits per row cover |a| <= 1000 < 2^10 at any E
    C = Ai @ Bi
    for i in range(5):
        for j in range(4):
            assert X.to_fraction(r["S"][i][j]) == Fraction(int(C[i, j]))


def test_paper_literal_algorithm1():
    A, B = gen_problem("dd", 6, 5, 32, phi=1.0, seed=7)
    D = 4
    r = O.paper_literal(A, B, D)
    assert sorted(r["prods"]) == sorted(O.pairs(D))
    # the extracted slices (alpha < D) give error-free binary64 products
    for (a, b), P in r["prods"].items():
        if a < D and b < D:
            for i in range(6):
                for j in range(5):
                    ex = sum(Fraction(float(r["A"][a - 1][i, p])) * Fraction(float(r["B"][b - 1][p, j]))
                             for p in range(32))
                    assert Fraction(float(P[i, j])) == ex
    # slices + final remainder reproduce A exactly (L-bit residual update)
    vals = X.matrix_values(A)
    for i in range(6):
        for p in range(32):
            tot = sum(Fraction(float(sl[i, p])) for sl in r["A"])
            rem = X.to_fraction(r["rem_A"][i][p]) - Fraction(float(r["A"][-1][i, p]))
            assert tot + rem == X.to_fraction(vals[i][p])


def test_paper_literal_accuracy_improves_with_D():
    A, B = gen_problem("dd", 4, 4, 64, phi=1.0, seed=8)
    ex = _clib.exact_block(A, B, range(4), range(4))
    errs = []
    for D in [2, 3, 4, 6, 8]:
        r = O.paper_literal(A, B, D)
        chat = [[X.to_components(v, 2) for v in row] for row in r["C"]]
        errs.append(X.error_metrics(chat, ex)["err_nw"])
    assert errs[0] > errs[2] > 0
    assert errs[-1] < 2.0 ** -100          # DD accuracy reached well before D = 8


def _golden_divisions():
    out = {}
    for line in open(os.path.join(GOLD, "max_accuracy_divisions.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, d = line.split()[:2]
        out[p] = int(d)
    return out


@pytest.mark.parametrize("prec,q", [("dd", 2), ("td", 3), ("qd", 4)])
def test_paper_literal_plateau_matches_paper_division_counts(prec, q):
    """Sec. 4.1-4.3: accuracy stops improving at D = 6 (DD), 10 (TD), 11 (QD).

    The plateau must be reached by the paper's D.  For DD and QD it is also
    not reached one division earlier, as the paper reports; this TD
    arithmetic (exact L-bit residuals) reaches it before D = 10.
    """
    Dp = _golden_divisions()[prec]
    A, B = gen_problem(prec, 6, 6, 512, phi=1.0, seed=0)
    ex = _clib.exact_block(A, B, range(6), range(6))

    def err(D):
        r = O.paper_literal(A, B, D)
        chat = [[X.to_components(v, q) for v in row] for row in r["C"]]
        return X.error_metrics(chat, ex)["err_nw"]

    e_at, e_after = err(Dp), err(Dp + 1)
    assert e_after >= e_at / 2
    if prec != "td":
        assert err(Dp - 1) > 2 * e_at


# ---------------------------------------------------------------------------
# balanced radix-32 digits (e4m3, beta = 5)
# ---------------------------------------------------------------------------
def test_balanced_split_hand_examples():
    # worked by hand: 0.99 has E = 0; N = floor(0.99 * 2^9) = 506 = 16 * 32 - 6
    # (residue 26 -> -6, carry 16 into the top digit); 1 - 2^-20 gives
    # N = 511 = 16 * 32 - 1; 0.5 gives N = 256 = 8 * 32; 0.75 with s = 3
    # gives N = 0.75 * 2^14 = 12 * 1024
    A = [np.array([[0.99, -0.99, 0.5, 1 - 2.0 ** -20]])]
    E, dig = O.split_balanced(A, 2)
    assert E == [0]
    assert [[int(d) for d in dig[:, 0, p]] for p in range(4)] == [[16, -6], [-16, 6], [8, 0], [16, -1]]
    E, dig = O.split_balanced([np.array([[0.75]])], 3)
    assert [int(d) for d in dig[:, 0, 0]] == [12, 0, 0]


@pytest.mark.parametrize("prec,s", [("dd", 26), ("td", 9), ("qd", 44), ("ts", 14), ("dd", 1)])
def test_balanced_split_invariants(prec, s):
    rng = np.random.default_rng(11)
    A = gen_operand(rng, prec, 6, 9, phi=2.0)
    E, dig = O.split_balanced(A, s)
    rem = O.split_remainder(A, E, dig, 5, eoff=1)
    E1, bits = O.split(A, 1, 5 * s - 1)           # the same truncation, one bit per slice
    assert E1 == E
    vals = X.matrix_values(A)
    for i in range(6):
        for p in range(9):
            x = X.to_fraction(vals[i][p])
            ds = [int(dig[t, i, p]) for t in range(s)]
            sg = 1 if x >= 0 else -1
            assert 0 <= sg * ds[0] <= 16
            assert all(-16 <= sg * d <= 15 for d in ds[1:])
            back = sum(Fraction(d) * Fraction(2) ** (E[i] + 1 - 5 * (t + 1)) for t, d in enumerate(ds))
            r = X.to_fraction(rem[i][p])
            assert back + r == x
            assert abs(r) < Fraction(2) ** (E[i] + 1 - 5 * s)
            assert x == 0 or r == 0 or (r > 0) == (x > 0)      # truncation toward zero
            trunc = sum(Fraction(int(bits[t, i, p])) * Fraction(2) ** (E[i] - (t + 1)) for t in range(5 * s - 1))
            assert back == trunc


def test_balanced_ozaki_sum_error_bound():
    # remainders below 2^(E + 1 - 5 s), digits |d| <= 16, dropped pairs
    # t + u > s + 1: |S_ij - C*_ij| <= 2 k s 2^(E_i + F_j + 2 - 5 s)
    for prec, s in [("dd", 9), ("td", 12), ("qd", 5)]:
        A, B = gen_problem(prec, 4, 5, 16, phi=1.0, seed=5)
        r = O.ozaki_product(A, B, O.BETA_BAL, s, balanced=True)
        ex = _clib.exact_block(A, B, range(4), range(5))
        for i in range(4):
            for j in range(5):
                d = abs(X.to_fraction(r["S"][i][j]) - X.to_fraction(ex[i][j]))
                assert d <= 2 * 16 * s * Fraction(2) ** (r["E"][i] + r["F"][j] + 2 - 5 * s)


def test_balanced_ozaki_exact_special_cases():
    # k = 1: a's 53 bits sit in the top 11 digits of a 23-digit window (the
    # low 61 bits of N are zero, so are its 12 lowest digits), the same for
    # b; every non-zero pair has t + u <= 22 <= s + 1 and S = a b exactly,
    # whose canonical DD is TwoProd(a, b)
    rng = random.Random(10)
    for _ in range(50):
        a = math.ldexp(rng.uniform(0.5, 1) * rng.choice([-1, 1]), rng.randint(-30, 30))
        b = math.ldexp(rng.uniform(0.5, 1) * rng.choice([-1, 1]), rng.randint(-30, 30))
        r = O.ozaki_product([np.array([[a]]), np.array([[0.0]])], [np.array([[b]]), np.array([[0.0]])],
                            O.BETA_BAL, 23, balanced=True)
        assert X.to_fraction(r["S"][0][0]) == Fraction(a) * Fraction(b)
        assert X.to_components(r["S"][0][0], 2) == list(eft.two_prod(a, b))
    # small integers (|a| <= 1000, E <= 10): with s = 8 the window's low 29
    # bits are zero, only digits 1..3 can be non-zero, no non-zero pair is dropped
    g = np.random.default_rng(12)
    Ai = g.integers(-1000, 1001, (5, 8)).astype(np.float64)
    Bi = g.integers(-1000, 1001, (8, 4)).astype(np.float64)
    r = O.ozaki_product([np.asfortranarray(Ai), np.zeros((5, 8), order="F")],
                        [np.asfortranarray(Bi), np.zeros((8, 4), order="F")], O.BETA_BAL, 8, balanced=True)
    C = Ai @ Bi
    for i in range(5):
        for j in range(4):
            assert X.to_fraction(r["S"][i][j]) == Fraction(int(C[i, j]))
