"""CPU Ozaki-scheme product (test infrastructure).

Follows Algorithm 1 (Sec. 3) of the paper: split A and B into slices whose
pairwise products are error-free, form the products of the slice pairs
alpha + beta <= D + 1, and add them in long (L-bit) arithmetic.

Two splits are provided.

* ``split`` -- exact truncating digit slices (the form the CUDA library
  computes).  Row i of an operand gets the exponent
  E_i = max_p E(x_ip), E(x) = floor(log2|x|) + 1 (the power-of-two shift of
  Algorithm 1's tau vectors, taken from the exact value), and
  |x| * 2^(beta*s - E_i) is truncated toward zero to an integer D of beta*s
  bits; slice t holds bits [beta*(s-t), beta*(s-t+1)) of D with the sign of
  x.  Hence x = sum_t d_t 2^(E_i - beta*t) + r exactly, |d_t| <= 2^beta - 1,
  |r| < 2^(E_i - beta*s).  The digits are found here from one exact big
  integer per element (a different algorithm from the library's).
* ``split_balanced`` -- the same truncated value written in balanced
  radix-32 digits (|d| <= 16, all exact in e4m3), found from the least
  significant end by residues in [-16, 15].
* ``paper_literal`` -- Algorithm 1 as printed: round-to-nearest extraction
  (A + S_A) - S_A in binary64, an exact (L-bit) residual update, and the
  last slice taken as the rounded remainder.

Slice products T_d = sum_{t+u=d} A_t B_u^T are exact integer matrices
(plain int64 triple loop); the long accumulation is exact dyadic arithmetic.
"""
from __future__ import annotations

import math

import numpy as np

from . import exact as X
from ._clib import int_gemm_tn

EXP_ZERO = X.EXP_ZERO


# ---------------------------------------------------------------------------
# digit widths (Algorithm 1, Sec. 3: each slice product must be exact in the
# short-precision product)
# ---------------------------------------------------------------------------
def beta_fp64(k: int) -> int:
    """Largest beta with k * (2^beta - 1)^2 <= 2^53: a binary64 dot product
    of k digit pairs then never rounds (the role of the
    ceil((S + log2 l)/2) shift with S = 53 in Algorithm 1)."""
    b = 1
    while k * ((1 << (b + 1)) - 1) ** 2 <= (1 << 53):
        b += 1
    return b


def beta_fp32(k: int) -> int:
    """Same rule for a binary32 accumulator (S = 24)."""
    b = 0
    while k * ((1 << (b + 1)) - 1) ** 2 <= (1 << 24):
        b += 1
    return b


BETA_INT8 = 7   # |d| <= 127: an int8 digit
BETA_FP8 = 4    # |d| <= 15: exactly representable in e4m3
BETA_BAL = 5    # balanced radix-32 digits, |d| <= 16: exactly representable in e4m3


def pairs(D: int):
    """Slice pairs (alpha, beta) with alpha + beta <= D + 1 (Algorithm 1's
    double loop), in the loop's order."""
    return [(a, b) for a in range(1, D + 1) for b in range(1, D - a + 2)]


# ---------------------------------------------------------------------------
# exact truncating digit split
# ---------------------------------------------------------------------------
def split(comps, beta: int, s: int):
    """Split the rows of a multi-component matrix (r x k components).

    Returns (E, digits): E is a list of r row exponents, digits an int64
    array of shape (s, r, k) with digits[t-1, i, p] = d_t(x_ip).
    """
    r, k = comps[0].shape
    vals = X.matrix_values(comps)
    E = []
    for i in range(r):
        e = max(X.exponent(v) for v in vals[i]) if k else EXP_ZERO
        E.append(e)
    dig = np.zeros((s, r, k), dtype=np.int64)
    mask = (1 << beta) - 1
    for i in range(r):
        Ei = E[i]
        if Ei == EXP_ZERO:
            continue
        for p in range(k):
            n, e = vals[i][p]
            if n == 0:
                continue
            sh = e + beta * s - Ei
            a = abs(n)
            D = a << sh if sh >= 0 else a >> (-sh)
            sg = 1 if n > 0 else -1
            for t in range(1, s + 1):
                dig[t - 1, i, p] = sg * ((D >> (beta * (s - t))) & mask)
    return E, dig


def split_balanced(comps, s: int):
    """Balanced radix-32 digits of the truncated value (the e4m3 form with
    beta = 5).

    Row exponents E_i as in ``split``.  The magnitude is truncated at
    2^(E_i + 1 - 5 s): N = floor(|x| 2^(5 s - 1 - E_i)), an integer below
    2^(5 s - 1).  Its digits are peeled off from the least significant end:
    d_s is the residue of N modulo 32 taken in [-16, 15], N := (N - d_s) / 32,
    and so on down to d_2; what is left is the top digit d_1, in [0, 16].
    Every digit then takes the sign of x, so
    x = sum_t d_t 2^(E_i + 1 - 5 t) + r with |d_t| <= 16,
    |r| < 2^(E_i + 1 - 5 s) and r of the sign of x (truncation toward zero):
    the same truncated value as ``split`` with beta = 1 and 5 s - 1 slices,
    written with a third fewer slices than beta = 4 needs for it.
    Returns (E, digits) shaped as ``split``'s.
    """
    r, k = comps[0].shape
    vals = X.matrix_values(comps)
    E = []
    for i in range(r):
        E.append(max(X.exponent(v) for v in vals[i]) if k else EXP_ZERO)
    dig = np.zeros((s, r, k), dtype=np.int64)
    for i in range(r):
        Ei = E[i]
        if Ei == EXP_ZERO:
            continue
        for p in range(k):
            n, e = vals[i][p]
            if n == 0:
                continue
            sh = e + 5 * s - 1 - Ei
            a = abs(n)
            N = a << sh if sh >= 0 else a >> (-sh)
            sg = 1 if n > 0 else -1
            for t in range(s, 1, -1):
                d = N % 32
                if d >= 16:
                    d -= 32
                dig[t - 1, i, p] = sg * d
                N = (N - d) // 32
            assert 0 <= N <= 16
            dig[0, i, p] = sg * N
    return E, dig


def split_remainder(comps, E, dig, beta: int, eoff: int = 0):
    """Exact remainders r = x - sum_t d_t 2^(E + eoff - beta t), as dyadics
    (eoff = 1 for the balanced digits of ``split_balanced``)."""
    r, k = comps[0].shape
    s = dig.shape[0]
    vals = X.matrix_values(comps)
    out = []
    for i in range(r):
        row = []
        for p in range(k):
            acc = vals[i][p]
            if E[i] != EXP_ZERO:
                for t in range(1, s + 1):
                    d = int(dig[t - 1, i, p])
                    if d:
                        acc = X.add(acc, (-d, E[i] + eoff - beta * t))
            row.append(acc)
        out.append(row)
    return out


# ---------------------------------------------------------------------------
# slice products and the long accumulation
# ---------------------------------------------------------------------------
def slice_products(Ad, Bd):
    """T_d = sum_{t+u=d} A_t B_u^T for d = 2..s+1 (exact int64).

    Ad: (s, m, k) digits of A's rows, Bd: (s, n, k) digits of B's columns.
    """
    s = Ad.shape[0]
    T = {}
    for d in range(2, s + 2):
        acc = None
        for t in range(1, d):
            u = d - t
            if u > s:
                continue
            P = int_gemm_tn(Ad[t - 1], Bd[u - 1])
            acc = P if acc is None else acc + P
        T[d] = acc
    return T


def ozaki_sum(E, F, T, beta: int, s: int, eoff: int = 0):
    """Exact S_ij = sum_{d=2}^{s+1} 2^(E_i + F_j + eoff - beta d) T_d(i, j)
    (Algorithm 1's final loop, summed without rounding; eoff = 2 for two
    operands in balanced digits)."""
    m, n = T[2].shape
    out = []
    for i in range(m):
        row = []
        for j in range(n):
            if E[i] == EXP_ZERO or F[j] == EXP_ZERO:
                row.append((0, 0))
                continue
            N = 0
            for d in range(2, s + 2):
                N += int(T[d][i, j]) << (beta * (s + 1 - d))
            row.append((N, E[i] + F[j] + eoff - beta * (s + 1)) if N else (0, 0))
        out.append(row)
    return out


def ozaki_product(A, B, beta: int, s: int, balanced: bool = False):
    """The whole CPU Ozaki product with exact truncating digits (balanced
    radix-32 digits of the truncated values when ``balanced``; beta is then 5).

    A: list of m x k component arrays; B: list of k x n component arrays.
    Returns a dict with E, F, digits, T and the exact Ozaki sum S.
    """
    Bt = [np.asfortranarray(b.T) for b in B]
    if balanced:
        assert beta == BETA_BAL
        E, Ad = split_balanced(A, s)
        F, Bd = split_balanced(Bt, s)
    else:
        E, Ad = split(A, beta, s)
        F, Bd = split(Bt, beta, s)
    T = slice_products(Ad, Bd)
    S = ozaki_sum(E, F, T, beta, s, 2 if balanced else 0)
    return {"E": E, "F": F, "Ad": Ad, "Bd": Bd, "T": T, "S": S}


# ---------------------------------------------------------------------------
# Algorithm 1 as printed (round-to-nearest extraction, S = 53)
# ---------------------------------------------------------------------------
def _ceil_log2_float(mu: float) -> int:
    m, e = math.frexp(mu)     # mu = m 2^e, 0.5 <= m < 1
    return e - 1 if m == 0.5 else e


def paper_literal(A, B, D: int):
    """Algorithm 1 with binary64 short precision (S = 53).

    Inputs are multi-component matrices; the L-bit working copies are exact
    dyadics.  Returns dict with slices A_alpha (float64 arrays), B_beta, the
    float64 slice products C_ab, their exact values, and the exact sum C.
    """
    S = 53
    m, l = A[0].shape
    n = B[0].shape[1]
    Av = X.matrix_values(A)
    Bv = X.matrix_values(B)
    # ceil((S + log2 l)/2) as the smallest integer c with 2^(2c - S) >= l
    c = (S + max(0, (l - 1).bit_length()) + 1) // 2
    As, Bs = [], []

    def rn(M):
        return np.array([[X.round_f64(v) for v in row] for row in M], dtype=np.float64)

    def extract(V, axis):
        Vs = rn(V)
        mu = np.max(np.abs(Vs), axis=axis)
        tau = np.array([0.0 if x == 0 else math.ldexp(1.0, _ceil_log2_float(float(x)) + c) for x in mu])
        T = tau[:, None] if axis == 1 else tau[None, :]
        sl = (Vs + T) - T                     # binary64, round to nearest
        newV = [[X.add(V[i][j], X.neg(X.decode(sl[i, j]))) for j in range(len(V[0]))]
                for i in range(len(V))]
        return sl, newV

    alpha = 1
    while alpha < D:
        a_sl, Av = extract(Av, 1)
        b_sl, Bv = extract(Bv, 0)
        As.append(a_sl)
        Bs.append(b_sl)
        alpha += 1
    As.append(rn(Av))          # A_D := A^(S)
    Bs.append(rn(Bv))
    prods = {}
    C = [[(0, 0)] * n for _ in range(m)]
    for (a, b) in pairs(D):
        P = As[a - 1] @ Bs[b - 1]
        prods[(a, b)] = P
        for i in range(m):
            for j in range(n):
                C[i][j] = X.add(C[i][j], X.decode(P[i, j]))
    rem_a = Av
    rem_b = Bv
    return {"A": As, "B": Bs, "prods": prods, "C": C, "rem_A": rem_a, "rem_B": rem_b, "c": c}
