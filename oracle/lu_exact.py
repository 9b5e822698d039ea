"""Exact LU factorisation without pivoting, as the paper's block iteration
defines it (test infrastructure; imported only by the tests).

Paper, Sec. 4.6 ("LU decomposition using matrix multiplication"): choose an
iteration width K, split A into A11 (K x K), A12, A21, A22; factor
A11 = L11 U11; turn A12 into U12 = L11^-1 A12 and A21 into
L21 = A21 U11^-1; set A22 := A22 - L21 U12; repeat on A22 while rows are
left.  No pivoting.

Here every step is carried out in exact rational arithmetic (Fractions), so
the result is the exact L U factorisation of the exact input: L unit lower
triangular, U upper triangular, L U = A.  Without pivoting that
factorisation is unique when it exists, so it does not depend on K; the
pins check both facts.  This is independent of the library's own recursion,
block size and reciprocal iteration: it is the value the library's rounded
factors approximate.
"""
from __future__ import annotations

from fractions import Fraction

from . import exact as X


class ZeroPivot(ZeroDivisionError):
    """A leading principal submatrix is singular: no LU without pivoting."""


def values(comps):
    """Exact Fractions of an n x n multi-component matrix (list of arrays)."""
    r, c = comps[0].shape
    return [[X.to_fraction(X.elem_value([x[i, j] for x in comps])) for j in range(c)] for i in range(r)]


def _factor_block(A, r0, w):
    """Unblocked exact LU of the w x w block at (r0, r0), in place (L strictly
    below the diagonal, U on and above it)."""
    for p in range(r0, r0 + w):
        piv = A[p][p]
        if piv == 0:
            raise ZeroPivot(p)
        for i in range(p + 1, r0 + w):
            A[i][p] = A[i][p] / piv
            lip = A[i][p]
            if lip:
                for j in range(p + 1, r0 + w):
                    A[i][j] -= lip * A[p][j]


def lu_blocked(A, K: int):
    """Exact LU without pivoting of the n x n Fraction matrix A with the
    block iteration of Sec. 4.6 and width K.

    Returns (L, U) as n x n lists of Fractions (L with unit diagonal).
    Raises ZeroPivot if a pivot is zero.
    """
    n = len(A)
    W = [list(row) for row in A]
    r0 = 0
    while r0 < n:
        w = min(K, n - r0)
        # A11 = L11 U11
        _factor_block(W, r0, w)
        hi = r0 + w
        # U12 = L11^-1 A12: forward substitution with the unit lower L11
        for j in range(hi, n):
            for i in range(r0, hi):
                s = W[i][j]
                for p in range(r0, i):
                    s -= W[i][p] * W[p][j]
                W[i][j] = s
        # L21 = A21 U11^-1: substitution with the upper U11, column by column
        for i in range(hi, n):
            for j in range(r0, hi):
                s = W[i][j]
                for p in range(r0, j):
                    s -= W[i][p] * W[p][j]
                W[i][j] = s / W[j][j]
        # A22 := A22 - L21 U12
        for i in range(hi, n):
            for j in range(hi, n):
                s = Fraction(0)
                for p in range(r0, hi):
                    s += W[i][p] * W[p][j]
                W[i][j] -= s
        r0 = hi
    L = [[Fraction(1) if i == j else (W[i][j] if i > j else Fraction(0)) for j in range(n)] for i in range(n)]
    U = [[W[i][j] if i <= j else Fraction(0) for j in range(n)] for i in range(n)]
    return L, U
