"""LU factorisation without pivoting with the Ozaki-scheme product -- the
CPU oracle of the LU application (test infrastructure; imported only by
the tests).

Paper, Sec. 4.6 ("LU decomposition using matrix multiplication"): factor
A11 = L11 U11, turn A12 into U12 = L11^-1 A12 and A21 into L21 = A21 U11^-1,
update A22 := A22 - L21 U12 with the Ozaki product, and repeat on A22.

The library applies this step recursively (leading half of the block, down
to 32 x 32) and solves the panels with recursive triangular solves whose
updates are Ozaki products too.  Every operation that is not an Ozaki
product is an exact value rounded once, canonically, into q binary64
components (exact.to_components); the Ozaki products are the exact Ozaki
sums (ozaki.ozaki_product with balanced radix-32 e4m3 digits, beta = 5,
the slice count of the precision's target) rounded the same way.  This module restates those
definitions with exact dyadic arithmetic, operation by operation, so that
its factors are the exact values the definitions give.
"""
from __future__ import annotations

import math

import numpy as np

from . import exact as X
from . import ozaki as O

NB = 32


def half(n: int) -> int:
    """Split point of an n-block: ceil(blocks / 2) base blocks."""
    return ((n + NB - 1) // NB + 1) // 2 * NB


def slices_for(q: int, k: int) -> int:
    """Automatic slice count of the balanced e4m3 form: target 2^(-50 q),
    guard log2 k + 16 bits, 5 s - 1 bits kept below 2^E."""
    lg = max(0, (k - 1).bit_length())
    return -(-(50 * q + lg + 16 + 1) // 5)


def newton_steps(q: int) -> int:
    return 0 if q <= 1 else (2 if q <= 2 else 3)


class Matrix:
    """n x n matrix of q-component values: M[i][j] = list of q floats."""

    def __init__(self, comps):
        self.q = len(comps)
        self.n = comps[0].shape[0]
        self.v = [[[float(c[i, j]) for c in comps] for j in range(comps[0].shape[1])] for i in range(self.n)]

    def comps(self):
        r, c = len(self.v), len(self.v[0])
        out = [np.zeros((r, c)) for _ in range(self.q)]
        for i in range(r):
            for j in range(c):
                for t in range(self.q):
                    out[t][i, j] = self.v[i][j][t]
        return [np.asfortranarray(o) for o in out]


def value(x):
    """Exact dyadic of a q-component value."""
    return X.elem_value(x)


def canon(a, q):
    return X.to_components(a, q, "f64")


def product(x, y):
    """Exact x * y of two q-component values."""
    return X.mul(value(x), value(y))


def recip(d, q):
    """1 / d to q components: x_0 = RN(1 / d_0), then x := x + x (1 - d x)
    with every operation exact and rounded canonically."""
    x = [1.0 / d[0]] + [0.0] * (q - 1)
    one = X.decode(1.0)
    for _ in range(newton_steps(q)):
        e = canon(X.add(one, X.neg(product(d, x))), q)
        x = canon(X.add(value(x), product(x, e)), q)
    return x


def base_lu(M, r0, n, q):
    """Crout order on the n x n block at (r0, r0): row k of U, then column k
    of L, each entry one exact dot product rounded once."""
    v = M.v
    for k in range(n):
        for j in range(k, n):
            acc = value(v[r0 + k][r0 + j])
            for t in range(k):
                acc = X.add(acc, X.neg(product(v[r0 + k][r0 + t], v[r0 + t][r0 + j])))
            v[r0 + k][r0 + j] = canon(acc, q)
        r = recip(v[r0 + k][r0 + k], q)
        for i in range(k + 1, n):
            acc = value(v[r0 + i][r0 + k])
            for t in range(k):
                acc = X.add(acc, X.neg(product(v[r0 + i][r0 + t], v[r0 + t][r0 + k])))
            num = canon(acc, q)
            v[r0 + i][r0 + k] = canon(product(num, r), q)


def block(M, r0, c0, rows, cols):
    """Component arrays of a sub-block (for the Ozaki product)."""
    return [np.asfortranarray(np.array([[M.v[r0 + i][c0 + j][t] for j in range(cols)] for i in range(rows)],
                                       dtype=np.float64).reshape(rows, cols)) for t in range(M.q)]


def gemm_sub(M, cr, cc, ar, ac, br, bc, m, n, k):
    """C (m x n at (cr, cc)) := RN_q(C - P), P the Ozaki product of the
    m x k block at (ar, ac) and the k x n block at (br, bc)."""
    if m == 0 or n == 0 or k == 0:
        return
    q = M.q
    A = block(M, ar, ac, m, k)
    B = block(M, br, bc, k, n)
    r = O.ozaki_product(A, B, O.BETA_BAL, slices_for(q, k), balanced=True)
    for i in range(m):
        for j in range(n):
            p = canon(r["S"][i][j], q)
            M.v[cr + i][cc + j] = canon(X.add(value(M.v[cr + i][cc + j]), X.neg(value(p))), q)


def trsm_ll(M, lr, lc, br, bc, m, w):
    """L X = B, L (m x m unit lower at (lr, lc)), B (m x w at (br, bc))."""
    if m == 0 or w == 0:
        return
    q = M.q
    v = M.v
    if m <= NB:
        for j in range(w):
            for i in range(m):
                acc = value(v[br + i][bc + j])
                for t in range(i):
                    acc = X.add(acc, X.neg(product(v[lr + i][lc + t], v[br + t][bc + j])))
                v[br + i][bc + j] = canon(acc, q)
        return
    m1 = half(m)
    trsm_ll(M, lr, lc, br, bc, m1, w)
    gemm_sub(M, br + m1, bc, lr + m1, lc, br, bc, m - m1, w, m1)
    trsm_ll(M, lr + m1, lc + m1, br + m1, bc, m - m1, w)


def trsm_ru(M, ur, uc, br, bc, m, h):
    """X U = B, U (m x m upper at (ur, uc)), B (h x m at (br, bc))."""
    if m == 0 or h == 0:
        return
    q = M.q
    v = M.v
    if m <= NB:
        rs = [recip(v[ur + j][uc + j], q) for j in range(m)]
        for i in range(h):
            for j in range(m):
                acc = value(v[br + i][bc + j])
                for t in range(j):
                    acc = X.add(acc, X.neg(product(v[br + i][bc + t], v[ur + t][uc + j])))
                v[br + i][bc + j] = canon(product(canon(acc, q), rs[j]), q)
        return
    m1 = half(m)
    trsm_ru(M, ur, uc, br, bc, m1, h)
    gemm_sub(M, br, bc + m1, br, bc, ur, uc + m1, h, m - m1, m1)
    trsm_ru(M, ur + m1, uc + m1, br, bc + m1, m - m1, h)


def trsm_lu(M, ur, uc, br, bc, m, w):
    """U X = B, U (m x m upper at (ur, uc)), B (m x w at (br, bc))."""
    if m == 0 or w == 0:
        return
    q = M.q
    v = M.v
    if m <= NB:
        rs = [recip(v[ur + i][uc + i], q) for i in range(m)]
        for j in range(w):
            for i in range(m - 1, -1, -1):
                acc = value(v[br + i][bc + j])
                for t in range(i + 1, m):
                    acc = X.add(acc, X.neg(product(v[ur + i][uc + t], v[br + t][bc + j])))
                v[br + i][bc + j] = canon(product(canon(acc, q), rs[i]), q)
        return
    m1 = half(m)
    trsm_lu(M, ur + m1, uc + m1, br + m1, bc, m - m1, w)
    gemm_sub(M, br, bc, ur, uc + m1, br + m1, bc, m1, w, m - m1)
    trsm_lu(M, ur, uc, br, bc, m1, w)


def _lu(M, r0, n):
    if n == 0:
        return
    if n <= NB:
        base_lu(M, r0, n, M.q)
        return
    n1 = half(n)
    n2 = n - n1
    _lu(M, r0, n1)
    trsm_ll(M, r0, r0, r0, r0 + n1, n1, n2)
    trsm_ru(M, r0, r0, r0 + n1, r0, n1, n2)
    gemm_sub(M, r0 + n1, r0 + n1, r0 + n1, r0, r0, r0 + n1, n2, n2, n1)
    _lu(M, r0 + n1, n2)


def lu(comps):
    """Factors of the library's LU (packed: U on and above the diagonal, L
    strictly below) as q component arrays."""
    M = Matrix(comps)
    _lu(M, 0, M.n)
    return M.comps()


def lu_solve(lu_comps, b_comps):
    """Solve with packed factors: L y = b, then U x = y (same operations as
    the library's solve)."""
    n = lu_comps[0].shape[0]
    w = b_comps[0].shape[1]
    q = len(lu_comps)
    big = [np.zeros((n, n + w)) for _ in range(q)]
    for t in range(q):
        big[t][:, :n] = lu_comps[t]
        big[t][:, n:] = b_comps[t]
    M = Matrix(big)
    trsm_ll(M, 0, 0, 0, n, n, w)
    trsm_lu(M, 0, 0, 0, n, n, w)
    out = M.comps()
    return [np.asfortranarray(o[:, n:]) for o in out]
