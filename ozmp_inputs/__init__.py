"""Seeded synthetic operands for the Ozaki-scheme product C = A*B.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle.  It holds no arithmetic of the method itself: it only draws random
matrices with the distribution of the paper's test matrices (Sec. 1, Eq. 1:
a_ij = (ru - 0.5) * exp(rn), ru ~ U[0,1), rn ~ N(0,1)) and extends them to
multi-component operands.

Generator definition (the recipe every test and benchmark uses):

* RNG: ``numpy.random.default_rng(seed)`` (PCG64).
* Draw order: operand A, then operand B.  For each operand: one U matrix,
  one N matrix, then one V matrix per tail component.  Every matrix is drawn
  as a flat vector and laid out column-major (the BLAS convention of the
  problem statement), so element (i, j) of an r x c matrix is draw i + j*r.
* Head component: ``(U - 0.5) * exp(phi * N)`` in float64; ``phi`` is the
  exponent spread (phi = 1 is Eq. 1).
* Tail component t >= 1: ``RN64(c_{t-1} * 2^-53 * V_t)`` with
  ``V_t ~ U(-1, 1)`` (the scaling by 2^-53 is exact, so one rounding).
* Triple-single (TS): head ``float32((U - 0.5) * exp(phi * N))`` and tail
  ``float32(float64(c_{t-1}) * 2^-24 * V_t)``.

Components are returned as a list of separate column-major arrays (one per
component), which is the layout of the C ABI.
"""
from __future__ import annotations

import numpy as np

__all__ = ["PRECISIONS", "components_of", "gen_operand", "gen_problem",
           "batched_problem_shapes", "digit_matrix"]

#: number of components and component dtype for each precision; "q<N>" is
#: N binary64 components (q2/q3/q4 draw exactly as dd/td/qd)
PRECISIONS = {
    "dd": (2, np.float64),
    "td": (3, np.float64),
    "qd": (4, np.float64),
    "ts": (3, np.float32),
}
PRECISIONS.update({f"q{q}": (q, np.float64) for q in range(2, 17)})


def components_of(prec: str):
    return PRECISIONS[prec]


def _colmajor(vec, rows, cols):
    return np.asfortranarray(vec.reshape(cols, rows).T)


def gen_operand(rng, prec: str, rows: int, cols: int, phi: float = 1.0):
    """Draw one multi-component operand (list of column-major arrays)."""
    q, dt = PRECISIONS[prec]
    n = rows * cols
    u = rng.random(n)
    nrm = rng.standard_normal(n)
    head = (u - 0.5) * np.exp(phi * nrm)
    if dt == np.float32:
        comps = [head.astype(np.float32)]
        scale = 2.0 ** -24
    else:
        comps = [head]
        scale = 2.0 ** -53
    for _ in range(1, q):
        v = rng.uniform(-1.0, 1.0, n)
        prev = comps[-1].astype(np.float64)
        nxt = (prev * scale) * v
        comps.append(nxt.astype(dt))
    return [_colmajor(c, rows, cols) for c in comps]


def gen_problem(prec: str, m: int, n: int, k: int, phi: float = 1.0, seed: int = 0):
    """A (m x k) and B (k x n) drawn from one generator: A first, then B."""
    rng = np.random.default_rng(seed)
    a = gen_operand(rng, prec, m, k, phi)
    b = gen_operand(rng, prec, k, n, phi)
    return a, b


def batched_problem_shapes(count: int = 512, seed: int = 1, lo: int = 32, hi: int = 768):
    """Uneven batched workload: per problem draw (m, n, k, prec) in that order.

    m, n, k = round(exp(U(ln lo, ln hi))); precision DD if U < 0.5 else TD.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dims = [int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi)))))) for _ in range(3)]
        prec = "dd" if rng.random() < 0.5 else "td"
        out.append((dims[0], dims[1], dims[2], prec))
    return out


def digit_matrix(rng, rows: int, cols: int, dmax: int):
    """Uniform random small integers in [-dmax, dmax] (int64, column-major)."""
    return _colmajor(rng.integers(-dmax, dmax + 1, rows * cols), rows, cols)
