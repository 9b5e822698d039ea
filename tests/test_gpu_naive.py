"""The paper's simple-matrix-multiplication baseline (ozmp_gemm_naive).

Not an exact product: it is checked against the exact product with the
error bound of recursive multi-component arithmetic, |err_ij| <= k * 2^-(wq
- 8) * sum_p |a_ip| |b_pj| (w = 53 for binary64 words, 24 for binary32),
and its components must be non-overlapping.
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import _clib
from oracle import exact as X
from ozmp_inputs import gen_problem

from _util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,q,w", [("dd", 2, 53), ("td", 3, 53), ("qd", 4, 53), ("ts", 3, 24)])
def test_naive_within_multicomponent_bound(prec, q, w):
    m, n, k = 37, 29, 100
    A, B = gen_problem(prec, m, n, k, phi=1.0, seed=21)
    dt = torch.float32 if prec == "ts" else torch.float64
    C = [torch.zeros((n, m), dtype=dt, device="cuda").T for _ in range(q)]
    oz.ozmp_gemm_naive(prec, to_dev(A), to_dev(B), C)
    torch.cuda.synchronize()
    Cg = from_dev(C)
    rows, cols = list(range(0, m, 3)), list(range(0, n, 3))
    ex = _clib.exact_block(A, B, rows, cols)
    Av, Bv = X.matrix_values(A), X.matrix_values(B)
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            got = sum(Fraction(float(c[i, j])) for c in Cg)
            err = abs(got - X.to_fraction(ex[a][b]))
            mag = sum(abs(X.to_fraction(Av[i][p]) * X.to_fraction(Bv[p][j])) for p in range(k))
            assert err <= k * mag * Fraction(1, 2 ** (w * q - 8))
            assert X.nonoverlapping([float(c[i, j]) for c in Cg], "f32" if prec == "ts" else "f64")
