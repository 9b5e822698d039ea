"""GPU parity of Algorithm 1 as printed (round-to-nearest binary64 slices,
binary64 slice products, exact sum) against oracle.ozaki.paper_literal.

* every slice of A and B: bit-exact (the extraction is a fixed sequence of
  binary64 round-to-nearest operations on exact remainders);
* the slice products without a rounded-remainder slice: bit-exact (their
  entries are integers below 2^53 at a common scale, so every summation
  order gives the exact value); those with one: within the binary64 GEMM
  bound 2 k u |A_a| |B_b| of the oracle's;
* C: the canonical rounding of the exact sum of the GPU's own products,
  bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import exact as X
from oracle import ozaki as O
from ozmp_inputs import gen_problem

from _util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,q,D", [("dd", 2, 3), ("dd", 2, 6), ("td", 3, 8), ("qd", 4, 11)])
def test_literal_matches_oracle(prec, q, D):
    m, n, k = 40, 36, 50
    A, B = gen_problem(prec, m, n, k, phi=1.0, seed=D)
    Ad, Bd = to_dev(A), to_dev(B)
    C = [torch.empty((n, m), dtype=torch.float64, device="cuda").T for _ in range(q)]
    SA = torch.empty((D, k, m), dtype=torch.float64, device="cuda")
    SB = torch.empty((D, n, k), dtype=torch.float64, device="cuda")
    npairs = D * (D + 1) // 2
    P = torch.empty((npairs, n, m), dtype=torch.float64, device="cuda")
    assert oz.ozmp_gemm_literal(Ad, Bd, C, D, SA, SB, P) == oz.Status.OK
    sa = SA.cpu().numpy().transpose(0, 2, 1)    # slice a: m x k
    sb = SB.cpu().numpy().transpose(0, 2, 1)    # slice b: k x n
    pg = P.cpu().numpy().transpose(0, 2, 1)     # product t: m x n
    Cg = from_dev(C)
    r = O.paper_literal(A, B, D)
    for a in range(D):
        np.testing.assert_array_equal(sa[a], r["A"][a])
        np.testing.assert_array_equal(sb[a], r["B"][a])
    u = 2.0 ** -53
    for t, (a, b) in enumerate(O.pairs(D)):
        want = r["prods"][(a, b)]
        if a < D and b < D:
            np.testing.assert_array_equal(pg[t], want)
        else:
            bound = 2 * k * u * (np.abs(r["A"][a - 1]) @ np.abs(r["B"][b - 1]))
            assert np.all(np.abs(pg[t] - want) <= bound), (a, b)
    for i in range(m):
        for j in range(n):
            s = (0, 0)
            for t in range(npairs):
                s = X.add(s, X.decode(pg[t][i, j]))
            assert [float(c[i, j]) for c in Cg] == X.to_components(s, q, "f64"), (i, j)


def test_literal_and_truncating_forms_reach_the_same_plateau():
    # at the paper's max-accuracy division count (DD: D = 6) both forms meet the
    # DD target against the exact product on a sampled block
    from fractions import Fraction
    m = n = k = 64
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=1)
    Ad, Bd = to_dev(A), to_dev(B)
    C1 = [torch.empty((n, m), dtype=torch.float64, device="cuda").T for _ in range(2)]
    assert oz.ozmp_gemm_literal(Ad, Bd, C1, 6) == oz.Status.OK
    C2, p = oz.gemm(Ad, Bd, "dd", "fp64", 6)
    torch.cuda.synchronize()
    for Cg in (from_dev(C1), from_dev(C2)):
        num, den = Fraction(0), Fraction(0)
        for i in range(0, m, 9):
            for j in range(0, n, 11):
                ex = X.exact_product_fraction(A, B, i, j)
                got = sum((Fraction(float(c[i, j])) for c in Cg), Fraction(0))
                num += (got - ex) ** 2
                den += ex * ex
        assert num <= den * Fraction(1, 2 ** 200)
