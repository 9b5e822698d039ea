"""GPU parity for more than four binary64 components (and digit windows
wider than the register-resident splitter's), against the CPU oracle.

* exponents and every e4m3 digit (4-bit or balanced radix-32): bit-exact
  against oracle.ozaki.split / split_balanced;
* the product: bit-exact against the canonical q-component rounding of the
  oracle's exact Ozaki sum, on whole small problems and on sampled blocks of
  multi-tile ones (row and column exponents are maxima over the full k, so a
  block of rows and columns splits exactly as in the whole matrices);
* the error: ||C - C*||_F / ||C*||_F <= 2^(-50 q) against the exact product
  (Fractions; a 512-bit reference cannot resolve errors below 2^-512).
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import exact as X
from oracle import ozaki as O
from ozmp_inputs import gen_problem

from _util import digits_to_int, from_dev, to_dev

pytestmark = pytest.mark.gpu


def _gemm(q, m, n, k, seed, nslices=0, prec=None, form="fp8"):
    prec = prec or f"q{q}"
    A, B = gen_problem(prec, m, n, k, phi=1.0, seed=seed)
    Ad, Bd = to_dev(A), to_dev(B)
    C, p = oz.gemm(Ad, Bd, prec, form, nslices)
    torch.cuda.synchronize()
    assert p.status() == oz.Status.OK
    return A, B, from_dev(C), p, Ad, Bd


def _osplit(comps, form, beta, s):
    return O.split_balanced(comps, s) if form == "fp8bal" else O.split(comps, beta, s)


def _oproduct(A, B, info):
    return O.ozaki_product(A, B, info.beta, info.nslices, balanced=(info.form == oz.Form.FP8_BAL))


def _auto_slices(q, k, form):
    bits = 50 * q + max(0, (k - 1).bit_length()) + 16
    return -(-(bits + 1) // 5) if form == "fp8bal" else -(-bits // 4)


def _rows_cols(A, B, rows, cols):
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    return As, Bs


def _fraction_error(A, B, Cg, rows, cols):
    num, den = Fraction(0), Fraction(0)
    for i in rows:
        for j in cols:
            ex = X.exact_product_fraction(A, B, i, j)
            got = sum((Fraction(float(c[i, j])) for c in Cg), Fraction(0))
            num += (got - ex) ** 2
            den += ex * ex
    return num, den


@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
@pytest.mark.parametrize("q,m,n,k", [(5, 70, 60, 50), (8, 70, 60, 50), (16, 40, 36, 30)])
def test_split_bit_exact(q, m, n, k, form):
    A, B = gen_problem(f"q{q}", m, n, k, phi=1.0, seed=21 + q)
    p = oz.Plan(q, m, n, k, form, _auto_slices(q, k, form))
    p.split(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    i = p.info
    assert i.nslices == _auto_slices(q, k, form)
    E, F = [t.cpu().numpy() for t in p.exponents()]
    ga, gb = [t.cpu().numpy() for t in p.digits()]
    Eo, dA = _osplit(A, form, i.beta, i.nslices)
    Fo, dB = _osplit([np.asfortranarray(b.T) for b in B], form, i.beta, i.nslices)
    assert list(E) == Eo and list(F) == Fo
    np.testing.assert_array_equal(digits_to_int(ga[:, :m, :k], form), dA)
    np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], form), dB)
    assert not digits_to_int(ga[:, m:, :], form).any() and not digits_to_int(ga[:, :, k:], form).any()
    assert not digits_to_int(gb[:, n:, :], form).any() and not digits_to_int(gb[:, :, k:], form).any()


@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
@pytest.mark.parametrize("q,m,n,k", [(5, 70, 60, 50), (8, 50, 40, 36), (16, 24, 20, 18)])
def test_product_bit_exact_and_within_target(q, m, n, k, form):
    A, B, Cg, p, _, _ = _gemm(q, m, n, k, seed=40 + q, form=form)
    i = p.info
    r = _oproduct(A, B, i)
    for a in range(m):
        for b in range(n):
            assert [float(c[a, b]) for c in Cg] == X.to_components(r["S"][a][b], q, "f64"), (a, b)
    rows, cols = list(range(0, m, max(1, m // 6))), list(range(0, n, max(1, n // 6)))
    num, den = _fraction_error(A, B, Cg, rows, cols)
    assert num <= den * Fraction(1, 2 ** (100 * q))


@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
def test_multi_tile_q8_sampled_blocks(form):
    # 300 x 520 x 260: two row tiles, three column tiles, ragged in every direction
    q, m, n, k = 8, 300, 520, 260
    A, B, Cg, p, _, _ = _gemm(q, m, n, k, seed=77, form=form)
    i = p.info
    rows, cols = [0, 1, 127, 128, 255, 256, 299], [0, 255, 256, 300, 511, 519]
    As, Bs = _rows_cols(A, B, rows, cols)
    r = _oproduct(As, Bs, i)
    for a_i, a in enumerate(rows):
        for b_j, b in enumerate(cols):
            assert [float(c[a, b]) for c in Cg] == X.to_components(r["S"][a_i][b_j], q, "f64"), (a, b)
    num, den = _fraction_error(A, B, Cg, rows[:4], cols[:4])
    assert num <= den * Fraction(1, 2 ** (100 * q))


@pytest.mark.parametrize("form,s", [("fp8", 120), ("fp8bal", 100)])
def test_wide_window_with_few_components(form, s):
    # DD with more slices than the register splitter writes (64 four-bit,
    # 63 balanced): the many-component splitter
    m, n, k = 130, 140, 100
    A, B, Cg, p, _, _ = _gemm(2, m, n, k, seed=5, nslices=s, prec="dd", form=form)
    i = p.info
    assert i.nslices == s
    rows, cols = [0, 17, 64, 129], [0, 33, 127, 139]
    As, Bs = _rows_cols(A, B, rows, cols)
    r = _oproduct(As, Bs, i)
    for a_i, a in enumerate(rows):
        for b_j, b in enumerate(cols):
            assert [float(c[a, b]) for c in Cg] == X.to_components(r["S"][a_i][b_j], 2, "f64"), (a, b)


def test_plain_entry_point_matches_plan():
    q, m, n, k = 6, 90, 70, 80
    A, B, Cg, p, Ad, Bd = _gemm(q, m, n, k, seed=3, form="auto")
    assert p.info.form == oz.Form.FP8_BAL
    C2 = [torch.empty((n, m), dtype=torch.float64, device="cuda").T for _ in range(q)]
    oz.ozmp_gemm_md(Ad, Bd, C2)
    torch.cuda.synchronize()
    assert oz.ozmp_last_status() == oz.Status.OK
    for x, y in zip(from_dev(C2), Cg):
        assert np.array_equal(x, y)


def test_many_components_need_the_tcgen05_form():
    with pytest.raises(oz.OzmpError) as e:
        oz.Plan(5, 64, 64, 64, "int8", 0)
    assert e.value.status == oz.Status.ERR_UNSUPPORTED
