"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (tcgen05 CTA-pair tiles, dynamic item feed, split tail
tiles), on outputs the oracle computes one by one.

Row exponents are maxima over the full k of a row (column exponents over a
column), so a set of sampled rows of A and columns of B splits exactly as in
the whole matrices: the oracle's exact Ozaki sum on those rows and columns,
with the same slice count, is the exact value of the sampled elements.  The
GPU elements must equal its canonical rounding bit for bit, and the sampled
block's normwise error against the exact product (Fractions) must meet the
precision's target.
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

from _util import to_dev

pytestmark = pytest.mark.gpu

TARGET_BITS = {"dd": 100, "td": 150, "qd": 200, "ts": 66}
Q = {"dd": 2, "td": 3, "qd": 4, "ts": 3}


def _sampled(prec, form, m, n, k, phi, seed, rows, cols, err_rows, err_cols, nslices=0):
    A, B = gen_problem(prec, m, n, k, phi=phi, seed=seed)
    Ad, Bd = to_dev(A), to_dev(B)
    C, p = oz.gemm(Ad, Bd, prec, form, nslices)
    torch.cuda.synchronize()
    assert p.status() == oz.Status.OK
    i = p.info
    sel_r = torch.tensor(rows, device="cuda")
    sel_c = torch.tensor(cols, device="cuda")
    Cg = [c.index_select(0, sel_r).index_select(1, sel_c).cpu().numpy() for c in C]
    del C, Ad, Bd, p
    torch.cuda.empty_cache()
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    r = O.ozaki_product(As, Bs, i.beta, i.nslices, balanced=(i.form == oz.Form.FP8_BAL))
    kind = "f32" if prec == "ts" else "f64"
    for a in range(len(rows)):
        for b in range(len(cols)):
            got = [float(c[a, b]) for c in Cg]
            assert got == X.to_components(r["S"][a][b], Q[prec], kind), (rows[a], cols[b])
    num, den = Fraction(0), Fraction(0)
    for a in err_rows:
        for b in err_cols:
            ex = X.exact_product_fraction(As, Bs, a, b)
            got = sum((Fraction(float(c[a, b])) for c in Cg), Fraction(0))
            num += (got - ex) ** 2
            den += ex * ex
    assert num <= den * Fraction(1, 2 ** (2 * TARGET_BITS[prec]))
    return i


def test_dd_4096_headline():
    # the bench workload: DD 4096^3, phi = 1, in 4-bit e4m3 digits
    rows = [0, 1, 255, 256, 2047, 2048, 4094, 4095]
    cols = [0, 255, 256, 1000, 3071, 4095]
    i = _sampled("dd", "fp8", 4096, 4096, 4096, 1.0, 0, rows, cols, [0, 3, 7], [0, 5])
    assert i.nslices <= 32      # chosen from the data; the fixed rule ceil((100 + 12 + 16) / 4) is 32


def test_dd_4096_balanced_digits():
    # the same workload in balanced radix-32 e4m3 digits
    rows = [0, 1, 255, 256, 2047, 2048, 4094, 4095]
    cols = [0, 255, 256, 1000, 3071, 4095]
    i = _sampled("dd", "fp8bal", 4096, 4096, 4096, 1.0, 0, rows, cols, [0, 3, 7], [0, 5])
    assert i.nslices <= 26 and i.beta == 5      # the fixed rule gives 26


def test_qd_4096_balanced_digits():
    rows = [0, 300, 2048, 4095]
    cols = [1, 2049, 4095]
    i = _sampled("qd", "fp8bal", 4096, 4096, 4096, 1.0, 0, rows, cols, [0, 3], [0, 2])
    assert i.nslices <= 46      # the fixed rule gives 46


def test_qd_4096():
    rows = [0, 300, 2048, 4095]
    cols = [1, 2049, 4095]
    _sampled("qd", "fp8", 4096, 4096, 4096, 1.0, 0, rows, cols, [0, 3], [0, 2])


def test_dd_128_binary64_slices_every_element():
    # DD 128^3, head (U - 0.5) exp(0.5 N), binary64 slices: the whole C
    rows = list(range(128))
    cols = list(range(128))
    i = _sampled("dd", "fp64", 128, 128, 128, 0.5, 0, rows, cols, list(range(0, 128, 16)), list(range(0, 128, 16)))
    assert i.beta == 23


@pytest.mark.parametrize("prec", ["td", "qd"])
def test_td_qd_1024_binary64_slices(prec):
    rows = [0, 511, 512, 1023]
    cols = [0, 100, 1023]
    i = _sampled(prec, "fp64", 1024, 1024, 1024, 1.0, 0, rows, cols, [0, 3], [0, 2])
    assert i.beta == 21


@pytest.mark.slow
@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
def test_qd_8192_8192_16384(form):
    rows = [0, 4097, 8191]
    cols = [0, 8191]
    _sampled("qd", form, 8192, 8192, 16384, 1.0, 0, rows, cols, [0], [0, 1])


@pytest.mark.slow
@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
def test_ts_8192(form):
    rows = [0, 4096, 8191]
    cols = [7, 8191]
    _sampled("ts", form, 8192, 8192, 8192, 1.0, 0, rows, cols, [0, 2], [0, 1])


@pytest.mark.slow
@pytest.mark.parametrize("form,k", [("fp8bal", 65536), ("fp8", 74565)])
def test_k_at_the_exact_accumulation_limit(form, k):
    # the largest k of each e4m3 form: a slice product of k terms reaches
    # 2^24 (k 16^2 or k 15^2 rounded down), so every drain holds one pair
    rows = [0, 37, 63]
    cols = [0, 50, 95]
    i = _sampled("dd", form, 64, 96, k, 1.0, 0, rows, cols, [0, 2], [0, 2])
    assert i.pairs_per_drain == 1
