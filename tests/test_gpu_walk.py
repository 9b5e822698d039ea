"""The two pair orders of the tcgen05 product kernel (csrc/walk.h) on the GPU.

The snake (two anti-diagonals interleaved, OZMP_TC_WALK=1) and the order of
one diagonal at a time (OZMP_TC_WALK=0) visit the same pairs of the triangle
t + u <= s + 1 (Sec. 3, Algorithm 1) and drain every accumulator group into
exact integer limbs, so the product must not depend on the order: both are
compared bit for bit with each other and, on sampled blocks, with the
oracle's exact Ozaki sum.  The shapes cover tail tiles split into pair-range
chunks, diagonals longer than one accumulator group (k = 8192: at most 8 or
9 pairs per group in e4m3 digits, 2 in binary16 ones), the single-CTA and
CTA-pair tile forms, the binary16
digits with the widest digit (beta = 10, drains that reach a limb before the
diagonal above them does), and the diagonal-only diagnostic launches.
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

from _util import digits_to_int, from_dev, to_dev

pytestmark = pytest.mark.gpu

Q = {"dd": 2, "td": 3, "qd": 4, "ts": 3}


def _gemm_both(monkeypatch, prec, form, A, B, pair="1"):
    monkeypatch.setenv("OZMP_TC_PAIR", pair)
    Ad, Bd = to_dev(A), to_dev(B)
    out = {}
    for walk in ("0", "1"):
        monkeypatch.setenv("OZMP_TC_WALK", walk)
        C, p = oz.gemm(Ad, Bd, prec, form, 0)
        torch.cuda.synchronize()
        assert p.status() == oz.Status.OK
        out[walk] = (C, p)
    for x, y in zip(out["0"][0], out["1"][0]):
        assert torch.equal(x, y)
    return out["1"]


def _sampled_oracle(A, B, C, p, prec, rows, cols):
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    # exponents are row/column maxima over k, so the sub-block split equals the full one
    r = O.ozaki_product(As, Bs, p.info.beta, p.info.nslices, balanced=(p.info.form == oz.Form.FP8_BAL))
    kind = "f32" if prec == "ts" else "f64"
    Cg = from_dev(C)
    for a_i, i in enumerate(rows):
        for b_j, j in enumerate(cols):
            assert [float(c[i, j]) for c in Cg] == X.to_components(r["S"][a_i][b_j], Q[prec], kind), (i, j)


@pytest.mark.parametrize("pair", ["1", "0"])
@pytest.mark.parametrize("form", ["fp8bal", "fp8"])
def test_walks_agree_on_split_tail_tiles(form, pair, monkeypatch):
    # 2560 x 2048: a wave of whole tiles plus tail tiles in pair-range chunks
    m, n, k = 2560, 2048, 192
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=21)
    C, p = _gemm_both(monkeypatch, "dd", form, A, B, pair)
    _sampled_oracle(A, B, C, p, "dd", list(range(0, m, 509)), list(range(0, n, 401)))


@pytest.mark.parametrize("prec,form", [("dd", "fp8bal"), ("dd", "fp8"), ("qd", "fp8bal"), ("dd", "fp16")])
def test_walks_agree_with_diagonals_longer_than_a_group(prec, form, monkeypatch):
    # k = 8192: a binary32 accumulator holds at most 2^24 / (8192 dmax^2) pairs,
    # fewer than the longest diagonals have, so the groups split inside them
    m, n, k = 512, 256, 8192
    A, B = gen_problem(prec, m, n, k, phi=1.0, seed=22)
    C, p = _gemm_both(monkeypatch, prec, form, A, B)
    if form != "fp16":
        assert p.info.nslices > 16
    _sampled_oracle(A, B, C, p, prec, [0, 131, 377, 511], [0, 97, 255])


@pytest.mark.parametrize("k", [10, 40])
def test_walks_agree_on_wide_binary16_digits(k, monkeypatch):
    # TS in binary16 digits at k = 10 (beta = 10) and 40 (beta = 9): drains of
    # neighbouring diagonals step by more than half a limb, so the snake can
    # write a limb before the diagonal above it has; full check against the oracle
    m, n = 300, 260
    A, B = gen_problem("ts", m, n, k, phi=1.0, seed=23)
    C, p = _gemm_both(monkeypatch, "ts", "fp16", A, B)
    assert p.info.beta == (10 if k == 10 else 9)
    _sampled_oracle(A, B, C, p, "ts", list(range(0, m, 7)), list(range(0, n, 5)))


@pytest.mark.parametrize("form", ["fp8bal", "fp16"])
def test_diagonals_in_the_snake_order(form, monkeypatch):
    # the diagnostic launches of one diagonal: with the snake a lone diagonal
    # alternates between the two accumulators; T_d must still be exact
    monkeypatch.setenv("OZMP_TC_WALK", "1")
    s = 16 if form == "fp8bal" else 11
    m, n, k = 200, 150, 130
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=24)
    p = oz.Plan("dd", m, n, k, form, s)
    p.split(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    # the oracle's digits (and the GPU's equal to them), then its exact products
    Bt = [np.asfortranarray(b.T) for b in B]
    if form == "fp8bal":
        (_, dA), (_, dB) = O.split_balanced(A, s), O.split_balanced(Bt, s)
    else:
        (_, dA), (_, dB) = O.split(A, p.info.beta, s), O.split(Bt, p.info.beta, s)
    ga, gb = [t.cpu().numpy() for t in p.digits()]
    np.testing.assert_array_equal(digits_to_int(ga[:, :m, :k], form), dA)
    np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], form), dB)
    T = O.slice_products(dA, dB)
    for d in sorted({2, 3, 4, s // 2 + 1, s + 1}):
        np.testing.assert_array_equal(p.diagonal(d).cpu().numpy(), T[d])
