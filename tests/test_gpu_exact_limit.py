"""Exactness of the e4m3 slice products at the limit of their binary32
accumulator.

Every slice product must be error-free (Sec. 3, Algorithm 1).  The e4m3
forms multiply small-integer digits on the tensor cores and accumulate them
in binary32, which holds every integer up to 2^24 exactly; the plan drains
the accumulator after `pairs_per_drain` slice pairs, the most for which
pairs * k * max|d|^2 <= 2^24.  Random Eq. 1 operands stay orders of
magnitude below that bound, so these tests build operands whose digits are
chosen in advance: every digit at or next to its largest magnitude and
every product of a drain's pairs with one sign.  A drain then sums to just
under 2^24 (up to exactly 2^24 for balanced digits), with odd low bits.

An element with the digits d_1 .. d_s is the exact value
  balanced radix-32 digits: x = sum_t d_t 2^(2 - 5 t)  (|x| in [1, 2), E = 1),
  4-bit digits:             x = sum_t d_t 2^(1 - 4 t)  (|x| in [1, 2), E = 1),
so its truncated split is exactly these digits; groups of 10 (12) digits
are one binary64 component each.  The test checks that the library's
splitter writes those digits, that the oracle's splitter finds them too,
and that every diagonal T_d = sum_{t+u=d} A_t B_u^T of ozmp_plan_diagonal
equals the oracle's exact int64 slice products, element by element, on
the CTA-pair tile, the single-CTA tile and the mma.sync (QMMA) engine, at a
k with many pairs per drain and at the form's largest k (one pair per
drain); and the same for binary16 digits of beta = 6 bits on kind::f16.
"""
import os
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import ozaki as O

from _util import E4M3

pytestmark = pytest.mark.gpu

# e4m3 code of each digit value (the non-zero digits here have one code each)
ENC = np.zeros(64, np.uint8)
for _b in range(128):
    _v = E4M3[_b]
    if _v == int(_v) and 1 <= _v <= 16:
        ENC[32 + int(_v)] = _b
        ENC[32 - int(_v)] = _b | 0x80


def _digits(rng, s, rows, k, balanced, beta=4):
    """Digits (s, rows, k) int16 at their largest magnitudes, one sign pattern.

    Balanced radix-32: top digit 16 and the others in {-16, -15} (mostly -16;
    the negative rest keeps |x| below 2).  Products of two non-top digits are
    then +256, +240 or +225.  beta-bit digits: all in {2^beta - 2,
    2^beta - 1} (mostly the largest), products up to (2^beta - 1)^2."""
    d = np.empty((s, rows, k), np.int16)
    if balanced:
        d[0] = 16
        for t in range(1, s):
            d[t] = np.where(rng.random((rows, k)) < 0.85, -16, -15)
    else:
        top = (1 << beta) - 1
        for t in range(s):
            d[t] = np.where(rng.random((rows, k)) < 0.75, top, top - 1)
    return d


def _group(balanced, beta):
    """Digits per binary64 component."""
    return 10 if balanced else 52 // beta


def _components(d, balanced, q, beta=4):
    """Exact binary64 components (q arrays rows x k) of the values whose
    digits are d: groups of g digits, each group one component."""
    s = d.shape[0]
    g = _group(balanced, beta)
    assert s == g * q
    radix, bits, e0 = (32, 5, 2) if balanced else (1 << beta, beta, 1)
    comps = []
    for c in range(q):
        acc = np.zeros(d.shape[1:], np.int64)
        for t in range(c * g, (c + 1) * g):
            acc = acc * radix + d[t].astype(np.int64)
        t_last = (c + 1) * g                      # 1-based index of the group's last digit
        comps.append(np.ldexp(acc.astype(np.float64), e0 - bits * t_last))   # |acc| < 2^51: exact
    return comps


CASES = [
    # id, q, form, m, n, k, single-CTA tile by environment
    ("bal-pair-k2048", 4, "fp8bal", 256, 200, 2048, False),
    ("bal-single-k2048", 4, "fp8bal", 256, 200, 2048, True),
    ("bal-pair-kmax", 2, "fp8bal", 256, 72, 65536, False),
    ("bal-single-kmax", 2, "fp8bal", 128, 72, 65536, False),     # 128 rows: single-CTA tile
    ("fp8-pair-k2048", 4, "fp8", 256, 200, 2048, False),
    ("fp8-single-kmax", 2, "fp8", 256, 72, 74565, True),
    ("qmma-k2048", 4, "fp8mma", 256, 200, 2048, False),
    ("qmma-kmax", 2, "fp8mma", 128, 72, 74565, False),
    # binary16 digits on kind::f16: beta = 6 at k = 2048 (two pairs a drain)
    # and at k = 4096 (one pair a drain, 4096 * 63^2 = 0.97 * 2^24)
    ("fp16-pair-k2048", 4, "fp16", 256, 200, 2048, False),
    ("fp16-single-k4096", 2, "fp16", 128, 72, 4096, False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_diagonals_exact_at_the_accumulator_limit(case):
    name, q, form, m, n, k, single = case
    balanced = form == "fp8bal"
    beta = O.beta_fp32(k) if form == "fp16" else (5 if balanced else 4)
    s = _group(balanced, beta) * q
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    dA = _digits(rng, s, m, k, balanced, beta)
    dB = _digits(rng, s, n, k, balanced, beta)
    A = _components(dA, balanced, q, beta)
    Bt = _components(dB, balanced, q, beta)           # rows of Bt = columns of B
    old = os.environ.get("OZMP_TC_PAIR")
    if single:
        os.environ["OZMP_TC_PAIR"] = "0"
    try:
        p = oz.Plan(f"q{q}" if q > 4 else {2: "dd", 4: "qd"}[q], m, n, k, form, s)
    finally:
        if single:
            if old is None:
                del os.environ["OZMP_TC_PAIR"]
            else:
                os.environ["OZMP_TC_PAIR"] = old
    i = p.info
    dmax2 = 256 if balanced else ((1 << beta) - 1) ** 2
    assert i.nslices == s and i.beta == beta and i.pairs_per_drain == (2 ** 24) // (k * dmax2)
    # the drains reach the binary32 limit: pairs_per_drain full pairs of the
    # largest products come to within 8 % of 2^24
    assert i.pairs_per_drain * k * dmax2 > 0.92 * 2 ** 24
    Ad = [oz.colmajor(a) for a in A]
    Bd = [oz.colmajor(np.asfortranarray(b.T)) for b in Bt]
    p.split(Ad, Bd)
    torch.cuda.synchronize()
    E, F = [t.cpu().numpy() for t in p.exponents()]
    assert (E == 1).all() and (F == 1).all()
    ga, gb = p.digits()
    # the library's digits are the chosen ones (e4m3 codes, or binary16 values)
    for t in range(s):
        if form == "fp16":
            np.testing.assert_array_equal(ga[t, :m, :k].cpu().numpy().astype(np.int16), dA[t])
            np.testing.assert_array_equal(gb[t, :n, :k].cpu().numpy().astype(np.int16), dB[t])
        else:
            np.testing.assert_array_equal(ga[t, :m, :k].cpu().numpy(), ENC[dA[t].astype(np.intp) + 32])
            np.testing.assert_array_equal(gb[t, :n, :k].cpu().numpy(), ENC[dB[t].astype(np.intp) + 32])
    rows = sorted({0, 1, 127, m // 2 + 3, m - 1})
    cols = sorted({0, 1, n // 2, n - 1})
    # the oracle's splitter finds the chosen digits as well (a sample)
    pc = slice(0, 96)
    sub = [a[rows][:, pc] for a in A]
    Eo, do = O.split_balanced(sub, s) if balanced else O.split(sub, beta, s)
    assert Eo == [1] * len(rows)
    np.testing.assert_array_equal(do, dA[:, rows][:, :, pc])
    # every diagonal against the oracle's exact slice products on sampled
    # rows and columns; three diagonals on whole row samples by exact float64
    # matrix products (integers below 2^53)
    To = O.slice_products(dA[:, rows].astype(np.int64), dB[:, cols].astype(np.int64))
    big = {2, s // 2 + 1, s + 1}
    rr = np.arange(0, m, max(1, m // 16))
    Af = dA[:, rr].astype(np.float64)
    Bf = dB.astype(np.float64)
    largest = 0
    for d in range(2, s + 2):
        T = p.diagonal(d)
        torch.cuda.synchronize()
        Tg = T.cpu().numpy()
        np.testing.assert_array_equal(Tg[np.ix_(rows, cols)], To[d], err_msg=f"{name} d={d}")
        if d in big:
            ref = sum(Af[t - 1] @ Bf[d - t - 1].T for t in range(1, d) if d - t <= s)
            np.testing.assert_array_equal(Tg[rr], ref.astype(np.int64), err_msg=f"{name} d={d} rows")
        if d == s + 1:
            # the middle pairs' products (the largest of one sign)
            t = s // 2
            largest = int(np.max(Af[t - 1] @ Bf[s - t].T))
    assert i.pairs_per_drain * largest > 0.85 * 2 ** 24
