"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a and loads, exports every entry point declared in include/ozmp.h,
validates arguments, and plans digit widths, slice counts and the exact
accumulation schedule as the paper's exactness condition requires."""
import os
import re

import pytest

import paper_2301_09960_gb300 as oz
from oracle import ozaki as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ozmp.h")).read()
    return sorted(set(re.findall(r"\b(ozmp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ["ozmp_gemm_dd", "ozmp_gemm_td", "ozmp_gemm_qd", "ozmp_gemm_ts", "ozmp_plan_create",
              "ozmp_plan_execute", "ozmp_plan_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol():
    L = oz.load()
    for s in declared_symbols():
        assert hasattr(L, s), s
    assert set(declared_symbols()) <= set(oz.SIGNATURES)
    assert "sm_103a" in oz.ozmp_version()


@pytest.mark.parametrize("form,beta", [("fp64", None), ("int8", 7), ("fp8", 4), ("fp8mma", 4)])
@pytest.mark.parametrize("k", [1, 128, 1000, 4096, 16384])
def test_plan_digit_width_and_schedule(form, beta, k):
    h = oz.ozmp_plan_create(oz.Prec.QD, 300, 200, k, oz.FORM_BY_NAME[form], 0, None)
    try:
        i = oz.ozmp_plan_get_info(h)
        b = O.beta_fp64(k) if form == "fp64" else beta
        assert i.beta == b
        dmax = 15 if form.startswith("fp8") else 2 ** b - 1
        limit = {"fp64": 2 ** 53, "int8": 2 ** 31 - 1, "fp8": 2 ** 24, "fp8mma": 2 ** 24}[form]
        # pairs summed in the tensor-core accumulator stay exact
        assert i.pairs_per_drain * k * dmax ** 2 <= limit < (i.pairs_per_drain + 1) * k * dmax ** 2
        assert i.npairs == i.nslices * (i.nslices + 1) // 2
        assert i.mp % 128 == 0 and i.np % (256 if form == "fp8" else 128) == 0 and i.kp % 128 == 0 and i.kp >= k
        # slice count from the target 2^-200 with log2(k) + 16 guard bits
        import math
        want = math.ceil((200 + math.ceil(math.log2(k)) + 16) / b)
        want = min(want, 36 if form == "int8" else 64)
        while want * b > 376:
            want -= 1
        assert i.nslices == want
        assert 1 <= i.ngroups <= i.nslices
        assert i.workspace_bytes >= i.nslices * (i.mp + i.np) * i.kp * i.digit_bytes
    finally:
        oz.ozmp_plan_destroy(h)


def test_plan_rejects_bad_arguments():
    for args in [(1, 10, 10, 10, 0, 0), (17, 10, 10, 10, 0, 0), (102, 10, 10, 10, 0, 0), (2, -1, 10, 10, 0, 0),
                 (2, 10, 10, 10, 9, 0), (2, 10, 10, 10, 0, 257)]:
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_create(*args, None)
        assert e.value.status == oz.Status.ERR_INVALID_ARG
    # valid arguments beyond a form's limits
    for args in [(2, 10, 10, 10, oz.Form.FP8, 240), (2, 10, 10, 10, oz.Form.FP8_MMA, 65),
                 (2, 10, 10, 10, oz.Form.INT8, 37), (5, 10, 10, 10, oz.Form.INT8, 0), (5, 10, 10, 10, oz.Form.FP64, 0)]:
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_create(*args, None)
        assert e.value.status == oz.Status.ERR_UNSUPPORTED
    # binary32 accumulation of e4m3 digits is exact only up to k = 2^24 / 225
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_plan_create(oz.Prec.DD, 8, 8, 80000, oz.Form.FP8, 0, None)
    assert e.value.status == oz.Status.ERR_UNSUPPORTED
    h = oz.ozmp_plan_create(oz.Prec.DD, 8, 8, 74565, oz.Form.FP8, 0, None)
    oz.ozmp_plan_destroy(h)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 8, 12, 16])
def test_component_count_plans(q):
    # q binary64 components: target 2^(-50 q) -> s = ceil((50 q + log2 k + 16) / 4) e4m3 digits,
    # the accumulator holds every diagonal's weight, and more than 4 components
    # take the tcgen05 form only
    k = 1000
    h = oz.ozmp_plan_create(q, 300, 200, k, oz.Form.FP8, 0, None)
    try:
        i = oz.ozmp_plan_get_info(h)
        assert i.form == oz.Form.FP8 and i.beta == 4
        assert i.nslices == -(-(50 * q + 10 + 16) // 4)
        assert i.nslices * 4 + 65 <= 1024
        top_bits = 4 * (i.nslices - 1) + 20 + 8 + 2      # weight of diagonal 2, the sum of s + 1 terms, sign
        assert 64 * i.acc_words >= top_bits
    finally:
        oz.ozmp_plan_destroy(h)


def test_timing_ring_argument_checks():
    # no CUDA call is made on these paths
    for bad in (-1, 4097):
        h = oz.ozmp_plan_create(oz.Prec.DD, 64, 64, 64, oz.Form.FP8, 0, None)
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_set_timing(h, bad)
        assert e.value.status == oz.Status.ERR_INVALID_ARG
        oz.ozmp_plan_set_timing(h, 0)
        assert oz.ozmp_plan_read_timing(h, 4) == []
        oz.ozmp_plan_destroy(h)
    with pytest.raises(oz.OzmpError):
        oz.ozmp_plan_set_timing(None, 1)


def test_group_schedule_keeps_horner_value_below_2_62():
    for prec in (oz.Prec.DD, oz.Prec.QD):
        for form in (oz.Form.FP8, oz.Form.INT8, oz.Form.FP64):
            for k in (64, 4096, 16384):
                h = oz.ozmp_plan_create(prec, 128, 128, k, form, 0, None)
                i = oz.ozmp_plan_get_info(h)
                oz.ozmp_plan_destroy(h)
                s, b = i.nslices, i.beta
                dmax = 15 if form == oz.Form.FP8 else 2 ** b - 1
                tb = lambda d: (d - 1) * k * dmax ** 2
                # re-derive the greedy grouping and check every group's bound
                groups, cur, first, hb = 0, [], None, 0
                for d in range(s + 1, 1, -1):
                    if first is not None and hb + (tb(d) << (b * (first - d))) < 2 ** 62 and b * (first - d) < 62:
                        hb += tb(d) << (b * (first - d))
                    else:
                        groups += 1
                        first, hb = d, tb(d)
                    assert hb < 2 ** 62
                assert groups == i.ngroups
                # the exact accumulator holds the largest possible Ozaki sum
                total = sum(tb(d) << (b * (s + 1 - d)) for d in range(2, s + 2))
                assert total.bit_length() + 1 <= 64 * i.acc_words


@pytest.mark.parametrize("prec,k", [(oz.Prec.DD, 4096), (oz.Prec.TD, 1024), (oz.Prec.QD, 4096), (oz.Prec.TS, 8192),
                                    (oz.Prec.DD, 1)])
def test_balanced_digit_plans(prec, k):
    # balanced radix-32 e4m3 digits keep 5 s - 1 bits below 2^E: the same
    # target bits (50 q or 66, + log2 k + 16 guard bits) in about a fifth
    # fewer slices, a third fewer pairs; digits |d| <= 16, so a slice pair
    # of k terms reaches k 2^8 and a drain holds 2^24 / (k 2^8) pairs
    h = oz.ozmp_plan_create(prec, 300, 200, k, oz.Form.FP8_BAL, 0, None)
    try:
        i = oz.ozmp_plan_get_info(h)
        assert i.form == oz.Form.FP8_BAL and i.beta == 5 and i.digit_bytes == 1
        bits = (66 if prec == oz.Prec.TS else 50 * int(prec)) + max(0, (k - 1).bit_length()) + 16
        assert 5 * i.nslices - 1 >= bits > 5 * (i.nslices - 1) - 1
        assert i.pairs_per_drain == min(2 ** 24 // (k * 256), 2 ** 20)
        top_bits = 5 * (i.nslices - 1) + (k * 256).bit_length() + 8 + 2
        assert 64 * i.acc_words >= top_bits
    finally:
        oz.ozmp_plan_destroy(h)


def test_balanced_digit_limits():
    # windows of 5 s + 65 <= 1024 bits (the many-component splitter's 16
    # words), so s <= 191, for any component count
    for q, s in [(2, 63), (2, 64), (2, 191), (5, 0), (16, 0)]:
        h = oz.ozmp_plan_create(q, 10, 10, 10, oz.Form.FP8_BAL, s, None)
        oz.ozmp_plan_destroy(h)
    for args in [(2, 10, 10, 10, oz.Form.FP8_BAL, 192), (2, 8, 8, 70000, oz.Form.FP8_BAL, 0)]:
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_create(*args, None)
        assert e.value.status == oz.Status.ERR_UNSUPPORTED
    h = oz.ozmp_plan_create(oz.Prec.DD, 8, 8, 65536, oz.Form.FP8_BAL, 0, None)
    oz.ozmp_plan_destroy(h)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_plan_create(oz.Prec.DD, 8, 8, 8, 7, 0, None)
    assert e.value.status == oz.Status.ERR_INVALID_ARG


def test_automatic_form_choice():
    # balanced radix-32 digits up to their largest slice count, else 4-bit digits
    for q, ns, want in [(2, 0, oz.Form.FP8_BAL), (4, 63, oz.Form.FP8_BAL), (2, 191, oz.Form.FP8_BAL),
                        (2, 192, oz.Form.FP8), (5, 0, oz.Form.FP8_BAL), (16, 0, oz.Form.FP8_BAL),
                        (oz.Prec.TS, 0, oz.Form.FP8_BAL)]:
        h = oz.ozmp_plan_create(q, 64, 64, 64, oz.Form.AUTO, ns, None)
        try:
            assert oz.ozmp_plan_get_info(h).form == want, (q, ns)
        finally:
            oz.ozmp_plan_destroy(h)


def test_triple_single_slice_limits():
    # binary32 components go through the register splitter only: up to 63
    # balanced or 64 four-bit slices
    for form, s in [(oz.Form.FP8_BAL, 63), (oz.Form.FP8, 64)]:
        h = oz.ozmp_plan_create(oz.Prec.TS, 10, 10, 10, form, s, None)
        oz.ozmp_plan_destroy(h)
    for form, s in [(oz.Form.FP8_BAL, 64), (oz.Form.FP8, 65)]:
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_create(oz.Prec.TS, 10, 10, 10, form, s, None)
        assert e.value.status == oz.Status.ERR_UNSUPPORTED


@pytest.mark.parametrize("k", [1, 2, 3, 128, 1000, 2048, 4096, 8192, 16384, 2 ** 24])
@pytest.mark.parametrize("prec", [oz.Prec.DD, oz.Prec.QD, oz.Prec.TS])
def test_binary16_digit_plans(prec, k):
    # the binary32-slice form: beta is the largest width with k (2^beta - 1)^2
    # <= 2^24 (the oracle's beta_fp32, the paper's S = 24), held in binary16,
    # so at most 11 bits; two-byte digits; a drain holds 2^24 / (k (2^beta - 1)^2)
    # pairs; the fixed slice count covers the target bits + log2 k + 16 where
    # the splitter's limits allow
    h = oz.ozmp_plan_create(prec, 300, 200, k, oz.Form.FP16, 0, None)
    try:
        i = oz.ozmp_plan_get_info(h)
        beta = min(11, O.beta_fp32(k))
        assert i.form == oz.Form.FP16 and i.beta == beta and i.digit_bytes == 2
        assert i.pairs_per_drain == min(2 ** 24 // (k * (2 ** beta - 1) ** 2), 2 ** 20)
        bits = (66 if prec == oz.Prec.TS else 50 * int(prec)) + max(0, (k - 1).bit_length()) + 16
        # (at most 64 slices of at most 376 bits in all: the register splitter's limits)
        assert beta * i.nslices >= min(bits, beta * min(64, 376 // beta)) and i.nslices * beta <= 376
        assert i.np % 256 == 0     # the tcgen05 engine's tile width
    finally:
        oz.ozmp_plan_destroy(h)


def test_binary16_digit_limits():
    # no digit width fits beyond k = 2^24; the register splitter holds at
    # most 4 components and windows of beta s <= 376 bits
    for args in [(oz.Prec.DD, 8, 8, 2 ** 24 + 1, 0), (5, 8, 8, 64, 0), (oz.Prec.DD, 8, 8, 64, 377 // 9 + 1)]:
        with pytest.raises(oz.OzmpError) as e:
            oz.ozmp_plan_create(args[0], args[1], args[2], args[3], oz.Form.FP16, args[4], None)
        assert e.value.status == oz.Status.ERR_UNSUPPORTED, args
    h = oz.ozmp_plan_create(oz.Prec.DD, 8, 8, 64, oz.Form.FP16, 376 // 9, None)   # beta 9 at k = 64
    assert oz.ozmp_plan_get_info(h).beta == 9
    oz.ozmp_plan_destroy(h)
