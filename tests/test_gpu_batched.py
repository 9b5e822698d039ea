"""Batched products (ozmp_gemm_batched) against single products.

Every product is exact up to one canonical rounding, so a batched result
must equal the single-problem result bit for bit, whatever tile widths the
autotuner chose and however the persistent schedule ordered the tiles.  A
second call reuses the plan with new data and new pointers.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from ozmp_inputs import batched_problem_shapes, gen_problem

from _util import to_dev

pytestmark = pytest.mark.gpu


def _make(shapes, seed0):
    out = []
    for idx, (m, n, k, prec) in enumerate(shapes):
        A, B = gen_problem(prec, m, n, k, phi=1.0, seed=seed0 + idx)
        dt = torch.float32 if prec == "ts" else torch.float64
        q = len(A)
        C = [torch.full((n, m), 7.0, dtype=dt, device="cuda").T for _ in range(q)]
        out.append((prec, to_dev(A) if k > 0 else [oz.colmajor(np.zeros((m, 0)))] * q,
                    to_dev(B) if k > 0 else [oz.colmajor(np.zeros((0, n)))] * q, C, 0))
    return out


def _single(prec, A, B, form):
    # a batch takes the precision's automatic count (no data-dependent choice
    # inside a graph): the single product with that count forced
    m, k = A[0].shape
    n = B[0].shape[1]
    s0 = oz.Plan(prec, m, n, k, form, 0, workspace=False).info.nslices
    C, p = oz.gemm(A, B, prec, form, s0)
    return C


@pytest.mark.parametrize("form", ["fp8", "fp8bal", "int8"])
def test_batched_equals_single_products(form):
    shapes = batched_problem_shapes(24, seed=1, lo=16, hi=300)
    shapes += [(70, 40, 0, "dd"), (0, 5, 9, "td"), (33, 290, 45, "qd"), (130, 260, 70, "ts"), (1, 1, 1, "dd")]
    probs = _make(shapes, 1000)
    plan = oz.ozmp_gemm_batched(probs, oz.FORM_BY_NAME[form])
    torch.cuda.synchronize()
    assert oz.ozmp_plan_get_status(plan) == oz.Status.OK
    for (prec, A, B, C, ns), (m, n, k, _) in zip(probs, shapes):
        if m == 0 or n == 0:
            continue
        if k == 0:
            assert all(float(c.abs().max()) == 0.0 for c in C)
            continue
        ref = _single(prec, A, B, form)
        for x, y in zip(C, ref):
            assert torch.equal(x, y), (prec, m, n, k)
    # replay with new data and new pointers
    probs2 = _make(shapes, 5000)
    plan2 = oz.ozmp_gemm_batched(probs2, oz.FORM_BY_NAME[form], plan=plan)
    torch.cuda.synchronize()
    for (prec, A, B, C, ns), (m, n, k, _) in zip(probs2, shapes):
        if m == 0 or n == 0 or k == 0:
            continue
        ref = _single(prec, A, B, form)
        for x, y in zip(C, ref):
            assert torch.equal(x, y), (prec, m, n, k)
    oz.ozmp_plan_destroy(plan)


def test_batched_plan_rejects_a_different_batch():
    shapes = [(40, 30, 20, "dd"), (20, 30, 40, "td")]
    probs = _make(shapes, 7)
    plan = oz.ozmp_gemm_batched(probs)
    other = _make([(41, 30, 20, "dd"), (20, 30, 40, "td")], 8)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_batched(other, plan=plan)
    assert e.value.status == oz.Status.ERR_INVALID_ARG
    # nor another digit form (the automatic one is the balanced radix-32 form here)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_batched(probs, oz.Form.FP8, plan=plan)
    assert e.value.status == oz.Status.ERR_INVALID_ARG
    oz.ozmp_plan_destroy(plan)


def test_batched_rejects_more_than_four_components_and_wide_windows():
    probs = _make([(40, 30, 20, "q5")], 3)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_batched(probs)
    assert e.value.status == oz.Status.ERR_UNSUPPORTED
    probs = _make([(40, 30, 20, "dd")], 3)
    probs = [(p[0], p[1], p[2], p[3], 120) for p in probs]     # beta s = 480 bits
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_batched(probs)
    assert e.value.status == oz.Status.ERR_UNSUPPORTED


@pytest.mark.parametrize("split,defer", [("1", "1"), ("0", "1"), ("1", "0")])
def test_few_large_problems_split_into_pair_ranges(split, defer, monkeypatch):
    # a batch of few tiles: the autotuner splits the tiles' pair walks into
    # chunks that add exactly into limb slots (OZMP_BATCH_SPLIT=0: whole
    # tiles); the split tiles are rounded by the rounding pass, or with
    # OZMP_BATCH_DEFER=0 by the last chunk to finish; every way the results
    # equal the single products bit for bit
    monkeypatch.setenv("OZMP_BATCH_SPLIT", split)
    monkeypatch.setenv("OZMP_BATCH_DEFER", defer)
    shapes = [(520, 600, 300, "dd"), (260, 300, 200, "td"), (130, 70, 90, "qd")]
    probs = _make(shapes, 300)
    plan = oz.ozmp_gemm_batched(probs)
    torch.cuda.synchronize()
    assert oz.ozmp_plan_get_status(plan) == oz.Status.OK
    for (prec, A, B, C, ns), (m, n, k, _) in zip(probs, shapes):
        ref = _single(prec, A, B, "auto")
        for x, y in zip(C, ref):
            assert torch.equal(x, y), (prec, m, n, k)
    oz.ozmp_plan_destroy(plan)


def test_batched_512_problems_sampled_against_the_oracle():
    # the batch of the benchmark (512 DD/TD problems, m, n, k log-uniform in
    # [32, 768], seed 1), run as one graph; 8 DD and 8 TD problems are
    # checked on a block of up to 32 x 32 entries (full k): bit for bit
    # against the canonical rounding of the oracle's exact Ozaki sum with the
    # automatic slice count, and within the precision's target against the
    # exact product rounded to 512 bits
    from oracle import _clib
    from oracle import exact as X
    from oracle import ozaki as O

    shapes = batched_problem_shapes(512, seed=1)
    host, probs = [], []
    for idx, (m, n, k, prec) in enumerate(shapes):
        A, B = gen_problem(prec, m, n, k, phi=1.0, seed=1000 + idx)
        host.append((A, B))
        C = [torch.full((n, m), 7.0, dtype=torch.float64, device="cuda").T for _ in A]
        probs.append((prec, to_dev(A), to_dev(B), C, 0))
    plan = oz.ozmp_gemm_batched(probs)
    torch.cuda.synchronize()
    assert oz.ozmp_plan_get_status(plan) == oz.Status.OK
    rng = np.random.default_rng(11)
    picks = []
    for want in ("dd", "td"):
        idx = [i for i, s in enumerate(shapes) if s[3] == want]
        picks += list(rng.choice(idx, 8, replace=False))
    target = {"dd": 2.0 ** -100, "td": 2.0 ** -150}
    for idx in picks:
        m, n, k, prec = shapes[idx]
        A, B = host[idx]
        q = len(A)
        rows = sorted(set(np.linspace(0, m - 1, min(m, 32)).astype(int).tolist()))
        cols = sorted(set(np.linspace(0, n - 1, min(n, 32)).astype(int).tolist()))
        info = oz.Plan(prec, m, n, k, "auto", 0, workspace=False).info
        assert info.form == oz.Form.FP8_BAL
        r = O.ozaki_product([a[rows] for a in A], [b[:, cols] for b in B], info.beta, info.nslices,
                            balanced=True)
        Cg = [c.cpu().numpy() for c in probs[idx][3]]
        for a, i in enumerate(rows):
            for b, j in enumerate(cols):
                got = [float(c[i, j]) for c in Cg]
                assert got == X.to_components(r["S"][a][b], q), (idx, prec, m, n, k, i, j)
        ex = _clib.exact_block(A, B, rows, cols)
        chat = [[[float(c[i, j]) for c in Cg] for j in cols] for i in rows]
        err = X.error_metrics(chat, ex)["err_nw"]
        assert err <= target[prec], (idx, prec, m, n, k, err)
    oz.ozmp_plan_destroy(plan)
