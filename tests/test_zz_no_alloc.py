"""The allocation-free double-double entry point (ozmp_gemm_dd_noalloc).

It exists for callers that cannot call cudaMalloc (code under CUDA stream
capture, programs whose device memory belongs to a pool allocator, serving
loops that cannot pay for an allocation).  It must give the same result as
the regular entry point ozmp_gemm_dd, bit for bit -- the tolerance of every
product test here -- on consecutive calls that share its fixed scratch, and
must reject problems larger than the scratch.  This file is collected last
and passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from ozmp_inputs import gen_problem

pytestmark = pytest.mark.gpu


def _dd(m, n, k, seed):
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=seed)
    return [oz.colmajor(a) for a in A], [oz.colmajor(b) for b in B]


def _zeros(m, n):
    return [torch.zeros((n, m), dtype=torch.float64, device="cuda").T for _ in range(2)]


def test_noalloc_matches_regular_entry_point_on_two_calls():
    # a larger problem first, then a smaller one: the second call must not
    # see anything the first left in the shared scratch
    for (m, n, k, seed) in [(300, 260, 200, 31), (130, 70, 90, 32)]:
        A, B = _dd(m, n, k, seed)
        ref = _zeros(m, n)
        oz.ozmp_set_stream(torch.cuda.current_stream())
        oz.ozmp_set_form(oz.Form.AUTO)
        oz.ozmp_gemm_dd(A, B, ref, 0)
        got = _zeros(m, n)
        oz.ozmp_gemm_dd_noalloc(A, B, got, 0, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert torch.equal(g, r)


def test_noalloc_rejects_problems_beyond_the_scratch():
    h = oz.ozmp_plan_create(oz.Prec.DD, 1024, 1024, 1024, oz.Form.AUTO, 0, None)
    need = oz.ozmp_plan_get_info(h).workspace_bytes
    oz.ozmp_plan_destroy(h)
    assert need > 64 * 2 ** 20
    A, B = _dd(1024, 1024, 1024, 33)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_dd_noalloc(A, B, _zeros(1024, 1024), 0, torch.cuda.current_stream())
    assert e.value.status == oz.Status.ERR_UNSUPPORTED
