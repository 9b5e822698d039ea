"""The plain entry points' per-thread plan (ozmp_gemm_dd with ozmp_set_form).

The cached plan must follow the form the caller asks for: after a call in
one form, a call in another form of the same shape and slice count must run
in the new form.  With a forced small slice count the 4-bit and balanced
e4m3 digits give different (both canonical) results, so each call is
compared bit for bit with an explicit plan of the requested form.
"""
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from ozmp_inputs import gen_problem

pytestmark = pytest.mark.gpu


def _zeros(m, n):
    return [torch.zeros((n, m), dtype=torch.float64, device="cuda").T for _ in range(2)]


def test_thread_plan_follows_the_requested_form():
    m, n, k, s = 200, 300, 260, 8
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=41)
    Ad, Bd = [oz.colmajor(a) for a in A], [oz.colmajor(b) for b in B]
    ref = {}
    for form in ("fp8bal", "fp8"):
        C, _ = oz.gemm(Ad, Bd, "dd", form, s)
        ref[form] = C
    torch.cuda.synchronize()
    assert not all(torch.equal(a, b) for a, b in zip(ref["fp8bal"], ref["fp8"]))
    oz.ozmp_set_stream(torch.cuda.current_stream())
    try:
        for form, want in [(oz.Form.AUTO, "fp8bal"), (oz.Form.FP8, "fp8"), (oz.Form.FP8_BAL, "fp8bal"),
                           (oz.Form.FP8_BAL, "fp8bal"), (oz.Form.AUTO, "fp8bal"), (oz.Form.FP8, "fp8")]:
            oz.ozmp_set_form(form)
            C = _zeros(m, n)
            oz.ozmp_gemm_dd(Ad, Bd, C, s)
            torch.cuda.synchronize()
            # 8 slices are far from the 2^-100 target: the check says so
            assert oz.ozmp_last_status() == oz.Status.ERR_ACCURACY
            for g, r in zip(C, ref[want]):
                assert torch.equal(g, r), (form, want)
    finally:
        oz.ozmp_set_form(oz.Form.AUTO)
