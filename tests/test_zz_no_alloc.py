"""The allocation-free double-double entry point (ozmp_gemm_dd_noalloc).

It serves callers that cannot call cudaMalloc: programs whose device memory
is all handed out by their own pool allocator (an allocation behind the
pool's back can fail, and cudaMalloc/cudaFree synchronise the device), and
plug-ins or real-time loops that may not allocate after start-up.  It must
give the same result as the regular entry point ozmp_gemm_dd, bit for bit --
the tolerance of every product test here -- on consecutive calls that share
its fixed scratch, and must reject exactly the problems whose whole-tile
workspace does not fit the scratch.  This file is collected last and passes
both alone in a fresh process and after the other tests.
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


def _auto_count(m, n, k):
    """The automatic slice count that nslices = 0 means here: the fixed rule
    (the regular entry point would choose from the data instead)."""
    h = oz.ozmp_plan_create(oz.Prec.DD, m, n, k, oz.Form.AUTO, 0, None)
    s = oz.ozmp_plan_get_info(h).nslices
    oz.ozmp_plan_destroy(h)
    return s


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
        oz.ozmp_gemm_dd(A, B, ref, _auto_count(m, n, k))
        got = _zeros(m, n)
        oz.ozmp_gemm_dd_noalloc(A, B, got, 0, torch.cuda.current_stream())
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert torch.equal(g, r)


SCRATCH = 64 * 2 ** 20


def _scratch_need(m, n, k):
    """Bytes the entry point needs: the whole-tile layout of a DD FORM_AUTO
    plan (exponents, both operands' digits, carry-save limbs), without the
    tile schedule and split-tile limbs of a regular plan's workspace."""
    h = oz.ozmp_plan_create(oz.Prec.DD, m, n, k, oz.Form.AUTO, 0, None)
    i = oz.ozmp_plan_get_info(h)
    oz.ozmp_plan_destroy(h)
    need = i.off_acc + (4 * i.acc_words + 1) * i.mp * i.np * 8
    return (need + 255) // 256 * 256, i.workspace_bytes


def test_noalloc_rejects_problems_beyond_the_scratch():
    need, ws = _scratch_need(1024, 1024, 1024)
    assert need > SCRATCH and ws > SCRATCH
    A, B = _dd(1024, 1024, 1024, 33)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_dd_noalloc(A, B, _zeros(1024, 1024), 0, torch.cuda.current_stream())
    assert e.value.status == oz.Status.ERR_UNSUPPORTED


def test_noalloc_limit_is_the_whole_tile_layout():
    # the largest m (multiple of 128, n = 512, k = 384) whose whole-tile
    # layout fits is accepted, whatever a regular plan's workspace (which adds
    # the tile schedule and split buffers) would be; the next row tile is
    # rejected
    n, k = 512, 384
    fit = None
    for m in range(128, 4096 + 1, 128):
        need, _ = _scratch_need(m, n, k)
        if need > SCRATCH:
            break
        fit = m
    assert fit is not None and m > fit
    m_fit = fit
    A, B = _dd(m_fit, n, k, 34)
    ref = _zeros(m_fit, n)
    oz.ozmp_set_stream(torch.cuda.current_stream())
    oz.ozmp_set_form(oz.Form.AUTO)
    oz.ozmp_gemm_dd(A, B, ref, _auto_count(m_fit, n, k))
    got = _zeros(m_fit, n)
    oz.ozmp_gemm_dd_noalloc(A, B, got, 0, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert torch.equal(g, r)
    A, B = _dd(m, n, k, 35)
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_gemm_dd_noalloc(A, B, _zeros(m, n), 0, torch.cuda.current_stream())
    assert e.value.status == oz.Status.ERR_UNSUPPORTED
