"""The bounded waits of the tcgen05 product kernel, made to run out on
purpose without any fault: with OZMP_TC_INJECT_STALL=1 every CTA's first
stage is never loaded, so the barrier it waits on is never completed; with a
small OZMP_TC_WAIT_LIMIT the waits give up quickly.  The kernel must return
with OZMP_ERR_TIMEOUT in the plan's status word, and the context must stay
usable: a following product on the same device is bit-exact."""
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


@pytest.mark.parametrize("pair", ["1", "0"])
def test_wait_runs_out_and_context_stays_usable(pair, monkeypatch):
    m, n, k = 512, 512, 256
    A, B = gen_problem("dd", m, n, k, seed=2)
    Ad, Bd = to_dev(A), to_dev(B)
    monkeypatch.setenv("OZMP_TC_PAIR", pair)
    monkeypatch.setenv("OZMP_TC_INJECT_STALL", "1")
    monkeypatch.setenv("OZMP_TC_WAIT_LIMIT", "20000")
    p = oz.Plan("dd", m, n, k, "fp8", 0)
    monkeypatch.delenv("OZMP_TC_INJECT_STALL")
    monkeypatch.delenv("OZMP_TC_WAIT_LIMIT")
    C = [torch.empty((n, m), dtype=torch.float64, device="cuda").T for _ in range(2)]
    p.execute(Ad, Bd, C)
    torch.cuda.synchronize()
    assert p.status() == oz.Status.ERR_TIMEOUT
    del p
    # the same device, a normal plan: bit-exact on a sampled block
    C2, p2 = oz.gemm(Ad, Bd, "dd", "fp8", 0)
    torch.cuda.synchronize()
    assert p2.status() == oz.Status.OK
    Cg = from_dev(C2)
    rows, cols = [0, 255, 256, 511], [0, 300, 511]
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    r = O.ozaki_product(As, Bs, p2.info.beta, p2.info.nslices)
    for a_i, i in enumerate(rows):
        for b_j, j in enumerate(cols):
            assert [float(c[i, j]) for c in Cg] == X.to_components(r["S"][a_i][b_j], 2)


def test_column_split_wait_runs_out_and_context_stays_usable(monkeypatch):
    # the one-pass column splitter waits (bounded) on the bulk copies of its
    # column; OZMP_SPLIT_INJECT_STALL=1 issues none, so the wait runs out and
    # the split reports OZMP_ERR_TIMEOUT; a following split is the oracle's
    m, n, k = 256, 64, 256          # 16-byte aligned columns: the one-pass kernel
    A, B = gen_problem("dd", m, n, k, seed=3)
    Ad, Bd = to_dev(A), to_dev(B)
    monkeypatch.setenv("OZMP_SPLIT_INJECT_STALL", "1")
    monkeypatch.setenv("OZMP_SPLIT_WAIT_LIMIT", "20000")
    p = oz.Plan("dd", m, n, k, "fp8bal", 0)
    monkeypatch.delenv("OZMP_SPLIT_INJECT_STALL")
    monkeypatch.delenv("OZMP_SPLIT_WAIT_LIMIT")
    p.split(Ad, Bd)
    torch.cuda.synchronize()
    assert p.status() == oz.Status.ERR_TIMEOUT
    del p
    p2 = oz.Plan("dd", m, n, k, "fp8bal", 0)
    p2.split(Ad, Bd)
    torch.cuda.synchronize()
    assert p2.status() == oz.Status.OK
    i = p2.info
    Fo, dB = O.split_balanced([np.asfortranarray(b.T) for b in B], i.nslices)
    assert list(p2.exponents()[1].cpu().numpy()) == Fo
    gb = p2.digits()[1].cpu().numpy()
    np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], "fp8bal"), dB)
