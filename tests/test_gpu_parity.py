"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

* exponents E, F and every digit: bit-exact against oracle.ozaki.split
  (oracle.ozaki.split_balanced for the balanced radix-32 e4m3 form);
* each diagonal T_d = sum_{t+u=d} A_t B_u^T from the tensor-core main loop:
  bit-exact against the oracle's int64 slice products;
* the product: bit-exact against the canonical component rounding of the
  oracle's exact Ozaki sum, and within the precision's normwise target of
  the exact product rounded to 512 bits when the slice count is automatic.
Shapes span several 128 x 128 tiles with ragged m, n and k tails.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2301_09960_gb300 as oz
from oracle import _clib
from oracle import exact as X
from oracle import ozaki as O
from ozmp_inputs import gen_problem

from _util import digits_to_int, from_dev, to_dev

pytestmark = pytest.mark.gpu

TARGET = {"dd": 2.0 ** -100, "td": 2.0 ** -150, "qd": 2.0 ** -200, "ts": 2.0 ** -66}
Q = {"dd": 2, "td": 3, "qd": 4, "ts": 3}


def _osplit(comps, form, beta, s):
    """The oracle's exponents and digits of a form (rows of comps)."""
    if form == "fp8bal":
        return O.split_balanced(comps, s)
    return O.split(comps, beta, s)


def _oproduct(A, B, info):
    return O.ozaki_product(A, B, info.beta, info.nslices, balanced=(info.form == oz.Form.FP8_BAL))


def _split_check(prec, form, m, n, k, phi, seed, nslices=0):
    A, B = gen_problem(prec, m, n, k, phi=phi, seed=seed)
    p = oz.Plan(prec, m, n, k, form, nslices)
    Ad, Bd = to_dev(A), to_dev(B)
    p.split(Ad, Bd)
    torch.cuda.synchronize()
    i = p.info
    E, F = [t.cpu().numpy() for t in p.exponents()]
    ga, gb = [t.cpu().numpy() for t in p.digits()]
    Eo, dA = _osplit(A, form, i.beta, i.nslices)
    Fo, dB = _osplit([np.asfortranarray(b.T) for b in B], form, i.beta, i.nslices)
    assert list(E) == Eo
    assert list(F) == Fo
    gA = digits_to_int(ga[:, :m, :k], form)
    gB = digits_to_int(gb[:, :n, :k], form)
    np.testing.assert_array_equal(gA, dA)
    np.testing.assert_array_equal(gB, dB)
    # the padded region carries zero digits
    assert not digits_to_int(ga[:, m:, :], form).any() and not digits_to_int(ga[:, :, k:], form).any()
    assert not digits_to_int(gb[:, n:, :], form).any() and not digits_to_int(gb[:, :, k:], form).any()
    return p, A, B, Ad, Bd, dA, dB


@pytest.mark.parametrize("form", ["fp8", "fp8bal", "int8", "fp64", "fp16"])
@pytest.mark.parametrize("prec", ["dd", "td", "qd", "ts"])
def test_split_bit_exact(prec, form):
    _split_check(prec, form, 150, 140, 130, phi=1.0, seed=1, nslices={"fp64": 6, "fp16": 10}.get(form, 14))


@pytest.mark.parametrize("k", [300, 1100, 4300])
@pytest.mark.parametrize("prec", ["dd", "ts"])
def test_split_bit_exact_binary16_widths(prec, k):
    # binary16 digits of 7, 6 and 5 bits (the widths of k = 300, 1100, 4300),
    # split four elements a thread with the width fixed at compile time, on
    # ragged row and column tiles; the automatic slice count
    p = _split_check(prec, "fp16", 70, 90, k, phi=1.0, seed=2, nslices=0)[0]
    assert p.info.beta == {300: 7, 1100: 6, 4300: 5}[k]


@pytest.mark.parametrize("form,s", [("fp8", 64), ("fp8", 65), ("fp8bal", 63), ("fp8bal", 1)])
def test_split_widest_register_windows(form, s):
    # the register splitter writes up to 64 e4m3 slices (63 balanced ones,
    # 5 s + 65 <= 384 bits); 65 slices go to the many-component splitter
    _split_check("dd", form, 70, 60, 50, phi=1.0, seed=7, nslices=s)


@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
@pytest.mark.parametrize("prec", ["dd", "qd", "ts"])
def test_column_digits_in_one_pass_and_in_two(prec, form):
    # columns of B with 16-byte aligned starts and lengths are copied whole into
    # shared memory and split there (one read of B); a leading dimension of
    # k + 1 takes the separate exponent and digit kernels (and m + 1 gives A
    # an unaligned leading dimension too): both give the oracle's exponents
    # and digits
    m, n, k = 70, 90, 136
    A, B = gen_problem(prec, m, n, k, phi=1.0, seed=11)
    dt = torch.float32 if prec == "ts" else torch.float64
    Eo = Fo = dA = dB = None
    for pad in (0, 1):
        p = oz.Plan(prec, m, n, k, form, 0)
        Bd = []
        for b in B:
            buf = torch.zeros((n, k + pad), dtype=dt, device="cuda")
            buf[:, :k] = torch.from_numpy(np.ascontiguousarray(b.T))
            Bd.append(buf.T[:k, :])                   # k x n, column stride k + pad
        Ad = []
        for a in A:
            buf = torch.zeros((k, m + pad), dtype=dt, device="cuda")
            buf[:, :m] = torch.from_numpy(np.ascontiguousarray(a.T))
            Ad.append(buf.T[:m, :])                   # m x k, column stride m + pad
        p.split(Ad, Bd)
        torch.cuda.synchronize()
        assert p.status() == oz.Status.OK
        i = p.info
        if dB is None:
            Eo, dA = _osplit(A, form, i.beta, i.nslices)
            Fo, dB = _osplit([np.asfortranarray(b.T) for b in B], form, i.beta, i.nslices)
        E, F = [t.cpu().numpy() for t in p.exponents()]
        ga, gb = [t.cpu().numpy() for t in p.digits()]
        assert list(E) == Eo and list(F) == Fo, pad
        np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], form), dB)
        np.testing.assert_array_equal(digits_to_int(ga[:, :m, :k], form), dA)
        assert not digits_to_int(gb[:, n:, :], form).any() and not digits_to_int(gb[:, :, k:], form).any()


@pytest.mark.parametrize("prec,kmax", [("dd", 7168), ("td", 4778), ("qd", 3584)])
def test_column_split_at_the_shared_memory_limit(prec, kmax):
    # a column of B goes through shared memory in one pass while its q
    # components hold at most 112 KB (k = kmax); two more values of k take the
    # separate exponent and digit kernels: both give the oracle's digits
    m, n = 8, 6
    for k in (kmax, kmax + 2):
        A, B = gen_problem(prec, m, n, k, phi=1.0, seed=12)
        p = oz.Plan(prec, m, n, k, "fp8bal", 0)
        p.split(to_dev(A), to_dev(B))
        torch.cuda.synchronize()
        assert p.status() == oz.Status.OK
        i = p.info
        Fo, dB = O.split_balanced([np.asfortranarray(b.T) for b in B], i.nslices)
        assert list(p.exponents()[1].cpu().numpy()) == Fo, k
        gb = p.digits()[1].cpu().numpy()
        np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], "fp8bal"), dB)
        assert not digits_to_int(gb[:, n:, :], "fp8bal").any() and not digits_to_int(gb[:, :, k:], "fp8bal").any()


@pytest.mark.parametrize("form", ["fp8", "fp8bal", "fp8mma", "int8", "fp64", "fp16"])
def test_diagonals_bit_exact(form):
    s = {"fp8": 20, "fp8bal": 16, "fp8mma": 20, "int8": 12, "fp64": 5, "fp16": 11}[form]
    p, A, B, Ad, Bd, dA, dB = _split_check("dd", form, 200, 150, 130, phi=1.0, seed=2, nslices=s)
    T = O.slice_products(dA, dB)
    for d in sorted({2, 3, s // 2 + 1, s + 1}):
        got = p.diagonal(d).cpu().numpy()
        np.testing.assert_array_equal(got, T[d])


def _product(prec, form, m, n, k, phi, seed, nslices):
    A, B = gen_problem(prec, m, n, k, phi=phi, seed=seed)
    C, p = oz.gemm(to_dev(A), to_dev(B), prec, form, nslices)
    torch.cuda.synchronize()
    assert p.status() == oz.Status.OK
    return A, B, from_dev(C), p


def _canonical_check(A, B, Cg, p, prec):
    r = _oproduct(A, B, p.info)
    kind = "f32" if prec == "ts" else "f64"
    m, n = Cg[0].shape
    for a in range(m):
        for b in range(n):
            want = X.to_components(r["S"][a][b], Q[prec], kind)
            got = [float(c[a, b]) for c in Cg]
            assert got == want, (a, b, got, want)
    return r


CASES = [("dd", "fp8", 130, 140, 150), ("dd", "fp8mma", 140, 130, 150), ("dd", "int8", 200, 150, 130),
         ("dd", "fp64", 150, 130, 140), ("dd", "fp8", 300, 520, 260), ("ts", "fp8mma", 130, 120, 100),
         ("td", "fp8", 130, 70, 100), ("td", "int8", 140, 130, 70), ("td", "fp64", 130, 140, 70),
         ("qd", "fp8", 70, 130, 64), ("qd", "int8", 130, 70, 90), ("qd", "fp64", 140, 70, 70),
         ("ts", "fp8", 150, 140, 130), ("ts", "int8", 140, 130, 150), ("ts", "fp64", 130, 150, 140),
         ("dd", "fp8bal", 130, 140, 150), ("dd", "fp8bal", 300, 520, 260), ("td", "fp8bal", 130, 70, 100),
         ("qd", "fp8bal", 70, 130, 64), ("ts", "fp8bal", 150, 140, 130),
         ("dd", "fp16", 300, 520, 260), ("td", "fp16", 130, 70, 100), ("qd", "fp16", 70, 130, 64),
         ("ts", "fp16", 150, 140, 130), ("ts", "fp16", 40, 36, 1100), ("dd", "fp16", 40, 36, 4300)]


@pytest.mark.parametrize("prec,form,m,n,k", CASES)
def test_product_bit_exact_and_within_target(prec, form, m, n, k):
    A, B, Cg, p = _product(prec, form, m, n, k, phi=1.0, seed=3, nslices=0)
    _canonical_check(A, B, Cg, p, prec)
    # error against the exact product on a sampled block
    rows = list(range(0, m, max(1, m // 12)))[:12]
    cols = list(range(0, n, max(1, n // 12)))[:12]
    ex = _clib.exact_block(A, B, rows, cols)
    chat = [[[float(c[a, b]) for c in Cg] for b in cols] for a in rows]
    err = X.error_metrics(chat, ex)["err_nw"]
    assert err <= TARGET[prec], err


def test_phi4_needs_more_slices_and_fixed_s_is_exact():
    # exponent spread phi = 4: the automatic count is not enough, a larger
    # forced count is; both are bit-exact to the oracle's Ozaki sum
    A, B, Cg, p = _product("dd", "fp8", 128, 130, 140, phi=4.0, seed=4, nslices=48)
    _canonical_check(A, B, Cg, p, "dd")
    A, B, Cg, p = _product("dd", "fp8bal", 128, 130, 140, phi=4.0, seed=4, nslices=40)
    _canonical_check(A, B, Cg, p, "dd")


@pytest.mark.parametrize("form", ["fp8", "fp8bal"])
def test_edge_shapes(form):
    for (m, n, k) in [(1, 1, 1), (1, 7, 3), (5, 1, 2), (129, 1, 65), (1, 129, 127)]:
        A, B, Cg, p = _product("dd", form, m, n, k, phi=1.0, seed=5, nslices=0)
        _canonical_check(A, B, Cg, p, "dd")


def test_k_zero_gives_zero():
    A = [oz.colmajor(np.zeros((5, 0)))] * 2
    B = [oz.colmajor(np.zeros((0, 4)))] * 2
    C = [oz.colmajor(np.full((5, 4), 3.0)) for _ in range(2)]
    p = oz.Plan("dd", 5, 4, 0, "fp8", 0)
    p.execute(A, B, C)
    torch.cuda.synchronize()
    assert all(float(c.abs().max()) == 0.0 for c in C)


def test_zero_rows_unnormalised_and_slow_path():
    m, n, k = 6, 5, 4
    hi = np.zeros((m, k))
    lo = np.zeros((m, k))
    hi[0] = [1.0, -3.0, 2.0 ** 60, 0.5]
    lo[0] = [-(2.0 ** -400), 1.0, -(2.0 ** 60), 2.0 ** -1074]     # tails far below the window
    hi[2] = [2.0 ** -1000, 1.0, 0.0, 0.0]
    hi[3] = [1.0, 1.0, 1.0, 1.0]
    lo[3] = [-1.0, 0.0, 0.0, 2.0 ** -53]                           # complete cancellation
    hi[4] = [2.0 ** 60, -(2.0 ** 200), 3.0, 0.0]
    lo[4] = [-(2.0 ** 60 - 1.0), 2.0 ** 200 - 2.0 ** 148, -(2.0 ** 55), 0.0]   # components far above the value
    # rows 1 and 5 are zero
    A = [np.asfortranarray(hi), np.asfortranarray(lo)]
    rng = np.random.default_rng(0)
    B = [np.asfortranarray(rng.standard_normal((k, n))), np.zeros((k, n), order="F")]
    B[0][:, 2] = 0.0
    for form in ["fp8", "fp8bal", "int8", "fp64"]:
        p = oz.Plan("dd", m, n, k, form, 0)
        Ad, Bd = to_dev(A), to_dev(B)
        p.split(Ad, Bd)
        torch.cuda.synchronize()
        E, F = [t.cpu().numpy() for t in p.exponents()]
        Eo, dA = _osplit(A, form, p.info.beta, p.info.nslices)
        assert list(E) == Eo and E[1] == oz.EXP_ZERO and F[2] == oz.EXP_ZERO
        ga = p.digits()[0].cpu().numpy()
        np.testing.assert_array_equal(digits_to_int(ga[:, :m, :k], form), dA)
        C = [oz.colmajor(np.zeros((m, n))) for _ in range(2)]
        p.execute(Ad, Bd, C)
        torch.cuda.synchronize()
        st = p.status()
        # 2^-1000 * b underflows the output range: reported, not silently wrong
        assert st in (oz.Status.OK, oz.Status.ERR_RANGE)
        Cg = from_dev(C)
        r = _oproduct(A, B, p.info)
        for a in [0, 1, 3, 4, 5]:
            for b in range(n):
                assert [float(c[a, b]) for c in Cg] == X.to_components(r["S"][a][b], 2)


def test_nonfinite_input_sets_status():
    A, B = gen_problem("dd", 40, 30, 20, seed=6)
    A[0][3, 4] = np.nan
    B[1][2, 2] = np.inf
    C, p = oz.gemm(to_dev(A), to_dev(B), "dd", "fp8", 0)
    assert p.status() == oz.Status.ERR_NONFINITE


def test_leading_dimensions_larger_than_rows():
    A, B = gen_problem("td", 70, 60, 50, seed=7)
    pad = lambda x, r: np.asfortranarray(np.vstack([x, np.full((r, x.shape[1]), 7.0)]))
    Ap = [torch.as_tensor(pad(a, 9)).cuda() for a in A]
    Bp = [torch.as_tensor(pad(b, 5)).cuda() for b in B]
    # column-major views with ld = rows + pad
    Av = [torch.empty((50, 79), dtype=torch.float64, device="cuda").T for _ in A]
    Bv = [torch.empty((60, 55), dtype=torch.float64, device="cuda").T for _ in B]
    for v, a in zip(Av, Ap):
        v.copy_(a)
    for v, b in zip(Bv, Bp):
        v.copy_(b)
    Cbig = [torch.full((60, 75), 5.0, dtype=torch.float64, device="cuda").T for _ in range(3)]
    p = oz.Plan("td", 70, 60, 50, "int8", 0)
    p.execute([v[:70] for v in Av], [v[:50] for v in Bv], [c[:70] for c in Cbig])
    torch.cuda.synchronize()
    Cg = [c[:70].cpu().numpy() for c in Cbig]
    _canonical_check(A, B, Cg, p, "td")
    assert all(float(c[70:].min()) == 5.0 and float(c[70:].max()) == 5.0 for c in Cbig)


def test_plain_entry_points_match_plan():
    for prec, fn in [("dd", oz.ozmp_gemm_dd), ("td", oz.ozmp_gemm_td), ("qd", oz.ozmp_gemm_qd),
                     ("ts", oz.ozmp_gemm_ts)]:
        A, B = gen_problem(prec, 90, 70, 80, seed=8)
        Ad, Bd = to_dev(A), to_dev(B)
        oz.ozmp_set_stream(None)
        dt = torch.float32 if prec == "ts" else torch.float64
        C1 = [torch.zeros((70, 90), dtype=dt, device="cuda").T for _ in range(Q[prec])]
        fn(Ad, Bd, C1, 0)
        assert oz.ozmp_last_status() == oz.Status.OK
        C2, p = oz.gemm(Ad, Bd, prec, "auto", 0)
        torch.cuda.synchronize()
        for x, y in zip(C1, C2):
            assert torch.equal(x, y)


def test_bad_arguments_are_rejected():
    A, B = gen_problem("dd", 8, 8, 8, seed=9)
    Ad, Bd = to_dev(A), to_dev(B)
    C = [oz.colmajor(np.zeros((8, 8))) for _ in range(2)]
    p = oz.Plan("dd", 8, 8, 8, "fp8", 0)
    Cs = [torch.zeros((8, 4), dtype=torch.float64, device="cuda").T for _ in range(2)]   # ld = 4 < m = 8
    with pytest.raises(oz.OzmpError) as e:
        oz.ozmp_plan_execute(p.h, Ad, Bd, Cs)
    assert e.value.status == oz.Status.ERR_INVALID_ARG


def test_nondefault_stream_and_repeat():
    A, B = gen_problem("dd", 300, 260, 200, seed=10)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Ad, Bd = to_dev(A), to_dev(B)
        p = oz.Plan("dd", 300, 260, 200, "fp8", 0, stream=s)
        C1, _ = oz.gemm(Ad, Bd, "dd", plan=p)
        C2, _ = oz.gemm(Ad, Bd, "dd", plan=p)
    s.synchronize()
    for x, y in zip(C1, C2):
        assert torch.equal(x, y)


@pytest.mark.parametrize("form", ["fp8", "int8"])
def test_kernel_timing_ring(form):
    # the plan's event ring times the product kernel alone: one duration per
    # multiply, the ring keeps the last nslots, and it never exceeds the stage
    A, B = gen_problem("dd", 520, 300, 260, seed=12)
    Ad, Bd = to_dev(A), to_dev(B)
    p = oz.Plan("dd", 520, 300, 260, form, 0)
    C = [torch.empty((300, 520), dtype=torch.float64, device="cuda").T for _ in range(2)]
    p.split(Ad, Bd)
    assert p.read_timing(4) == []
    p.set_timing(3)
    stage = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p.multiply(C)
        e1.record()
        torch.cuda.synchronize()
        stage.append(e0.elapsed_time(e1))
    t = p.read_timing(8)
    assert len(t) == 3 and all(0 < x <= y + 1e-3 for x, y in zip(t, stage[2:]))
    p.set_timing(0)
    assert p.read_timing(8) == []
    with pytest.raises(oz.OzmpError):
        p.set_timing(-1)


def _adversarial(q, rows, cols, seed, dtype=np.float64):
    """Components at exact powers of two with tiny tails of either sign,
    spans far beyond 128 bits, cancelling leading pairs and zeros: every
    fast/slow boundary of the exponent and digit windows."""
    rng = np.random.default_rng(seed)
    tiny = 2.0 ** -140 if dtype == np.float32 else 2.0 ** -1000
    comps = [np.zeros((rows, cols)) for _ in range(q)]
    for i in range(rows):
        for j in range(cols):
            kind = rng.integers(0, 6)
            e = int(rng.integers(-30, 30))
            hi = float(rng.choice([-1.0, 1.0])) * 2.0 ** e
            if kind == 1:
                hi *= 1.0 + float(rng.integers(1, 2 ** 20)) * 2.0 ** -52 if dtype == np.float64 else 1.0
            vals = [hi]
            for t in range(1, q):
                gap = int(rng.integers(1, 400 if dtype == np.float64 else 100))
                v = float(rng.choice([-1.0, 1.0])) * 2.0 ** (e - gap)
                if kind == 2:
                    v = -vals[-1] if t == 1 else v          # cancelling pair
                if kind == 3:
                    v = max(v, tiny) if v > 0 else min(v, -tiny)
                vals.append(v)
            if kind == 4:
                vals = [0.0] * q
            for t in range(q):
                comps[t][i, j] = vals[t]
    return [np.asfortranarray(c.astype(dtype)) for c in comps]


@pytest.mark.parametrize("form", ["fp8", "fp8bal", "int8", "fp64"])
@pytest.mark.parametrize("prec", ["dd", "qd", "ts"])
def test_split_adversarial_boundaries(prec, form):
    q = {"dd": 2, "qd": 4, "ts": 3}[prec]
    dt = np.float32 if prec == "ts" else np.float64
    m, n, k = 40, 36, 33
    A = _adversarial(q, m, k, 11, dt)
    B = _adversarial(q, k, n, 12, dt)
    p = oz.Plan(prec, m, n, k, form, 6 if form == "fp64" else 20)
    p.split(to_dev(A), to_dev(B))
    torch.cuda.synchronize()
    i = p.info
    E, F = [t.cpu().numpy() for t in p.exponents()]
    ga, gb = [t.cpu().numpy() for t in p.digits()]
    Eo, dA = _osplit(A, form, i.beta, i.nslices)
    Fo, dB = _osplit([np.asfortranarray(b.T) for b in B], form, i.beta, i.nslices)
    assert list(E) == Eo and list(F) == Fo
    np.testing.assert_array_equal(digits_to_int(ga[:, :m, :k], form), dA)
    np.testing.assert_array_equal(digits_to_int(gb[:, :n, :k], form), dB)


@pytest.mark.parametrize("pair", ["1", "0"])
def test_tail_tiles_split_across_ctas_match_other_engine(pair, monkeypatch):
    # 2560 x 2048: 160 tiles of 128 x 256 on 152 SMs, or 80 tiles of 256 x 256
    # on the CTA pairs (about 76 clusters): a wave of whole tiles plus tail
    # tiles split into pair-range chunks that add atomically.  Exactness makes
    # the result independent of the split and of the tile form: it must equal
    # the mma.sync e4m3 engine bit for bit.
    monkeypatch.setenv("OZMP_TC_PAIR", pair)
    m, n, k = 2560, 2048, 192
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=13)
    Ad, Bd = to_dev(A), to_dev(B)
    C1, p1 = oz.gemm(Ad, Bd, "dd", "fp8", 0)
    C2, p2 = oz.gemm(Ad, Bd, "dd", "fp8mma", 0)
    torch.cuda.synchronize()
    assert p1.status() == oz.Status.OK and p2.status() == oz.Status.OK
    for x, y in zip(C1, C2):
        assert torch.equal(x, y)
    # and a sampled block against the oracle's Ozaki sum
    rows = list(range(0, m, 397))
    cols = list(range(0, n, 311))
    Cg = from_dev(C1)
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    # exponents are row/column maxima over k, so the sub-block split equals the full one
    r = O.ozaki_product(As, Bs, p1.info.beta, p1.info.nslices)
    for a_i, i in enumerate(rows):
        for b_j, j in enumerate(cols):
            assert [float(c[i, j]) for c in Cg] == X.to_components(r["S"][a_i][b_j], 2)


def test_balanced_digits_on_split_tail_tiles(monkeypatch):
    # the balanced form on the same tail-split schedules: single-CTA and
    # CTA-pair tiles agree bit for bit, and a sampled block equals the
    # oracle's Ozaki sum of the balanced digits
    m, n, k = 2560, 2048, 192
    A, B = gen_problem("dd", m, n, k, phi=1.0, seed=14)
    Ad, Bd = to_dev(A), to_dev(B)
    out = {}
    for pair in ("1", "0"):
        monkeypatch.setenv("OZMP_TC_PAIR", pair)
        C, p = oz.gemm(Ad, Bd, "dd", "fp8bal", 0)
        torch.cuda.synchronize()
        assert p.status() == oz.Status.OK and p.info.form == oz.Form.FP8_BAL and p.info.beta == 5
        out[pair] = (C, p)
    for x, y in zip(out["1"][0], out["0"][0]):
        assert torch.equal(x, y)
    C, p = out["1"]
    rows = list(range(0, m, 397))
    cols = list(range(0, n, 311))
    Cg = from_dev(C)
    As = [np.asfortranarray(a[rows, :]) for a in A]
    Bs = [np.asfortranarray(b[:, cols]) for b in B]
    r = _oproduct(As, Bs, p.info)
    for a_i, i in enumerate(rows):
        for b_j, j in enumerate(cols):
            assert [float(c[i, j]) for c in Cg] == X.to_components(r["S"][a_i][b_j], 2)
