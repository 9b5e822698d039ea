"""Pins of the oracle's error metrics (oracle.exact.error_metrics).

Every "within 2^-100 / 2^-150 / 2^-200 / 2^-66" assertion of the GPU tests,
smoke() and the bench's error keys goes through error_metrics, so it is
pinned here against values worked out by hand or in exact rationals:
  err_nw  = ||Chat - C*||_F / ||C*||_F (normwise relative error),
  err_max = max |Chat_ij - C*_ij| / |C*_ij| (Sec. 1's largest relative
            error over all elements; an error on an exact zero is infinite).
"""
import math
import random
from fractions import Fraction

from oracle import exact as X

D = X.decode


def _frac_sqrt(f: Fraction) -> float:
    """sqrt of a positive Fraction, correct to about 2^-100 relative."""
    e = 0
    while f * Fraction(4) ** e < 2 ** 200:
        e += 16
    while f * Fraction(4) ** e > 2 ** 216:
        e -= 16
    r = math.isqrt(int(f * Fraction(4) ** e))
    return math.ldexp(float(r), -e) if r else 0.0


def _cplx(vals):
    """Exact dyadics of plain floats."""
    return [[D(v) for v in row] for row in vals]


def test_hand_computed_2x2():
    # C* = [[3, 4], [12, 0]]: ||C*||_F = 13.  Errors 3 2^-110 and 4 2^-110 on
    # the first row: ||Chat - C*||_F = 5 2^-110, so err_nw = (5 / 13) 2^-110
    # and err_max = 2^-110.  The exact zero entry carries no error.
    cstar = _cplx([[3.0, 4.0], [12.0, 0.0]])
    chat = [[[3.0, 3 * 2.0 ** -110], [4.0, 4 * 2.0 ** -110]],
            [[12.0, 0.0], [0.0, 0.0]]]
    m = X.error_metrics(chat, cstar)
    assert math.isclose(m["err_nw"], 5.0 / 13.0 * 2.0 ** -110, rel_tol=1e-15)
    assert m["err_max"] == 2.0 ** -110


def test_error_on_an_exact_zero():
    # a wrong value where C* is exactly zero: err_max is infinite, err_nw is
    # the error over ||C*||_F = 1
    cstar = _cplx([[1.0, 0.0]])
    chat = [[[1.0, 0.0], [2.0 ** -80, 0.0]]]
    m = X.error_metrics(chat, cstar)
    assert m["err_max"] == math.inf
    assert m["err_nw"] == 2.0 ** -80


def test_entries_far_apart_in_scale():
    # C* = [2^600, 2^-600]: relative errors 2^-100 on the big entry and 2^-50
    # on the small one.  err_nw is the big entry's (the small one adds
    # 2^-1300 relative); err_max is the small entry's 2^-50.
    cstar = _cplx([[2.0 ** 600, 2.0 ** -600]])
    chat = [[[2.0 ** 600, 2.0 ** 500], [2.0 ** -600, 2.0 ** -650]]]
    m = X.error_metrics(chat, cstar)
    assert math.isclose(m["err_nw"], 2.0 ** -100, rel_tol=1e-15)
    assert m["err_max"] == 2.0 ** -50


def test_errors_below_the_square_range_of_binary64():
    # a relative error of 2^-800 (the size a 16-component result has) squares
    # to 2^-1600, below every binary64; it must still be measured
    cstar = _cplx([[1.0, -3.0]])
    chat = [[[1.0, 2.0 ** -800], [-3.0, 0.0]]]
    m = X.error_metrics(chat, cstar)
    assert math.isclose(m["err_nw"], 2.0 ** -800 / math.sqrt(10.0), rel_tol=1e-15)
    assert m["err_max"] == 2.0 ** -800


def test_exact_and_all_zero():
    cstar = _cplx([[1.5, -2.25], [0.0, 7.0]])
    chat = [[[1.5, 0.0], [-2.25, 0.0]], [[0.0, 0.0], [7.0, 0.0]]]
    assert X.error_metrics(chat, cstar) == {"err_nw": 0.0, "err_max": 0.0}
    z = _cplx([[0.0, 0.0]])
    assert X.error_metrics([[[0.0], [0.0]]], z) == {"err_nw": 0.0, "err_max": 0.0}


def test_random_blocks_against_fractions():
    # 5 x 4 blocks of exact values over a wide exponent range, each computed
    # entry off by a few components; err_nw and err_max against Fractions
    rng = random.Random(7)
    for trial in range(20):
        cstar, chat = [], []
        num = Fraction(0)
        den = Fraction(0)
        emax = Fraction(0)
        for i in range(5):
            rs, rh = [], []
            for j in range(4):
                v = rng.uniform(-1, 1) * 2.0 ** rng.randint(-300, 300)
                err = [rng.uniform(-1, 1) * abs(v) * 2.0 ** -rng.randint(40, 200) for _ in range(2)]
                rs.append(D(v))
                rh.append([v] + err)
                d = Fraction(err[0]) + Fraction(err[1])
                num += d * d
                den += Fraction(v) * Fraction(v)
                emax = max(emax, abs(d) / abs(Fraction(v)))
            cstar.append(rs)
            chat.append(rh)
        m = X.error_metrics(chat, cstar)
        assert math.isclose(m["err_nw"], _frac_sqrt(num / den), rel_tol=1e-14)
        assert math.isclose(m["err_max"], float(emax), rel_tol=1e-15)
