"""Error-free transformations on binary64 (test infrastructure).

The multi-component formats the paper uses (DD, TD, QD; Sec. 1) are built
on error-free transformations: for floating-point a, b the rounded sum or
product together with its exactly representable error equals the exact
result.  These are the textbook forms, written here for the oracle's own
checks of multi-component outputs; the tests pin them against exact
rational arithmetic.
"""
from __future__ import annotations


def two_sum(a: float, b: float):
    """s = fl(a + b) and e with s + e = a + b exactly (no magnitude order)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def fast_two_sum(a: float, b: float):
    """Same as two_sum under the precondition |a| >= |b| (or a == 0)."""
    s = a + b
    e = b - (s - a)
    return s, e


_SPLITTER = 134217729.0   # 2^27 + 1


def veltkamp_split(a: float):
    """a = hi + lo with hi, lo of at most 26 significant bits each."""
    t = _SPLITTER * a
    hi = t - (t - a)
    return hi, a - hi


def two_prod(a: float, b: float):
    """p = fl(a * b) and e with p + e = a * b exactly (Dekker's product;
    valid while no intermediate overflows or underflows)."""
    p = a * b
    ah, al = veltkamp_split(a)
    bh, bl = veltkamp_split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e
