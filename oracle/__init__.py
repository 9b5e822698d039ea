"""CPU oracle for the Ozaki-scheme multi-component product (test infrastructure).

This package is test infrastructure.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the library path never does and shares no code with it.

Contents (each function cites the passage of the paper it follows):

* ``_clib``   -- build/load of ``mp512.c``: exact (Kulisch) dot products
                 rounded to a self-written 512-bit float, the naive 512-bit
                 triple loop, 512-bit add/mul, exact int64 slice products.
* ``exact``   -- exact dyadic arithmetic on multi-component numbers, the
                 exponent and digit split, canonical component rounding,
                 error metrics.
* ``ozaki``   -- the CPU Ozaki product (Algorithm 1 with exact truncating
                 digit slices) and the paper-literal round-to-nearest form.
* ``eft``     -- error-free transformations (TwoSum, FastTwoSum, TwoProd).

Every function is pinned by ``tests/test_oracle_*.py`` against exact
rational brute force, closed forms, invariants or values the paper prints.
"""
