"""Host logic of bench.py that the JSON line rests on: the splitter's
algorithmic bytes and the count of kernel launches per step."""
import os
import sys
import types

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import paper_2301_09960_gb300 as oz  # noqa: E402


def test_splitter_bytes_are_one_read_of_the_operands_and_one_write_of_the_digits():
    # DD 4096^3 with 26 one-byte slices: 2 x 8 x (mk + kn) + 26 x (mk + kn)
    n = 4096
    assert bench.splitter_bytes(2, 8, n, n, n, 26, 1) == (2 * 8 + 26) * 2 * n * n == 1409286144
    # binary64 digits (8 bytes each), rectangular
    assert bench.splitter_bytes(3, 8, 100, 30, 70, 9, 8) == (3 * 8 + 9 * 8) * (100 * 70 + 70 * 30)


class _Col:
    """A stand-in for a column-major device tensor: stride(1) and data_ptr()."""

    def __init__(self, ld, ptr):
        self.ld, self.ptr = ld, ptr

    def stride(self, i):
        return self.ld if i == 1 else 1

    def data_ptr(self):
        return self.ptr


@pytest.mark.parametrize("form,k,ld,ptr,q,want", [
    (oz.Form.FP8_BAL, 4096, 4096, 256, 2, 7),   # aligned DD columns: one pass over B
    (oz.Form.FP8_BAL, 4095, 4095, 256, 2, 8),   # k * 8 not a multiple of 16: two kernels
    (oz.Form.FP8_BAL, 4096, 4097, 256, 2, 8),   # leading dimension unaligned
    (oz.Form.FP8_BAL, 4096, 4096, 264, 2, 8),   # base not 16-byte aligned
    (oz.Form.FP8_BAL, 7168, 7168, 256, 2, 7),   # 112 KB a column: still one pass
    (oz.Form.FP8_BAL, 7170, 7170, 256, 2, 8),   # past 112 KB
    (oz.Form.FP8, 4096, 4096, 256, 4, 8),       # QD: 128 KB a column
    (oz.Form.FP16, 4096, 4096, 256, 2, 8),      # binary16 digits: two kernels for B, rounding pass
    (oz.Form.FP8_MMA, 4096, 4096, 256, 2, 7),   # mma.sync engine: no rounding pass, a check pass
    (oz.Form.INT8, 4096, 4096, 256, 2, 8),      # int8 digits: two kernels for B, a check pass
    (oz.Form.FP64, 4096, 4096, 256, 2, 8),
])
def test_launches_per_step_with_a_fixed_slice_count(form, k, ld, ptr, q, want):
    # exponent init, row exponents, (column exponents,) row and column
    # digits, the check's exponent statistics, the product, then the rounding
    # pass (tcgen05, which runs the check) or the check pass
    info = types.SimpleNamespace(form=form)
    Bd = [_Col(ld, ptr + c * 1024 * 1024) for c in range(q)]
    assert bench.launches_per_step(oz, info, Bd, k, 8, adaptive=False) == want


@pytest.mark.parametrize("form,want", [(oz.Form.FP8_BAL, 7), (oz.Form.FP8, 7), (oz.Form.FP16, 8),
                                       (oz.Form.FP8_MMA, 7), (oz.Form.INT8, 8), (oz.Form.FP64, 8)])
def test_launches_per_step_with_the_data_dependent_count(form, want):
    # exponent init, the row exponent pass with the norms, the one-pass
    # column digits with B's exponents and norms (e4m3 forms) or a column
    # exponent pass and later the column digits, the choice, the row digits,
    # the product, the rounding or the check pass
    info = types.SimpleNamespace(form=form)
    Bd = [_Col(4096, 256 + c * 1024 * 1024) for c in range(2)]
    assert bench.launches_per_step(oz, info, Bd, 4096, 8) == want
