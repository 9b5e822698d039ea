"""Build and call the oracle's C library (``mp512.c``); test infrastructure.

The library is compiled with gcc on first use into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mp512.c")
_OUT = os.path.join(_HERE, "_build", "libozoracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mp512.c (gcc, OpenMP) and return the shared-object path."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            for name in ("oz_exact_block", "oz_naive512_block"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64,
                              vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, vp]
            L.oz_mp_binop.restype = None
            L.oz_mp_binop.argtypes = [ctypes.c_int, i64] + [vp] * 9
            L.oz_int_gemm_tn.restype = None
            L.oz_int_gemm_tn.argtypes = [i64, i64, i64, vp, vp, vp]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _unpack(sgn, ex, limbs):
    """(sign, exponent, 8 limbs) arrays -> list of (N, e) with value N*2^e."""
    out = []
    lb = limbs.reshape(-1, 8)
    for s, e, row in zip(sgn.tolist(), ex.tolist(), lb):
        if s == 0:
            out.append((0, 0))
        else:
            n = int.from_bytes(row.astype("<u8").tobytes(), "little")
            out.append((n if s > 0 else -n, int(e)))
    return out


def _block(fn_name, A, B, rows, cols):
    L = lib()
    is_float = int(A[0].dtype == np.float32)
    m, k = A[0].shape
    k2, n = B[0].shape
    assert k == k2
    Ac = [np.asfortranarray(a) for a in A]
    Bc = [np.asfortranarray(b) for b in B]
    pa = (ctypes.c_void_p * len(Ac))(*[a.ctypes.data for a in Ac])
    pb = (ctypes.c_void_p * len(Bc))(*[b.ctypes.data for b in Bc])
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    cnt = len(rows) * len(cols)
    sgn = np.zeros(cnt, np.int8)
    ex = np.zeros(cnt, np.int64)
    limbs = np.zeros(cnt * 8, np.uint64)
    getattr(L, fn_name)(len(Ac), len(Bc), is_float, k,
                        ctypes.cast(pa, ctypes.c_void_p), m, ctypes.cast(pb, ctypes.c_void_p), k,
                        _ptr(rows), len(rows), _ptr(cols), len(cols),
                        _ptr(sgn), _ptr(ex), _ptr(limbs))
    vals = _unpack(sgn, ex, limbs)
    # column-major block: element (r, c) at r + c*nrows
    return [[vals[r + c * len(rows)] for c in range(len(cols))] for r in range(len(rows))]


def exact_block(A, B, rows, cols):
    """Exact product entries, rounded once to 512 bits (RNE).

    Returns a nested list [r][c] of (N, e) pairs, value N*2^e, |N| < 2^512.
    Follows the problem statement C := AB (Sec. 1) with each operand element
    equal to the exact sum of its components.
    """
    return _block("oz_exact_block", A, B, rows, cols)


def naive512_block(A, B, rows, cols):
    """The plain triple loop with every operation rounded to 512 bits."""
    return _block("oz_naive512_block", A, B, rows, cols)


def mp_binop(op: str, xs, ys):
    """Elementwise RN512(x op y) for lists of (N, e) operands, |N| < 2^512."""
    L = lib()
    cnt = len(xs)

    def pack(vs):
        s = np.zeros(cnt, np.int8); e = np.zeros(cnt, np.int64); m = np.zeros(cnt * 8, np.uint64)
        for i, (n, ee) in enumerate(vs):
            if n:
                s[i] = 1 if n > 0 else -1
                e[i] = ee
                m[8 * i:8 * i + 8] = np.frombuffer(abs(n).to_bytes(64, "little"), dtype="<u8")
        return s, e, m

    s1, e1, m1 = pack(xs); s2, e2, m2 = pack(ys)
    so = np.zeros(cnt, np.int8); eo = np.zeros(cnt, np.int64); mo = np.zeros(cnt * 8, np.uint64)
    L.oz_mp_binop(0 if op == "add" else 1, cnt, _ptr(s1), _ptr(e1), _ptr(m1),
                  _ptr(s2), _ptr(e2), _ptr(m2), _ptr(so), _ptr(eo), _ptr(mo))
    return _unpack(so, eo, mo)


def int_gemm_tn(X, Y):
    """T[i, j] = sum_p X[i, p] * Y[j, p] exactly in int64 (X: m x k, Y: n x k)."""
    L = lib()
    X = np.ascontiguousarray(X, dtype=np.int64)
    Y = np.ascontiguousarray(Y, dtype=np.int64)
    m, k = X.shape
    n, k2 = Y.shape
    assert k == k2
    T = np.zeros((n, m), np.int64)          # T[j, i] at i + j*m: column-major m x n
    L.oz_int_gemm_tn(m, n, k, _ptr(X), _ptr(Y), _ptr(T))
    return T.T
