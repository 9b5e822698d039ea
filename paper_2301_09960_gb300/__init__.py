"""ozmp: Ozaki-scheme multiple-precision matrix product on GB300 (sm_103a).

Thin Python binding of the C ABI declared in ``include/ozmp.h``.  It only
marshals arguments: every step of the product runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the CUDA library cannot be built or loaded, calls raise.

Matrices follow the BLAS convention of the paper's problem C := AB
(column-major).  A torch matrix is passed as a tensor of shape (rows, cols)
whose column stride is its leading dimension and whose row stride is 1
(``colmajor`` makes one).  Multi-component operands are lists of such
tensors (2/3/4 float64 for DD/TD/QD, 3 float32 for TS).
"""
from __future__ import annotations

import ctypes
import os
import threading
from enum import IntEnum

from . import _build

__all__ = [
    "Status", "Prec", "Form", "OzmpError", "PlanInfo", "Plan", "load", "colmajor",
    "ozmp_plan_create", "ozmp_plan_destroy", "ozmp_plan_get_info", "ozmp_plan_set_workspace",
    "ozmp_plan_set_stream", "ozmp_plan_execute", "ozmp_plan_get_status", "ozmp_plan_split",
    "ozmp_plan_diagonal", "ozmp_plan_multiply", "ozmp_plan_set_timing", "ozmp_plan_read_timing", "ozmp_gemm_dd", "ozmp_gemm_td", "ozmp_gemm_qd", "ozmp_gemm_ts", "ozmp_gemm_md", "ozmp_lu", "ozmp_lu_solve", "ozmp_gemm_literal", "prec_code", "MAX_COMPONENTS", "ozmp_gemm_dd_noalloc", "ozmp_gemm_batched", "Problem", "ozmp_gemm_naive",
    "ozmp_set_stream", "ozmp_set_form", "ozmp_last_status", "ozmp_version", "gemm", "EXP_ZERO",
]

EXP_ZERO = -(2 ** 31)


class Status(IntEnum):
    OK = 0
    ERR_INVALID_ARG = 1
    ERR_NONFINITE = 2
    ERR_RANGE = 3
    ERR_NOMEM = 4
    ERR_CUDA = 5
    ERR_UNSUPPORTED = 6
    ERR_TIMEOUT = 7
    ERR_ACCURACY = 8


class Prec(IntEnum):
    DD = 2
    TD = 3
    QD = 4
    TS = 103


class Form(IntEnum):
    AUTO = 0
    FP64 = 1
    INT8 = 2
    FP8 = 3
    FP8_MMA = 4
    FP8_BAL = 5
    FP16 = 6


MAX_COMPONENTS = 16
# "dd"/"td"/"qd"/"ts" and "q2" .. "q16" (q binary64 components)
PREC_BY_NAME = {"dd": Prec.DD, "td": Prec.TD, "qd": Prec.QD, "ts": Prec.TS}
PREC_BY_NAME.update({f"q{q}": q for q in range(2, MAX_COMPONENTS + 1)})
FORM_BY_NAME = {"auto": Form.AUTO, "fp64": Form.FP64, "int8": Form.INT8, "fp8": Form.FP8,
                "fp8mma": Form.FP8_MMA, "fp8bal": Form.FP8_BAL, "fp16": Form.FP16}
NCOMP = {Prec.DD: 2, Prec.TD: 3, Prec.QD: 4, Prec.TS: 3}
NCOMP.update({q: q for q in range(5, MAX_COMPONENTS + 1)})


def prec_code(prec) -> int:
    """The C ABI precision code of a name ("dd", "q8", ...) or code."""
    if isinstance(prec, str):
        return int(PREC_BY_NAME[prec])
    p = int(prec)
    if p not in NCOMP:
        raise ValueError(f"unknown precision {prec!r}")
    return p


class OzmpError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = Status(status)
        super().__init__(f"{where}: {self.status.name}")


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int), ("form", ctypes.c_int), ("beta", ctypes.c_int), ("nslices", ctypes.c_int),
        ("npairs", ctypes.c_int64),
        ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
        ("mp", ctypes.c_int64), ("np", ctypes.c_int64), ("kp", ctypes.c_int64),
        ("digit_bytes", ctypes.c_int), ("acc_words", ctypes.c_int), ("ngroups", ctypes.c_int),
        ("pairs_per_drain", ctypes.c_int),
        ("workspace_bytes", ctypes.c_size_t),
        ("off_E", ctypes.c_size_t), ("off_F", ctypes.c_size_t), ("off_status", ctypes.c_size_t),
        ("off_Adig", ctypes.c_size_t), ("off_Bdig", ctypes.c_size_t), ("off_acc", ctypes.c_size_t),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(ctypes.Structure):
    """ozmp_problem: one product of a batch."""
    _fields_ = [("prec", ctypes.c_int), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("ldb", ctypes.c_int64), ("ldc", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p), ("nslices", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_PP = ctypes.POINTER(ctypes.c_void_p)

#: exported symbols and their argument types (every entry of include/ozmp.h)
SIGNATURES = {
    "ozmp_plan_create": [ctypes.POINTER(_VP), ctypes.c_int, _I64, _I64, _I64, ctypes.c_int, ctypes.c_int, _VP],
    "ozmp_plan_destroy": [_VP],
    "ozmp_plan_get_info": [_VP, ctypes.POINTER(PlanInfo)],
    "ozmp_plan_set_workspace": [_VP, _VP, ctypes.c_size_t],
    "ozmp_plan_set_stream": [_VP, _VP],
    "ozmp_plan_execute": [_VP, _PP, _I64, _PP, _I64, _PP, _I64],
    "ozmp_plan_get_status": [_VP, ctypes.POINTER(ctypes.c_int)],
    "ozmp_plan_split": [_VP, _PP, _I64, _PP, _I64],
    "ozmp_plan_diagonal": [_VP, ctypes.c_int, _VP],
    "ozmp_plan_multiply": [_VP, _PP, _I64],
    "ozmp_plan_set_timing": [_VP, ctypes.c_int],
    "ozmp_plan_read_timing": [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "ozmp_gemm_dd": [_I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int],
    "ozmp_gemm_td": [_I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int],
    "ozmp_gemm_qd": [_I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int],
    "ozmp_gemm_ts": [_I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int],
    "ozmp_gemm_md": [ctypes.c_int, _I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int],
    "ozmp_lu": [ctypes.c_int, _I64, _PP, _I64, _VP],
    "ozmp_gemm_literal": [ctypes.c_int, ctypes.c_int, _I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64,
                          _VP, _VP, _VP, _VP],
    "ozmp_lu_solve": [ctypes.c_int, _I64, _I64, _PP, _I64, _PP, _I64, _VP],
    "ozmp_gemm_dd_noalloc": [_I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, ctypes.c_int, _VP],
    "ozmp_set_stream": [_VP],
    "ozmp_set_form": [ctypes.c_int],
    "ozmp_last_status": [ctypes.POINTER(ctypes.c_int)],
    "ozmp_version": [],
    "ozmp_gemm_naive": [ctypes.c_int, _I64, _I64, _I64, _PP, _I64, _PP, _I64, _PP, _I64, _VP],
    "ozmp_gemm_batched": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_VP)],
}


def load(build: bool = True):
    """Build (if needed) and load libozmp.so; raises if it is unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise OSError(f"ozmp library missing: {path}")
            L = ctypes.CDLL(path)
            for name, args in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name == "ozmp_version" else ctypes.c_int
            _lib = L
    return _lib


def _check(st, where):
    if st != 0:
        raise OzmpError(st, where)


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return ctypes.cast(arr, _PP), arr


def _stream_handle(stream):
    """cudaStream_t of a torch stream (None: torch's current stream, or the
    legacy default stream when CUDA is not initialised)."""
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


def colmajor(x, device="cuda", dtype=None):
    """Column-major device copy of a 2-D array (numpy or torch)."""
    import numpy as np
    import torch
    t = torch.as_tensor(np.asarray(x)) if not isinstance(x, torch.Tensor) else x
    if dtype is not None:
        t = t.to(dtype)
    r, c = t.shape
    out = torch.empty((c, r), dtype=t.dtype, device=device).T
    out.copy_(t)
    return out


def _ld(t):
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("matrices must be column-major (row stride 1)")
    return max(t.stride(1), t.shape[0], 1)


# ---------------------------------------------------------------------------
# C ABI, one Python function per entry point
# ---------------------------------------------------------------------------
def ozmp_version() -> str:
    return load().ozmp_version().decode()


def ozmp_plan_create(prec, m, n, k, form=Form.AUTO, nslices=0, stream=None):
    L = load()
    h = ctypes.c_void_p()
    st = L.ozmp_plan_create(ctypes.byref(h), int(prec), m, n, k, int(form), nslices, _stream_handle(stream))
    _check(st, "ozmp_plan_create")
    return h


def ozmp_plan_destroy(h):
    _check(load().ozmp_plan_destroy(h), "ozmp_plan_destroy")


def ozmp_plan_get_info(h) -> PlanInfo:
    info = PlanInfo()
    _check(load().ozmp_plan_get_info(h, ctypes.byref(info)), "ozmp_plan_get_info")
    return info


def ozmp_plan_set_workspace(h, ptr: int, nbytes: int):
    _check(load().ozmp_plan_set_workspace(h, ctypes.c_void_p(ptr), nbytes), "ozmp_plan_set_workspace")


def ozmp_plan_set_stream(h, stream=None):
    _check(load().ozmp_plan_set_stream(h, _stream_handle(stream)), "ozmp_plan_set_stream")


def ozmp_plan_execute(h, A, B, C):
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    st = load().ozmp_plan_execute(h, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]))
    _check(st, "ozmp_plan_execute")


def ozmp_plan_get_status(h) -> Status:
    v = ctypes.c_int()
    _check(load().ozmp_plan_get_status(h, ctypes.byref(v)), "ozmp_plan_get_status")
    return Status(v.value)


def ozmp_plan_split(h, A, B):
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    _check(load().ozmp_plan_split(h, pa, _ld(A[0]), pb, _ld(B[0])), "ozmp_plan_split")


def ozmp_plan_multiply(h, C):
    pc, kc = _ptrs(C)
    _check(load().ozmp_plan_multiply(h, pc, _ld(C[0])), "ozmp_plan_multiply")


def ozmp_plan_set_timing(h, nslots: int):
    _check(load().ozmp_plan_set_timing(h, nslots), "ozmp_plan_set_timing")


def ozmp_plan_read_timing(h, n: int):
    """Durations (ms) of the last product kernels, oldest first."""
    buf = (ctypes.c_float * max(n, 1))()
    cnt = ctypes.c_int(0)
    _check(load().ozmp_plan_read_timing(h, buf, n, ctypes.byref(cnt)), "ozmp_plan_read_timing")
    return [float(buf[i]) for i in range(cnt.value)]


def ozmp_plan_diagonal(h, d: int, T):
    _check(load().ozmp_plan_diagonal(h, d, ctypes.c_void_p(T.data_ptr())), "ozmp_plan_diagonal")


def _plain(name, A, B, C, nslices):
    m, k = A[0].shape
    n = B[0].shape[1]
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    st = getattr(load(), name)(m, n, k, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]), nslices)
    _check(st, name)


def ozmp_gemm_dd(A, B, C, nslices=0):
    _plain("ozmp_gemm_dd", A, B, C, nslices)


def ozmp_gemm_td(A, B, C, nslices=0):
    _plain("ozmp_gemm_td", A, B, C, nslices)


def ozmp_gemm_qd(A, B, C, nslices=0):
    _plain("ozmp_gemm_qd", A, B, C, nslices)


def ozmp_gemm_ts(A, B, C, nslices=0):
    _plain("ozmp_gemm_ts", A, B, C, nslices)


def ozmp_gemm_literal(A, B, C, D, slices_A=None, slices_B=None, products=None, stream=None):
    """Algorithm 1 as printed: binary64 round-to-nearest slices (D of each
    operand), DGEMM slice products, exact sum rounded into C.  Optional
    torch outputs: slices_A (D, k, m) / slices_B (D, n, k) / products
    (D(D+1)/2, n, m) contiguous tensors (each slice column-major)."""
    m, k = A[0].shape
    n = B[0].shape[1]
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    vp = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
    st = load().ozmp_gemm_literal(len(A), D, m, n, k, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]),
                                  vp(slices_A), vp(slices_B), vp(products), _stream_handle(stream))
    if st in (Status.ERR_INVALID_ARG, Status.ERR_NOMEM, Status.ERR_CUDA, Status.ERR_UNSUPPORTED):
        _check(st, "ozmp_gemm_literal")
    return Status(st)


def ozmp_lu(A, stream=None):
    """In-place LU without pivoting of the n x n q-component matrix A (list of
    q column-major torch tensors); returns the device status."""
    n = A[0].shape[0]
    pa, ka = _ptrs(A)
    st = load().ozmp_lu(len(A), n, pa, _ld(A[0]), _stream_handle(stream))
    if st in (Status.ERR_INVALID_ARG, Status.ERR_NOMEM, Status.ERR_CUDA, Status.ERR_UNSUPPORTED):
        _check(st, "ozmp_lu")
    return Status(st)


def ozmp_lu_solve(LU, B, stream=None):
    """Solve with the factors of ozmp_lu, in place in B (n x nrhs)."""
    n = LU[0].shape[0]
    nrhs = B[0].shape[1]
    pa, ka = _ptrs(LU)
    pb, kb = _ptrs(B)
    st = load().ozmp_lu_solve(len(LU), n, nrhs, pa, _ld(LU[0]), pb, _ld(B[0]), _stream_handle(stream))
    if st in (Status.ERR_INVALID_ARG, Status.ERR_NOMEM, Status.ERR_CUDA, Status.ERR_UNSUPPORTED):
        _check(st, "ozmp_lu_solve")
    return Status(st)


def ozmp_gemm_md(A, B, C, nslices=0):
    """q binary64 components (q = len(A), 2 <= q <= 16)."""
    m, k = A[0].shape
    n = B[0].shape[1]
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    st = load().ozmp_gemm_md(len(A), m, n, k, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]), nslices)
    _check(st, "ozmp_gemm_md")


def ozmp_gemm_dd_noalloc(A, B, C, nslices=0, stream=None):
    """Double-double product that allocates nothing (a fixed 64 MiB scratch
    inside the library), for callers that cannot call cudaMalloc, such as
    programs whose device memory is all held by their own pool allocator."""
    m, k = A[0].shape
    n = B[0].shape[1]
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    st = load().ozmp_gemm_dd_noalloc(m, n, k, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]), nslices,
                                     _stream_handle(stream))
    _check(st, "ozmp_gemm_dd_noalloc")


def ozmp_gemm_batched(problems, form=Form.AUTO, stream=None, plan=None):
    """Run a batch of products; problems is a list of (prec, A, B, C, nslices)
    with column-major torch operands.  Returns the (reusable) batched plan."""
    n = len(problems)
    arr = (Problem * n)()
    keep = []
    for i, (prec, A, B, C, ns) in enumerate(problems):
        prec = PREC_BY_NAME[prec] if isinstance(prec, str) else Prec(prec)
        m, k = A[0].shape
        nn = B[0].shape[1]
        pa, ka = _ptrs(A)
        pb, kb = _ptrs(B)
        pc, kc = _ptrs(C)
        keep += [ka, kb, kc]
        arr[i] = Problem(int(prec), m, nn, k, _ld(A[0]), _ld(B[0]), _ld(C[0]),
                         ctypes.cast(ka, ctypes.c_void_p), ctypes.cast(kb, ctypes.c_void_p),
                         ctypes.cast(kc, ctypes.c_void_p), ns)
    h = plan if plan is not None else ctypes.c_void_p()
    st = load().ozmp_gemm_batched(ctypes.cast(arr, ctypes.c_void_p), n, int(form), _stream_handle(stream),
                                  ctypes.byref(h))
    _check(st, "ozmp_gemm_batched")
    return h


def ozmp_gemm_naive(prec, A, B, C, stream=None):
    """The triple-loop multi-component product (the paper's baseline)."""
    prec = prec_code(prec)
    m, k = A[0].shape
    n = B[0].shape[1]
    pa, ka = _ptrs(A)
    pb, kb = _ptrs(B)
    pc, kc = _ptrs(C)
    st = load().ozmp_gemm_naive(int(prec), m, n, k, pa, _ld(A[0]), pb, _ld(B[0]), pc, _ld(C[0]),
                                _stream_handle(stream))
    _check(st, "ozmp_gemm_naive")


def ozmp_set_stream(stream=None):
    _check(load().ozmp_set_stream(_stream_handle(stream)), "ozmp_set_stream")


def ozmp_set_form(form):
    _check(load().ozmp_set_form(int(form)), "ozmp_set_form")


def ozmp_last_status() -> Status:
    v = ctypes.c_int()
    _check(load().ozmp_last_status(ctypes.byref(v)), "ozmp_last_status")
    return Status(v.value)


# ---------------------------------------------------------------------------
# object wrapper
# ---------------------------------------------------------------------------
class Plan:
    """A plan (precision, shape, digit form, slice count) with a torch-owned
    workspace on the current CUDA device."""

    def __init__(self, prec, m, n, k, form=Form.AUTO, nslices=0, stream=None, workspace=True):
        import torch
        self.prec = prec_code(prec)
        self.form_req = FORM_BY_NAME[form] if isinstance(form, str) else Form(form)
        self.h = ozmp_plan_create(self.prec, m, n, k, self.form_req, nslices, stream)
        self.ws = None
        if workspace:
            nb = max(256, int(self.info.workspace_bytes))
            self.ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
            base = self.ws.data_ptr()
            self.ws_off = (-base) % 256
            ozmp_plan_set_workspace(self.h, base + self.ws_off, nb)

    @property
    def info(self) -> PlanInfo:
        """The plan's description; with nslices = 0 the slice count is the one
        the last split chose from the data."""
        return ozmp_plan_get_info(self.h)

    @property
    def q(self):
        return NCOMP[self.prec]

    def set_stream(self, stream=None):
        ozmp_plan_set_stream(self.h, stream)

    def execute(self, A, B, C):
        ozmp_plan_execute(self.h, A, B, C)

    def status(self) -> Status:
        return ozmp_plan_get_status(self.h)

    def split(self, A, B):
        ozmp_plan_split(self.h, A, B)

    def multiply(self, C):
        ozmp_plan_multiply(self.h, C)

    def set_timing(self, nslots: int):
        ozmp_plan_set_timing(self.h, nslots)

    def read_timing(self, n: int):
        return ozmp_plan_read_timing(self.h, n)

    def diagonal(self, d):
        import torch
        T = torch.empty((self.info.n, self.info.m), dtype=torch.int64, device="cuda").T
        ozmp_plan_diagonal(self.h, d, T)
        return T

    # views of the workspace (valid after split/execute)
    def _region(self, off, count, dtype):
        import torch
        itemsize = torch.empty((), dtype=dtype).element_size()
        start = self.ws_off + off
        return self.ws[start:start + count * itemsize].view(dtype)

    def exponents(self):
        import torch
        i = self.info
        return (self._region(i.off_E, i.m, torch.int32), self._region(i.off_F, i.n, torch.int32))

    def digits(self):
        """(A digits [s, mp, kp], B digits [s, np, kp]) in the stored encoding."""
        import torch
        i = self.info
        dt = {8: torch.float64, 2: torch.float16}.get(i.digit_bytes, torch.uint8)
        a = self._region(i.off_Adig, i.nslices * i.mp * i.kp, dt).view(i.nslices, i.mp, i.kp)
        b = self._region(i.off_Bdig, i.nslices * i.np * i.kp, dt).view(i.nslices, i.np, i.kp)
        return a, b

    def close(self):
        if self.h:
            ozmp_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gemm(A, B, prec, form="auto", nslices=0, C=None, plan=None):
    """C := A B for multi-component column-major torch operands."""
    import torch
    m, k = A[0].shape
    n = B[0].shape[1]
    p = plan or Plan(prec, m, n, k, form, nslices)
    if C is None:
        dt = torch.float32 if p.prec == Prec.TS else torch.float64
        C = [torch.empty((n, m), dtype=dt, device="cuda").T for _ in range(p.q)]
    p.execute(A, B, C)
    return C, p
