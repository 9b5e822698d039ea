"""Helpers shared by the tests: operand transfer and digit decoding."""
import numpy as np

E4M3 = {}
for b in range(256):
    s = -1.0 if b & 0x80 else 1.0
    e = (b >> 3) & 15
    m = b & 7
    E4M3[b] = s * (m / 8.0) * 2.0 ** -6 if e == 0 else s * (1 + m / 8.0) * 2.0 ** (e - 7)


def digits_to_int(arr, form):
    """Stored digits (numpy) -> signed integers."""
    if form == "fp64":
        v = arr.astype(np.float64)
        assert np.all(v == np.round(v))
        return v.astype(np.int64)
    if form == "fp16":
        v = arr.astype(np.float16).astype(np.float64)
        assert np.all(v == np.round(v))
        return v.astype(np.int64)
    if form == "int8":
        return arr.astype(np.uint8).view(np.int8).astype(np.int64)
    assert form in ("fp8", "fp8mma", "fp8bal")
    lut = np.array([E4M3[b] for b in range(256)])
    v = lut[arr.astype(np.uint8)]
    assert np.all(v == np.round(v))
    return v.astype(np.int64)


def to_dev(comps):
    import paper_2301_09960_gb300 as oz
    return [oz.colmajor(c) for c in comps]


def from_dev(ts):
    return [t.detach().cpu().numpy() for t in ts]
