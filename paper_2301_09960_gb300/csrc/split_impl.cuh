// Splitter: exponent reduce (K1) and exact truncating digit split (K2).
//
// Paper, Sec. 3, Algorithm 1: mu_A / mu_B (row / column maxima), the
// power-of-two shifts tau_A / tau_B, and the extraction of the slices
// A_alpha, B_alpha.  Here the shift of row i is 2^E_i with
// E_i = max_p floor(log2|a_ip|) + 1 of the exact element values, and the
// slices are the base-2^beta digits of |a_ip| 2^(beta s - E_i) truncated
// toward zero (sign of a_ip), found with exact integer arithmetic on the
// IEEE encodings.  The balanced e4m3 form writes the same truncated value,
// floor(|a_ip| 2^(5 s - 1 - E_i)), in balanced radix-32 digits.
#pragma once
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include "ozmp_internal.cuh"
#include "kernels.h"
#include "bound.cuh"

namespace ozmp {

template <typename T>
struct Operand {
    const T* c[4];
    int64_t ld;
    int q;
};

static __global__ void k_init_exponents(int32_t* E, int64_t mp, int32_t* F, int64_t np, uint32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < mp) E[i] = OZMP_EXP_ZERO;
    if (i < np) F[i] = OZMP_EXP_ZERO;
    if (i == 0) *status = 0u;
}

template <typename T>
__device__ __forceinline__ bool load_elem(const Operand<T>& op, int64_t idx, T (&v)[4], Comp (&c)[4], int& Ptop) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (i < op.q) ? op.c[i][idx] : (T)0;
    return decode_all<T>(v, op.q, c, Ptop);
}

// the components of element idx (zeros when !inside), loaded without any
// arithmetic so that a thread's loads of several elements are all in flight
// before the first one is decoded
template <typename T>
__device__ __forceinline__ void load_raw(const Operand<T>& op, int q, bool inside, int64_t idx, T (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (inside && i < q) ? op.c[i][idx] : (T)0;
}

// exponent of one loaded element; false for a non-finite component.  The
// encodings alone settle almost every element (exponent_fast); the others
// are decoded and summed exactly.
template <typename T>
__device__ __forceinline__ bool exponent_loaded(const T (&v)[4], int q, int& e) {
    if (exponent_fast<T>(v, q, e)) return true;
    Comp c[4];
    int Ptop;
    const bool ok = decode_all<T>(v, q, c, Ptop);
    e = exponent_of<T>(c, v, q, Ptop);
    return ok;
}

// ---------------------------------------------------------------------------
// K1: exponents
// ---------------------------------------------------------------------------
// rows of a column-major m x k matrix: one thread per row, a chunk of
// columns per block row; consecutive threads read consecutive addresses.
// Q > 0: the component count known at compile time (the loops over the
// components and their registers shrink to it); Q = 0: a.q at run time.
template <typename T, int Q = 0>
__device__ __forceinline__ void exp_rows_body(Operand<T> a, int64_t m, int64_t k, int kchunk, int32_t* E,
                                                  uint32_t* status, int64_t bx, int64_t by) {
    const int q = Q ? Q : a.q;
    int64_t i = bx * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t p0 = by * kchunk;
    int64_t p1 = p0 + kchunk < k ? p0 + kchunk : k;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    constexpr int U = 4;   // elements whose loads are issued together
    for (int64_t p = p0; p < p1; p += U) {
        T v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) load_raw<T>(a, q, p + u < p1, i + (p + u) * a.ld, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int e;
            ok &= exponent_loaded<T>(v[u], q, e);
            emax = e > emax ? e : emax;
        }
    }
    if (emax != OZMP_EXP_ZERO) atomicMax(&E[i], emax);
    if (!ok) atomicOr(status, ST_NONFINITE);
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_exp_rows(Operand<T> a, int64_t m, int64_t k, int kchunk, int32_t* E,
                                                  uint32_t* status) {
    exp_rows_body<T, Q>(a, m, k, kchunk, E, status, (int64_t)blockIdx.x, (int64_t)blockIdx.y);
}

// columns of a column-major k x n matrix (contiguous): `split` warps per
// column (consecutive warps, each a contiguous part of k), warp-shuffle max
// reduction, atomicMax across the parts (F starts at OZMP_EXP_ZERO).
template <typename T, int Q = 0>
__device__ __forceinline__ void exp_cols_body(Operand<T> b, int64_t k, int64_t n, int32_t* F, uint32_t* status,
                                              int64_t bx, int64_t by, int split = 1) {
    const int q = Q ? Q : b.q;
    int warps = blockDim.x >> 5;
    int64_t gw = bx * warps + (threadIdx.x >> 5);
    int64_t j = gw / split;
    int part = (int)(gw % split);
    int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int64_t plen = ((k + split - 1) / split + 31) / 32 * 32;
    const int64_t pa = part * plen, pb = pa + plen < k ? pa + plen : k;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    constexpr int U = 4;   // elements whose loads are issued together
    for (int64_t p = pa + lane; p < pb; p += 32 * U) {
        T v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) load_raw<T>(b, q, p + 32 * u < pb, p + 32 * u + j * b.ld, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int e;
            ok &= exponent_loaded<T>(v[u], q, e);
            emax = e > emax ? e : emax;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int v = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = v > emax ? v : emax;
    }
    unsigned bad = __ballot_sync(0xffffffffu, !ok);
    if (lane == 0) {
        if (split == 1) F[j] = emax;
        else if (emax != OZMP_EXP_ZERO) atomicMax(&F[j], emax);
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_exp_cols(Operand<T> b, int64_t k, int64_t n, int32_t* F, uint32_t* status,
                                                  int split) {
    exp_cols_body<T, Q>(b, k, n, F, status, (int64_t)blockIdx.x, (int64_t)blockIdx.y, split);
}

// ---------------------------------------------------------------------------
// K1 with the statistics of the data-dependent slice count (bound.cuh): the
// same exponents, and beside them the squared norms of the elements (each
// magnitude estimated from its exact exponent and leading component, in
// binary32: mag_est_f32), unscaled (the caller falls back to scaled norms
// when the exponents leave +-BOUND_RAW_EXP, where no square or sum of squares
// can overflow or vanish in binary32): colA[p] += sum_i a_ip^2 over the
// block's rows, rowB[p] += sum_j b_pj^2 over the block's columns (both zeroed
// before).
__device__ __forceinline__ int xmax_warp(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// |x| of an element as a binary32 from bit operations only (the binary64
// pipe is slow on this GPU): the leading component when its exponent is the
// element's exact exponent e (2^(e-1) <= |x| < 2^e), else 2^(e-1), a lower
// bound (components that cancel cannot inflate it).  0 for a zero element or
// below the binary32 normal range; saturated above it (exponents beyond
// +-BOUND_RAW_EXP send the caller to the scaled norms anyway).
template <typename T>
__device__ __forceinline__ float mag_est_f32(const T (&v)[4], int e) {
    if (e == OZMP_EXP_ZERO) return 0.f;
    int fe;            // binary32 exponent field of the estimate
    unsigned man = 0;  // its mantissa bits
    if constexpr (sizeof(T) == 8) {
        const unsigned long long b = (unsigned long long)__double_as_longlong((double)v[0]);
        const int ef = (int)((b >> 52) & 0x7ff);
        if (ef != 0 && ef - 1022 == e) { fe = ef - 1023 + 127; man = (unsigned)((b >> 29) & 0x7fffffu); }
        else fe = e - 1 + 127;
    } else {
        const unsigned b = __float_as_uint((float)v[0]);
        const int ef = (int)((b >> 23) & 0xff);
        if (ef != 0 && ef - 126 == e) { fe = ef; man = b & 0x7fffffu; }
        else fe = e - 1 + 127;
    }
    if (fe <= 0) return 0.f;
    if (fe >= 255) { fe = 254; man = 0x7fffffu; }
    return __uint_as_float(((unsigned)fe << 23) | man);
}

// 16 per-lane values v[c] (c = column) summed over the 32 lanes of a warp by
// recursive halving: each step hands half of the columns to the partner lane;
// at the end lanes 2c and 2c + 1 hold the sum of column c (16 shuffle steps
// per warp instead of a 5-step reduction per column)
__device__ __forceinline__ float xsum16_warp(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;   // this lane keeps the upper half of the columns
#pragma unroll
        for (int c = 0; c < h; ++c) {
            const float give = up ? v[c] : v[c + h];
            const float got = __shfl_xor_sync(0xffffffffu, give, o);
            v[c] = (up ? v[c + h] : v[c]) + got;
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// rows of A: one thread per row, KC = 16 columns per block row (as
// k_exp_rows); a thread keeps its 16 squares in registers, the warp sums them
// by recursive halving, the block in shared memory, then one global atomic
// per block and column
template <typename T, int Q>
__global__ void __launch_bounds__(256) k_exp_rows_norm(Operand<T> a, int64_t m, int64_t k, int32_t* E,
                                                       uint32_t* status, double* colA) {
    constexpr int KC = 16, U = 4;
    __shared__ double sc[KC];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = i < m;
    const int64_t p0 = (int64_t)blockIdx.y * KC;
    const int64_t p1 = p0 + KC < k ? p0 + KC : k;
    if (threadIdx.x < KC) sc[threadIdx.x] = 0.0;
    __syncthreads();
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    float sq[KC];
#pragma unroll
    for (int g = 0; g < KC / U; ++g) {
        const int64_t p = p0 + g * U;
        T v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) load_raw<T>(a, Q, in && p + u < p1, i + (p + u) * a.ld, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int e;
            ok &= exponent_loaded<T>(v[u], Q, e);   // zeros outside the matrix: no exponent
            emax = e > emax ? e : emax;
            const float x = mag_est_f32<T>(v[u], e);
            sq[g * U + u] = x * x;
        }
    }
    const float w = xsum16_warp(sq);
    const int lane = threadIdx.x & 31;
    if ((lane & 1) == 0 && (lane >> 1) < p1 - p0) atomicAdd(&sc[lane >> 1], (double)w);
    __syncthreads();
    if (threadIdx.x < p1 - p0) atomicAdd(&colA[p0 + threadIdx.x], sc[threadIdx.x]);
    if (in && emax != OZMP_EXP_ZERO) atomicMax(&E[i], emax);
    if (!ok) atomicOr(status, ST_NONFINITE);
}

// columns of B: one thread per row p (coalesced along the column), JB
// columns per block; a column's exponent is reduced over the warp and the
// block (one global atomicMax per block and column), a row's squares are
// summed in the thread (one global atomicAdd per thread)
template <typename T, int Q>
__global__ void __launch_bounds__(256) k_exp_cols_norm(Operand<T> b, int64_t k, int64_t n, int32_t* F,
                                                       uint32_t* status, double* rowB) {
    constexpr int JB = 64, U = 4;
    __shared__ int sf[JB];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < k;
    const int64_t j0 = (int64_t)blockIdx.y * JB;
    const int64_t j1 = j0 + JB < n ? j0 + JB : n;
    if (threadIdx.x < JB) sf[threadIdx.x] = OZMP_EXP_ZERO;
    __syncthreads();
    float acc = 0.f;
    bool ok = true;
    for (int64_t j = j0; j < j1; j += U) {
        T v[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) load_raw<T>(b, Q, in && j + u < j1, p + (j + u) * b.ld, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j + u >= j1) break;   // uniform over the block
            int e;
            ok &= exponent_loaded<T>(v[u], Q, e);
            const int w = xmax_warp(e);
            if ((threadIdx.x & 31) == 0 && w != OZMP_EXP_ZERO) atomicMax(&sf[j + u - j0], w);
            const float x = mag_est_f32<T>(v[u], e);
            acc += x * x;
        }
    }
    __syncthreads();
    if (threadIdx.x < j1 - j0 && sf[threadIdx.x] != OZMP_EXP_ZERO) atomicMax(&F[j0 + threadIdx.x], sf[threadIdx.x]);
    if (in && acc != 0.f) atomicAdd(&rowB[p], (double)acc);
    if (!ok) atomicOr(status, ST_NONFINITE);
}

// ---------------------------------------------------------------------------
// K2: digits
// ---------------------------------------------------------------------------
// encodings: FORM_INT8 -> two's complement int8, FORM_FP8 -> e4m3,
// FORM_FP64 -> binary64 integer value.
template <int FORM>
struct DigitTraits;
template <> struct DigitTraits<OZMP_FORM_INT8> { static constexpr int BETA = 7; static constexpr int MAXS = 36; };
template <> struct DigitTraits<OZMP_FORM_FP8> { static constexpr int BETA = 4; static constexpr int MAXS = 64; };
template <> struct DigitTraits<OZMP_FORM_FP8_BAL> { static constexpr int BETA = 5; static constexpr int MAXS = 63; };

// the digit windows of four elements -> one 32-bit word of slice t
template <int FORM, int NW>
__device__ __forceinline__ uint32_t pack4(const uint64_t (&w)[4][NW], const int (&sign)[4], int t) {
    constexpr int BETA = DigitTraits<FORM>::BETA;
    uint32_t m4 = 0, neg = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        m4 |= digit_of<NW, BETA>(w[e], t) << (8 * e);
        if (sign[e] < 0) neg |= (FORM == OZMP_FORM_INT8 ? 0xFFu : 0x80u) << (8 * e);
    }
    return (FORM == OZMP_FORM_INT8) ? int8x4(m4, neg) : e4m3x4(m4, neg);
}

// The e4m3 digits of four elements (consecutive k), all slices: calls
// put(t, word) for t = 1 .. s with byte e of `word` = e4m3 code of digit t of
// element e.  The windows are shifted left one bit so that digit t becomes
// the nibble at bits [64 NW - 4 t, 64 NW - 4 t + 4): each 32-bit half-word
// then holds 8 whole digits, encoded 4 at a time by table lookup and
// transposed across the elements in registers.
template <int NW, typename Put>
__device__ __forceinline__ void pack_fp8_quad(uint64_t (&w)[4][NW], const int (&sign)[4], int s, Put&& put) {
    constexpr int MAXS = DigitTraits<OZMP_FORM_FP8>::MAXS;
    uint32_t negm[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        mw_shl<NW>(w[e], 1);
        negm[e] = sign[e] < 0 ? 0x80808080u : 0u;
    }
#pragma unroll
    for (int h = 0; h < 2 * NW && 8 * h < MAXS; ++h) {
        if (8 * h >= s) break;
        const int wi = NW - 1 - (h >> 1);
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t X = (h & 1) ? (uint32_t)w[e][wi] : (uint32_t)(w[e][wi] >> 32);
            lo[e] = e4m3_nibbles4(X, negm[e]);         // digits 8h+8, 8h+7, 8h+6, 8h+5 in bytes 0..3
            hi[e] = e4m3_nibbles4(X >> 16, negm[e]);   // digits 8h+4 .. 8h+1
        }
        uint32_t th[4], tl[4];
        transpose4(hi, th);
        transpose4(lo, tl);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (8 * h + 4 - b <= s) put(8 * h + 4 - b, th[b]);
            if (8 * h + 8 - b <= s) put(8 * h + 8 - b, tl[b]);
        }
    }
}

// 32-bit word i of a multiword value (zero outside it)
template <int NW>
__device__ __forceinline__ uint32_t word32_of(const uint64_t (&w)[NW], int i) {
    return (i < 0 || i >= 2 * NW) ? 0u : (uint32_t)(w[i >> 1] >> (32 * (i & 1)));
}

// bits [pos, pos + 32) of a multiword value, zeros outside it (pos >= -32).
// With pos a compile-time constant (an unrolled digit loop) the two words are
// fixed registers and this is a single funnel shift.
template <int NW>
__device__ __forceinline__ uint32_t bits32_at(const uint64_t (&w)[NW], int pos) {
    const int i = (pos + 32) / 32 - 1;     // floor(pos / 32) for pos >= -32
    const int r = pos - 32 * i;
    return __funnelshift_r(word32_of<NW>(w, i), word32_of<NW>(w, i + 1), r);
}

// The balanced radix-32 e4m3 digits of four elements (consecutive k), all
// slices: calls put(t, word) for t = 1 .. s with byte e of `word` = e4m3 code
// of digit t of element e.  The magnitude window holds
// floor(|x| 2^(64 NW - 1 - E)) with at least GUARD bits below the lowest
// group; group t of its top 5 s bits is digit t of
// N = floor(|x| 2^(5 s - 1 - E)) in plain radix 32.  Adding 16 to every
// group (G = window + sum_t 16 2^(64 NW - 5 t), nothing added below the
// lowest group, so no carry enters it) makes the groups of G the balanced
// digits plus 16: d_t = g_t - 16 in [-16, 15], and the carry out of the top
// group turns d_1 into 16.  Each g goes through binary16 as 1024 + g (exact),
// one fused multiply-add applies -16 and the element's sign (exact: the
// result is an integer of magnitude <= 16, a zero digit comes out +0), and
// the conversion to e4m3 is exact for these integers.  Two elements share
// one binary16 pair: element 2h's group is cut out at bit 0 and element
// 2h + 1's at bit 16, each by one funnel shift.
template <int NW, int GUARD, typename Put>
__device__ __forceinline__ void pack_bal_quad(uint64_t (&w)[4][NW], const int (&sign)[4], int s, Put&& put) {
    constexpr int TMAX = (64 * NW - GUARD) / 5;
    const int lo = 64 * NW - 5 * s;   // lowest bit of the lowest group (>= GUARD)
    constexpr BalSixteens<NW> P16;
    uint64_t H[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint64_t keep = (lo <= 64 * j) ? ~0ull : (lo >= 64 * j + 64 ? 0ull : (~0ull << (lo - 64 * j)));
        H[j] = P16.w[j] & keep;
    }
    uint32_t top[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        // the top word gets bit 63 of H and never equals its old value: it
        // wrapped (the carry out of the top group) iff it came out smaller
        const uint64_t before = w[e][NW - 1];
        mw_add<NW>(w[e], H);
        if (w[e][NW - 1] < before) top[e >> 1] |= (e & 1) ? 0x200000u : 0x20u;
    }
    // per pair of elements: binary16 multipliers (+-1) and addends (-+1040)
    __half2 mul[2], add[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float s0 = sign[2 * h] < 0 ? -1.f : 1.f, s1 = sign[2 * h + 1] < 0 ? -1.f : 1.f;
        mul[h] = __floats2half2_rn(s0, s1);
        add[h] = __floats2half2_rn(-1040.f * s0, -1040.f * s1);
    }
#pragma unroll
    for (int t = 1; t <= TMAX; ++t) {
        if (t > s) break;
        const int pos = 64 * NW - 5 * t;
        uint32_t c[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t x0 = bits32_at<NW>(w[2 * h], pos);         // group at bits 0..4
            const uint32_t x1 = bits32_at<NW>(w[2 * h + 1], pos - 16);  // group at bits 16..20
            uint32_t bits = (x0 & 0x1Fu) | (x1 & 0x1F0000u) | 0x64006400u;   // 1024 + g, two lanes
            if (t == 1) bits |= top[h];
            __half2 v = *reinterpret_cast<const __half2*>(&bits);
            v = __hfma2(v, mul[h], add[h]);
            c[h] = (uint32_t)__nv_cvt_halfraw2_to_fp8x2(static_cast<__half2_raw>(v), __NV_SATFINITE, __NV_E4M3);
        }
        put(t, __byte_perm(c[0], c[1], 0x5410));
    }
}

template <typename T, int NW>
__device__ __forceinline__ int window_of(const Operand<T>& op, bool inside, int64_t idx, int Erow, uint64_t (&w)[NW]) {
    Comp c[4];
    T v[4] = {(T)0, (T)0, (T)0, (T)0};
    int Ptop = -100000;
    if (inside) load_elem<T>(op, idx, v, c, Ptop);
    if (!inside || Ptop == -100000 || Erow == OZMP_EXP_ZERO) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        return 0;
    }
    return digit_window<NW, T>(c, v, op.q, Erow, w);
}

// bits [o, o + 64) of the 128-bit value s1:s0 (zeros outside it)
__device__ __forceinline__ uint64_t bits128(uint64_t s0, uint64_t s1, int o) {
    if (o <= -64 || o >= 128) return 0ull;
    if (o < 0) return s0 << (-o);
    if (o == 0) return s0;
    if (o < 64) return (s0 >> o) | (s1 << (64 - o));
    if (o == 64) return s1;
    return s1 >> (o - 64);
}

// Two binary64 components whose exponents differ by at most 74: their exact
// sum S as a signed 128-bit integer at the smaller one's exponent, then
// floor(|S| 2^(e - L)) placed in the window in one shift (the exact
// truncated magnitude, every word exact).  Returns false, leaving w alone,
// when the components are further apart.
template <int NW>
__device__ __forceinline__ bool window_two(double hi, double lo, int Erow, uint64_t (&w)[NW], int& sg) {
    Comp a, b;
    decode(hi, a);
    decode(lo, b);
    if (b.M && (!a.M || b.e > a.e)) { const Comp t = a; a = b; b = t; }   // a: the larger exponent
    if (!a.M || Erow == OZMP_EXP_ZERO) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        sg = 0;
        return true;
    }
    unsigned __int128 S;
    int es;
    bool neg;
    if (!b.M) {
        S = a.M; es = a.e; neg = a.neg != 0;
    } else {
        const int d = a.e - b.e;
        if (d > 74) return false;   // 53 + 74 bits fit the signed 128-bit sum
        __int128 sa = (__int128)((unsigned __int128)a.M << d);
        if (a.neg) sa = -sa;
        __int128 sb = (__int128)b.M;
        if (b.neg) sb = -sb;
        const __int128 t = sa + sb;
        neg = t < 0;
        S = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
        es = b.e;
    }
    const int L = Erow - (64 * NW - 1);   // weight of window bit 0
    const int sh = es - L;
    const uint64_t s0 = (uint64_t)S, s1 = (uint64_t)(S >> 64);
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = bits128(s0, s1, 64 * j - sh);
    sg = S == 0 ? 0 : (neg ? -1 : 1);
    return true;
}

// the same on components already loaded (zeros outside the matrix); two
// binary64 components known at compile time (Q = 2) first try the 128-bit frame
template <typename T, int NW, int Q = 0>
__device__ __forceinline__ int window_loaded(const T (&v)[4], int q, int Erow, uint64_t (&w)[NW]) {
    if constexpr (Q == 2 && sizeof(T) == 8) {
        int sg;
        if (window_two<NW>((double)v[0], (double)v[1], Erow, w, sg)) return sg;
    }
    Comp c[4];
    int Ptop;
    decode_all<T>(v, q, c, Ptop);
    if (Ptop == -100000 || Erow == OZMP_EXP_ZERO) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        return 0;
    }
    return digit_window<NW, T>(c, v, q, Erow, w);
}

// Two binary64 components: the top three words of the four-word window, that
// is floor(|x| 2^(191 - E)) with no guard bits, which is all that balanced
// digits of up to 38 slices read.  The 128-bit frame gives it directly;
// components more than 74 binades apart take the general window.
template <typename T>
__device__ __forceinline__ int window_top3(const T (&v)[4], int Erow, uint64_t (&w3)[3]) {
    int sg;
    if (window_two<3>((double)v[0], (double)v[1], Erow, w3, sg)) return sg;
    uint64_t w4[4];
    sg = window_loaded<T, 4, 0>(v, 2, Erow, w4);
    w3[0] = w4[1];
    w3[1] = w4[2];
    w3[2] = w4[3];
    return sg;
}

// balanced digits of two binary64 components read a three-word window
template <typename T, int FORM, int NW, int Q>
constexpr bool DIGITS_DD3 = FORM == OZMP_FORM_FP8_BAL && Q == 2 && sizeof(T) == 8 && NW == 4;

// the digits of four loaded elements (consecutive k) that share the exponent
// Ex: put(t, word) for t = 1 .. s, byte e of word = digit t of element e
template <typename T, int FORM, int NW, int Q, typename Put>
__device__ __forceinline__ void quad_digits(const T (&v)[4][4], int q, int Ex, int s, Put&& put) {
    int sign[4];
    if constexpr (DIGITS_DD3<T, FORM, NW, Q>) {
        uint64_t w3[4][3];
#pragma unroll
        for (int e = 0; e < 4; ++e) sign[e] = window_top3<T>(v[e], Ex, w3[e]);
        pack_bal_quad<3, 0>(w3, sign, s, put);
    } else {
        uint64_t w[4][NW];
#pragma unroll
        for (int e = 0; e < 4; ++e) sign[e] = window_loaded<T, NW, Q>(v[e], q, Ex, w[e]);
        if constexpr (FORM == OZMP_FORM_FP8) {
            pack_fp8_quad<NW>(w, sign, s, put);
        } else if constexpr (FORM == OZMP_FORM_FP8_BAL) {
            pack_bal_quad<NW, 65>(w, sign, s, put);
        } else {
#pragma unroll
            for (int t = 1; t <= DigitTraits<FORM>::MAXS; ++t)
                if (t <= s) put(t, pack4<FORM, NW>(w, sign, t));
        }
    }
}

// Rows of A (column-major) -> Adig[(t * mp + i) * kp + p], 1-byte digits.
// Tile: 32 rows x 64 columns, 256 threads; thread (row ri, quad) handles
// 4 consecutive columns of one row (two quads per thread); the 4 digits of
// a slice go to shared memory as one word, then the tile is written
// K-contiguous in 16-byte pieces.  Word qd of tile row ri sits at position
// qd ^ (ri >> 1) of its 16-word row: the 32 rows of a warp's store then fall
// in 32 different banks, and so do the words of a warp's read-out.
template <typename T, int FORM, int NW, int Q = 0>
__device__ __forceinline__ void split_rows_b1_body(Operand<T> a, int64_t m, int64_t k, const int32_t* E,
                                                       uint8_t* dig, int64_t mp, int64_t kp, int s, int64_t bx, int64_t by) {
    const int q = Q ? Q : a.q;
    constexpr int TI = 32, TP = 64, QW = TP / 4;    // 16 words per tile row
    extern __shared__ __align__(16) uint32_t sw[];  // [s][TI][QW], swizzled rows
    const int64_t i0 = bx * TI, p0 = by * TP;
    const int ri = threadIdx.x & 31;
    const int64_t i = i0 + ri;
    const int Erow = (i < m) ? E[i] : OZMP_EXP_ZERO;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int qd = (threadIdx.x >> 5) + 8 * h;
        uint32_t* const srow = sw + ri * QW + (qd ^ (ri >> 1));
        T v[4][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t p = p0 + 4 * qd + e;
            load_raw<T>(a, q, i < m && p < k, i + p * a.ld, v[e]);
        }
        quad_digits<T, FORM, NW, Q>(v, q, Erow, s, [&](int t, uint32_t word) { srow[(t - 1) * TI * QW] = word; });
    }
    __syncthreads();
    // 16 bytes (four words) per thread and step: a warp covers 8 rows x 4 pieces
    const int total = s * TI * 4;
    for (int x = threadIdx.x; x < total; x += 256) {
        const int t = x / (TI * 4), r = (x >> 2) % TI, c4 = x & 3;
        const uint32_t* row = sw + (t * TI + r) * QW;
        const int z = r >> 1;
        uint4 u;
        u.x = row[(4 * c4 + 0) ^ z];
        u.y = row[(4 * c4 + 1) ^ z];
        u.z = row[(4 * c4 + 2) ^ z];
        u.w = row[(4 * c4 + 3) ^ z];
        *reinterpret_cast<uint4*>(dig + ((size_t)t * mp + (i0 + r)) * kp + p0 + 16 * c4) = u;
    }
}

template <typename T, int FORM, int NW, int Q>
__global__ void __launch_bounds__(256) k_split_rows_b1(Operand<T> a, int64_t m, int64_t k, const int32_t* E,
                                                       uint8_t* dig, int64_t mp, int64_t kp, int s) {
    split_rows_b1_body<T, FORM, NW, Q>(a, m, k, E, dig, mp, kp, s, (int64_t)blockIdx.x, (int64_t)blockIdx.y);
}

// Columns of B (contiguous along k) -> Bdig[(t * np + j) * kp + p], 1-byte
// digits: 4 consecutive k per thread, one 32-bit store per slice.  Thread g
// takes column g / quads, quads = kp / 4 (the whole padded workspace), or
// the given count (columns j < n and k < kp only, when the padding of the
// workspace is known to hold zero digits already).
template <typename T, int FORM, int NW, int Q = 0>
__device__ __forceinline__ void split_cols_b1_body(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                       uint8_t* dig, int64_t np, int64_t kp, int s, int64_t bx, int64_t by,
                                                       int64_t quads_only = 0) {
    const int q = Q ? Q : b.q;
    const int64_t quads = quads_only > 0 ? quads_only : kp / 4;
    int64_t g = bx * blockDim.x + threadIdx.x;
    if (g >= quads * (quads_only > 0 ? n : np)) return;
    const int64_t j = g / quads;
    const int64_t p0 = (g % quads) * 4;
    const int Ecol = (j < n) ? F[j] : OZMP_EXP_ZERO;
    T v[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) load_raw<T>(b, q, j < n && p0 + e < k, p0 + e + j * b.ld, v[e]);
    uint8_t* const base = dig + (size_t)j * kp + p0;
    const size_t slice = (size_t)np * kp;
    quad_digits<T, FORM, NW, Q>(v, q, Ecol, s, [&](int t, uint32_t word) {
        *reinterpret_cast<uint32_t*>(base + (size_t)(t - 1) * slice) = word;
    });
}

template <typename T, int FORM, int NW, int Q>
__global__ void __launch_bounds__(256) k_split_cols_b1(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                       uint8_t* dig, int64_t np, int64_t kp, int s) {
    split_cols_b1_body<T, FORM, NW, Q>(b, k, n, F, dig, np, kp, s, (int64_t)blockIdx.x, (int64_t)blockIdx.y);
}

// ---------------------------------------------------------------------------
// K1 + K2 for the columns of B in one pass: a block takes one column, copies
// its components into shared memory with one bulk copy each (the whole column
// in flight at once, no registers held), reduces the column exponent there and
// writes the column's digits from shared memory, so B is read once.
// ---------------------------------------------------------------------------
namespace colbulk {
constexpr long long WAIT_POLLS = 1ll << 24;   // try_wait polls before giving up

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16) from a 16-byte aligned global address
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     saddr(dst)),
                 "l"(src), "r"(bytes), "r"(saddr(b))
                 : "memory");
}
__device__ __forceinline__ bool wait(uint64_t* b, long long polls) {
    for (long long it = 0; it < polls; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(saddr(b))
            : "memory");
        if (ok) return true;
    }
    return false;
}
}  // namespace colbulk

// With rowBf set, the exponent pass also adds each element's squared
// magnitude estimate (mag_est_f32) into rowBf[p], coalesced along the column:
// the row norms of B for the data-dependent slice count, without a pass of
// its own over B.
template <typename T, int FORM, int NW, int Q>
__global__ void __launch_bounds__(256, 3) k_split_cols_fused(Operand<T> b, int64_t k, int64_t n, int32_t* F,
                                                          uint32_t* status, uint8_t* dig, int64_t np, int64_t kp,
                                                          int s, long long polls, int stall, float* rowBf) {
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
    const T* col = reinterpret_cast<const T*>(smraw + 16);   // [Q][k]
    __shared__ int red[8];
    __shared__ int bad_any;
    const int64_t j = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool live = j < n;   // padding columns get zero digits
    int Ecol = OZMP_EXP_ZERO;
    if (live) {
        if (tid == 0) {
            bad_any = 0;
            colbulk::bar_init(bar);
            const uint32_t bytes = (uint32_t)(k * (int64_t)sizeof(T));
            if (!stall) {   // (the test hook leaves the barrier incomplete, nothing in flight)
                colbulk::expect_tx(bar, bytes * Q);
#pragma unroll
                for (int c = 0; c < Q; ++c)
                    colbulk::copy(smraw + 16 + (size_t)c * bytes, b.c[c] + j * b.ld, bytes, bar);
            }
        }
        __syncthreads();
        // every thread sees the copies complete (bounded); the verdict is uniform
        const bool arrived = colbulk::wait(bar, polls);
        if (!__syncthreads_and(arrived)) {
            if (tid == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        int emax = OZMP_EXP_ZERO;
        bool ok = true;
        for (int64_t p = tid; p < k; p += 256) {
            T v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = (c < Q) ? col[(size_t)c * k + p] : (T)0;
            int e;
            ok &= exponent_loaded<T>(v, Q, e);
            emax = e > emax ? e : emax;
            if (rowBf) {
                const float x = mag_est_f32<T>(v, e);
                if (x != 0.f) atomicAdd(&rowBf[p], x * x);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int x = __shfl_xor_sync(0xffffffffu, emax, o);
            emax = x > emax ? x : emax;
        }
        if (lane == 0) red[wid] = emax;
        if (!ok) bad_any = 1;
        __syncthreads();
        Ecol = red[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) Ecol = red[w] > Ecol ? red[w] : Ecol;
        if (tid == 0) {
            F[j] = Ecol;
            if (bad_any) atomicOr(status, ST_NONFINITE);
        }
    }
    const int64_t quads = kp / 4;
    uint8_t* const cbase = dig + (size_t)j * kp;
    const size_t slice = (size_t)np * kp;
    for (int64_t g = tid; g < quads; g += 256) {
        const int64_t p0 = 4 * g;
        T v[4][4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                v[e][c] = (live && c < Q && p0 + e < k) ? col[(size_t)c * k + p0 + e] : (T)0;
        quad_digits<T, FORM, NW, Q>(v, Q, Ecol, s, [&](int t, uint32_t word) {
            *reinterpret_cast<uint32_t*>(cbase + (size_t)(t - 1) * slice + p0) = word;
        });
    }
}

// binary64 digits, rows of A: 16 x 16 tile staged in shared memory
// a digit of magnitude `mag` (at most 26 bits) and the element's sign in the
// stored type: binary64, or binary16 for the binary16-digit form (|d| <= 2047
// there), converted from the integer directly (exact; no binary64 arithmetic,
// whose pipe is narrow on this GPU; a zero digit is +0)
template <typename DT>
__device__ __forceinline__ DT digit_value(uint32_t mag, int sign) {
    const double d = (double)mag;
    return (DT)(sign < 0 ? -d : d);
}
template <>
__device__ __forceinline__ __half digit_value<__half>(uint32_t mag, int sign) {
    const int v = (int)mag;
    return __int2half_rn(sign < 0 ? -v : v);
}

template <typename T, int NW, typename DT = double>
__global__ void __launch_bounds__(256) k_split_rows_f64(Operand<T> a, int64_t m, int64_t k, const int32_t* E,
                                                        DT* dig, int64_t mp, int64_t kp, int s, int beta) {
    constexpr int TI = 16, TP = 16;
    extern __shared__ __align__(16) unsigned char sd_raw[];
    DT* sd = reinterpret_cast<DT*>(sd_raw);         // [s][TI][TP]
    const int64_t i0 = (int64_t)blockIdx.x * TI, p0 = (int64_t)blockIdx.y * TP;
    const int ri = threadIdx.x % TI, pi = threadIdx.x / TI;
    const int64_t i = i0 + ri, p = p0 + pi;
    const int Erow = (i < m) ? E[i] : OZMP_EXP_ZERO;
    uint64_t w[NW];
    const int sign = window_of<T, NW>(a, i < m && p < k, i + p * a.ld, Erow, w);
    for (int t = 1; t <= s; ++t) {
        sd[((t - 1) * TI + ri) * TP + pi] = digit_value<DT>(digit_of_rt<NW>(w, t, beta), sign);
    }
    __syncthreads();
    const int total = s * TI * TP;
    for (int x = threadIdx.x; x < total; x += 256) {
        const int t = x / (TI * TP), r = (x / TP) % TI, c = x % TP;
        dig[((size_t)t * mp + (i0 + r)) * kp + p0 + c] = sd[x];
    }
}

// binary64 digits, columns of B: one element per thread
template <typename T, int NW, typename DT = double>
__global__ void __launch_bounds__(256) k_split_cols_f64(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                        DT* dig, int64_t np, int64_t kp, int s, int beta) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= kp * np) return;
    const int64_t j = g / kp, p = g % kp;
    const int Ecol = (j < n) ? F[j] : OZMP_EXP_ZERO;
    uint64_t w[NW];
    const int sign = window_of<T, NW>(b, j < n && p < k, p + j * b.ld, Ecol, w);
    for (int t = 1; t <= s; ++t) {
        dig[((size_t)(t - 1) * np + j) * kp + p] = digit_value<DT>(digit_of_rt<NW>(w, t, beta), sign);
    }
}

// Binary16 digits of a width BETA known at compile time (5, 6 or 7 bits:
// the widths of 259 <= k <= 17459), four consecutive k of one row or column
// per thread as in the 1-byte digit kernels: digit t of element e is a fixed
// bit field of its exact window, converted from the integer to binary16
// directly (exact: |d| < 2^BETA), a zero digit +0.
template <int NW, int BETA>
__device__ __forceinline__ uint2 halves4(const uint64_t (&w)[4][NW], const int (&sg)[4], int t) {
    uint32_t h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int d = (int)digit_of<NW, BETA>(w[e], t);
        h[e] = (uint32_t)__half_as_ushort(__int2half_rn(sg[e] < 0 ? -d : d));
    }
    return make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
}

// Rows of A -> Adig[(t * mp + i) * kp + p] (binary16): tile 32 rows x 64
// columns, thread (row, quad) takes 4 consecutive columns of one row (two
// quads a thread); a slice's 4 digits go to shared memory as 8 bytes, quad qd
// of tile row r at position qd ^ (r & 15) of its 16 (a warp's 32 rows then
// fall on 16 distinct 8-byte slots: two wavefronts, the least for 256 bytes),
// and the tile is written K-contiguous in 16-byte pieces.
template <typename T, int NW, int Q, int BETA>
__global__ void __launch_bounds__(256) k_split_rows_h(Operand<T> a, int64_t m, int64_t k, const int32_t* E,
                                                      __half* dig, int64_t mp, int64_t kp, int s) {
    constexpr int TI = 32, TP = 64, MAXS = (64 * NW - 65) / BETA;
    extern __shared__ __align__(16) uint2 sq[];   // [s][TI][16]
    const int64_t i0 = (int64_t)blockIdx.x * TI, p0 = (int64_t)blockIdx.y * TP;
    const int ri = threadIdx.x & 31;
    const int64_t i = i0 + ri;
    const int Erow = (i < m) ? E[i] : OZMP_EXP_ZERO;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int qd = (threadIdx.x >> 5) + 8 * h;
        T v[4][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t p = p0 + 4 * qd + e;
            load_raw<T>(a, Q, i < m && p < k, i + p * a.ld, v[e]);
        }
        uint64_t w[4][NW];
        int sg[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) sg[e] = window_loaded<T, NW, Q>(v[e], Q, Erow, w[e]);
        uint2* const dst = sq + ri * 16 + (qd ^ (ri & 15));
#pragma unroll
        for (int t = 1; t <= MAXS; ++t) {
            if (t > s) break;
            dst[(t - 1) * TI * 16] = halves4<NW, BETA>(w, sg, t);
        }
    }
    __syncthreads();
    const int total = s * TI * 8;   // 16-byte pieces: 8 a tile row and slice
    for (int x = threadIdx.x; x < total; x += 256) {
        const int t = x / (TI * 8), r = (x >> 3) % TI, c8 = x & 7;
        const uint2* row = sq + (t * TI + r) * 16;
        const int z = r & 15;
        const uint2 lo = row[(2 * c8) ^ z], hi = row[(2 * c8 + 1) ^ z];
        *reinterpret_cast<uint4*>(dig + ((size_t)t * mp + (i0 + r)) * kp + p0 + 8 * c8) =
            make_uint4(lo.x, lo.y, hi.x, hi.y);
    }
}

// Columns of B -> Bdig[(t * np + j) * kp + p] (binary16): thread g takes 4
// consecutive k of column g / (kp / 4), one 8-byte store per slice (the
// padding of the workspace gets zero digits).
template <typename T, int NW, int Q, int BETA>
__global__ void __launch_bounds__(256) k_split_cols_h(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                      __half* dig, int64_t np, int64_t kp, int s) {
    constexpr int MAXS = (64 * NW - 65) / BETA;
    const int64_t quads = kp / 4;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= quads * np) return;
    const int64_t j = g / quads, p0 = (g % quads) * 4;
    const int Ecol = (j < n) ? F[j] : OZMP_EXP_ZERO;
    T v[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) load_raw<T>(b, Q, j < n && p0 + e < k, p0 + e + j * b.ld, v[e]);
    uint64_t w[4][NW];
    int sg[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) sg[e] = window_loaded<T, NW, Q>(v[e], Q, Ecol, w[e]);
    uint2* const base = reinterpret_cast<uint2*>(dig + (size_t)j * kp + p0);
    const size_t slice = (size_t)np * kp / 4;   // uint2 units
#pragma unroll
    for (int t = 1; t <= MAXS; ++t) {
        if (t > s) break;
        base[(size_t)(t - 1) * slice] = halves4<NW, BETA>(w, sg, t);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
static inline Operand<T> make_op(const void* const* comps, int q, int64_t ld) {
    Operand<T> o;
    for (int i = 0; i < 4; ++i) o.c[i] = (i < q) ? (const T*)comps[i] : nullptr;
    o.ld = ld;
    o.q = q;
    return o;
}

// words of the digit window: word 0 below every digit, sign bit on top
static inline int digit_words(int beta, int s) { return (beta * s + 65 + 63) / 64; }

// shared memory of the one-pass column kernel, or 0 where it does not apply:
// e4m3 digits, whole columns of at most 112 KB (two blocks per SM), and
// 16-byte aligned column starts and lengths for the bulk copies
static inline size_t cols_fused_smem(const SplitArgs& g) {
    if (g.big || !(g.form == OZMP_FORM_FP8 || g.form == OZMP_FORM_FP8_MMA)) return 0;
    if (g.is_f32 ? g.q != 3 : (g.q < 2 || g.q > 4)) return 0;
    if (g.n <= 0 || g.k <= 0) return 0;
    const size_t es = g.is_f32 ? 4 : 8;
    const size_t bytes = (size_t)g.k * es;
    if (bytes % 16 != 0 || ((size_t)g.ldb * es) % 16 != 0) return 0;
    for (int c = 0; c < g.q; ++c)
        if ((uintptr_t)g.B[c] % 16 != 0) return 0;
    const size_t total = 16 + bytes * (size_t)g.q;
    return total <= 112 * 1024 + 16 ? total : 0;
}

template <typename T, int FORM, int NW, int Q>
static cudaError_t digits_b1_q(const SplitArgs& g, cudaStream_t st) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    cudaError_t e = cudaSuccess;
    if (g.parts != 2) {
        dim3 gr((unsigned)(g.mp / 32), (unsigned)(g.kp / 64));
        size_t sm = (size_t)g.s * 32 * 16 * 4;
        auto kr = k_split_rows_b1<T, FORM, NW, Q>;
        e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        kr<<<gr, 256, sm, st>>>(a, g.m, g.k, g.E, (uint8_t*)g.Adig, g.mp, g.kp, g.s);
    }
    if (g.parts == 1) return cudaGetLastError();
    if constexpr ((FORM == OZMP_FORM_FP8 || FORM == OZMP_FORM_FP8_BAL) && Q > 0) {
        const size_t fsm = cols_fused_smem(g);
        if (fsm) {
            auto kf = k_split_cols_fused<T, FORM, NW, Q>;
            e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
            if (e != cudaSuccess) return e;
            const long long polls = g.wait_limit > 0 ? g.wait_limit : colbulk::WAIT_POLLS;
            kf<<<(unsigned)g.np, 256, fsm, st>>>(b, g.k, g.n, g.F, g.status, (uint8_t*)g.Bdig, g.np, g.kp, g.s,
                                                 polls, g.inject_stall, g.rowBf);
            return cudaGetLastError();
        }
    }
    if (g.rowBf) return cudaErrorInvalidValue;   // only the one-pass column kernel sums the norms
    int64_t tot = (g.kp / 4) * g.np;
    k_split_cols_b1<T, FORM, NW, Q><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, g.k, g.n, g.F,
                                                                                 (uint8_t*)g.Bdig, g.np, g.kp, g.s);
    return cudaGetLastError();
}

// the e4m3 form (the product path) is specialised on the component count;
// the int8 form keeps it a run-time value
template <typename T, int FORM, int NW>
static cudaError_t digits_b1(const SplitArgs& g, cudaStream_t st) {
    constexpr bool e4m3 = (FORM == OZMP_FORM_FP8 || FORM == OZMP_FORM_FP8_BAL);
    if constexpr (e4m3 && sizeof(T) == 8) {
        if (g.q == 2) return digits_b1_q<T, FORM, NW, 2>(g, st);
        if (g.q == 3) return digits_b1_q<T, FORM, NW, 3>(g, st);
        return digits_b1_q<T, FORM, NW, 4>(g, st);
    } else if constexpr (e4m3) {
        return digits_b1_q<T, FORM, NW, 3>(g, st);
    } else {
        return digits_b1_q<T, FORM, NW, 0>(g, st);
    }
}

// general-beta digits as binary64 (DT = double) or binary16 (DT = __half)
// values: the same exact windows, one element per thread
template <typename T, int NW, typename DT = double>
static cudaError_t digits_f64(const SplitArgs& g, cudaStream_t st) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    dim3 gr((unsigned)(g.mp / 16), (unsigned)(g.kp / 16));
    size_t sm = (size_t)g.s * 16 * 16 * sizeof(DT);
    auto kr = k_split_rows_f64<T, NW, DT>;
    cudaError_t e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kr<<<gr, 256, sm, st>>>(a, g.m, g.k, g.E, (DT*)g.Adig, g.mp, g.kp, g.s, g.beta);
    int64_t tot = g.kp * g.np;
    k_split_cols_f64<T, NW, DT><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, g.k, g.n, g.F, (DT*)g.Bdig,
                                                                              g.np, g.kp, g.s, g.beta);
    return cudaGetLastError();
}

// binary16 digits of compile-time width BETA (k_split_rows_h, k_split_cols_h)
template <typename T, int NW, int Q, int BETA>
static cudaError_t digits_h(const SplitArgs& g, cudaStream_t st) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    const size_t sm = (size_t)g.s * 32 * 16 * sizeof(uint2);
    auto kr = k_split_rows_h<T, NW, Q, BETA>;
    cudaError_t e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kr<<<dim3((unsigned)(g.mp / 32), (unsigned)(g.kp / 64)), 256, sm, st>>>(a, g.m, g.k, g.E, (__half*)g.Adig, g.mp,
                                                                          g.kp, g.s);
    const int64_t tot = (g.kp / 4) * g.np;
    k_split_cols_h<T, NW, Q, BETA><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, g.k, g.n, g.F, (__half*)g.Bdig,
                                                                                  g.np, g.kp, g.s);
    return cudaGetLastError();
}

// digits of both operands for one form (the padded region gets zero digits)
template <typename T, int FORM>
static cudaError_t digits_impl(const SplitArgs& g, cudaStream_t st) {
    const int nw = digit_words(g.beta, g.s);
    if constexpr (FORM == OZMP_FORM_FP64) {
        if (nw <= 4) return digits_f64<T, 4>(g, st);
        return digits_f64<T, 7>(g, st);
    } else if constexpr (FORM == OZMP_FORM_FP16) {
        if (nw <= 4) {
            // the common widths and component counts: four digits a thread
            // with the width known at compile time (DD, TS)
            constexpr int QH = sizeof(T) == 8 ? 2 : 3;
            if (g.q == QH && g.beta == 5) return digits_h<T, 4, QH, 5>(g, st);
            if (g.q == QH && g.beta == 6) return digits_h<T, 4, QH, 6>(g, st);
            if (g.q == QH && g.beta == 7) return digits_h<T, 4, QH, 7>(g, st);
            return digits_f64<T, 4, __half>(g, st);
        }
        return digits_f64<T, 7, __half>(g, st);
    } else {
        if (nw <= 4) return digits_b1<T, FORM, 4>(g, st);
        return digits_b1<T, FORM, 6>(g, st);
    }
}

}  // namespace ozmp
