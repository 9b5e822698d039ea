// Internal device helpers of the ozmp library (not part of the C ABI).
//
// All arithmetic that decides a digit, an exponent or an output component is
// exact integer arithmetic on the IEEE-754 encodings: on GB300 the integer
// ALU is far faster than the binary64 pipe, and exactness makes every stage
// reproducible bit for bit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ozmp.h"

namespace ozmp {

// ----------------------------------------------------------------------------
// status word bits (device) -> ozmp_status (host picks the first set bit)
// ----------------------------------------------------------------------------
enum : uint32_t { ST_NONFINITE = 1u, ST_RANGE = 2u, ST_TIMEOUT = 4u, ST_ACCURACY = 8u };

// ----------------------------------------------------------------------------
// 64-bit shifts that are defined for every count (0 for counts >= 64)
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint64_t shl(uint64_t x, int n) { return (n >= 64 || n < 0) ? 0ull : (x << n); }
__device__ __forceinline__ uint64_t shr(uint64_t x, int n) { return (n >= 64 || n < 0) ? 0ull : (x >> n); }

// ----------------------------------------------------------------------------
// decoding one component: value = (-1)^neg * M * 2^e, M < 2^53 (0 = zero)
// ----------------------------------------------------------------------------
struct Comp {
    uint64_t M;
    int e;
    int neg;
};

__device__ __forceinline__ bool decode(double x, Comp& c) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7ff);
    uint64_t fr = b & 0xFFFFFFFFFFFFFull;
    c.neg = (int)(b >> 63);
    if (ex == 0x7ff) { c.M = 0; c.e = 0; return false; }
    if (ex == 0) { c.M = fr; c.e = -1074; }
    else { c.M = fr | (1ull << 52); c.e = ex - 1075; }
    return true;
}

__device__ __forceinline__ bool decode(float x, Comp& c) {
    uint32_t b = __float_as_uint(x);
    int ex = (int)((b >> 23) & 0xff);
    uint32_t fr = b & 0x7fffffu;
    c.neg = (int)(b >> 31);
    if (ex == 0xff) { c.M = 0; c.e = 0; return false; }
    if (ex == 0) { c.M = fr; c.e = -149; }
    else { c.M = fr | (1u << 23); c.e = ex - 150; }
    return true;
}

__device__ __forceinline__ int bitlen(uint64_t x) { return 64 - __clzll((long long)x); }

// bit 4 of every 5-bit digit group t = 1, 2, ... of a top-aligned window
// (group t at bits [64 NW - 5 t, 64 NW - 5 t + 5)), word j
__host__ __device__ constexpr uint64_t bal_sixteens(int nw, int j) {
    uint64_t r = 0;
    for (int t = 1; 64 * nw - 5 * t >= 0; ++t) {
        const int b = 64 * nw - 5 * t + 4;
        if (b >= 64 * j && b < 64 * j + 64) r |= 1ull << (b - 64 * j);
    }
    return r;
}

// the words of that pattern as a constant table (evaluated by the compiler:
// a constexpr function called in a run-time expression need not be)
template <int NW>
struct BalSixteens {
    uint64_t w[NW];
    constexpr BalSixteens() : w() {
        for (int j = 0; j < NW; ++j) w[j] = bal_sixteens(NW, j);
    }
};

// ----------------------------------------------------------------------------
// multiword two's complement helpers (NW words, word 0 least significant)
// ----------------------------------------------------------------------------
// (the carries travel in 128-bit sums, so the compiler owns the carry chain:
// separate inline-asm add.cc / addc.cc statements carry no dependency on the
// condition code and may be interleaved with other chains)
template <int NW>
__device__ __forceinline__ void mw_add(uint64_t (&w)[NW], const uint64_t (&p)[NW]) {
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const unsigned __int128 t = (unsigned __int128)w[j] + p[j] + c;
        w[j] = (uint64_t)t;
        c = (uint64_t)(t >> 64);
    }
}

template <int NW>
__device__ __forceinline__ void mw_sub(uint64_t (&w)[NW], const uint64_t (&p)[NW]) {
    uint64_t b = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const unsigned __int128 t = (unsigned __int128)w[j] - p[j] - b;
        w[j] = (uint64_t)t;
        b = (uint64_t)(t >> 64) & 1u;   // a borrow wraps the 128-bit difference
    }
}

template <int NW>
__device__ __forceinline__ void mw_neg(uint64_t (&w)[NW]) {
    uint64_t z[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) z[j] = 0;
    mw_sub<NW>(z, w);
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = z[j];
}

template <int NW>
__device__ __forceinline__ bool mw_is_zero(const uint64_t (&w)[NW]) {
    uint64_t o = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) o |= w[j];
    return o == 0;
}

// index of the highest set bit, -1 for zero
template <int NW>
__device__ __forceinline__ int mw_top(const uint64_t (&w)[NW]) {
    int t = -1;
#pragma unroll
    for (int j = 0; j < NW; ++j)
        if (w[j]) t = 64 * j + 63 - __clzll((long long)w[j]);
    return t;
}

// the unsigned value v placed with its bit 0 at window bit `sh` (may be < 0:
// bits below the window are dropped), as NW words
template <int NW>
__device__ __forceinline__ void mw_place(uint64_t (&p)[NW], uint64_t v, int sh) {
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        int o = sh - 64 * j;
        p[j] = (o >= 0) ? shl(v, o) : shr(v, -o);
    }
}

// logical left shift by n bits (0 <= n), static word indices only
template <int NW>
__device__ __forceinline__ void mw_shl(uint64_t (&w)[NW], int n) {
    if (n >= 64 * NW) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        return;
    }
    int ws = n >> 6, b = n & 63;
#pragma unroll
    for (int step = 1; step < NW; step <<= 1) {
        if (ws & step) {
#pragma unroll
            for (int j = NW - 1; j >= 0; --j) w[j] = (j - step >= 0) ? w[j - step] : 0ull;
        }
    }
    if (b) {
#pragma unroll
        for (int j = NW - 1; j >= 0; --j) w[j] = (w[j] << b) | ((j > 0) ? (w[j - 1] >> (64 - b)) : 0ull);
    }
}

// logical right shift by n bits (0 <= n)
template <int NW>
__device__ __forceinline__ void mw_shr(uint64_t (&w)[NW], int n) {
    if (n >= 64 * NW) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        return;
    }
    int ws = n >> 6, b = n & 63;
#pragma unroll
    for (int step = 1; step < NW; step <<= 1) {
        if (ws & step) {
#pragma unroll
            for (int j = 0; j < NW; ++j) w[j] = (j + step < NW) ? w[j + step] : 0ull;
        }
    }
    if (b) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = (w[j] >> b) | ((j + 1 < NW) ? (w[j + 1] << (64 - b)) : 0ull);
    }
}

// ----------------------------------------------------------------------------
// exact sum of up to Q components into a fixed window
// ----------------------------------------------------------------------------
// Adds every component, truncated toward zero at window bit 0 (weight 2^L),
// into the two's complement window w.  Returns true if some component has a
// non-zero bit below the window (then w is not the exact sum).
template <int NW>
__device__ __forceinline__ bool window_sum(uint64_t (&w)[NW], const Comp (&c)[4], int q, int L) {
    bool tail = false;
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i >= q || c[i].M == 0) continue;
        int sh = c[i].e - L;
        if (sh < 0) {
            int r = -sh;
            uint64_t mask = (r >= 64) ? ~0ull : ((1ull << r) - 1ull);
            if (c[i].M & mask) tail = true;
        }
        uint64_t p[NW];
        mw_place<NW>(p, c[i].M, sh);
        if (c[i].neg) mw_sub<NW>(w, p); else mw_add<NW>(w, p);
    }
    return tail;
}

// Window of the wide (slow) path: covers every binary64 and binary32 bit.
constexpr int SLOW_NW = 36;
constexpr int SLOW_L = -1152;
constexpr int FAST_NW = 6;    // 384 bits

// Exact magnitude of x = sum of components, normalised so that the bit of
// weight 2^(E_top - 1) sits at bit 383 of a 384-bit window `out`
// (truncating whatever falls below bit 0).  Returns sign (-1, 0, +1).
// If E_top is OZMP_EXP_ZERO-like (x == 0) the window is zero.
// Also returns the exact exponent E(x) = floor(log2|x|) + 1 (or EXP_ZERO).
struct Exact {
    int sign;
    int E;          // floor(log2|x|) + 1
};

// magnitude in an NW-word window with LSB weight 2^L; sign and E computed
template <int NW>
__device__ __forceinline__ Exact window_magnitude(uint64_t (&w)[NW], int L) {
    Exact r;
    r.sign = 0;
    r.E = OZMP_EXP_ZERO;
    if (mw_is_zero<NW>(w)) return r;
    bool neg = (w[NW - 1] >> 63) != 0;
    if (neg) mw_neg<NW>(w);
    r.sign = neg ? -1 : 1;
    r.E = L + mw_top<NW>(w) + 1;
    return r;
}

template <typename T>
__device__ __forceinline__ int mant_bits();
template <> __device__ __forceinline__ int mant_bits<double>() { return 53; }
template <> __device__ __forceinline__ int mant_bits<float>() { return 24; }

// Decode q components (q <= 4) of type T; returns false on a non-finite one.
template <typename T>
__device__ __forceinline__ bool decode_all(const T (&v)[4], int q, Comp (&c)[4], int& Ptop) {
    bool ok = true;
    Ptop = -100000;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        c[i].M = 0; c[i].e = 0; c[i].neg = 0;
        if (i >= q) continue;
        ok &= decode(v[i], c[i]);
        if (c[i].M) {
            int p = c[i].e + bitlen(c[i].M);
            Ptop = p > Ptop ? p : Ptop;
        }
    }
    return ok;
}

// Slow paths (a component has bits below the fast window): exact sums over
// the whole binary64 range in a local-memory array, with rolled loops so
// their register footprint stays small.  They take the component values
// (binary32 ones widened exactly) so the common path never takes the address
// of its register-resident component array.
static __device__ __noinline__ int slow_sum(double v0, double v1, double v2, double v3, int q, uint64_t* W) {
    const double v[4] = {v0, v1, v2, v3};
#pragma unroll 1
    for (int j = 0; j < SLOW_NW; ++j) W[j] = 0;
#pragma unroll 1
    for (int i = 0; i < q; ++i) {
        Comp c;
        decode(v[i], c);
        if (c.M == 0) continue;
        const int sh = c.e - SLOW_L;          // >= 0 for every finite double
        const int wi = sh >> 6, b = sh & 63;
        const uint64_t lo = c.M << b, hi = b ? (c.M >> (64 - b)) : 0ull;
        uint64_t carry = 0;
#pragma unroll 1
        for (int j = wi; j < SLOW_NW; ++j) {
            const uint64_t a = (j == wi) ? lo : ((j == wi + 1) ? hi : 0ull);
            if (!c.neg) {
                const uint64_t t = W[j] + a;
                const uint64_t c1 = t < a;
                const uint64_t t2 = t + carry;
                carry = c1 | (t2 < t);
                W[j] = t2;
            } else {
                const uint64_t t = W[j] - a;
                const uint64_t b1 = W[j] < a;
                const uint64_t t2 = t - carry;
                carry = b1 | (t < carry);
                W[j] = t2;
            }
            if (j > wi + 1 && carry == 0) break;
        }
    }
    // magnitude and sign
    int sign = 0;
#pragma unroll 1
    for (int j = 0; j < SLOW_NW; ++j) if (W[j]) sign = 1;
    if (!sign) return 0;
    if (W[SLOW_NW - 1] >> 63) {
        uint64_t c = 1;
#pragma unroll 1
        for (int j = 0; j < SLOW_NW; ++j) {
            const uint64_t x = ~W[j] + c;
            c = (c && x == 0) ? 1ull : 0ull;
            W[j] = x;
        }
        return -1;
    }
    return 1;
}

static __device__ __noinline__ Exact exact_exponent_slow(double v0, double v1, double v2, double v3, int q) {
    uint64_t W[SLOW_NW];
    Exact r;
    r.sign = slow_sum(v0, v1, v2, v3, q, W);
    r.E = OZMP_EXP_ZERO;
    if (r.sign) {
        int top = -1;
#pragma unroll 1
        for (int j = SLOW_NW - 1; j >= 0 && top < 0; --j)
            if (W[j]) top = 64 * j + 63 - __clzll((long long)W[j]);
        r.E = SLOW_L + top + 1;
    }
    return r;
}

// NW words of |x| with the bit of weight 2^(Erow - 1) at bit `toppos`
static __device__ __noinline__ int slow_window(double v0, double v1, double v2, double v3, int q, int Erow, int nw,
                                               int toppos, uint64_t* out) {
    uint64_t W[SLOW_NW];
    const int sign = slow_sum(v0, v1, v2, v3, q, W);
    const int lo = (Erow - 1 - SLOW_L) - toppos;   // bit of W that becomes bit 0
#pragma unroll 1
    for (int j = 0; j < nw; ++j) {
        const int b = lo + 64 * j;
        const int li = b >> 6;
        const int sh = b - 64 * li;
        const uint64_t a0 = (li >= 0 && li < SLOW_NW) ? W[li] : 0ull;
        const uint64_t a1 = (li + 1 >= 0 && li + 1 < SLOW_NW) ? W[li + 1] : 0ull;
        out[j] = sign ? (sh ? ((a0 >> sh) | (a1 << (64 - sh))) : a0) : 0ull;
    }
    return sign;
}

static __device__ __noinline__ int aligned_slow(double v0, double v1, double v2, double v3, int q, int Erow,
                                                uint64_t* out) {
    return slow_window(v0, v1, v2, v3, q, Erow, FAST_NW, 383, out);
}

// the component values, widened to binary64 (exact)
template <typename T>
__device__ __forceinline__ double comp_value(const T (&v)[4], int i) { return (double)v[i]; }

// Exact exponent E(x) and sign of the sum of the decoded components (v are
// the raw component values, used only by the slow path).
template <typename T>
__device__ __forceinline__ Exact exact_exponent(const Comp (&c)[4], const T (&v)[4], int q, int Ptop) {
    Exact r;
    r.sign = 0;
    r.E = OZMP_EXP_ZERO;
    if (Ptop == -100000) return r;
    int L = Ptop + 3 - 64 * FAST_NW;
    uint64_t w[FAST_NW];
    bool tail = window_sum<FAST_NW>(w, c, q, L);
    if (!tail) return window_magnitude<FAST_NW>(w, L);
    return exact_exponent_slow((double)v[0], (double)v[1], (double)v[2], (double)v[3], q);
}

// Exact |x| placed so that weight 2^(Erow - 1) is window bit 383 (bits
// below bit 0 truncated).  Erow must satisfy |x| < 2^Erow.  Returns sign.
template <typename T>
__device__ __forceinline__ int aligned_magnitude(const Comp (&c)[4], const T (&v)[4], int q, int Ptop, int Erow,
                                                 uint64_t (&out)[FAST_NW]) {
#pragma unroll
    for (int j = 0; j < FAST_NW; ++j) out[j] = 0;
    if (Ptop == -100000) return 0;
    int L = Ptop + 3 - 64 * FAST_NW;
    bool tail = window_sum<FAST_NW>(out, c, q, L);
    if (!tail) {
        Exact ex = window_magnitude<FAST_NW>(out, L);
        if (ex.sign == 0) return 0;
        int pos = Erow - 1 - L;          // window bit of weight 2^(Erow - 1)
        int left = 383 - pos;
        if (left >= 0) mw_shl<FAST_NW>(out, left); else mw_shr<FAST_NW>(out, -left);
        return ex.sign;
    }
    uint64_t tmp[FAST_NW];
    int sg = aligned_slow((double)v[0], (double)v[1], (double)v[2], (double)v[3], q, Erow, tmp);
#pragma unroll
    for (int j = 0; j < FAST_NW; ++j) out[j] = tmp[j];
    return sg;
}

// ----------------------------------------------------------------------------
// exponent E(x) with a 128-bit window anchored at the largest component
// ----------------------------------------------------------------------------
// Components are added, truncated toward zero at the window LSB 2^L, into a
// two's complement 128-bit integer V (L = Ptop - 125 leaves room for the
// carries of four terms).  Without bits below the window V is exact.  With
// them, x = V 2^L + T, |T| < q 2^L, and the top bit of |x| is that of |V|
// unless |V| is within q of a power of two (or |V| < 2^64); those rare cases
// take the exact full-range path.
// Fast exponent from the encodings alone.  Let the top component have the
// largest exponent field, |top| in [2^(e-1), 2^e).  If every other component
// is below 2^(e - P - g) (P = 53 or 24 significand bits, 2^g >= q - 1), the
// others sum to less than an ulp of top, so |x| stays in (2^(e-1), 2^e) and
// E(x) = e -- unless top is a power of two, when x drops below 2^(e-1) iff
// the others sum to the opposite sign (decided here only for q = 2).
// Returns false when these conditions do not settle E(x) (then the exact
// window decides); zero, subnormal and non-finite tops also return false.
template <typename T>
__device__ __forceinline__ bool exponent_fast(const T (&v)[4], int q, int& E) {
    constexpr int P = (sizeof(T) == 8) ? 53 : 24;
    constexpr int EB = (sizeof(T) == 8) ? 1022 : 126;     // frexp exponent = field - EB
    constexpr int EMAXF = (sizeof(T) == 8) ? 0x7ff : 0xff;
    uint64_t bits[4];
    int ef[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (sizeof(T) == 8) {
            bits[i] = (uint64_t)__double_as_longlong((double)v[i]);
            ef[i] = (int)((bits[i] >> 52) & 0x7ff);
        } else {
            bits[i] = __float_as_uint((float)v[i]);
            ef[i] = (int)((bits[i] >> 23) & 0xff);
        }
        if (i >= q) ef[i] = 0;
    }
    int top = 0;
#pragma unroll
    for (int i = 1; i < 4; ++i) top = ef[i] > ef[top] ? i : top;
    const int et = ef[top];
    if (et == 0 || et == EMAXF) return false;
    int eo = 0;   // largest exponent field among the others (0: zero or subnormal)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i == top) continue;
        if (ef[i] == EMAXF) return false;
        const bool nonzero = (sizeof(T) == 8) ? ((bits[i] << 1) != 0) : ((bits[i] << 33) != 0);
        if (nonzero) eo = (ef[i] > eo) ? ef[i] : (eo ? eo : 1);   // a subnormal counts as field 1
    }
    const int g = q <= 2 ? 0 : (q <= 3 ? 1 : 2);
    if (eo && eo > et - P - g) return false;
    const uint64_t mant = (sizeof(T) == 8) ? (bits[top] & 0xFFFFFFFFFFFFFull) : (bits[top] & 0x7FFFFFull);
    E = et - EB;
    if (mant == 0 && eo) {
        if (q != 2) return false;
        const bool opposite = (sizeof(T) == 8) ? (((bits[0] ^ bits[1]) >> 63) != 0) : (((bits[0] ^ bits[1]) >> 31) != 0);
        if (opposite) E -= 1;
    }
    return true;
}

template <typename T>
__device__ __forceinline__ int exponent_of(const Comp (&c)[4], const T (&v)[4], int q, int Ptop) {
    if (Ptop == -100000) return OZMP_EXP_ZERO;
    {
        int Ef;
        if (exponent_fast<T>(v, q, Ef)) return Ef;
    }
    const int L = Ptop - 125;
    unsigned __int128 V = 0;
    bool tail = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i >= q || c[i].M == 0) continue;
        int sh = c[i].e - L;                      // <= 125 - bitlen(M)
        unsigned __int128 part;
        if (sh >= 0) {
            part = (unsigned __int128)c[i].M << sh;
        } else {
            int r = -sh;
            uint64_t mask = (r >= 64) ? ~0ull : ((1ull << r) - 1ull);
            if (c[i].M & mask) tail = true;
            part = (unsigned __int128)((r >= 64) ? 0ull : (c[i].M >> r));
        }
        V = c[i].neg ? V - part : V + part;
    }
    const bool negv = (uint64_t)(V >> 127) != 0;
    unsigned __int128 A = negv ? (unsigned __int128)0 - V : V;
    const uint64_t hi = (uint64_t)(A >> 64), lo = (uint64_t)A;
    int top = hi ? 64 + 63 - __clzll((long long)hi) : (lo ? 63 - __clzll((long long)lo) : -1);
    if (!tail) return top < 0 ? OZMP_EXP_ZERO : L + top + 1;
    if (top >= 64) {
        unsigned __int128 pw = (unsigned __int128)1 << top;
        unsigned __int128 below = A - pw;                                  // >= 0
        unsigned __int128 above = (top < 127) ? ((unsigned __int128)1 << (top + 1)) - A : (unsigned __int128)1;
        if (below >= (unsigned __int128)q && above > (unsigned __int128)q) return L + top + 1;
    }
    return exact_exponent_slow((double)v[0], (double)v[1], (double)v[2], (double)v[3], q).E;
}

// ----------------------------------------------------------------------------
// digit window anchored at the row exponent
// ----------------------------------------------------------------------------
// NW words; weight 2^(Erow - 1) sits at bit 64 NW - 2 (the top bit is the
// sign), so digit t occupies bits [64 NW - 1 - beta t, 64 NW - 1 - beta (t-1))
// at positions known at compile time.  Word 0 lies below every digit
// (64 NW >= beta s + 65) and absorbs truncation: with bits of some component
// below the window the truncated |x| differs from |V| only by a borrow or
// carry out of word 0, which can reach the digits only when word 0 is
// within q of 0 or of 2^64 -- those cases take the exact full-range path.
template <int NW, typename T>
__device__ __forceinline__ int digit_window(const Comp (&c)[4], const T (&v)[4], int q, int Erow,
                                            uint64_t (&w)[NW]) {
    const int L = Erow - (64 * NW - 1);
    bool tail = window_sum<NW>(w, c, q, L);
    bool neg = (w[NW - 1] >> 63) != 0;
    if (neg) mw_neg<NW>(w);
    if (!tail) return mw_is_zero<NW>(w) ? 0 : (neg ? -1 : 1);
    if (w[0] >= (uint64_t)q && w[0] <= ~0ull - (uint64_t)q) return neg ? -1 : 1;
    uint64_t tmp[NW];
    int sg = slow_window((double)v[0], (double)v[1], (double)v[2], (double)v[3], q, Erow, NW, 64 * NW - 2, tmp);
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = tmp[j];
    return sg;
}

// digit t (1-based) of a digit window (BETA known at compile time)
template <int NW, int BETA>
__device__ __forceinline__ uint32_t digit_of(const uint64_t (&w)[NW], int t) {
    const int p = 64 * NW - 1 - BETA * t;
    const int wi = p >> 6, off = p & 63;
    uint64_t x = w[wi] >> off;
    if (off + BETA > 64 && wi + 1 < NW) x |= w[wi + 1] << (64 - off);
    return (uint32_t)(x & ((1ull << BETA) - 1ull));
}

// digit t with a run-time beta (binary64 digits)
template <int NW>
__device__ __forceinline__ uint32_t digit_of_rt(const uint64_t (&w)[NW], int t, int beta) {
    const int p = 64 * NW - 1 - beta * t;
    const int wi = p >> 6, off = p & 63;
    uint64_t a0 = 0, a1 = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        if (j == wi) a0 = w[j];
        if (j == wi + 1) a1 = w[j];
    }
    uint64_t x = (a0 >> off) | (off ? (a1 << (64 - off)) : 0ull);
    return (uint32_t)(x & ((1ull << beta) - 1ull));
}

// four e4m3 codes of four magnitudes 0..15 (one per byte of m4), signs in
// negmask (0x80 per negative byte; zero digits stay +0)
__device__ __forceinline__ uint32_t e4m3x4(uint32_t m4, uint32_t negmask) {
    // codes of 0..7 and 8..15 (integers below 16 are exact in e4m3)
    const uint32_t lo0 = 0x44403800u, lo1 = 0x4E4C4A48u, hi0 = 0x53525150u, hi1 = 0x57565554u;
    const uint32_t sel = (m4 & 7u) | ((m4 >> 4) & 0x70u) | ((m4 >> 8) & 0x700u) | ((m4 >> 12) & 0x7000u);
    const uint32_t a = __byte_perm(lo0, lo1, sel), b = __byte_perm(hi0, hi1, sel);
    const uint32_t big = ((m4 >> 3) & 0x01010101u) * 0xFFu;
    const uint32_t code = (a & ~big) | (b & big);
    return code | (negmask & __vcmpne4(code, 0u));
}

// prmt in its default mode: each selector nibble picks one of the 8 bytes of
// {b, a} with its low 3 bits and, when its bit 3 is set, replicates that
// byte's sign bit instead of copying it
__device__ __forceinline__ uint32_t prmt_sign(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

// e4m3 codes of the four digit magnitudes held in the low 16 bits of x (one
// nibble each, nibble i -> byte i), with the sign bit set on the non-zero
// codes when negm = 0x80808080.  Two table lookups: codes of 0..7 where the
// nibble is below 8 (the bytes selected for 8..15 replicate a clear sign bit
// and give 0) and codes of 8..15 on the nibbles with bit 3 flipped.
__device__ __forceinline__ uint32_t e4m3_nibbles4(uint32_t x, uint32_t negm) {
    const uint32_t a = prmt_sign(0x44403800u, 0x4E4C4A48u, x);
    const uint32_t b = prmt_sign(0x53525150u, 0x57565554u, x ^ 0x8888u);
    const uint32_t code = a | b;
    // 0x80 in every non-zero byte: (code & 0x78) is 0 or at least 0x38
    return code | (((code & 0x78787878u) + 0x78787878u) & negm);
}

// 4 x 4 byte transpose: out[b] byte e = in[e] byte b
__device__ __forceinline__ void transpose4(const uint32_t (&in)[4], uint32_t (&out)[4]) {
    const uint32_t a = __byte_perm(in[0], in[1], 0x5140), b = __byte_perm(in[0], in[1], 0x7362);
    const uint32_t c = __byte_perm(in[2], in[3], 0x5140), d = __byte_perm(in[2], in[3], 0x7362);
    out[0] = __byte_perm(a, c, 0x5410);
    out[1] = __byte_perm(a, c, 0x7632);
    out[2] = __byte_perm(b, d, 0x5410);
    out[3] = __byte_perm(b, d, 0x7632);
}

// four int8 digits (two's complement) of four magnitudes 0..127, sign bytes
// 0xFF in negmask for negative ones
__device__ __forceinline__ uint32_t int8x4(uint32_t m4, uint32_t negmask) {
    return __vsub4(m4 ^ negmask, negmask);
}

// Digit t (1-based) of the aligned window: bits [384 - beta t, 384 - beta (t-1)).
template <int BETA>
__device__ __forceinline__ uint32_t digit_at(const uint64_t (&w)[FAST_NW], int t) {
    int p = 384 - BETA * t;
    int wi = p >> 6, off = p & 63;
    uint64_t v = w[wi] >> off;
    if (off + BETA > 64 && wi + 1 < FAST_NW) v |= w[wi + 1] << (64 - off);
    return (uint32_t)(v & ((1ull << BETA) - 1ull));
}

// runtime beta: top beta bits of the window, then shift the window left
__device__ __forceinline__ uint32_t take_top(uint64_t (&w)[FAST_NW], int beta) {
    uint32_t d = (uint32_t)(w[FAST_NW - 1] >> (64 - beta));
    mw_shl<FAST_NW>(w, beta);
    return d;
}

// e4m3 encoding of a small integer |d| <= 15 (exact: 4-bit integers have at
// most 4 significant bits and e4m3 stores 1 + 3 of them).
__device__ __forceinline__ uint32_t e4m3_of_int(int d) {
    uint32_t a = (uint32_t)(d < 0 ? -d : d);
    if (a == 0) return 0u;
    int e = 31 - __clz(a);                       // 0..3
    uint32_t m = ((a << (3 - e)) & 7u);           // 3 mantissa bits below the leading one
    uint32_t code = ((uint32_t)(e + 7) << 3) | m;
    return code | (d < 0 ? 0x80u : 0u);
}

// ----------------------------------------------------------------------------
// canonical rounding of an exact two's complement accumulator into q words
// ----------------------------------------------------------------------------
// value = acc * 2^U.  Emits c_0 = RN(value), c_t = RN(value - c_0 - ...)
// through put(t, c_t) for t = 0 .. q-1.
// Returns false if a non-zero component would leave the normal range.
template <int NW, typename T, typename Put>
__device__ __forceinline__ bool canonical_round_put(uint64_t (&acc)[NW], int U, int q, Put&& put) {
    constexpr int P = (sizeof(T) == 8) ? 53 : 24;
    constexpr int EBIAS = (sizeof(T) == 8) ? 1023 : 127;
    constexpr int EMAX = (sizeof(T) == 8) ? 2046 : 254;
    bool ok = true;
    int sgn = 1;
    if ((acc[NW - 1] >> 63) != 0) { mw_neg<NW>(acc); sgn = -1; }
    int scale = U;
#pragma unroll 4
    for (int c = 0; c < q; ++c) {
        int top = mw_top<NW>(acc);
        if (top < 0) { put(c, (T)0); continue; }
        int z = 64 * NW - 1 - top;
        mw_shl<NW>(acc, z);
        scale -= z;
        uint64_t hi = acc[NW - 1];
        uint64_t mant = hi >> (64 - P);
        uint64_t rb = (hi >> (63 - P)) & 1ull;
        uint64_t low = hi & ((1ull << (63 - P)) - 1ull);
#pragma unroll
        for (int j = 0; j < NW - 1; ++j) low |= acc[j];
        bool up = rb && (low != 0 || (mant & 1ull));
        // residual in the normalised frame
        acc[NW - 1] = hi & ((1ull << (64 - P)) - 1ull);
        if (up) {
            mant += 1;
            // residual := 2^(64 NW - P) - residual, and the sign flips
            uint64_t one[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) one[j] = 0;
            one[NW - 1] = 1ull << (64 - P);
            mw_sub<NW>(one, acc);
#pragma unroll
            for (int j = 0; j < NW; ++j) acc[j] = one[j];
        }
        // component = sgn * mant * 2^(scale + 64 NW - P), mant in [2^(P-1), 2^P]
        int ex = scale + 64 * NW - P;
        if (mant >> P) { mant >>= 1; ex += 1; }
        int be = ex + (P - 1) + EBIAS;             // biased exponent of 1.f x 2^(ex + P - 1)
        if (be < 1 || be > EMAX) {
            ok = false;
            put(c, (T)0);
        } else if (sizeof(T) == 8) {
            uint64_t bits = ((uint64_t)(sgn < 0) << 63) | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1ull));
            double dv = __longlong_as_double((long long)bits);
            put(c, (T)dv);
        } else {
            uint32_t bits = ((uint32_t)(sgn < 0) << 31) | ((uint32_t)be << 23) | ((uint32_t)mant & 0x7fffffu);
            float fv = __uint_as_float(bits);
            put(c, (T)fv);
        }
        if (up) sgn = -sgn;
    }
    return ok;
}


// the same into out[0 .. q-1]
template <int NW, typename T>
__device__ __forceinline__ bool canonical_round(uint64_t (&acc)[NW], int U, int q, T* out) {
    return canonical_round_put<NW, T>(acc, U, q, [&](int c, T v) { out[c] = v; });
}

}  // namespace ozmp
