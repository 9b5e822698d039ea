// Exact accumulator for the operations of the LU application: sums of
// products of binary64 components, held exactly in a fixed-point two's
// complement integer of KW 64-bit words (LSB weight 2^KL), then rounded
// canonically into q components (c_0 = RN(v), c_t = RN(v - c_0 - ...)).
//
// Every product of two binary64 components whose exact value lies in
// [2^KL, 2^(KL + 64 KW - 2)) is added without rounding (53 x 53-bit integer
// product, placed at its exponent); a product outside that range sets the
// range flag.  The accumulator lives in local memory (one per thread); the
// loops are rolled to keep the code small.
#pragma once
#include <cstdint>
#include "ozmp_internal.cuh"

namespace ozmp {
namespace xacc {

constexpr int KW = 48;       // 3072 bits
constexpr int KL = -1600;    // products of magnitude down to 2^-1600 are exact

struct Acc {
    uint64_t w[KW];
    bool range_bad;
};

__device__ __forceinline__ void clear(Acc& a) {
#pragma unroll 1
    for (int j = 0; j < KW; ++j) a.w[j] = 0;
    a.range_bad = false;
}

// add (neg ? -1 : 1) * (hi:lo) * 2^e, hi:lo a 128-bit magnitude
static __device__ __noinline__ void add128(Acc& a, uint64_t hi, uint64_t lo, int e, bool neg) {
    if (hi == 0 && lo == 0) return;
    int sh = e - KL;
    if (sh < 0) {
        // bits below the window are allowed only if they are all zero
        const int r = -sh;
        bool lost;
        if (r >= 128) lost = true;
        else if (r >= 64) lost = (lo != 0) || (r > 64 && (hi << (128 - r)) != 0);
        else lost = (lo << (64 - r)) != 0;
        if (lost) { a.range_bad = true; return; }
        if (r >= 64) { lo = hi >> (r - 64); hi = 0; }
        else { lo = (lo >> r) | (hi << (64 - r)); hi >>= r; }
        sh = 0;
    }
    if (sh + 128 > 64 * KW - 2) { a.range_bad = true; return; }
    const int wi = sh >> 6, b = sh & 63;
    uint64_t p0 = lo << b;
    uint64_t p1 = b ? ((hi << b) | (lo >> (64 - b))) : hi;
    uint64_t p2 = b ? (hi >> (64 - b)) : 0ull;
    uint64_t carry = 0;
#pragma unroll 1
    for (int j = wi; j < KW; ++j) {
        const uint64_t v = (j == wi) ? p0 : (j == wi + 1) ? p1 : (j == wi + 2) ? p2 : 0ull;
        if (!neg) {
            const uint64_t t = a.w[j] + v;
            const uint64_t c1 = t < v;
            const uint64_t t2 = t + carry;
            carry = c1 | (t2 < t);
            a.w[j] = t2;
        } else {
            const uint64_t t = a.w[j] - v;
            const uint64_t b1 = a.w[j] < v;
            const uint64_t t2 = t - carry;
            carry = b1 | (t < carry);
            a.w[j] = t2;
        }
        if (j > wi + 2 && carry == 0) break;
    }
}

// a += x (one binary64 value)
__device__ __forceinline__ void add_value(Acc& a, double x) {
    Comp c;
    decode(x, c);
    if (c.M) add128(a, 0, c.M, c.e, c.neg != 0);
}

// a += s * x * y exactly (s = +1 or -1)
__device__ __forceinline__ void add_product(Acc& a, double x, double y, bool negate) {
    Comp cx, cy;
    decode(x, cx);
    decode(y, cy);
    if (!cx.M || !cy.M) return;
    const uint64_t lo = cx.M * cy.M, hi = __umul64hi(cx.M, cy.M);
    add128(a, hi, lo, cx.e + cy.e, ((cx.neg ^ cy.neg) != 0) != negate);
}

// canonical rounding into q binary64 components (the accumulator is used up)
static __device__ __noinline__ void round_q(Acc& a, int q, double* out) {
    int sgn = 1;
    if (a.w[KW - 1] >> 63) {
        // negate in place
        uint64_t c = 1;
#pragma unroll 1
        for (int j = 0; j < KW; ++j) {
            const uint64_t x = ~a.w[j] + c;
            c = (c && x == 0) ? 1ull : 0ull;
            a.w[j] = x;
        }
        sgn = -1;
    }
#pragma unroll 1
    for (int t = 0; t < q; ++t) {
        int top = -1;
#pragma unroll 1
        for (int j = KW - 1; j >= 0; --j)
            if (a.w[j]) { top = 64 * j + 63 - __clzll((long long)a.w[j]); break; }
        if (top < 0) { out[t] = 0.0; continue; }
        // the 53 bits below and including `top`, the round bit and the sticky bits
        const int lsb = top - 52;   // window bit of the last kept bit
        uint64_t mant = 0;
#pragma unroll 1
        for (int b = 0; b < 53; ++b) {
            const int pos = top - b;
            const uint64_t bit = pos >= 0 ? (a.w[pos >> 6] >> (pos & 63)) & 1ull : 0ull;
            mant = (mant << 1) | bit;
        }
        bool rb = false, sticky = false;
        if (lsb - 1 >= 0) {
            rb = ((a.w[(lsb - 1) >> 6] >> ((lsb - 1) & 63)) & 1ull) != 0;
#pragma unroll 1
            for (int j = 0; j <= ((lsb - 2) >> 6) && lsb - 2 >= 0; ++j) {
                uint64_t word = a.w[j];
                if (j == ((lsb - 2) >> 6)) {
                    const int hb = (lsb - 2) & 63;
                    word &= (hb == 63) ? ~0ull : ((2ull << hb) - 1ull);
                }
                if (word) { sticky = true; break; }
            }
        }
        const bool up = rb && (sticky || (mant & 1ull));
        // residual: v - c_t, computed as (v - mant 2^lsb) then -2^lsb if rounded up
        // (clear the kept bits, then subtract one unit at lsb when rounding up)
#pragma unroll 1
        for (int b = 0; b < 53; ++b) {
            const int pos = top - b;
            if (pos >= 0) a.w[pos >> 6] &= ~(1ull << (pos & 63));
        }
        const int ex = KL + lsb;    // c_t = sgn * mant * 2^ex
        if (up) {
            mant += 1;
            // residual := residual - 2^lsb (two's complement in the window; lsb >= 1 here)
            const int p = lsb;
            uint64_t borrow = 1ull << (p & 63);
#pragma unroll 1
            for (int j = p >> 6; j < KW; ++j) {
                const uint64_t old = a.w[j];
                a.w[j] = old - borrow;
                borrow = (old < borrow) ? 1ull : 0ull;
                if (!borrow) break;
            }
        }
        // value of this component: sgn * mant * 2^ex (mant may be 2^53 after
        // rounding up); outside the normal binary64 range the range flag is set
        const int topexp = ex + 63 - __clzll((long long)mant);   // exponent of the leading bit
        double v = 0.0;
        if (topexp < -1022 || topexp > 1023) a.range_bad = true;
        else v = ldexp((double)mant, ex);                        // exact: mant <= 2^53, result normal
        out[t] = sgn > 0 ? v : -v;
        // the residual may now be negative (rounded up): continue with its sign
        if (a.w[KW - 1] >> 63) {
            uint64_t c = 1;
#pragma unroll 1
            for (int j = 0; j < KW; ++j) {
                const uint64_t x = ~a.w[j] + c;
                c = (c && x == 0) ? 1ull : 0ull;
                a.w[j] = x;
            }
            sgn = -sgn;
        }
    }
}

// ---------------------------------------------------------------------------
// The same operation with a register-resident window (the fast path).  A
// term generator gen(v) calls v.value(x) and v.product(x, y, negate) for
// every term; it is walked twice: once for the largest leading-bit position
// and the term count, which fix a window of NW words whose top leaves room
// for the carries, and once to add the terms exactly.  If a term has bits
// below the window the register sum is not exact and the local-memory
// accumulator above evaluates the terms instead.  Either way the result is
// the exact value rounded canonically into q components.
// ---------------------------------------------------------------------------
struct TopVisitor {
    int top = -100000;   // largest leading-bit position (weight 2^top)
    int count = 0;
    __device__ __forceinline__ void value(double x) {
        Comp c;
        decode(x, c);
        if (!c.M) return;
        const int t = c.e + 63 - __clzll((long long)c.M);
        top = t > top ? t : top;
        ++count;
    }
    __device__ __forceinline__ void product(double x, double y, bool) {
        Comp cx, cy;
        decode(x, cx);
        decode(y, cy);
        if (!cx.M || !cy.M) return;
        const int t = cx.e + cy.e + (63 - __clzll((long long)cx.M)) + (63 - __clzll((long long)cy.M)) + 1;
        top = t > top ? t : top;
        ++count;
    }
};

template <int NW>
struct RegVisitor {
    uint64_t w[NW];
    int L;               // weight of window bit 0
    bool tail;           // some term had bits below the window

    __device__ __forceinline__ void init(int top, int count) {
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = 0;
        int g = 1;
        while ((1 << g) <= count) ++g;          // |sum| < 2^(top + 1 + g)
        L = top + 1 + g - (64 * NW - 1);        // bit 64 NW - 1 is the sign
        tail = false;
    }
    __device__ __forceinline__ void add128(uint64_t hi, uint64_t lo, int e, bool neg) {
        int sh = e - L;
        if (sh < 0) {
            const int r = -sh;
            bool lost;
            if (r >= 128) lost = (hi | lo) != 0;
            else if (r >= 64) lost = (lo != 0) || (r > 64 && (hi << (128 - r)) != 0);
            else lost = (lo << (64 - r)) != 0;
            if (lost) { tail = true; return; }
            if (r >= 128) return;
            if (r >= 64) { lo = hi >> (r - 64); hi = 0; }
            else { lo = (lo >> r) | (hi << (64 - r)); hi >>= r; }
            sh = 0;
        }
        const int wi = sh >> 6, b = sh & 63;
        const uint64_t p0 = lo << b;
        const uint64_t p1 = b ? ((hi << b) | (lo >> (64 - b))) : hi;
        const uint64_t p2 = b ? (hi >> (64 - b)) : 0ull;
        uint64_t p[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) p[j] = (j == wi) ? p0 : (j == wi + 1) ? p1 : (j == wi + 2) ? p2 : 0ull;
        if (neg) mw_sub<NW>(w, p); else mw_add<NW>(w, p);
    }
    __device__ __forceinline__ void value(double x) {
        Comp c;
        decode(x, c);
        if (c.M) add128(0, c.M, c.e, c.neg != 0);
    }
    __device__ __forceinline__ void product(double x, double y, bool negate) {
        Comp cx, cy;
        decode(x, cx);
        decode(y, cy);
        if (!cx.M || !cy.M) return;
        add128(__umul64hi(cx.M, cy.M), cx.M * cy.M, cx.e + cy.e, ((cx.neg ^ cy.neg) != 0) != negate);
    }
};

struct KulVisitor {
    Acc a;
    __device__ __forceinline__ void value(double x) { add_value(a, x); }
    __device__ __forceinline__ void product(double x, double y, bool negate) { add_product(a, x, y, negate); }
};

// out[0 .. q-1] = canonical rounding of the exact sum of gen's terms; `bad`
// is set when a term or a component leaves the representable range
template <int NW, typename Gen>
__device__ __forceinline__ void exact_round(int q, Gen&& gen, double* out, bool& bad) {
    TopVisitor tv;
    gen(tv);
    if (tv.count == 0) {
        for (int c = 0; c < q; ++c) out[c] = 0.0;
        return;
    }
    RegVisitor<NW> rv;
    rv.init(tv.top, tv.count);
    gen(rv);
    if (!rv.tail) {
        if (!canonical_round<NW, double>(rv.w, rv.L, q, out)) bad = true;
        return;
    }
    KulVisitor kv;
    clear(kv.a);
    gen(kv);
    bad |= kv.a.range_bad;
    round_q(kv.a, q, out);
    bad |= kv.a.range_bad;
}

// Warp-cooperative form: gen(v, part) yields the terms of part `part`
// (0 .. 31); lane l adds part l into its own register window (all lanes
// share the anchor from the warp-wide largest leading bit and term count),
// the 32 windows are summed exactly with xor shuffles, and every lane
// rounds the total.  If some lane's terms have bits below the window, one
// lane evaluates all parts in the local-memory accumulator and broadcasts
// the result.  All 32 lanes of the warp must call this together.
template <int NW, typename Gen>
__device__ __forceinline__ void warp_exact_round(int q, Gen&& gen, double* out, bool& bad) {
    const int lane = threadIdx.x & 31;
    TopVisitor tv;
    gen(tv, lane);
    const int top = __reduce_max_sync(0xffffffffu, tv.top);
    const int count = (int)__reduce_add_sync(0xffffffffu, (unsigned)tv.count);
    if (count == 0) {
        for (int c = 0; c < q; ++c) out[c] = 0.0;
        return;
    }
    RegVisitor<NW> rv;
    rv.init(top, count);
    gen(rv, lane);
    if (!__any_sync(0xffffffffu, rv.tail)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            uint64_t other[NW];
#pragma unroll
            for (int j = 0; j < NW; ++j) other[j] = __shfl_xor_sync(0xffffffffu, rv.w[j], o);
            mw_add<NW>(rv.w, other);
        }
        if (!canonical_round<NW, double>(rv.w, rv.L, q, out)) bad = true;
        return;
    }
    double res[8];
    bool b = false;
    if (lane == 0) {
        KulVisitor kv;
        clear(kv.a);
        for (int part = 0; part < 32; ++part) gen(kv, part);
        b = kv.a.range_bad;
        round_q(kv.a, q, res);
        b |= kv.a.range_bad;
    }
    for (int c = 0; c < q; ++c) out[c] = __shfl_sync(0xffffffffu, res[c], 0);
    bad |= __shfl_sync(0xffffffffu, (int)b, 0) != 0;
}

}  // namespace xacc
}  // namespace ozmp
