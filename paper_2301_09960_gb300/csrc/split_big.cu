// Splitter for many components: exponent reduce (K1) and exact truncating
// e4m3 digit split (K2, 4-bit or balanced radix-32 digits) for operands of up
// to OZMP_MAX_COMPONENTS binary64 components, or more slices than the
// register-resident path writes (64 four-bit, 63 balanced).
//
// Paper, Sec. 3, Algorithm 1 (mu, tau and the slice extraction), carried to
// the multiple precisions of Sec. 5.  Same definitions as the q <= 4 path:
// E_i = max_p floor(log2|a_ip|) + 1 of the exact values, and the s digits
// of |a_ip| 2^(beta s - E_i) truncated toward zero (sign of a_ip).  Here the
// component count is a run-time loop, the window has 8, 12 or 16 64-bit
// words, and the digits of a 16 x 32 tile are staged in shared memory so
// that both the component loads and the digit stores are coalesced.
#include "kernels.h"
#include "ozmp_internal.cuh"

namespace ozmp {
namespace big {

constexpr int QB = OZMP_MAX_COMPONENTS;
constexpr int TR = 16, TC = 32;   // tile: 16 (row / column) lines x 32 k
constexpr int NT = 256;

struct Op {
    const double* c[QB];
    int64_t ld;
    int q;
};

__device__ __forceinline__ void load_comps(const Op& op, bool inside, int64_t idx, double (&v)[QB]) {
#pragma unroll
    for (int c = 0; c < QB; ++c) v[c] = (inside && c < op.q) ? op.c[c][idx] : 0.0;
}

// Exact sum of q binary64 values over the whole binary64 range (local
// memory, rolled loops): two's complement words W, returns the sign and
// leaves the magnitude in W.
static __device__ __noinline__ int slow_sum_n(const double* v, int q, uint64_t* W) {
#pragma unroll 1
    for (int j = 0; j < SLOW_NW; ++j) W[j] = 0;
#pragma unroll 1
    for (int i = 0; i < q; ++i) {
        Comp c;
        decode(v[i], c);
        if (c.M == 0) continue;
        const int sh = c.e - SLOW_L;
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
    int nz = 0;
#pragma unroll 1
    for (int j = 0; j < SLOW_NW; ++j) if (W[j]) nz = 1;
    if (!nz) return 0;
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

static __device__ __noinline__ int slow_exponent_n(const double* v, int q) {
    uint64_t W[SLOW_NW];
    if (!slow_sum_n(v, q, W)) return OZMP_EXP_ZERO;
    int top = -1;
#pragma unroll 1
    for (int j = SLOW_NW - 1; j >= 0 && top < 0; --j)
        if (W[j]) top = 64 * j + 63 - __clzll((long long)W[j]);
    return SLOW_L + top + 1;
}

// nw words of |x| with the bit of weight 2^(Erow - 1) at bit `toppos`
static __device__ __noinline__ int slow_window_n(const double* v, int q, int Erow, int nw, int toppos,
                                                 uint64_t* out) {
    uint64_t W[SLOW_NW];
    const int sign = slow_sum_n(v, q, W);
    const int lo = (Erow - 1 - SLOW_L) - toppos;
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

// E(x) = floor(log2|x|) + 1 of x = v[0] + ... + v[q-1]; `ok` cleared for a
// non-finite component.  A 128-bit window anchored 123 bits below the top
// component's leading bit holds the sum of up to 16 truncated components
// exactly; bits below it move the top bit only when |V| lies within q of a
// power of two (then the full-range sum decides).
__device__ __forceinline__ int exponent_n(const double (&v)[QB], int q, bool& ok) {
    int Ptop = -100000;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
        if (i >= q) continue;
        Comp c;
        ok &= decode(v[i], c);
        if (c.M) {
            const int p = c.e + bitlen(c.M);
            Ptop = p > Ptop ? p : Ptop;
        }
    }
    if (Ptop == -100000) return OZMP_EXP_ZERO;
    const int L = Ptop - 123;
    unsigned __int128 V = 0;
    bool tail = false;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
        if (i >= q) continue;
        Comp c;
        decode(v[i], c);
        if (c.M == 0) continue;
        const int sh = c.e - L;   // <= 123 - bitlen(M)
        unsigned __int128 part;
        if (sh >= 0) {
            part = (unsigned __int128)c.M << sh;
        } else {
            const int r = -sh;
            const uint64_t mask = (r >= 64) ? ~0ull : ((1ull << r) - 1ull);
            if (c.M & mask) tail = true;
            part = (unsigned __int128)((r >= 64) ? 0ull : (c.M >> r));
        }
        V = c.neg ? V - part : V + part;
    }
    const bool negv = (uint64_t)(V >> 127) != 0;
    const unsigned __int128 A = negv ? (unsigned __int128)0 - V : V;
    const uint64_t hi = (uint64_t)(A >> 64), lo = (uint64_t)A;
    const int top = hi ? 64 + 63 - __clzll((long long)hi) : (lo ? 63 - __clzll((long long)lo) : -1);
    if (!tail) return top < 0 ? OZMP_EXP_ZERO : L + top + 1;
    if (top >= 64) {
        const unsigned __int128 pw = (unsigned __int128)1 << top;
        const unsigned __int128 below = A - pw;
        const unsigned __int128 above = (top < 127) ? ((unsigned __int128)1 << (top + 1)) - A : (unsigned __int128)1;
        if (below >= (unsigned __int128)q && above > (unsigned __int128)q) return L + top + 1;
    }
    return slow_exponent_n(v, q);
}

// |x| in an NW-word window whose bit 64 NW - 1 has weight 2^(Erow - 1) (with
// NIB; 2^Erow without), so that 4-bit digit t (1-based) is the nibble at bits
// [64 NW - 4 t, 64 NW - 4 t + 4), or balanced radix-32 group t is at bits
// [64 NW - 5 t, 64 NW - 5 t + 5).
// Word 0 lies below every digit (64 NW >= 4 s + 65) and absorbs truncation:
// bits of components below the window change the truncated magnitude only
// through a borrow or carry out of word 0, possible only when word 0 is
// within q of 0 or of 2^64; those cases take the full-range sum.
// Returns the sign of x (0 for zero or an all-zero row).
template <int NW, bool NIB = true>
__device__ __forceinline__ int window_n(const double (&v)[QB], int q, int Erow, uint64_t (&w)[NW]) {
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = 0;
    if (Erow == OZMP_EXP_ZERO) return 0;
    const int L = Erow - (64 * NW - 1);   // window bit 0 has weight 2^L; 2^(Erow-1) at bit 64 NW - 2
    bool tail = false;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
        if (i >= q) continue;
        Comp c;
        decode(v[i], c);
        if (c.M == 0) continue;
        const int sh = c.e - L;
        if (sh < 0) {
            const int r = -sh;
            const uint64_t mask = (r >= 64) ? ~0ull : ((1ull << r) - 1ull);
            if (c.M & mask) tail = true;
        }
        uint64_t p[NW];
        mw_place<NW>(p, c.M, sh);
        if (c.neg) mw_sub<NW>(w, p); else mw_add<NW>(w, p);
    }
    const bool neg = (w[NW - 1] >> 63) != 0;
    if (neg) mw_neg<NW>(w);
    int sg;
    if (!tail || (w[0] >= (uint64_t)q && w[0] <= ~0ull - (uint64_t)q)) {
        sg = mw_is_zero<NW>(w) ? 0 : (neg ? -1 : 1);
    } else {
        uint64_t tmp[NW];
        sg = slow_window_n(v, q, Erow, NW, 64 * NW - 2, tmp);
#pragma unroll
        for (int j = 0; j < NW; ++j) w[j] = tmp[j];
    }
    if (NIB) mw_shl<NW>(w, 1);   // nibble-align the digits (the top bit is 0 for a magnitude below 2^Erow)
    return sg;
}

// e4m3 code of a digit magnitude 0..15 (all exact in e4m3), sign bit for a
// negative non-zero digit
__device__ __forceinline__ uint32_t e4m3_nibble(uint32_t d, bool neg) {
    const uint32_t code = __byte_perm(d < 8 ? 0x44403800u : 0x53525150u, d < 8 ? 0x4E4C4A48u : 0x57565554u, d & 7u) & 0xFFu;
    return (neg && d) ? (code | 0x80u) : code;
}

// the s digits of one element into shared memory, slice t at out[(t-1) * stride]
template <int NW>
__device__ __forceinline__ void emit_digits(const uint64_t (&w)[NW], int sg, int s, uint8_t* out, int stride) {
    const bool neg = sg < 0;
#pragma unroll
    for (int jj = 0; jj < NW; ++jj) {
        const uint64_t word = w[NW - 1 - jj];
#pragma unroll
        for (int nb = 0; nb < 16; ++nb) {
            const int t = jj * 16 + nb + 1;
            if (t <= s) out[(t - 1) * stride] = (uint8_t)e4m3_nibble((uint32_t)(word >> (60 - 4 * nb)) & 15u, neg);
        }
    }
}

// e4m3 code of a digit d in [-16, 16] (all exact in e4m3; zero is +0)
__device__ __forceinline__ uint32_t e4m3_small(int d) {
    const uint32_t m = (uint32_t)(d < 0 ? -d : d);
    const uint32_t code = m == 16u ? 0x58u : e4m3_nibble(m, false);
    return (d < 0) ? (code | 0x80u) : code;
}

// the s balanced radix-32 digits of one element into shared memory: the
// groups of the magnitude window plus 16 at every group (nothing added below
// the lowest one) are the balanced digits plus 16, the carry out of the top
// group making the top digit 16; each digit then takes the sign of x
template <int NW>
__device__ __forceinline__ void emit_digits_bal(uint64_t (&w)[NW], int sg, int s, uint8_t* out, int stride) {
    constexpr int TMAX = (64 * NW - 65) / 5;
    const int lo = 64 * NW - 5 * s;
    constexpr BalSixteens<NW> P16;
    uint64_t H[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        const uint64_t keep = (lo <= 64 * j) ? ~0ull : (lo >= 64 * j + 64 ? 0ull : (~0ull << (lo - 64 * j)));
        H[j] = P16.w[j] & keep;
    }
    const uint64_t before = w[NW - 1];
    mw_add<NW>(w, H);
    const int top = (w[NW - 1] < before) ? 32 : 0;   // the top word carries bit 63 of H
    const int sgn = sg < 0 ? -1 : 1;
#pragma unroll
    for (int t = 1; t <= TMAX; ++t) {
        if (t > s) break;
        const int pos = 64 * NW - 5 * t;
        const int wi = pos >> 6, off = pos & 63;
        uint64_t x = w[wi] >> off;
        if (off > 59) x |= w[wi + 1] << (64 - off);
        const int g = (int)((uint32_t)x & 31u) + (t == 1 ? top : 0);
        out[(t - 1) * stride] = (uint8_t)e4m3_small(sgn * (g - 16));
    }
}

// ---------------------------------------------------------------------------
// K1: exponents
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_exp_rows_n(Op a, int64_t m, int64_t k, int kchunk, int32_t* E,
                                                   uint32_t* status) {
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (i >= m) return;
    const int64_t p0 = (int64_t)blockIdx.y * kchunk;
    const int64_t p1 = p0 + kchunk < k ? p0 + kchunk : k;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    for (int64_t p = p0; p < p1; ++p) {
        double v[QB];
        load_comps(a, true, i + p * a.ld, v);
        const int e = exponent_n(v, a.q, ok);
        emax = e > emax ? e : emax;
    }
    if (emax != OZMP_EXP_ZERO) atomicMax(&E[i], emax);
    if (!ok) atomicOr(status, ST_NONFINITE);
}

__global__ void __launch_bounds__(NT) k_exp_cols_n(Op b, int64_t k, int64_t n, int32_t* F, uint32_t* status) {
    const int64_t j = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    for (int64_t p = lane; p < k; p += 32) {
        double v[QB];
        load_comps(b, true, p + j * b.ld, v);
        const int e = exponent_n(v, b.q, ok);
        emax = e > emax ? e : emax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int x = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = x > emax ? x : emax;
    }
    const unsigned bad = __ballot_sync(0xffffffffu, !ok);
    if (lane == 0) {
        F[j] = emax;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

// ---------------------------------------------------------------------------
// K2: digits.  A tile is TR lines (rows of A / columns of B) x TC values of k;
// the digits go to shared memory [s][TR][TC] and then to dig[t][line][k] as
// 32-byte line segments.
//   ROWS: A (column-major m x k, element (i, p) at i + p lda), lines = rows;
//   else: B (column-major k x n, element (p, j) at p + j ldb), lines = columns.
// ---------------------------------------------------------------------------
template <int NW, bool ROWS, bool BAL>
__global__ void __launch_bounds__(NT) k_split_n(Op op, int64_t lines, int64_t k, const int32_t* Ex, uint8_t* dig,
                                                int64_t lp, int64_t kp, int s) {
    extern __shared__ __align__(16) uint8_t sd[];
    const int64_t l0 = (int64_t)blockIdx.x * TR, p0 = (int64_t)blockIdx.y * TC;
#pragma unroll 1
    for (int h = 0; h < (TR * TC) / NT; ++h) {
        const int e = threadIdx.x + NT * h;
        // consecutive threads walk the contiguous direction of the operand
        const int rl = ROWS ? (e % TR) : (e / TC);
        const int cp = ROWS ? (e / TR) : (e % TC);
        const int64_t line = l0 + rl, p = p0 + cp;
        const bool inside = line < lines && p < k;
        double v[QB];
        load_comps(op, inside, ROWS ? (line + p * op.ld) : (p + line * op.ld), v);
        const int Er = (line < lines) ? Ex[line] : OZMP_EXP_ZERO;
        uint64_t w[NW];
        const int sg = window_n<NW, !BAL>(v, op.q, inside ? Er : OZMP_EXP_ZERO, w);
        if (BAL) emit_digits_bal<NW>(w, sg, s, sd + rl * TC + cp, TR * TC);
        else emit_digits<NW>(w, sg, s, sd + rl * TC + cp, TR * TC);
    }
    __syncthreads();
    const int words = s * TR * (TC / 4);
    for (int x = threadIdx.x; x < words; x += NT) {
        const int t = x / (TR * (TC / 4)), r = (x / (TC / 4)) % TR, c = x % (TC / 4);
        *reinterpret_cast<uint32_t*>(dig + ((size_t)t * lp + (l0 + r)) * kp + p0 + 4 * c) =
            reinterpret_cast<const uint32_t*>(sd)[x];
    }
}

static Op make_op(const void* const* comps, int q, int64_t ld) {
    Op o;
    for (int c = 0; c < QB; ++c) o.c[c] = (c < q) ? (const double*)comps[c] : nullptr;
    o.ld = ld;
    o.q = q;
    return o;
}

template <int NW, bool BAL>
static cudaError_t digits(const SplitArgs& g, cudaStream_t st) {
    const size_t smem = (size_t)g.s * TR * TC;
    cudaError_t e =
        cudaFuncSetAttribute(k_split_n<NW, true, BAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_split_n<NW, false, BAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (g.m > 0) {
        const Op a = make_op(g.A, g.q, g.lda);
        dim3 gr((unsigned)(g.mp / TR), (unsigned)(g.kp / TC));
        k_split_n<NW, true, BAL><<<gr, NT, smem, st>>>(a, g.m, g.k, g.E, (uint8_t*)g.Adig, g.mp, g.kp, g.s);
    }
    if (g.n > 0) {
        const Op b = make_op(g.B, g.q, g.ldb);
        dim3 gr((unsigned)(g.np / TR), (unsigned)(g.kp / TC));
        k_split_n<NW, false, BAL><<<gr, NT, smem, st>>>(b, g.n, g.k, g.F, (uint8_t*)g.Bdig, g.np, g.kp, g.s);
    }
    return cudaGetLastError();
}

}  // namespace big

// exponents of both operands (the E/F arrays and the status word are
// initialised by the caller)
cudaError_t launch_exponents_big(const SplitArgs& g, cudaStream_t st) {
    if (g.m > 0 && g.k > 0) {
        const big::Op a = big::make_op(g.A, g.q, g.lda);
        const int kchunk = 64;
        dim3 gr((unsigned)((g.m + big::NT - 1) / big::NT), (unsigned)((g.k + kchunk - 1) / kchunk));
        big::k_exp_rows_n<<<gr, big::NT, 0, st>>>(a, g.m, g.k, kchunk, g.E, g.status);
    }
    if (g.n > 0 && g.k > 0) {
        const big::Op b = big::make_op(g.B, g.q, g.ldb);
        big::k_exp_cols_n<<<(unsigned)((g.n + 7) / 8), big::NT, 0, st>>>(b, g.k, g.n, g.F, g.status);
    }
    return cudaGetLastError();
}

// e4m3 digits (4-bit, or balanced radix-32 with g.bal); the window has 8,
// 12 or 16 words (beta s + 65 bits at least)
cudaError_t launch_digits_big(const SplitArgs& g, cudaStream_t st) {
    const int need = (g.beta * g.s + 65 + 63) / 64;
    if (g.form != OZMP_FORM_FP8 && g.form != OZMP_FORM_FP8_MMA) return cudaErrorInvalidValue;
    if (g.is_f32 || need > 16 || (g.bal && g.beta != 5)) return cudaErrorInvalidValue;
    if (g.bal) {
        if (need <= 8) return big::digits<8, true>(g, st);
        if (need <= 12) return big::digits<12, true>(g, st);
        return big::digits<16, true>(g, st);
    }
    if (need <= 8) return big::digits<8, false>(g, st);
    if (need <= 12) return big::digits<12, false>(g, st);
    return big::digits<16, false>(g, st);
}

}  // namespace ozmp
