// Splitter: exponent reduce (K1) and exact truncating digit split (K2).
//
// Paper, Sec. 3, Algorithm 1: mu_A / mu_B (row / column maxima), the
// power-of-two shifts tau_A / tau_B, and the extraction of the slices
// A_alpha, B_alpha.  Here the shift of row i is 2^E_i with
// E_i = max_p floor(log2|a_ip|) + 1 of the exact element values, and the
// slices are the base-2^beta digits of |a_ip| 2^(beta s - E_i) truncated
// toward zero (sign of a_ip), found with exact integer arithmetic on the
// IEEE encodings.
#pragma once
#include "ozmp_internal.cuh"
#include "kernels.h"

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
__device__ __forceinline__ bool load_elem(const Operand<T>& op, int64_t idx, Comp* c, int& Ptop) {
    T v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (i < op.q) ? op.c[i][idx] : (T)0;
    return decode_all<T>(v, op.q, c, Ptop);
}

// ---------------------------------------------------------------------------
// K1: exponents
// ---------------------------------------------------------------------------
// rows of a column-major m x k matrix: one thread per row, a chunk of
// columns per block row; consecutive threads read consecutive addresses.
template <typename T>
__global__ void k_exp_rows(Operand<T> a, int64_t m, int64_t k, int kchunk, int32_t* E, uint32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    int64_t p0 = (int64_t)blockIdx.y * kchunk;
    int64_t p1 = p0 + kchunk < k ? p0 + kchunk : k;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    for (int64_t p = p0; p < p1; ++p) {
        Comp c[4];
        int Ptop;
        ok &= load_elem<T>(a, i + p * a.ld, c, Ptop);
        Exact ex = exact_exponent(c, a.q, Ptop);
        emax = ex.E > emax ? ex.E : emax;
    }
    if (emax != OZMP_EXP_ZERO) atomicMax(&E[i], emax);
    if (!ok) atomicOr(status, ST_NONFINITE);
}

// columns of a column-major k x n matrix (contiguous): one warp per column,
// warp-shuffle max reduction.
template <typename T>
__global__ void k_exp_cols(Operand<T> b, int64_t k, int64_t n, int32_t* F, uint32_t* status) {
    int warps = blockDim.x >> 5;
    int64_t j = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (j >= n) return;
    int emax = OZMP_EXP_ZERO;
    bool ok = true;
    for (int64_t p = lane; p < k; p += 32) {
        Comp c[4];
        int Ptop;
        ok &= load_elem<T>(b, p + j * b.ld, c, Ptop);
        Exact ex = exact_exponent(c, b.q, Ptop);
        emax = ex.E > emax ? ex.E : emax;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int v = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = v > emax ? v : emax;
    }
    unsigned bad = __ballot_sync(0xffffffffu, !ok);
    if (lane == 0) {
        F[j] = emax;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
}

// ---------------------------------------------------------------------------
// K2: digits
// ---------------------------------------------------------------------------
// digit encodings: FORM_INT8 -> two's complement int8, FORM_FP8 -> e4m3,
// FORM_FP64 -> binary64 integer value.
template <int FORM>
struct DigitTraits;
template <> struct DigitTraits<OZMP_FORM_INT8> { typedef uint8_t T; static constexpr int BETA = 7; static constexpr int MAXS = 36; };
template <> struct DigitTraits<OZMP_FORM_FP8> { typedef uint8_t T; static constexpr int BETA = 4; static constexpr int MAXS = 64; };
template <> struct DigitTraits<OZMP_FORM_FP64> { typedef double T; static constexpr int BETA = 0; static constexpr int MAXS = 64; };

template <int FORM>
__device__ __forceinline__ uint8_t encode_byte(int sign, uint32_t d) {
    int v = sign < 0 ? -(int)d : (int)d;
    if (FORM == OZMP_FORM_INT8) return (uint8_t)(int8_t)v;
    return (uint8_t)e4m3_of_int(v);
}

// Rows of A: 32 x 32 element tile (1-byte digits) or 16 x 16 (binary64),
// digits staged in shared memory [s][TI][TP] and written K-contiguous:
// Adig[(t * mp + i) * kp + p].
template <typename T, int FORM, int TI, int TP>
__global__ void __launch_bounds__(256) k_split_rows(Operand<T> a, int64_t m, int64_t k, const int32_t* E,
                                                    void* dig, int64_t mp, int64_t kp, int s, int beta) {
    typedef typename DigitTraits<FORM>::T DT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DT* sd = reinterpret_cast<DT*>(smem_raw);
    const int64_t i0 = (int64_t)blockIdx.x * TI;
    const int64_t p0 = (int64_t)blockIdx.y * TP;
    constexpr int EPT = (TI * TP) / 256;   // elements per thread
#pragma unroll 1
    for (int e = 0; e < EPT; ++e) {
        int lin = threadIdx.x + 256 * e;
        int ri = lin % TI, pi = lin / TI;   // consecutive threads: consecutive rows (coalesced reads)
        int64_t i = i0 + ri, p = p0 + pi;
        Comp c[4];
        int Ptop = -100000;
        if (i < m && p < k) load_elem<T>(a, i + p * a.ld, c, Ptop);
        int Erow = (i < m) ? E[i] : OZMP_EXP_ZERO;
        uint64_t w[FAST_NW];
        int sign = (Erow == OZMP_EXP_ZERO) ? 0 : aligned_magnitude(c, a.q, Ptop, Erow, w);
        if (FORM == OZMP_FORM_FP64) {
            for (int t = 1; t <= s; ++t) {
                uint32_t d = sign ? take_top(w, beta) : 0u;
                double v = (double)d;
                ((double*)sd)[((t - 1) * TI + ri) * TP + pi] = sign < 0 ? -v : v;
            }
        } else {
            constexpr int BETA = DigitTraits<FORM>::BETA;
#pragma unroll
            for (int t = 1; t <= DigitTraits<FORM>::MAXS; ++t) {
                if (t <= s) {
                    uint32_t d = sign ? digit_at<BETA>(w, t) : 0u;
                    ((uint8_t*)sd)[((t - 1) * TI + ri) * TP + pi] = encode_byte<FORM>(sign, d);
                }
            }
        }
    }
    __syncthreads();
    // write out: each slice is a TI x TP tile, rows of TP digits
    constexpr int WORD = 4;                                   // bytes per store
    constexpr int ROWBYTES = TP * (int)sizeof(DT);
    constexpr int WPR = ROWBYTES / WORD;                      // words per row
    const int total = s * TI * WPR;
    for (int w = threadIdx.x; w < total; w += 256) {
        int t = w / (TI * WPR);
        int r = (w / WPR) % TI;
        int c = w % WPR;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(smem_raw + ((size_t)(t * TI + r) * TP) * sizeof(DT)) + c;
        unsigned char* dst = (unsigned char*)dig + (((size_t)t * mp + (i0 + r)) * kp + p0) * sizeof(DT) + (size_t)c * WORD;
        *reinterpret_cast<uint32_t*>(dst) = *src;
    }
}

// Columns of B (contiguous along k): 1-byte digits, 4 consecutive k per
// thread (one 32-bit store per slice); Bdig[(t * np + j) * kp + p].
template <typename T, int FORM>
__global__ void __launch_bounds__(256) k_split_cols_b1(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                       uint8_t* dig, int64_t np, int64_t kp, int s) {
    constexpr int BETA = DigitTraits<FORM>::BETA;
    const int64_t quads = kp / 4;
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= quads * np) return;
    int64_t j = g / quads;
    int64_t p0 = (g % quads) * 4;
    int Ecol = (j < n) ? F[j] : OZMP_EXP_ZERO;
    uint64_t w[4][FAST_NW];
    int sign[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        int64_t p = p0 + e;
        Comp c[4];
        int Ptop = -100000;
        if (j < n && p < k) load_elem<T>(b, p + j * b.ld, c, Ptop);
        sign[e] = (Ecol == OZMP_EXP_ZERO) ? 0 : aligned_magnitude(c, b.q, Ptop, Ecol, w[e]);
    }
#pragma unroll
    for (int t = 1; t <= DigitTraits<FORM>::MAXS; ++t) {
        if (t <= s) {
            uint32_t word = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                uint32_t d = sign[e] ? digit_at<BETA>(w[e], t) : 0u;
                word |= (uint32_t)encode_byte<FORM>(sign[e], d) << (8 * e);
            }
            *reinterpret_cast<uint32_t*>(dig + ((size_t)(t - 1) * np + j) * kp + p0) = word;
        }
    }
}

// Columns of B, binary64 digits: one element per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_split_cols_f64(Operand<T> b, int64_t k, int64_t n, const int32_t* F,
                                                        double* dig, int64_t np, int64_t kp, int s, int beta) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= kp * np) return;
    int64_t j = g / kp, p = g % kp;
    int Ecol = (j < n) ? F[j] : OZMP_EXP_ZERO;
    Comp c[4];
    int Ptop = -100000;
    if (j < n && p < k) load_elem<T>(b, p + j * b.ld, c, Ptop);
    uint64_t w[FAST_NW];
    int sign = (Ecol == OZMP_EXP_ZERO) ? 0 : aligned_magnitude(c, b.q, Ptop, Ecol, w);
    for (int t = 1; t <= s; ++t) {
        uint32_t d = sign ? take_top(w, beta) : 0u;
        double v = (double)d;
        dig[((size_t)(t - 1) * np + j) * kp + p] = sign < 0 ? -v : v;
    }
}

template <typename T>
static inline Operand<T> make_op(const void* const* comps, int q, int64_t ld) {
    Operand<T> o;
    for (int i = 0; i < 4; ++i) o.c[i] = (i < q) ? (const T*)comps[i] : nullptr;
    o.ld = ld;
    o.q = q;
    return o;
}

// digits of both operands for one form (the padded region gets zero digits)
template <typename T, int FORM>
static cudaError_t digits_impl(const SplitArgs& g, cudaStream_t st) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    if (FORM == OZMP_FORM_FP64) {
        dim3 gr((unsigned)(g.mp / 16), (unsigned)(g.kp / 16));
        size_t sm = (size_t)g.s * 16 * 16 * 8;
        auto kr = k_split_rows<T, OZMP_FORM_FP64, 16, 16>;
        cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kr<<<gr, 256, sm, st>>>(a, g.m, g.k, g.E, g.Adig, g.mp, g.kp, g.s, g.beta);
        int64_t tot = g.kp * g.np;
        k_split_cols_f64<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b, g.k, g.n, g.F, (double*)g.Bdig,
                                                                         g.np, g.kp, g.s, g.beta);
    } else {
        dim3 gr((unsigned)(g.mp / 32), (unsigned)(g.kp / 32));
        size_t sm = (size_t)g.s * 32 * 32;
        int64_t tot = (g.kp / 4) * g.np;
        auto kr = k_split_rows<T, FORM, 32, 32>;
        cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kr<<<gr, 256, sm, st>>>(a, g.m, g.k, g.E, g.Adig, g.mp, g.kp, g.s, g.beta);
        k_split_cols_b1<T, FORM><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
            b, g.k, g.n, g.F, (uint8_t*)g.Bdig, g.np, g.kp, g.s);
    }
    return cudaGetLastError();
}

}  // namespace ozmp
