// Error bound of the truncated slice split, the data-dependent slice count
// and the a-posteriori check of a product (bound.cu).
//
// Sec. 3 notes that the number of slices a product needs depends on the
// data.  With exact truncating digits (weights 2^(E_i + eo - beta t),
// |d_t| <= D, remainder |r| < 2^(E_i + eo - beta s)) the computed sum S of the
// pairs t + u <= s + 1 satisfies, per element,
//   |S_ij - C*_ij| <= k c(s) 2^(E_i + F_j - W(s)),   W(s) = beta s - eo,
//   c(s) = 2 + 2^(eo - beta s) + (s - 1) D^2 2^(eo - 2 beta) / (1 - 2^-beta):
// the two cross terms a^ r_b and r_a b^ (each below 2^(E + F - W) per term,
// as |a^| <= |a| < 2^E), the product of the remainders, and the dropped pairs
// t + u >= s + 2 (at most 2 s + 1 - d pairs on diagonal d, a geometric tail).
// Summed over the elements of C, in the Frobenius norm,
//   ||S - C*||_F <= k c(s) 2^-W(s) ||2^E||_2 ||2^F||_2.
//
// A-priori choice: ||C*||_F is estimated by sqrt(sum_p ||A(:,p)||^2
// ||B(p,:)||^2) (exact in expectation for independent signs); s is the
// smallest count whose bound is 2^-(target + 1) of that estimate.  The
// exponent passes take each element's magnitude as its leading component
// when that component carries the element's exponent, else 2^(e-1), and sum
// the squares in binary32; the scaled fallback launches take the binary64
// sum of the components.
// A-posteriori check: with the result's first components c0,
// ||C*||_F >= ||S||_F - bound, and the canonical rounding into q components
// adds at most u_q ||S||_F; the check flags the result when
// (bound + u_q N) / (N - bound) > 2^-target, N a lower bound of ||S||_F.
//
// All sums are scaled by 2^-(GE + GF), GE = max E_i, GF = max F_j, so no
// square overflows; rows far below the largest (4^(E_i - GE) below the
// binary64 range) contribute nothing measurable to either norm.
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ozmp.h"

namespace ozmp {

// digit form of the bound: weights 2^(E + eo - beta t), |d| <= dmax
struct BoundForm {
    int beta, eo, dmax;
    int target;     // normwise target 2^-target
    double uq;      // relative error of the canonical rounding into the output components
    int64_t k;
};

// workspace statistics of one product (off_stats)
struct BoundStats {
    int GE, GF;          // largest row / column exponent (OZMP_EXP_ZERO: all rows / columns zero)
    int s_needed;        // the a-priori slice count
    unsigned int done;   // blocks of the check launch that have finished
    double SE, SF;       // sum_i 4^(E_i - GE), sum_j 4^(F_j - GF)
    double est;          // sum_p ||A(:,p)||^2 ||B(p,:)||^2, scaled by 4^-(GE + GF)
    double normS2;       // sum of the squared first output components, scaled likewise
};

// c(s) and W(s) of the bound (see the file comment)
__host__ __device__ inline double bound_coeff(const BoundForm& f, int s) {
    const double D = (double)f.dmax;
    const double tail = D * D * ldexp(1.0, f.eo - 2 * f.beta) / (1.0 - ldexp(1.0, -f.beta));
    return 2.0 + ldexp(1.0, f.eo - f.beta * s) + (double)(s - 1) * tail;
}
__host__ __device__ inline int bound_W(const BoundForm& f, int s) { return f.beta * s - f.eo; }

// log2 of the bound relative to 2^(GE + GF): log2(k c(s)) - W(s) + log2(sqrt(SE SF))
__host__ __device__ inline double bound_log2(const BoundForm& f, int s, double SE, double SF) {
    return log2((double)f.k * bound_coeff(f, s)) - (double)bound_W(f, s) + 0.5 * (log2(SE) + log2(SF));
}

// The largest exponent magnitude for which the unscaled squared norms of the
// exponent pass (launch_split_exponents_norm), summed in binary32, stay
// inside its normal range: squares below 2^80, their sums over up to 2^31
// rows below 2^111, the row maxima's squares above 2^-80.
constexpr int BOUND_RAW_EXP = 40;

#ifdef __CUDACC__
// (x 2^-g)^2, exact scaling where 2^-g is a normal number
__device__ __forceinline__ double bound_sq_scaled(double x, int g) {
    const double y = (g > -1000 && g < 1000) ? x * __longlong_as_double((long long)(1023 - g) << 52) : ldexp(x, -g);
    return y * y;
}

// |x| 2^-g as a binary32 from the bits of x with integer operations only (no
// binary64 arithmetic, which is slow on this GPU): the mantissa is truncated
// to 24 bits, so the value is never above |x| 2^-g; 0 below the binary32
// normal range (those squares do not count against the sums they enter)
__device__ __forceinline__ float bound_abs_scaled_f32(double x, int g) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int fe = (int)((b >> 52) & 0x7ff) - 1023 - g + 127;
    if (((b >> 52) & 0x7ff) == 0 || fe <= 0) return 0.f;
    const unsigned fb = ((unsigned)(fe < 254 ? fe : 254) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    return __uint_as_float(fb);
}

// Thread 0 of each block of a check: adds the block's sum of squared first
// components (scaled by 4^-(GE + GF)); the last of the nblocks blocks decides
// whether the bound certifies the target (else `flag` into *status) and
// resets the accumulators for the next check of the same split.
__device__ __forceinline__ void bound_finish_block(BoundStats* st, double bsum, unsigned nblocks, const BoundForm& f,
                                                   int s, uint32_t* status, uint32_t flag) {
    atomicAdd(&st->normS2, bsum);
    __threadfence();
    if (atomicAdd(&st->done, 1u) != nblocks - 1) return;
    __threadfence();
    const double n2 = atomicAdd(&st->normS2, 0.0);
    st->normS2 = 0.0;
    st->done = 0u;
    if (st->GE == OZMP_EXP_ZERO || st->GF == OZMP_EXP_ZERO) return;   // C* = 0 exactly
    // N: a lower bound of ||S||_F (the first components are within 2^-53 of
    // S, scaled and truncated below their value; the binary32 partial sums of
    // at most a few thousand squares are within far less than 2^-10)
    const double N = sqrt(n2) * (1.0 - ldexp(1.0, -10));
    const double B = exp2(bound_log2(f, s, st->SE, st->SF));
    bool ok = N > B;
    if (ok) ok = (B + f.uq * N) / (N - B) <= ldexp(1.0, -f.target);
    if (!ok) atomicOr(status, flag);
}
#endif

// Statistics of the exponents (and, when `norms`, the zeroed row-norm array).
cudaError_t launch_bound_scale(const int32_t* E, int64_t m, const int32_t* F, int64_t n, BoundStats* st,
                               double* rowB, int64_t k, bool norms, cudaStream_t stream);
// Column norms of A and row norms of B (elements as binary64 sums of their
// components), then the a-priori slice count in [s_lo, s_hi] into st->s_needed.
cudaError_t launch_bound_choose(const void* const* A, int64_t lda, const void* const* B, int64_t ldb, int q,
                                bool is_f32, int64_t m, int64_t n, int64_t k, BoundStats* st, double* colA,
                                double* rowB, const BoundForm& f, int s_lo, int s_hi, cudaStream_t stream);
// After launch_split_exponents_norm: the exponent statistics and the slice
// count from the unscaled norms in one launch (resets the check's
// accumulators too); st->s_needed = -1 when an exponent lies beyond
// BOUND_RAW_EXP (then the scaled launches above decide).  B's row norms come
// from rowBf (binary32, summed by the one-pass column digit kernel) when it is
// set, else from rowB.  s_hi - s_lo < 256 (one block of 256 threads, a candidate
// count each).
cudaError_t launch_bound_choose_raw(const int32_t* E, int64_t m, const int32_t* F, int64_t n, const double* colA,
                                    const double* rowB, const float* rowBf, int64_t k, BoundStats* st,
                                    const BoundForm& f, int s_lo, int s_hi, cudaStream_t stream);
// The a-posteriori check of a result with s slices (first output component C0,
// column-major m x n, leading dimension ldc): sets `flag` in *status when the
// bound does not certify the target.
cudaError_t launch_bound_check(const void* C0, bool is_f32, int64_t m, int64_t n, int64_t ldc, BoundStats* st,
                               const BoundForm& f, int s, uint32_t* status, uint32_t flag, cudaStream_t stream);

}  // namespace ozmp
