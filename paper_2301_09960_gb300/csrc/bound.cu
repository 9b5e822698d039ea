// Data-dependent slice count and a-posteriori error check (definitions in
// bound.cuh).  Small launches beside the product: one block for the exponent
// statistics, one pass over the columns of A and one over the rows of B for
// the a-priori estimate of ||C||_F, one pass over C's first component for the
// check.
#include <cfloat>
#include "bound.cuh"
#include "ozmp_internal.cuh"

namespace ozmp {
namespace {

struct Ptrs {
    const void* p[OZMP_MAX_COMPONENTS];
};

template <typename T>
__device__ __forceinline__ double elem(const Ptrs& a, int q, size_t at) {
    double x = 0.0;
    for (int c = 0; c < q; ++c) x += (double)((const T*)a.p[c])[at];
    return x;
}

// 2^e as a double (exact; e outside the normal range falls back to ldexp)
__device__ __forceinline__ double pow2(int e) {
    if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(1.0, e);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block-wide sum of one double per thread (blockDim.x a multiple of 32); the
// result is valid in thread 0
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

__device__ int block_max(int v, int* sh) {
    v = warp_max(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : OZMP_EXP_ZERO;
    if (w == 0) v = warp_max(v);
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = v;
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

// GE, GF, SE, SF; resets the check's accumulators (and zeroes rowB)
__global__ void __launch_bounds__(1024) k_bound_scale(const int32_t* E, int64_t m, const int32_t* F, int64_t n,
                                                      BoundStats* st, double* rowB, int64_t k) {
    __shared__ int shi[32];
    __shared__ double shd[32];
    int ge = OZMP_EXP_ZERO, gf = OZMP_EXP_ZERO;   // the zero sentinel is the smallest int
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) ge = max(ge, E[i]);
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) gf = max(gf, F[j]);
    ge = block_max(ge, shi);
    gf = block_max(gf, shi);
    double se = 0.0, sf = 0.0;
    if (ge != OZMP_EXP_ZERO)
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
            if (E[i] != OZMP_EXP_ZERO) se += ldexp(1.0, 2 * (E[i] - ge));
    if (gf != OZMP_EXP_ZERO)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            if (F[j] != OZMP_EXP_ZERO) sf += ldexp(1.0, 2 * (F[j] - gf));
    se = block_sum(se, shd);
    __syncthreads();
    sf = block_sum(sf, shd);
    if (threadIdx.x == 0) {
        st->GE = ge;
        st->GF = gf;
        st->SE = se;
        st->SF = sf;
        st->est = 0.0;
        st->normS2 = 0.0;
        st->done = 0u;
        st->s_needed = 0;
    }
    if (rowB)
        for (int64_t p = threadIdx.x; p < k; p += blockDim.x) rowB[p] = 0.0;
}

// x 2^-g, exact unless it leaves the normal range (then as ldexp)
__device__ __forceinline__ double scaled(double x, int g, double sc, bool plain) {
    return plain ? x * sc : ldexp(x, -g);
}

// ||A(:,p)||^2 scaled by 4^-GE: one warp per column, coalesced along the
// column, eight loads of a lane in flight at a time
template <typename T>
__global__ void __launch_bounds__(256) k_bound_colnorm(Ptrs a, int q, int64_t lda, int64_t m, int64_t k,
                                                       const BoundStats* st, double* colA) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= k) return;
    const int ge = st->GE;
    const bool plain = ge > -1000 && ge < 1000;   // 2^-ge normal, and no product leaves the range
    const double sc = plain ? pow2(-ge) : 1.0;
    double acc = 0.0;
    if (ge != OZMP_EXP_ZERO) {
        constexpr int U = 8;
        for (int64_t i0 = lane; i0 < m; i0 += 32 * U) {
            double x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + 32 * u;
                x[u] = i < m ? elem<T>(a, q, (size_t)(i + p * lda)) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const double y = scaled(x[u], ge, sc, plain);
                acc += y * y;
            }
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) colA[p] = acc;
}

// ||B(p,:)||^2 scaled by 4^-GF: threads along p (coalesced), 64 columns a
// block, eight loads in flight at a time
template <typename T>
__global__ void __launch_bounds__(256) k_bound_rownorm(Ptrs b, int q, int64_t ldb, int64_t k, int64_t n,
                                                       const BoundStats* st, double* rowB) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k) return;
    const int gf = st->GF;
    if (gf == OZMP_EXP_ZERO) return;
    const bool plain = gf > -1000 && gf < 1000;
    const double sc = plain ? pow2(-gf) : 1.0;
    const int64_t j0 = (int64_t)blockIdx.y * 64;
    const int64_t j1 = j0 + 64 < n ? j0 + 64 : n;
    double acc = 0.0;
    constexpr int U = 8;
    for (int64_t j = j0; j < j1; j += U) {
        double x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = (j + u < j1) ? elem<T>(b, q, (size_t)(p + (j + u) * ldb)) : 0.0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const double y = scaled(x[u], gf, sc, plain);
            acc += y * y;
        }
    }
    atomicAdd(&rowB[p], acc);
}

// est = sum_p colA[p] rowB[p]; the smallest s in [s_lo, s_hi] whose bound is
// 2^-(target + 1) of sqrt(est) (s_hi when none is)
__global__ void __launch_bounds__(1024) k_bound_choose(BoundStats* st, const double* colA, const double* rowB,
                                                       int64_t k, BoundForm f, int s_lo, int s_hi) {
    __shared__ double shd[32];
    double v = 0.0;
    for (int64_t p = threadIdx.x; p < k; p += blockDim.x) v += colA[p] * rowB[p];
    v = block_sum(v, shd);
    if (threadIdx.x != 0) return;
    st->est = v;
    int s = s_lo;
    if (st->GE != OZMP_EXP_ZERO && st->GF != OZMP_EXP_ZERO && v > 0.0) {
        const double rhs = -(double)(f.target + 1) + 0.5 * log2(v);
        s = s_hi;
        for (int t = s_lo; t <= s_hi; ++t)
            if (bound_log2(f, t, st->SE, st->SF) <= rhs) { s = t; break; }
    }
    st->s_needed = s;
}

// sum of the squared first components (scaled by 4^-(GE + GF)), blocks over
// columns; the last block to finish decides
template <typename T>
__global__ void __launch_bounds__(256) k_bound_check(const T* C0, int64_t m, int64_t n, int64_t ldc, BoundStats* st,
                                                     BoundForm f, int s, uint32_t* status, uint32_t flag) {
    __shared__ double shd[32];
    const int ge = st->GE, gf = st->GF;
    const bool zero = (ge == OZMP_EXP_ZERO || gf == OZMP_EXP_ZERO);
    double acc = 0.0;
    if (!zero)
        for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
            float col = 0.f;   // binary32 partial sums: one column part of at most m / 256 squares
            for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
                const float y = bound_abs_scaled_f32((double)C0[i + j * ldc], ge + gf);
                col += y * y;
            }
            acc += (double)col;
        }
    acc = block_sum(acc, shd);
    if (threadIdx.x == 0) bound_finish_block(st, acc, gridDim.x, f, s, status, flag);
}

// GE, GF, SE, SF from the exponents, est from the unscaled norms of the
// exponent pass, and the slice count (-1: an exponent beyond the raw range).
// One block; its latency is a fixed cost of every product, so the loads go
// in two passes (maxima and est, then SE and SF) and each pass's values are
// reduced together: warp shuffles, one shared-memory round, warp 0.
__global__ void __launch_bounds__(256) k_bound_choose_raw(const int32_t* E, int64_t m, const int32_t* F, int64_t n,
                                                           const double* colA, const double* rowB,
                                                           const float* rowBf, int64_t k, BoundStats* st,
                                                           BoundForm f, int s_lo, int s_hi) {
    __shared__ int shi[2][32];
    __shared__ double shd[3][32];
    __shared__ double bc[3];   // SE, SF, est to every thread
    __shared__ int bg[2];      // GE, GF to every thread
    __shared__ int best;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // pass 1: the largest exponents and est = sum_p colA[p] rowB[p]
    int ge = OZMP_EXP_ZERO, gf = OZMP_EXP_ZERO;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) ge = max(ge, E[i]);
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) gf = max(gf, F[j]);
    for (int64_t p = threadIdx.x; p < k; p += blockDim.x) v += colA[p] * (rowBf ? (double)rowBf[p] : rowB[p]);
    ge = warp_max(ge);
    gf = warp_max(gf);
    v = warp_sum(v);
    if (lane == 0) {
        shi[0][wid] = ge;
        shi[1][wid] = gf;
        shd[2][wid] = v;
    }
    __syncthreads();
    if (wid == 0) {
        ge = lane < nw ? shi[0][lane] : OZMP_EXP_ZERO;
        gf = lane < nw ? shi[1][lane] : OZMP_EXP_ZERO;
        v = lane < nw ? shd[2][lane] : 0.0;
        ge = warp_max(ge);
        gf = warp_max(gf);
        v = warp_sum(v);
        if (lane == 0) {
            bg[0] = ge;
            bg[1] = gf;
            bc[2] = v;
            best = s_hi;
        }
    }
    __syncthreads();
    ge = bg[0];
    gf = bg[1];
    v = bc[2];
    // pass 2: SE = sum_i 4^(E_i - GE), SF = sum_j 4^(F_j - GF)
    double se = 0.0, sf = 0.0;
    if (ge != OZMP_EXP_ZERO)
        for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
            if (E[i] != OZMP_EXP_ZERO) se += pow2(2 * (E[i] - ge));
    if (gf != OZMP_EXP_ZERO)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            if (F[j] != OZMP_EXP_ZERO) sf += pow2(2 * (F[j] - gf));
    se = warp_sum(se);
    sf = warp_sum(sf);
    if (lane == 0) {
        shd[0][wid] = se;
        shd[1][wid] = sf;
    }
    __syncthreads();
    const bool zero = (ge == OZMP_EXP_ZERO || gf == OZMP_EXP_ZERO || !(v > 0.0));
    const bool raw = !(ge > BOUND_RAW_EXP || ge < -BOUND_RAW_EXP || gf > BOUND_RAW_EXP || gf < -BOUND_RAW_EXP);
    __shared__ double blest;
    if (wid == 0) {
        se = warp_sum(lane < nw ? shd[0][lane] : 0.0);
        sf = warp_sum(lane < nw ? shd[1][lane] : 0.0);
        if (lane == 0) {
            bc[0] = se;
            bc[1] = sf;
            // log2 of est scaled by 4^-(GE + GF), once (binary64 is slow on this GPU)
            blest = zero ? 0.0 : log2(v) - 2.0 * (double)(ge + gf);
        }
    }
    __syncthreads();
    se = bc[0];
    sf = bc[1];
    const double lest = blest;
    // candidate s_lo + x in thread x (the binary64 logarithms are slow one after another)
    const int t = s_lo + (int)threadIdx.x;
    if (!zero && raw && t <= s_hi && bound_log2(f, t, se, sf) <= -(double)(f.target + 1) + 0.5 * lest)
        atomicMin(&best, t);
    __syncthreads();
    if (threadIdx.x != 0) return;
    st->GE = ge;
    st->GF = gf;
    st->SE = se;
    st->SF = sf;
    st->normS2 = 0.0;
    st->done = 0u;
    st->est = zero || !raw ? 0.0 : exp2(lest);
    st->s_needed = zero ? s_lo : (!raw ? -1 : best);
}

Ptrs make_ptrs(const void* const* v, int q) {
    Ptrs p;
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) p.p[c] = (c < q) ? v[c] : nullptr;
    return p;
}

}  // namespace

cudaError_t launch_bound_scale(const int32_t* E, int64_t m, const int32_t* F, int64_t n, BoundStats* st,
                               double* rowB, int64_t k, bool norms, cudaStream_t stream) {
    k_bound_scale<<<1, 1024, 0, stream>>>(E, m, F, n, st, norms ? rowB : nullptr, k);
    return cudaGetLastError();
}

cudaError_t launch_bound_choose(const void* const* A, int64_t lda, const void* const* B, int64_t ldb, int q,
                                bool is_f32, int64_t m, int64_t n, int64_t k, BoundStats* st, double* colA,
                                double* rowB, const BoundForm& f, int s_lo, int s_hi, cudaStream_t stream) {
    if (m > 0 && n > 0 && k > 0) {
        const Ptrs a = make_ptrs(A, q), b = make_ptrs(B, q);
        const unsigned gc = (unsigned)((k * 32 + 255) / 256);
        const dim3 gr((unsigned)((k + 255) / 256), (unsigned)((n + 63) / 64));
        // each element as the binary64 sum of its components: components
        // that cancel would mislead an estimate from the leading one alone
        if (is_f32) {
            k_bound_colnorm<float><<<gc, 256, 0, stream>>>(a, q, lda, m, k, st, colA);
            k_bound_rownorm<float><<<gr, 256, 0, stream>>>(b, q, ldb, k, n, st, rowB);
        } else {
            k_bound_colnorm<double><<<gc, 256, 0, stream>>>(a, q, lda, m, k, st, colA);
            k_bound_rownorm<double><<<gr, 256, 0, stream>>>(b, q, ldb, k, n, st, rowB);
        }
    }
    k_bound_choose<<<1, 1024, 0, stream>>>(st, colA, rowB, (m > 0 && n > 0) ? k : 0, f, s_lo, s_hi);
    return cudaGetLastError();
}

cudaError_t launch_bound_choose_raw(const int32_t* E, int64_t m, const int32_t* F, int64_t n, const double* colA,
                                    const double* rowB, const float* rowBf, int64_t k, BoundStats* st,
                                    const BoundForm& f, int s_lo, int s_hi, cudaStream_t stream) {
    k_bound_choose_raw<<<1, 256, 0, stream>>>(E, m, F, n, colA, rowB, rowBf, (m > 0 && n > 0) ? k : 0, st, f, s_lo,
                                               s_hi);
    return cudaGetLastError();
}

cudaError_t launch_bound_check(const void* C0, bool is_f32, int64_t m, int64_t n, int64_t ldc, BoundStats* st,
                               const BoundForm& f, int s, uint32_t* status, uint32_t flag, cudaStream_t stream) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(n < 1216 ? n : 1216);
    if (is_f32)
        k_bound_check<float><<<grid, 256, 0, stream>>>((const float*)C0, m, n, ldc, st, f, s, status, flag);
    else
        k_bound_check<double><<<grid, 256, 0, stream>>>((const double*)C0, m, n, ldc, st, f, s, status, flag);
    return cudaGetLastError();
}

}  // namespace ozmp
