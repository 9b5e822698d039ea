// The "simple matrix multiplication" baseline of Sec. 4: the triple loop in
// multi-component arithmetic (DD / TD / QD in binary64 words, TS in binary32
// words), on the GPU with shared-memory tiles (the paper's GPU comparison runs
// a simple TS/DD GEMM with and without shared memory, Sec. 4.4).
//
// Arithmetic: each product a_i * b_j of components is split exactly with
// TwoProd (fma), the terms of one multiply-add are added into the q-word
// accumulator with TwoSum chains, and the accumulator is renormalised after
// every multiply-add (a bottom-up TwoSum pass and a top-down FastTwoSum pass).
// This is not an Ozaki-scheme product; it is the yardstick the paper compares
// the scheme against.
#include <cstring>
#include "kernels.h"
#include "ozmp_internal.cuh"
#include "plan.h"

namespace ozmp {
namespace naive {

template <typename T> __device__ __forceinline__ T fma_(T a, T b, T c);
template <> __device__ __forceinline__ double fma_<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float fma_<float>(float a, float b, float c) { return fmaf(a, b, c); }

// s + e = a + b exactly
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b|
template <typename T>
__device__ __forceinline__ void fast_two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    e = b - (s - a);
}
// p + e = a * b exactly
template <typename T>
__device__ __forceinline__ void two_prod(T a, T b, T& p, T& e) {
    p = a * b;
    e = fma_<T>(a, b, -p);
}

template <int Q, typename T>
__device__ __forceinline__ void add_term(T (&x)[Q], T t) {
    T e = t;
#pragma unroll
    for (int l = 0; l < Q; ++l) two_sum<T>(x[l], e, x[l], e);
}

template <int Q, typename T>
__device__ __forceinline__ void renorm(T (&x)[Q]) {
#pragma unroll
    for (int l = Q - 1; l > 0; --l) two_sum<T>(x[l - 1], x[l], x[l - 1], x[l]);
#pragma unroll
    for (int l = 0; l < Q - 1; ++l) fast_two_sum<T>(x[l], x[l + 1], x[l], x[l + 1]);
}

// acc += a * b (q-word operands)
template <int Q, typename T>
__device__ __forceinline__ void mul_add(T (&acc)[Q], const T (&a)[Q], const T (&b)[Q]) {
    // terms of weight level i + j < Q, with the TwoProd error one level lower
#pragma unroll
    for (int lvl = Q - 1; lvl >= 0; --lvl) {
#pragma unroll
        for (int i = 0; i <= lvl; ++i) {
            const int j = lvl - i;
            T p, e;
            two_prod<T>(a[i], b[j], p, e);
            if (lvl + 1 < Q) add_term<Q, T>(acc, e);
            add_term<Q, T>(acc, p);
        }
    }
    renorm<Q, T>(acc);
}

constexpr int TB = 16;   // 16 x 16 threads, one element each; 16-wide k tiles in shared memory

template <int Q, typename T>
struct Ptrs {
    const T* a[Q];
    const T* b[Q];
    T* c[Q];
};

template <int Q, typename T>
__global__ void __launch_bounds__(TB * TB) k_naive(int64_t m, int64_t n, int64_t k, const Ptrs<Q, T> P,
                                                    int64_t lda, int64_t ldb, int64_t ldc) {
    __shared__ T sa[Q][TB][TB + 1];
    __shared__ T sb[Q][TB][TB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t i = (int64_t)blockIdx.x * TB + tx;
    const int64_t j = (int64_t)blockIdx.y * TB + ty;
    T acc[Q];
#pragma unroll
    for (int c = 0; c < Q; ++c) acc[c] = (T)0;
    for (int64_t p0 = 0; p0 < k; p0 += TB) {
        // A tile: rows i (tx), columns p0 + ty; B tile: rows p0 + tx, columns j (ty)
        const int64_t ia = (int64_t)blockIdx.x * TB + tx, pa = p0 + ty;
        const int64_t pb = p0 + tx, jb = (int64_t)blockIdx.y * TB + ty;
#pragma unroll
        for (int c = 0; c < Q; ++c) {
            sa[c][ty][tx] = (ia < m && pa < k) ? P.a[c][ia + pa * lda] : (T)0;
            sb[c][ty][tx] = (pb < k && jb < n) ? P.b[c][pb + jb * ldb] : (T)0;
        }
        __syncthreads();
        const int kk = (int)((k - p0) < TB ? (k - p0) : TB);
        for (int p = 0; p < kk; ++p) {
            T a[Q], b[Q];
#pragma unroll
            for (int c = 0; c < Q; ++c) { a[c] = sa[c][p][tx]; b[c] = sb[c][ty][p]; }
            mul_add<Q, T>(acc, a, b);
        }
        __syncthreads();
    }
    if (i < m && j < n) {
#pragma unroll
        for (int c = 0; c < Q; ++c) P.c[c][i + j * ldc] = acc[c];
    }
}

template <int Q, typename T>
cudaError_t run(int64_t m, int64_t n, int64_t k, const void* const* A, int64_t lda, const void* const* B,
                int64_t ldb, void* const* C, int64_t ldc, cudaStream_t st) {
    Ptrs<Q, T> P;
    for (int c = 0; c < Q; ++c) {
        P.a[c] = (const T*)A[c];
        P.b[c] = (const T*)B[c];
        P.c[c] = (T*)C[c];
    }
    dim3 grid((unsigned)((m + TB - 1) / TB), (unsigned)((n + TB - 1) / TB));
    k_naive<Q, T><<<grid, dim3(TB, TB), 0, st>>>(m, n, k, P, lda, ldb, ldc);
    return cudaGetLastError();
}

}  // namespace naive
}  // namespace ozmp

using namespace ozmp_plan_detail;

extern "C" ozmp_status ozmp_gemm_naive(ozmp_prec prec, int64_t m, int64_t n, int64_t k, const void* const* A,
                                       int64_t lda, const void* const* B, int64_t ldb, void* const* C, int64_t ldc,
                                       ozmp_stream stream) {
    const int q = prec_q(prec);
    if (!q || m < 0 || n < 0 || k < 0) return OZMP_ERR_INVALID_ARG;
    if (lda < (m > 1 ? m : 1) || ldb < (k > 1 ? k : 1) || ldc < (m > 1 ? m : 1)) return OZMP_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return OZMP_OK;
    if (!ptrs_ok(C, q) || (k > 0 && (!ptrs_ok(A, q) || !ptrs_ok(B, q)))) return OZMP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const void* none[4] = {C[0], C[0], C[0], C[0]};   // k = 0: the loop never reads A or B
    const void* const* a = k > 0 ? A : none;
    const void* const* b = k > 0 ? B : none;
    cudaError_t e;
    switch (prec) {
        case OZMP_DD: e = ozmp::naive::run<2, double>(m, n, k, a, lda, b, ldb, C, ldc, st); break;
        case OZMP_TD: e = ozmp::naive::run<3, double>(m, n, k, a, lda, b, ldb, C, ldc, st); break;
        case OZMP_QD: e = ozmp::naive::run<4, double>(m, n, k, a, lda, b, ldb, C, ldc, st); break;
        default: e = ozmp::naive::run<3, float>(m, n, k, a, lda, b, ldb, C, ldc, st); break;
    }
    return e == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}
