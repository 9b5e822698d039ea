// Algorithm 1 as printed (paper, Sec. 3): round-to-nearest extraction of
// binary64 slices with a per-step shift tau, the rounded remainder as the
// last slice, binary64 slice products, and the sum of the products.  It is
// kept beside the truncating-digit form so that the two can be compared in
// accuracy and slice count (the paper's D).
//
// For each operand and alpha = 1 .. D-1 (A by rows, B by columns):
//   V_s = RN64(V), V = the exact remainder (the input's components minus the
//         slices so far);
//   mu  = max |V_s| over the row (column);
//   tau = 2^(ceil(log2 mu) + c), c = ceil((53 + log2 l) / 2) (the smallest
//         c with 2^(2c - 53) >= l, l the inner dimension);
//   slice_alpha = (V_s + tau) - tau in binary64 round-to-nearest;
// and slice_D = RN64(V).  The products A_alpha B_beta (alpha + beta <= D+1)
// are binary64 GEMMs (the paper's GPU path called cuBLAS DGEMM; here they run
// on this library's own binary64 tensor-core kernel, DMMA m8n8k4); they are
// error-free except those of the rounded remainders.  The products are
// summed exactly and rounded canonically into the q output components.
#include <cstring>
#include <vector>
#include "exact_acc.cuh"
#include "kernels.h"

namespace ozmp {
namespace lit {

constexpr int QL = OZMP_MAX_COMPONENTS;
constexpr int NWR = 12;   // register window of the remainders and of the product sums (768 bits)

struct Comps {
    const double* c[QL];
    int q;
};

// V_s = RN64(a - sum_{t < nsl} slice_t) for element (i, p) of an r x l
// operand; `row` selects the reduction of mu (rows of A, columns of B).
// mu is kept as the bit pattern of |V_s| (non-negative doubles order as
// their bits).
__global__ void __launch_bounds__(256) k_rn(Comps a, int64_t lda, const double* slices, int nsl, int64_t r,
                                            int64_t l, bool by_row, double* Vs, unsigned long long* mu,
                                            uint32_t* status) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= r * l) return;
    const int64_t i = x % r, p = x / r;   // element (i, p), column-major r x l
    bool bad = false;
    double v;
    xacc::exact_round<NWR>(1, [&](auto& vis) {
        for (int c = 0; c < a.q; ++c) vis.value(a.c[c][i + p * lda]);
        for (int t = 0; t < nsl; ++t) vis.value(-slices[(size_t)t * r * l + x]);
    }, &v, bad);
    bool finite = true;
    for (int c = 0; c < a.q; ++c) {
        Comp cc;
        finite &= decode(a.c[c][i + p * lda], cc);
    }
    if (!finite) atomicOr(status, ST_NONFINITE);
    if (bad) atomicOr(status, ST_RANGE);
    Vs[x] = v;
    if (mu) atomicMax(&mu[by_row ? i : p], (unsigned long long)__double_as_longlong(fabs(v)));
}

// slice = (V_s + tau) - tau, tau = 2^(ceil(log2 mu) + c) (tau = 0 for mu = 0)
__global__ void __launch_bounds__(256) k_slice(const double* Vs, const unsigned long long* mu, int64_t r, int64_t l,
                                               bool by_row, int cshift, double* slice) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= r * l) return;
    const int64_t i = x % r, p = x / r;
    const double m = __longlong_as_double((long long)mu[by_row ? i : p]);
    double tau = 0.0;
    if (m != 0.0) {
        int e;
        const double f = frexp(m, &e);            // m = f 2^e, 0.5 <= f < 1
        const int cl = (f == 0.5) ? e - 1 : e;    // ceil(log2 m)
        tau = ldexp(1.0, cl + cshift);
    }
    slice[x] = __dsub_rn(__dadd_rn(Vs[x], tau), tau);
}

// C(i, j) = canonical q-component rounding of sum over the pairs of P_pair(i, j)
__global__ void __launch_bounds__(256) k_sum(const double* P, int npairs, int64_t m, int64_t n, Comps C_, double* const* Cw,
                                             int64_t ldc, uint32_t* status) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= m * n) return;
    const int64_t i = x % m, j = x / m;
    bool bad = false;
    double out[QL];
    xacc::exact_round<NWR>(C_.q, [&](auto& vis) {
        for (int t = 0; t < npairs; ++t) vis.value(P[(size_t)t * m * n + x]);
    }, out, bad);
    for (int c = 0; c < C_.q; ++c) Cw[c][i + j * ldc] = out[c];
    if (bad) atomicOr(status, ST_RANGE);
}

// P = X Y for column-major X (m x k, ld ldx), Y (k x n, ld ldy), P (m x n,
// ld m) in binary64 on the tensor cores (mma.sync m8n8k4 f64, fp64
// accumulation).  A 64 x 64 tile of P per block of four warps (32 x 32 each),
// k in steps of 16 through shared memory; ragged edges are zero-filled.
namespace dg {
constexpr int BM = 64, BN = 64, BK = 16, NT = 128;
constexpr int LDA = BM + 8;   // sA[kk][row]: the four k columns of a fragment fall in two bank halves
constexpr int LDB = BK + 4;   // sB[col][kk]
}

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(128) k_dgemm(const double* X, int64_t ldx, const double* Y, int64_t ldy, double* P,
                                               int64_t m, int64_t n, int64_t k) {
    using namespace dg;
    __shared__ double sA[BK * LDA];
    __shared__ double sB[BN * LDB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    double acc[16][2];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e][0] = acc[e][1] = 0.0;
    for (int64_t p0 = 0; p0 < k; p0 += BK) {
#pragma unroll
        for (int r = 0; r < BM * BK / NT; ++r) {
            const int x = tid + NT * r;
            const int row = x % BM, kk = x / BM;            // along the columns of X: coalesced
            const int64_t i = i0 + row, p = p0 + kk;
            sA[kk * LDA + row] = (i < m && p < k) ? X[i + p * ldx] : 0.0;
            const int kb = x % BK, col = x / BK;            // along the columns of Y
            const int64_t pb = p0 + kb, j = j0 + col;
            sB[col * LDB + kb] = (pb < k && j < n) ? Y[pb + j * ldy] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k4 = 0; k4 < BK / 4; ++k4) {
            double af[4], bf[4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) af[mt] = sA[(k4 * 4 + tq) * LDA + wm * 32 + mt * 8 + gq];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) bf[nt] = sB[(wn * 32 + nt * 8 + gq) * LDB + k4 * 4 + tq];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) dmma(acc[mt * 4 + nt], af[mt], bf[nt]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int64_t i = i0 + wm * 32 + mt * 8 + gq;
                const int64_t j = j0 + wn * 32 + nt * 8 + 2 * tq + v;
                if (i < m && j < n) P[i + j * m] = acc[mt * 4 + nt][v];
            }
}

struct State {
    void* buf = nullptr;
    size_t bytes = 0;
    double* cptr_dev = nullptr;   // device copy of the output pointers
};
thread_local State tl;

static unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace lit
}  // namespace ozmp

using namespace ozmp;

extern "C" ozmp_status ozmp_gemm_literal(int q, int D, int64_t m, int64_t n, int64_t k, const double* const* A,
                                         int64_t lda, const double* const* B, int64_t ldb, double* const* C,
                                         int64_t ldc, double* slices_A, double* slices_B, double* products,
                                         ozmp_stream stream) {
    if (q < 2 || q > OZMP_MAX_COMPONENTS || D < 1 || D > 32 || m < 0 || n < 0 || k < 0) return OZMP_ERR_INVALID_ARG;
    if (lda < (m > 1 ? m : 1) || ldb < (k > 1 ? k : 1) || ldc < (m > 1 ? m : 1)) return OZMP_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return OZMP_OK;
    if (!C) return OZMP_ERR_INVALID_ARG;
    for (int c = 0; c < q; ++c)
        if (!C[c] || (k > 0 && (!A || !B || !A[c] || !B[c]))) return OZMP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int npairs = D * (D + 1) / 2;
    // workspace: slices of A and B (unless supplied), V_s, mu, products (unless
    // supplied), status, output pointer table
    const size_t sa = (size_t)D * m * k, sb = (size_t)D * k * n, vs = (size_t)(m > n ? m : n) * k,
                 pr = (size_t)npairs * m * n;
    size_t need = 256;
    auto take = [&](size_t bytes) { size_t o = need; need = (need + bytes + 255) & ~(size_t)255; return o; };
    const size_t o_sa = slices_A ? 0 : take(sa * 8), o_sb = slices_B ? 0 : take(sb * 8), o_vs = take(vs * 8),
                 o_mu = take((size_t)(m > n ? m : n) * 8), o_pr = products ? 0 : take(pr * 8), o_st = take(16),
                 o_cp = take((size_t)OZMP_MAX_COMPONENTS * 8);
    if (need > lit::tl.bytes) {
        if (lit::tl.buf) { cudaStreamSynchronize(st); cudaFree(lit::tl.buf); lit::tl.buf = nullptr; lit::tl.bytes = 0; }
        if (cudaMalloc(&lit::tl.buf, need) != cudaSuccess) { cudaGetLastError(); return OZMP_ERR_NOMEM; }
        lit::tl.bytes = need;
    }
    char* w = (char*)lit::tl.buf;
    double* SA = slices_A ? slices_A : (double*)(w + o_sa);
    double* SB = slices_B ? slices_B : (double*)(w + o_sb);
    double* Vs = (double*)(w + o_vs);
    unsigned long long* mu = (unsigned long long*)(w + o_mu);
    double* P = products ? products : (double*)(w + o_pr);
    uint32_t* status = (uint32_t*)(w + o_st);
    double** Cp = (double**)(w + o_cp);
    if (cudaMemsetAsync(status, 0, 16, st) != cudaSuccess) return OZMP_ERR_CUDA;
    if (cudaMemcpyAsync(Cp, C, (size_t)q * sizeof(double*), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return OZMP_ERR_CUDA;
    const int cshift = (53 + (k > 1 ? 64 - __builtin_clzll((unsigned long long)(k - 1)) : 0) + 1) / 2;
    lit::Comps a, b, cc;
    memset(&a, 0, sizeof(a)); memset(&b, 0, sizeof(b)); memset(&cc, 0, sizeof(cc));
    a.q = b.q = cc.q = q;
    for (int c = 0; c < q; ++c) { a.c[c] = k > 0 ? A[c] : nullptr; b.c[c] = k > 0 ? B[c] : nullptr; }
    if (k > 0) {
        // slices of A (rows) and B (columns)
        for (int pass = 0; pass < 2; ++pass) {
            const bool isA = pass == 0;
            const int64_t r = isA ? m : k, l = isA ? k : n;
            double* S = isA ? SA : SB;
            const lit::Comps& op = isA ? a : b;
            const int64_t ld = isA ? lda : ldb;
            for (int al = 1; al <= D; ++al) {
                const bool last = (al == D);
                if (!last && cudaMemsetAsync(mu, 0, (size_t)(isA ? m : n) * 8, st) != cudaSuccess) return OZMP_ERR_CUDA;
                double* dst = last ? S + (size_t)(al - 1) * r * l : Vs;
                lit::k_rn<<<lit::blocks(r * l), 256, 0, st>>>(op, ld, S, al - 1, r, l, isA, dst, last ? nullptr : mu,
                                                              status);
                if (!last)
                    lit::k_slice<<<lit::blocks(r * l), 256, 0, st>>>(Vs, mu, r, l, isA, cshift,
                                                                      S + (size_t)(al - 1) * r * l);
            }
        }
        // binary64 slice products, pairs alpha + beta <= D + 1 (alpha outer)
        const dim3 grid((unsigned)((m + lit::dg::BM - 1) / lit::dg::BM), (unsigned)((n + lit::dg::BN - 1) / lit::dg::BN));
        int t = 0;
        for (int al = 1; al <= D; ++al)
            for (int be = 1; be <= D + 1 - al; ++be, ++t)
                lit::k_dgemm<<<grid, lit::dg::NT, 0, st>>>(SA + (size_t)(al - 1) * m * k, m,
                                                           SB + (size_t)(be - 1) * k * n, k, P + (size_t)t * m * n,
                                                           m, n, k);
        if (cudaGetLastError() != cudaSuccess) return OZMP_ERR_CUDA;
    } else {
        if (cudaMemsetAsync(P, 0, pr * 8, st) != cudaSuccess) return OZMP_ERR_CUDA;
    }
    lit::k_sum<<<lit::blocks(m * n), 256, 0, st>>>(P, npairs, m, n, cc, Cp, ldc, status);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return OZMP_ERR_CUDA;
    uint32_t sw = 0;
    if (cudaMemcpy(&sw, status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZMP_ERR_CUDA;
    if (sw & ST_NONFINITE) return OZMP_ERR_NONFINITE;
    if (sw & ST_RANGE) return OZMP_ERR_RANGE;
    return OZMP_OK;
}
