// LU factorisation without pivoting with the Ozaki-scheme product (paper,
// Sec. 4.6 "LU decomposition using matrix multiplication"): A = L U for q
// binary64 components (2 <= q <= 4), L unit lower, both stored in place.
//
// The paper's step is: factor A11 = L11 U11, turn A12 into U12 and A21 into
// L21, and update A22 := A22 - L21 U12 with the Ozaki product, then repeat
// on A22.  Here the same step is applied recursively (A11 is the leading half
// of the block, factored the same way down to 32 x 32), and the two panel
// transformations are triangular solves, themselves recursive, whose
// off-diagonal updates are also Ozaki products.  Every operation that is not
// an Ozaki product -- the 32 x 32 factorisations and solves, the
// subtractions C - P -- computes its exact value (integer accumulator of
// binary64 component products) and rounds it once, canonically, into q
// components; the pivots' reciprocals come from a fixed Newton sequence of
// such operations.  All O(n^3) work is in the Ozaki products on the tensor
// cores; the binary64 pipe (slow on GB300) is not used for arithmetic.
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>
#include "exact_acc.cuh"
#include "kernels.h"
#include "plan.h"

namespace ozmp {
namespace lu {

constexpr int NB = 32;      // base block
constexpr int QL = 4;       // largest component count of the LU path

struct Mat {
    double* c[QL];
    int64_t ld;
};

// number of Newton steps for q components: 53 correct bits doubled each step
__host__ __device__ constexpr int newton_steps(int q) { return q <= 1 ? 0 : (q <= 2 ? 2 : 3); }

// register window of the exact operations: 2 q + 2 words hold every term of
// the products of q-component values of similar size
template <int Q>
struct W { static constexpr int NW = 2 * Q + 2; };

// r = 1 / d to Q components: x_0 = RN(1 / d_0); x := x + x (1 - d x), each
// operation evaluated exactly and rounded canonically
template <int Q>
__device__ void recip_q(const double* d, double* r, bool& bad) {
    double x[Q], e[Q];
#pragma unroll
    for (int c = 0; c < Q; ++c) x[c] = 0.0;
    x[0] = 1.0 / d[0];
    for (int it = 0; it < newton_steps(Q); ++it) {
        xacc::exact_round<W<Q>::NW>(Q, [&](auto& v) {
            v.value(1.0);
            for (int i = 0; i < Q; ++i)
                for (int j = 0; j < Q; ++j) v.product(d[i], x[j], true);
        }, e, bad);
        double y[Q];
        xacc::exact_round<W<Q>::NW>(Q, [&](auto& v) {
            for (int i = 0; i < Q; ++i) v.value(x[i]);
            for (int i = 0; i < Q; ++i)
                for (int j = 0; j < Q; ++j) v.product(x[i], e[j], false);
        }, y, bad);
#pragma unroll
        for (int c = 0; c < Q; ++c) x[c] = y[c];
    }
#pragma unroll
    for (int c = 0; c < Q; ++c) r[c] = x[c];
}

// RN_Q(n * r) for Q-component n and r
template <int Q>
__device__ __forceinline__ void mul_round(const double* n, const double* r, double* out, bool& bad) {
    xacc::exact_round<W<Q>::NW>(Q, [&](auto& v) {
        for (int i = 0; i < Q; ++i)
            for (int j = 0; j < Q; ++j) v.product(n[i], r[j], false);
    }, out, bad);
}

// shared-memory copy of an n x n block: S[(c * NB + j) * NB + i] = component c of (i, j)
template <int Q>
__device__ __forceinline__ void stage(const Mat& A, int n, double* S) {
    for (int x = threadIdx.x; x < Q * NB * NB; x += blockDim.x) {
        const int c = x / (NB * NB), j = (x / NB) % NB, i = x % NB;
        S[x] = (i < n && j < n) ? A.c[c][i + (int64_t)j * A.ld] : 0.0;
    }
}
#define SIDX(c, i, j) (((c) * NB + (j)) * NB + (i))

// 32 x 32 (or smaller) LU in one CTA, Crout order: for k = 0 .. n-1, row k
// of U then column k of L, each entry one exact dot product rounded once
// (a warp per entry, its lanes sharing the terms);
// l_ik = RN_q(RN_q(a_ik - sum) * RN_q(1 / u_kk)).
// The numerators of column k use only finished entries (l_it, u_tk, t < k),
// so one pass computes them beside row k of U; the warp that finishes u_kk
// computes its reciprocal while the other warps go on, and every l_ik is
// then one multiplication, all in parallel.  The values are those of the
// sequential order.
// warps of the base LU: 32 (a phase of up to 63 entries in two rounds) for
// two components, 16 where the exact windows need more registers
template <int Q>
struct LuWarps { static constexpr int N = Q == 2 ? 32 : 16; };

template <int Q>
__global__ void __launch_bounds__(32 * LuWarps<Q>::N) k_base_lu(Mat A, int n, uint32_t* status) {
    constexpr int LU_WARPS = LuWarps<Q>::N;
    __shared__ double S[Q * NB * NB];
    __shared__ double R[Q];
    __shared__ int bad_any;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) bad_any = 0;
    stage<Q>(A, n, S);
    __syncthreads();
    bool bad = false;
    double out[Q];
    for (int k = 0; k < n; ++k) {
        // entries e < n - k: u_kj, j = k + e (e = 0 first: its warp then takes
        // the reciprocal); entries e >= n - k: the numerator of l_ik,
        // i = k + 1 + (e - (n - k)), stored in place of a_ik
        const int nu = n - k, ne = 2 * (n - k) - 1;
        for (int e = warp; e < ne; e += LU_WARPS) {
            const bool urow = e < nu;
            const int i = urow ? k : k + 1 + (e - nu);
            const int j = urow ? k + e : k;
            xacc::warp_exact_round<W<Q>::NW>(Q, [&](auto& v, int part) {
                if (part == 0)
                    for (int c = 0; c < Q; ++c) v.value(S[SIDX(c, i, j)]);
                for (int t = part; t < k; t += 32)
                    for (int c1 = 0; c1 < Q; ++c1)
                        for (int c2 = 0; c2 < Q; ++c2) v.product(S[SIDX(c1, i, t)], S[SIDX(c2, t, j)], true);
            }, out, bad);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < Q; ++c) S[SIDX(c, i, j)] = out[c];
                if (e == 0) {
                    if (out[0] == 0.0) bad = true;
                    else recip_q<Q>(out, R, bad);
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // column k of L: l_ik = RN_q(num_ik * r), one thread per entry
        for (int i = k + 1 + (int)threadIdx.x; i < n; i += (int)blockDim.x) {
            double num[Q], rr[Q];
#pragma unroll
            for (int c = 0; c < Q; ++c) { num[c] = S[SIDX(c, i, k)]; rr[c] = R[c]; }
            mul_round<Q>(num, rr, out, bad);
#pragma unroll
            for (int c = 0; c < Q; ++c) S[SIDX(c, i, k)] = out[c];
        }
        __syncthreads();
    }
    if (bad) atomicOr(&bad_any, 1);
    __syncthreads();
    for (int x = threadIdx.x; x < Q * NB * NB; x += blockDim.x) {
        const int c = x / (NB * NB), j = (x / NB) % NB, i = x % NB;
        if (i < n && j < n) A.c[c][i + (int64_t)j * A.ld] = S[x];
    }
    if (threadIdx.x == 0 && bad_any) atomicOr(status, ST_RANGE);
}

constexpr int TS_WARPS = 4;   // warps (right-hand sides) per CTA of the triangular-solve bases

// L X = B, L n x n unit lower (n <= 32), B n x w: one warp per column,
// x_ij = RN_q(b_ij - sum_{t<i} l_it x_tj), in place in B
template <int Q>
__global__ void __launch_bounds__(32 * TS_WARPS) k_base_trsm_ll(Mat L, Mat B, int n, int64_t w, uint32_t* status) {
    __shared__ double S[Q * NB * NB];
    __shared__ double Xs[TS_WARPS][Q * NB];
    stage<Q>(L, n, S);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * TS_WARPS + warp;
    if (j >= w) return;   // the whole warp
    double* X = Xs[warp];
    bool bad = false;
    for (int i = 0; i < n; ++i) {
        double out[Q];
        xacc::warp_exact_round<W<Q>::NW>(Q, [&](auto& v, int part) {
            if (part == 0)
                for (int c = 0; c < Q; ++c) v.value(B.c[c][i + j * B.ld]);
            for (int t = part; t < i; t += 32)
                for (int c1 = 0; c1 < Q; ++c1)
                    for (int c2 = 0; c2 < Q; ++c2) v.product(S[SIDX(c1, i, t)], X[c2 * NB + t], true);
        }, out, bad);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < Q; ++c) X[c * NB + i] = out[c];
        __syncwarp();
    }
    if (lane < n)
#pragma unroll
        for (int c = 0; c < Q; ++c) B.c[c][lane + j * B.ld] = X[c * NB + lane];
    if (bad && lane == 0) atomicOr(status, ST_RANGE);
}

// reciprocals of the diagonal of an n x n upper block into Sr[c * NB + j]
template <int Q>
__device__ __forceinline__ void diag_recips(const double* S, int n, double* Sr, bool& bad) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double d[Q], r[Q];
#pragma unroll
        for (int c = 0; c < Q; ++c) d[c] = S[SIDX(c, j, j)];
        if (d[0] == 0.0) {
            bad = true;
#pragma unroll
            for (int c = 0; c < Q; ++c) r[c] = 0.0;
        } else {
            recip_q<Q>(d, r, bad);
        }
#pragma unroll
        for (int c = 0; c < Q; ++c) Sr[c * NB + j] = r[c];
    }
}

// X U = B, U n x n upper (n <= 32), B h x n: one warp per row,
// x_ij = RN_q(RN_q(b_ij - sum_{t<j} x_it u_tj) * RN_q(1 / u_jj)), in place
template <int Q>
__global__ void __launch_bounds__(32 * TS_WARPS) k_base_trsm_ru(Mat U, Mat B, int n, int64_t h, uint32_t* status) {
    __shared__ double S[Q * NB * NB];
    __shared__ double Sr[Q * NB];
    __shared__ double Xs[TS_WARPS][Q * NB];
    stage<Q>(U, n, S);
    __syncthreads();
    bool bad = false;
    diag_recips<Q>(S, n, Sr, bad);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * TS_WARPS + warp;
    if (i < h) {   // the whole warp
        double* X = Xs[warp];
        for (int j = 0; j < n; ++j) {
            double num[Q], out[Q], rr[Q];
            xacc::warp_exact_round<W<Q>::NW>(Q, [&](auto& v, int part) {
                if (part == 0)
                    for (int c = 0; c < Q; ++c) v.value(B.c[c][i + (int64_t)j * B.ld]);
                for (int t = part; t < j; t += 32)
                    for (int c1 = 0; c1 < Q; ++c1)
                        for (int c2 = 0; c2 < Q; ++c2) v.product(X[c1 * NB + t], S[SIDX(c2, t, j)], true);
            }, num, bad);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < Q; ++c) rr[c] = Sr[c * NB + j];
                mul_round<Q>(num, rr, out, bad);
#pragma unroll
                for (int c = 0; c < Q; ++c) X[c * NB + j] = out[c];
            }
            __syncwarp();
        }
        if (lane < n)
#pragma unroll
            for (int c = 0; c < Q; ++c) B.c[c][i + (int64_t)lane * B.ld] = X[c * NB + lane];
    }
    if (bad) atomicOr(status, ST_RANGE);
}

// U X = B, U n x n upper (n <= 32), B n x w: one warp per column, back
// substitution x_ij = RN_q(RN_q(b_ij - sum_{t>i} u_it x_tj) * RN_q(1 / u_ii))
template <int Q>
__global__ void __launch_bounds__(32 * TS_WARPS) k_base_trsm_lu(Mat U, Mat B, int n, int64_t w, uint32_t* status) {
    __shared__ double S[Q * NB * NB];
    __shared__ double Sr[Q * NB];
    __shared__ double Xs[TS_WARPS][Q * NB];
    stage<Q>(U, n, S);
    __syncthreads();
    bool bad = false;
    diag_recips<Q>(S, n, Sr, bad);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * TS_WARPS + warp;
    if (j < w) {   // the whole warp
        double* X = Xs[warp];
        for (int i = n - 1; i >= 0; --i) {
            double num[Q], out[Q], rr[Q];
            xacc::warp_exact_round<W<Q>::NW>(Q, [&](auto& v, int part) {
                if (part == 0)
                    for (int c = 0; c < Q; ++c) v.value(B.c[c][i + j * B.ld]);
                for (int t = i + 1 + part; t < n; t += 32)
                    for (int c1 = 0; c1 < Q; ++c1)
                        for (int c2 = 0; c2 < Q; ++c2) v.product(S[SIDX(c1, i, t)], X[c2 * NB + t], true);
            }, num, bad);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < Q; ++c) rr[c] = Sr[c * NB + i];
                mul_round<Q>(num, rr, out, bad);
#pragma unroll
                for (int c = 0; c < Q; ++c) X[c * NB + i] = out[c];
            }
            __syncwarp();
        }
        if (lane < n)
#pragma unroll
            for (int c = 0; c < Q; ++c) B.c[c][lane + j * B.ld] = X[c * NB + lane];
    }
    if (bad) atomicOr(status, ST_RANGE);
}

// C := RN_q(C - P) elementwise, C m x n (ld C.ld), P m x n (ld P.ld)
template <int Q>
__global__ void __launch_bounds__(256) k_sub(Mat C, Mat P, int64_t m, int64_t n, uint32_t* status) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= m * n) return;
    const int64_t i = x % m, j = x / m;
    bool bad = false;
    double out[Q];
    xacc::exact_round<W<Q>::NW>(Q, [&](auto& v) {
        for (int c = 0; c < Q; ++c) {
            v.value(C.c[c][i + j * C.ld]);
            v.value(-P.c[c][i + j * P.ld]);
        }
    }, out, bad);
#pragma unroll
    for (int c = 0; c < Q; ++c) C.c[c][i + j * C.ld] = out[c];
    if (bad) atomicOr(status, ST_RANGE);
}

// ---------------------------------------------------------------------------
// host: the recursion
// ---------------------------------------------------------------------------
struct Ctx {
    int q;
    cudaStream_t st;
    uint32_t* status;                   // device word of the base kernels
    Mat P;                              // product buffer of pcap doubles per component
    int64_t pcap;
    std::map<std::tuple<int64_t, int64_t, int64_t>, ozmp_plan> plans;
    bool failed;
    bool dry;                           // walk the recursion only, recording the largest product
    int64_t need;
    // the second stream of the factorisation (its own product buffer and
    // plans): X U11 = A21 runs there beside L11 X = A12
    Ctx* side;
    cudaEvent_t ev_fork, ev_join;
};

static Mat host_sub(const Mat& M, int64_t i, int64_t j, int q) {
    Mat r;
    for (int c = 0; c < QL; ++c) r.c[c] = (c < q && M.c[c]) ? M.c[c] + i + j * M.ld : nullptr;
    r.ld = M.ld;
    return r;
}

static unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static int64_t half(int64_t n) { return ((n + NB - 1) / NB + 1) / 2 * NB; }

// C (m x n) := C - A (m x k) B (k x n), the product by the Ozaki scheme
static void gemm_sub(Ctx& x, const Mat& C, const Mat& A, const Mat& B, int64_t m, int64_t n, int64_t k) {
    if (x.failed || m == 0 || n == 0 || k == 0) return;
    if (x.dry) {
        if (m * n > x.need) x.need = m * n;
        return;
    }
    if (m * n > x.pcap) { x.failed = true; return; }   // never write past the product buffer
    auto key = std::make_tuple(m, n, k);
    ozmp_plan p;
    auto it = x.plans.find(key);
    if (it == x.plans.end()) {
        // the automatic slice count of the precision (no data-dependent choice, no check):
        // the factorisation is defined with it
        if (plan_create_internal(&p, OZMP_PREC_Q(x.q), m, n, k, OZMP_FORM_FP8_BAL, 0, x.st, false, false) != OZMP_OK) {
            x.failed = true;
            return;
        }
        x.plans[key] = p;
    } else {
        p = it->second;
    }
    Mat Pm = x.P;
    Pm.ld = m;
    if (ozmp_plan_execute(p, (const void* const*)A.c, A.ld, (const void* const*)B.c, B.ld, (void* const*)Pm.c, m) !=
        OZMP_OK) {
        x.failed = true;
        return;
    }
    switch (x.q) {
        case 2: k_sub<2><<<blocks(m * n, 256), 256, 0, x.st>>>(C, Pm, m, n, x.status); break;
        case 3: k_sub<3><<<blocks(m * n, 256), 256, 0, x.st>>>(C, Pm, m, n, x.status); break;
        default: k_sub<4><<<blocks(m * n, 256), 256, 0, x.st>>>(C, Pm, m, n, x.status); break;
    }
}

// L X = B (L m x m unit lower, B m x w), in place
static void trsm_ll(Ctx& x, const Mat& L, const Mat& B, int64_t m, int64_t w) {
    if (x.failed || m == 0 || w == 0) return;
    if (m <= NB) {
        if (!x.dry) {
            switch (x.q) {
                case 2: k_base_trsm_ll<2><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(L, B, (int)m, w, x.status); break;
                case 3: k_base_trsm_ll<3><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(L, B, (int)m, w, x.status); break;
                default: k_base_trsm_ll<4><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(L, B, (int)m, w, x.status); break;
            }
        }
        return;
    }
    const int64_t m1 = half(m);
    trsm_ll(x, L, B, m1, w);
    gemm_sub(x, host_sub(B, m1, 0, x.q), host_sub(L, m1, 0, x.q), B, m - m1, w, m1);
    trsm_ll(x, host_sub(L, m1, m1, x.q), host_sub(B, m1, 0, x.q), m - m1, w);
}

// X U = B (U m x m upper, B h x m), in place
static void trsm_ru(Ctx& x, const Mat& U, const Mat& B, int64_t m, int64_t h) {
    if (x.failed || m == 0 || h == 0) return;
    if (m <= NB) {
        if (!x.dry) {
            switch (x.q) {
                case 2: k_base_trsm_ru<2><<<blocks(h, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, h, x.status); break;
                case 3: k_base_trsm_ru<3><<<blocks(h, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, h, x.status); break;
                default: k_base_trsm_ru<4><<<blocks(h, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, h, x.status); break;
            }
        }
        return;
    }
    const int64_t m1 = half(m);
    trsm_ru(x, U, B, m1, h);
    gemm_sub(x, host_sub(B, 0, m1, x.q), B, host_sub(U, 0, m1, x.q), h, m - m1, m1);
    trsm_ru(x, host_sub(U, m1, m1, x.q), host_sub(B, 0, m1, x.q), m - m1, h);
}

// U X = B (U m x m upper, B m x w), in place
static void trsm_lu(Ctx& x, const Mat& U, const Mat& B, int64_t m, int64_t w) {
    if (x.failed || m == 0 || w == 0) return;
    if (m <= NB) {
        if (!x.dry) {
            switch (x.q) {
                case 2: k_base_trsm_lu<2><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, w, x.status); break;
                case 3: k_base_trsm_lu<3><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, w, x.status); break;
                default: k_base_trsm_lu<4><<<blocks(w, TS_WARPS), 32 * TS_WARPS, 0, x.st>>>(U, B, (int)m, w, x.status); break;
            }
        }
        return;
    }
    const int64_t m1 = half(m);
    trsm_lu(x, host_sub(U, m1, m1, x.q), host_sub(B, m1, 0, x.q), m - m1, w);
    gemm_sub(x, B, host_sub(U, 0, m1, x.q), host_sub(B, m1, 0, x.q), m1, w, m - m1);
    trsm_lu(x, U, B, m1, w);
}

static void lu_rec(Ctx& x, const Mat& A, int64_t n) {
    if (x.failed || n == 0) return;
    if (n <= NB) {
        if (!x.dry) {
            switch (x.q) {
                case 2: k_base_lu<2><<<1, 32 * LuWarps<2>::N, 0, x.st>>>(A, (int)n, x.status); break;
                case 3: k_base_lu<3><<<1, 32 * LuWarps<3>::N, 0, x.st>>>(A, (int)n, x.status); break;
                default: k_base_lu<4><<<1, 32 * LuWarps<4>::N, 0, x.st>>>(A, (int)n, x.status); break;
            }
        }
        return;
    }
    const int64_t n1 = half(n), n2 = n - n1;
    lu_rec(x, A, n1);
    // the two panel solves read only L11 / U11 and write disjoint blocks:
    // A21 on the second stream, A12 on this one, joined before the update
    Ctx& y = x.side ? *x.side : x;
    if (x.side && !x.dry) {
        if (cudaEventRecord(x.ev_fork, x.st) != cudaSuccess || cudaStreamWaitEvent(y.st, x.ev_fork, 0) != cudaSuccess) {
            x.failed = true;
            return;
        }
    }
    trsm_ru(y, A, host_sub(A, n1, 0, x.q), n1, n2);                  // A21 := A21 U11^-1 = L21
    trsm_ll(x, A, host_sub(A, 0, n1, x.q), n1, n2);                  // A12 := L11^-1 A12 = U12
    if (x.side && !x.dry) {
        if (cudaEventRecord(x.ev_join, y.st) != cudaSuccess || cudaStreamWaitEvent(x.st, x.ev_join, 0) != cudaSuccess)
            x.failed = true;
    }
    if (y.failed) x.failed = true;
    gemm_sub(x, host_sub(A, n1, n1, x.q), host_sub(A, n1, 0, x.q), host_sub(A, 0, n1, x.q), n2, n2, n1);
    lu_rec(x, host_sub(A, n1, n1, x.q), n2);
}

// buffers shared by the calls of one thread
struct State {
    int64_t pcap = 0;           // doubles per component of the product buffer
    double* P = nullptr;        // q * pcap doubles
    int64_t pcap2 = 0;          // the same for the second stream
    double* P2 = nullptr;
    uint32_t* status = nullptr;
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Ctx ctx;
    Ctx side;
};
thread_local State tl;

static void reset_ctx(Ctx& x, int q, cudaStream_t st) {
    if (x.q != q || x.st != st) {
        for (auto& kv : x.plans) ozmp_plan_destroy(kv.second);
        x.plans.clear();
    }
    x.q = q;
    x.st = st;
    x.status = tl.status;
    x.failed = false;
    x.dry = true;
    x.need = 1;
    x.side = nullptr;
}

static bool size_buffer(double*& P, int64_t& pcap, int64_t need, cudaStream_t st) {
    if (need <= pcap) return true;
    if (P) { cudaStreamSynchronize(st); cudaFree(P); P = nullptr; }
    if (cudaMalloc(&P, (size_t)QL * need * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        pcap = 0;
        return false;
    }
    pcap = need;
    return true;
}

// prepare(q, st) then a dry walk of the same recursion gives the largest
// product; allocate() then sizes the product buffer for it
// two_streams: the factorisation's panel solves of A21 go to a second
// stream (the triangular solves of ozmp_lu_solve run on one)
static ozmp_status prepare(int q, cudaStream_t st, bool two_streams) {
    if (!tl.status) {
        if (cudaMalloc(&tl.status, 16) != cudaSuccess) { cudaGetLastError(); return OZMP_ERR_NOMEM; }
    }
    reset_ctx(tl.ctx, q, st);
    if (two_streams) {
        if (!tl.st2) {
            if (cudaStreamCreateWithFlags(&tl.st2, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&tl.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&tl.ev_join, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return OZMP_ERR_CUDA;
            }
        }
        reset_ctx(tl.side, q, tl.st2);
        tl.ctx.side = &tl.side;
        tl.ctx.ev_fork = tl.ev_fork;
        tl.ctx.ev_join = tl.ev_join;
    }
    return OZMP_OK;
}

static ozmp_status allocate(cudaStream_t st) {
    Ctx& x = tl.ctx;
    x.dry = false;
    if (x.failed || (x.side && x.side->failed)) return OZMP_ERR_CUDA;
    if (!size_buffer(tl.P, tl.pcap, x.need, st)) return OZMP_ERR_NOMEM;
    for (int c = 0; c < QL; ++c) x.P.c[c] = tl.P + (size_t)c * tl.pcap;
    x.P.ld = 0;
    x.pcap = tl.pcap;
    if (x.side) {
        Ctx& y = *x.side;
        y.dry = false;
        if (!size_buffer(tl.P2, tl.pcap2, y.need, y.st)) return OZMP_ERR_NOMEM;
        for (int c = 0; c < QL; ++c) y.P.c[c] = tl.P2 + (size_t)c * tl.pcap2;
        y.P.ld = 0;
        y.pcap = tl.pcap2;
    }
    return cudaMemsetAsync(tl.status, 0, 16, st) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}

static ozmp_status finish(cudaStream_t st) {
    Ctx& x = tl.ctx;
    if (cudaGetLastError() != cudaSuccess) return OZMP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OZMP_ERR_CUDA;
    if (x.side && cudaStreamSynchronize(x.side->st) != cudaSuccess) return OZMP_ERR_CUDA;
    if (x.failed || (x.side && x.side->failed)) return OZMP_ERR_CUDA;
    uint32_t w = 0;
    if (cudaMemcpy(&w, tl.status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZMP_ERR_CUDA;
    ozmp_status worst = OZMP_OK;
    for (Ctx* c : {&x, x.side}) {
        if (!c) continue;
        for (auto& kv : c->plans) {
            ozmp_status s = OZMP_OK;
            if (ozmp_plan_get_status(kv.second, &s) != OZMP_OK) return OZMP_ERR_CUDA;
            if (s != OZMP_OK && worst == OZMP_OK) worst = s;
        }
    }
    if (w & ST_NONFINITE) return OZMP_ERR_NONFINITE;
    if (w & ST_RANGE) return OZMP_ERR_RANGE;
    return worst;
}

static bool ptrs(const void* const* v, int q) {
    if (!v) return false;
    for (int c = 0; c < q; ++c)
        if (!v[c]) return false;
    return true;
}

static Mat make(const void* const* v, int q, int64_t ld) {
    Mat M;
    for (int c = 0; c < QL; ++c) M.c[c] = c < q ? (double*)v[c] : nullptr;
    M.ld = ld;
    return M;
}

}  // namespace lu
}  // namespace ozmp

using namespace ozmp;

extern "C" ozmp_status ozmp_lu(int q, int64_t n, double* const* A, int64_t lda, ozmp_stream stream) {
    if (q < 2 || q > lu::QL || n < 0 || lda < (n > 1 ? n : 1)) return OZMP_ERR_INVALID_ARG;
    if (n == 0) return OZMP_OK;
    if (!lu::ptrs((const void* const*)A, q)) return OZMP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const lu::Mat M = lu::make((const void* const*)A, q, lda);
    ozmp_status s = lu::prepare(q, st, true);
    if (s != OZMP_OK) return s;
    lu::lu_rec(lu::tl.ctx, M, n);   // dry walk: the largest product of each stream
    s = lu::allocate(st);
    if (s != OZMP_OK) return s;
    lu::lu_rec(lu::tl.ctx, M, n);
    return lu::finish(st);
}

extern "C" ozmp_status ozmp_lu_solve(int q, int64_t n, int64_t nrhs, const double* const* LU, int64_t lda,
                                     double* const* B, int64_t ldb, ozmp_stream stream) {
    if (q < 2 || q > lu::QL || n < 0 || nrhs < 0 || lda < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1))
        return OZMP_ERR_INVALID_ARG;
    if (n == 0 || nrhs == 0) return OZMP_OK;
    if (!lu::ptrs((const void* const*)LU, q) || !lu::ptrs((const void* const*)B, q)) return OZMP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const lu::Mat L = lu::make((const void* const*)LU, q, lda);
    const lu::Mat X = lu::make((const void* const*)B, q, ldb);
    ozmp_status s = lu::prepare(q, st, false);
    if (s != OZMP_OK) return s;
    for (int pass = 0; pass < 2; ++pass) {      // dry walk, then the solve
        lu::trsm_ll(lu::tl.ctx, L, X, n, nrhs);   // L y = b
        lu::trsm_lu(lu::tl.ctx, L, X, n, nrhs);   // U x = y
        if (pass == 0) {
            s = lu::allocate(st);
            if (s != OZMP_OK) return s;
        }
    }
    return lu::finish(st);
}
