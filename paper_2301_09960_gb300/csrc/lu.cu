// LU factorisation without pivoting with the Ozaki-scheme product (paper,
// Sec. 5 "LU decomposition using matrix multiplication"): A = L U for q
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

using xacc::Acc;
constexpr int NB = 32;      // base block
constexpr int QL = 4;       // largest component count of the LU path

struct Mat {
    double* c[QL];
    int64_t ld;
};

// number of Newton steps for q components: 53 correct bits doubled each step
__host__ __device__ constexpr int newton_steps(int q) { return q <= 1 ? 0 : (q <= 2 ? 2 : 3); }

// r = 1 / d to q components: x_0 = RN(1 / d_0); x := x + x (1 - d x), each
// operation evaluated exactly and rounded canonically
__device__ void recip_q(const double* d, int q, double* r, bool& bad) {
    double x[QL] = {0, 0, 0, 0}, e[QL] = {0, 0, 0, 0};
    x[0] = 1.0 / d[0];
    Acc a;
    for (int it = 0; it < newton_steps(q); ++it) {
        xacc::clear(a);
        xacc::add_value(a, 1.0);
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) xacc::add_product(a, d[i], x[j], true);
        bad |= a.range_bad;
        xacc::round_q(a, q, e);
        bad |= a.range_bad;
        xacc::clear(a);
        for (int i = 0; i < q; ++i) xacc::add_value(a, x[i]);
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) xacc::add_product(a, x[i], e[j], false);
        bad |= a.range_bad;
        xacc::round_q(a, q, x);
        bad |= a.range_bad;
    }
    for (int i = 0; i < q; ++i) r[i] = x[i];
}

// a += sum_{t} sign * X[t] Y[t] for q-component values (component-major)
__device__ __forceinline__ void dot_into(Acc& a, const double* xs, int xstride, const double* ys, int ystride,
                                         int cstride_x, int cstride_y, int len, int q) {
    for (int t = 0; t < len; ++t)
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j)
                xacc::add_product(a, xs[t * xstride + i * cstride_x], ys[t * ystride + j * cstride_y], true);
}

// shared-memory copy of an n x n block: S[(c * NB + j) * NB + i] = component c of (i, j)
__device__ __forceinline__ void stage(const Mat& A, int n, int q, double* S) {
    for (int x = threadIdx.x; x < q * NB * NB; x += blockDim.x) {
        const int c = x / (NB * NB), j = (x / NB) % NB, i = x % NB;
        S[x] = (i < n && j < n) ? A.c[c][i + (int64_t)j * A.ld] : 0.0;
    }
}

// 32 x 32 (or smaller) LU in one CTA, Crout order: for k = 0 .. n-1, row k
// of U then column k of L, each entry one exact dot product rounded once;
// l_ik = RN_q(RN_q(a_ik - sum) * RN_q(1 / u_kk)).
__global__ void __launch_bounds__(64) k_base_lu(Mat A, int n, int q, uint32_t* status) {
    __shared__ double S[QL * NB * NB];
    __shared__ double R[QL];
    __shared__ int bad_any;
    if (threadIdx.x == 0) bad_any = 0;
    stage(A, n, q, S);
    __syncthreads();
    bool bad = false;
    Acc a;
    double out[QL];
    for (int k = 0; k < n; ++k) {
        // row k of U: u_kj = a_kj - sum_{t<k} l_kt u_tj, j = k .. n-1
        for (int j = k + (int)threadIdx.x; j < n; j += blockDim.x) {
            xacc::clear(a);
            for (int c = 0; c < q; ++c) xacc::add_value(a, S[(c * NB + j) * NB + k]);
            dot_into(a, &S[k], NB, &S[j * NB], 1, NB * NB, NB * NB, k, q);
            bad |= a.range_bad;
            xacc::round_q(a, q, out);
            bad |= a.range_bad;
            for (int c = 0; c < q; ++c) S[(c * NB + j) * NB + k] = out[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double d[QL];
            for (int c = 0; c < q; ++c) d[c] = S[(c * NB + k) * NB + k];
            if (d[0] == 0.0) bad = true;
            else recip_q(d, q, R, bad);
        }
        __syncthreads();
        // column k of L: l_ik = (a_ik - sum_{t<k} l_it u_tk) / u_kk, i = k+1 .. n-1
        for (int i = k + 1 + (int)threadIdx.x; i < n; i += blockDim.x) {
            xacc::clear(a);
            for (int c = 0; c < q; ++c) xacc::add_value(a, S[(c * NB + k) * NB + i]);
            dot_into(a, &S[i], NB, &S[k * NB], 1, NB * NB, NB * NB, k, q);
            bad |= a.range_bad;
            double num[QL];
            xacc::round_q(a, q, num);
            xacc::clear(a);
            for (int c1 = 0; c1 < q; ++c1)
                for (int c2 = 0; c2 < q; ++c2) xacc::add_product(a, num[c1], R[c2], false);
            bad |= a.range_bad;
            xacc::round_q(a, q, out);
            bad |= a.range_bad;
            for (int c = 0; c < q; ++c) S[(c * NB + k) * NB + i] = out[c];
        }
        __syncthreads();
    }
    if (bad) atomicOr(&bad_any, 1);
    __syncthreads();
    for (int x = threadIdx.x; x < q * NB * NB; x += blockDim.x) {
        const int c = x / (NB * NB), j = (x / NB) % NB, i = x % NB;
        if (i < n && j < n) A.c[c][i + (int64_t)j * A.ld] = S[x];
    }
    if (threadIdx.x == 0 && bad_any) atomicOr(status, ST_RANGE);
}

// L X = B, L n x n unit lower (n <= 32), B n x w: one thread per column,
// x_ij = RN_q(b_ij - sum_{t<i} l_it x_tj), in place in B
__global__ void __launch_bounds__(128) k_base_trsm_ll(Mat L, Mat B, int n, int64_t w, int q, uint32_t* status) {
    __shared__ double S[QL * NB * NB];
    stage(L, n, q, S);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= w) return;
    bool bad = false;
    Acc a;
    double out[QL];
    double X[QL * NB];   // column j of the solution, [c][i]
    for (int i = 0; i < n; ++i) {
        xacc::clear(a);
        for (int c = 0; c < q; ++c) xacc::add_value(a, B.c[c][i + j * B.ld]);
        for (int t = 0; t < i; ++t)
            for (int c1 = 0; c1 < q; ++c1)
                for (int c2 = 0; c2 < q; ++c2)
                    xacc::add_product(a, S[(c1 * NB + t) * NB + i], X[c2 * NB + t], true);
        bad |= a.range_bad;
        xacc::round_q(a, q, out);
        bad |= a.range_bad;
        for (int c = 0; c < q; ++c) X[c * NB + i] = out[c];
    }
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < q; ++c) B.c[c][i + j * B.ld] = X[c * NB + i];
    if (bad) atomicOr(status, ST_RANGE);
}

// reciprocals of the diagonal of an n x n upper block into S_r[c * NB + j]
__device__ __forceinline__ void diag_recips(const double* S, int n, int q, double* Sr, bool& bad) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double d[QL], r[QL];
        for (int c = 0; c < q; ++c) d[c] = S[(c * NB + j) * NB + j];
        if (d[0] == 0.0) { bad = true; for (int c = 0; c < q; ++c) r[c] = 0.0; }
        else recip_q(d, q, r, bad);
        for (int c = 0; c < q; ++c) Sr[c * NB + j] = r[c];
    }
}

// X U = B, U n x n upper (n <= 32), B h x n: one thread per row,
// x_ij = RN_q(RN_q(b_ij - sum_{t<j} x_it u_tj) * RN_q(1 / u_jj)), in place
__global__ void __launch_bounds__(128) k_base_trsm_ru(Mat U, Mat B, int n, int64_t h, int q, uint32_t* status) {
    __shared__ double S[QL * NB * NB];
    __shared__ double Sr[QL * NB];
    stage(U, n, q, S);
    __syncthreads();
    bool bad = false;
    diag_recips(S, n, q, Sr, bad);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < h) {
        Acc a;
        double out[QL], num[QL];
        double X[QL * NB];   // row i of the solution, [c][j]
        for (int j = 0; j < n; ++j) {
            xacc::clear(a);
            for (int c = 0; c < q; ++c) xacc::add_value(a, B.c[c][i + (int64_t)j * B.ld]);
            for (int t = 0; t < j; ++t)
                for (int c1 = 0; c1 < q; ++c1)
                    for (int c2 = 0; c2 < q; ++c2)
                        xacc::add_product(a, X[c1 * NB + t], S[(c2 * NB + j) * NB + t], true);
            bad |= a.range_bad;
            xacc::round_q(a, q, num);
            xacc::clear(a);
            for (int c1 = 0; c1 < q; ++c1)
                for (int c2 = 0; c2 < q; ++c2) xacc::add_product(a, num[c1], Sr[c2 * NB + j], false);
            bad |= a.range_bad;
            xacc::round_q(a, q, out);
            bad |= a.range_bad;
            for (int c = 0; c < q; ++c) X[c * NB + j] = out[c];
        }
        for (int j = 0; j < n; ++j)
            for (int c = 0; c < q; ++c) B.c[c][i + (int64_t)j * B.ld] = X[c * NB + j];
    }
    if (bad) atomicOr(status, ST_RANGE);
}

// U X = B, U n x n upper (n <= 32), B n x w: one thread per column, back
// substitution x_ij = RN_q(RN_q(b_ij - sum_{t>i} u_it x_tj) * RN_q(1 / u_ii))
__global__ void __launch_bounds__(128) k_base_trsm_lu(Mat U, Mat B, int n, int64_t w, int q, uint32_t* status) {
    __shared__ double S[QL * NB * NB];
    __shared__ double Sr[QL * NB];
    stage(U, n, q, S);
    __syncthreads();
    bool bad = false;
    diag_recips(S, n, q, Sr, bad);
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < w) {
        Acc a;
        double out[QL], num[QL];
        double X[QL * NB];
        for (int i = n - 1; i >= 0; --i) {
            xacc::clear(a);
            for (int c = 0; c < q; ++c) xacc::add_value(a, B.c[c][i + j * B.ld]);
            for (int t = i + 1; t < n; ++t)
                for (int c1 = 0; c1 < q; ++c1)
                    for (int c2 = 0; c2 < q; ++c2)
                        xacc::add_product(a, S[(c1 * NB + t) * NB + i], X[c2 * NB + t], true);
            bad |= a.range_bad;
            xacc::round_q(a, q, num);
            xacc::clear(a);
            for (int c1 = 0; c1 < q; ++c1)
                for (int c2 = 0; c2 < q; ++c2) xacc::add_product(a, num[c1], Sr[c2 * NB + i], false);
            bad |= a.range_bad;
            xacc::round_q(a, q, out);
            bad |= a.range_bad;
            for (int c = 0; c < q; ++c) X[c * NB + i] = out[c];
        }
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < q; ++c) B.c[c][i + j * B.ld] = X[c * NB + i];
    }
    if (bad) atomicOr(status, ST_RANGE);
}

// C := RN_q(C - P) elementwise, C m x n (ld C.ld), P m x n (ld P.ld)
__global__ void __launch_bounds__(256) k_sub(Mat C, Mat P, int64_t m, int64_t n, int q, uint32_t* status) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= m * n) return;
    const int64_t i = x % m, j = x / m;
    Acc a;
    xacc::clear(a);
    for (int c = 0; c < q; ++c) {
        xacc::add_value(a, C.c[c][i + j * C.ld]);
        xacc::add_value(a, -P.c[c][i + j * P.ld]);
    }
    double out[QL];
    xacc::round_q(a, q, out);
    for (int c = 0; c < q; ++c) C.c[c][i + j * C.ld] = out[c];
    if (a.range_bad) atomicOr(status, ST_RANGE);
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
        if (ozmp_plan_create(&p, OZMP_PREC_Q(x.q), m, n, k, OZMP_FORM_FP8, 0, x.st) != OZMP_OK) { x.failed = true; return; }
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
    k_sub<<<blocks(m * n, 256), 256, 0, x.st>>>(C, Pm, m, n, x.q, x.status);
}

// L X = B (L m x m unit lower, B m x w), in place
static void trsm_ll(Ctx& x, const Mat& L, const Mat& B, int64_t m, int64_t w) {
    if (x.failed || m == 0 || w == 0) return;
    if (m <= NB) {
        if (!x.dry) k_base_trsm_ll<<<blocks(w, 128), 128, 0, x.st>>>(L, B, (int)m, w, x.q, x.status);
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
        if (!x.dry) k_base_trsm_ru<<<blocks(h, 128), 128, 0, x.st>>>(U, B, (int)m, h, x.q, x.status);
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
        if (!x.dry) k_base_trsm_lu<<<blocks(w, 128), 128, 0, x.st>>>(U, B, (int)m, w, x.q, x.status);
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
        if (!x.dry) k_base_lu<<<1, 64, 0, x.st>>>(A, (int)n, x.q, x.status);
        return;
    }
    const int64_t n1 = half(n), n2 = n - n1;
    lu_rec(x, A, n1);
    trsm_ll(x, A, host_sub(A, 0, n1, x.q), n1, n2);                  // A12 := L11^-1 A12 = U12
    trsm_ru(x, A, host_sub(A, n1, 0, x.q), n1, n2);                  // A21 := A21 U11^-1 = L21
    gemm_sub(x, host_sub(A, n1, n1, x.q), host_sub(A, n1, 0, x.q), host_sub(A, 0, n1, x.q), n2, n2, n1);
    lu_rec(x, host_sub(A, n1, n1, x.q), n2);
}

// buffers shared by the calls of one thread
struct State {
    int64_t pcap = 0;           // doubles per component of the product buffer
    double* P = nullptr;        // q * pcap doubles
    uint32_t* status = nullptr;
    Ctx ctx;
};
thread_local State tl;

// prepare(q, st) then a dry walk of the same recursion gives the largest
// product; allocate() then sizes the product buffer for it
static ozmp_status prepare(int q, cudaStream_t st) {
    if (!tl.status) {
        if (cudaMalloc(&tl.status, 16) != cudaSuccess) { cudaGetLastError(); return OZMP_ERR_NOMEM; }
    }
    Ctx& x = tl.ctx;
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
    return OZMP_OK;
}

static ozmp_status allocate(cudaStream_t st) {
    Ctx& x = tl.ctx;
    x.dry = false;
    if (x.failed) return OZMP_ERR_CUDA;
    if (x.need > tl.pcap) {
        if (tl.P) { cudaStreamSynchronize(st); cudaFree(tl.P); tl.P = nullptr; }
        if (cudaMalloc(&tl.P, (size_t)QL * x.need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            tl.pcap = 0;
            return OZMP_ERR_NOMEM;
        }
        tl.pcap = x.need;
    }
    for (int c = 0; c < QL; ++c) x.P.c[c] = tl.P + (size_t)c * tl.pcap;
    x.P.ld = 0;
    x.pcap = tl.pcap;
    return cudaMemsetAsync(tl.status, 0, 16, st) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}

static ozmp_status finish(cudaStream_t st) {
    Ctx& x = tl.ctx;
    if (cudaGetLastError() != cudaSuccess) return OZMP_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OZMP_ERR_CUDA;
    if (x.failed) return OZMP_ERR_CUDA;
    uint32_t w = 0;
    if (cudaMemcpy(&w, tl.status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZMP_ERR_CUDA;
    ozmp_status worst = OZMP_OK;
    for (auto& kv : x.plans) {
        ozmp_status s = OZMP_OK;
        if (ozmp_plan_get_status(kv.second, &s) != OZMP_OK) return OZMP_ERR_CUDA;
        if (s != OZMP_OK && worst == OZMP_OK) worst = s;
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
    ozmp_status s = lu::prepare(q, st);
    if (s != OZMP_OK) return s;
    lu::lu_rec(lu::tl.ctx, M, n);   // dry walk: the largest product
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
    ozmp_status s = lu::prepare(q, st);
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
