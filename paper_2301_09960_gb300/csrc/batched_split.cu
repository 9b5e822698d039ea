// Split kernels of the batched products (declarations in batched_split.cuh):
// exponents and digits of every problem of a group in one launch per step,
// block b serving the problem whose block range holds b.  Each group shares
// its component type and count, so the kernels take the count at compile
// time (the per-element windows and loops shrink to it, and two binary64
// components take the three-word window of the balanced digits).
#include "batched_split.cuh"
#include "split_impl.cuh"

namespace ozmp {

template <typename T>
__device__ __forceinline__ Operand<T> bs_opA(const BSplit& s) {
    Operand<T> o;
    for (int i = 0; i < 4; ++i) o.c[i] = (const T*)s.A[i];
    o.ld = s.lda;
    o.q = s.q;
    return o;
}
template <typename T>
__device__ __forceinline__ Operand<T> bs_opB(const BSplit& s) {
    Operand<T> o;
    for (int i = 0; i < 4; ++i) o.c[i] = (const T*)s.B[i];
    o.ld = s.ldb;
    o.q = s.q;
    return o;
}

__global__ void k_b_init(const BSplit* P, const int* pre, int count) {
    const int p = find_prob(pre, count, blockIdx.x);
    const BSplit& s = P[p];
    const int64_t i = (int64_t)(blockIdx.x - pre[p]) * blockDim.x + threadIdx.x;
    if (i < s.mp) s.E[i] = OZMP_EXP_ZERO;
    if (i < s.np) s.F[i] = OZMP_EXP_ZERO;
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_b_exp_rows(const BSplit* P, const int* pre, int count, uint32_t* status) {
    const int p = find_prob(pre, count, blockIdx.x);
    const BSplit& s = P[p];
    const int lb = blockIdx.x - pre[p];
    const int nbx = (int)((s.m + 255) / 256);
    exp_rows_body<T, Q>(bs_opA<T>(s), s.m, s.k, B_EXP_KCHUNK, s.E, status, (int64_t)(lb % nbx), (int64_t)(lb / nbx));
}

template <typename T, int Q>
__global__ void __launch_bounds__(256) k_b_exp_cols(const BSplit* P, const int* pre, int count, uint32_t* status) {
    const int p = find_prob(pre, count, blockIdx.x);
    const BSplit& s = P[p];
    exp_cols_body<T, Q>(bs_opB<T>(s), s.k, s.n, s.F, status, (int64_t)(blockIdx.x - pre[p]), (int64_t)0);
}

// The digit launches cover only the tiles that hold values: rows i < m
// (tiles of 32) and values p < k (chunks of 64) of A, columns j < n and
// values p < k (quads) of B.  The batched workspace is zeroed when the plan
// is built, so the rest of the padding keeps zero digits without being
// written.
template <typename T, int NW, int FORM, int Q>
__global__ void __launch_bounds__(256) k_b_split_rows(const BSplit* P, const int* pre, int count) {
    const int p = find_prob(pre, count, blockIdx.x);
    const BSplit& s = P[p];
    const int lb = blockIdx.x - pre[p];
    const int nbx = (int)((s.m + 31) / 32);
    split_rows_b1_body<T, FORM, NW, Q>(bs_opA<T>(s), s.m, s.k, s.E, s.Adig, s.mp, s.kp, s.s,
                                       (int64_t)(lb % nbx), (int64_t)(lb / nbx));
}

template <typename T, int NW, int FORM, int Q>
__global__ void __launch_bounds__(256) k_b_split_cols(const BSplit* P, const int* pre, int count) {
    const int p = find_prob(pre, count, blockIdx.x);
    const BSplit& s = P[p];
    split_cols_b1_body<T, FORM, NW, Q>(bs_opB<T>(s), s.k, s.n, s.F, s.Bdig, s.np, s.kp, s.s,
                                       (int64_t)(blockIdx.x - pre[p]), (int64_t)0, (s.k + 3) / 4);
}

template <typename T, int NW, int FORM, int Q>
static cudaError_t set_smem_t(size_t sm) {
    return cudaFuncSetAttribute(k_b_split_rows<T, NW, FORM, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename T, int NW, int FORM, int Q>
static cudaError_t launch_t(const BSplitGroup& g, cudaStream_t cs, cudaStream_t cs_b, cudaEvent_t ev_init) {
    k_b_init<<<g.blocks[0], 256, 0, cs>>>(g.sp, g.pre[0], g.count);
    if (cs_b != cs) {
        cudaError_t e = cudaEventRecord(ev_init, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs_b, ev_init, 0);
        if (e != cudaSuccess) return e;
    }
    k_b_exp_rows<T, Q><<<g.blocks[1], 256, 0, cs>>>(g.sp, g.pre[1], g.count, g.status);
    k_b_split_rows<T, NW, FORM, Q><<<g.blocks[3], 256, g.smem, cs>>>(g.sp, g.pre[3], g.count);
    k_b_exp_cols<T, Q><<<g.blocks[2], 256, 0, cs_b>>>(g.sp, g.pre[2], g.count, g.status);
    k_b_split_cols<T, NW, FORM, Q><<<g.blocks[4], 256, 0, cs_b>>>(g.sp, g.pre[4], g.count);
    return cudaGetLastError();
}


struct Streams {
    cudaStream_t a, b;
    cudaEvent_t ev;
};

template <typename T, int NW, int FORM, int Q>
static cudaError_t one(const BSplitGroup& g, const Streams* st) {
    return st ? launch_t<T, NW, FORM, Q>(g, st->a, st->b, st->ev) : set_smem_t<T, NW, FORM, Q>(g.smem);
}

template <typename T, int Q>
static cudaError_t by_form(const BSplitGroup& g, const Streams* st) {
    if (g.bal) return g.nw == 4 ? one<T, 4, OZMP_FORM_FP8_BAL, Q>(g, st) : one<T, 6, OZMP_FORM_FP8_BAL, Q>(g, st);
    return g.nw == 4 ? one<T, 4, OZMP_FORM_FP8, Q>(g, st) : one<T, 6, OZMP_FORM_FP8, Q>(g, st);
}

// st == nullptr: raise the shared-memory limit only
static cudaError_t dispatch(const BSplitGroup& g, const Streams* st) {
    if (g.is_f32) return by_form<float, 3>(g, st);
    if (g.q == 2) return by_form<double, 2>(g, st);
    if (g.q == 3) return by_form<double, 3>(g, st);
    return by_form<double, 4>(g, st);
}

cudaError_t bsplit_set_smem(const BSplitGroup& g) { return dispatch(g, nullptr); }
cudaError_t bsplit_launch(const BSplitGroup& g, cudaStream_t cs, cudaStream_t cs_b, cudaEvent_t ev_init) {
    const Streams st = {cs, cs_b, ev_init};
    return dispatch(g, &st);
}

}  // namespace ozmp
