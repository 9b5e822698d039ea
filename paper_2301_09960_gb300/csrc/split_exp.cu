// Exponent reduce (K1) and the split dispatcher; kernels in split_impl.cuh.
#include "split_impl.cuh"

namespace ozmp {

cudaError_t launch_digits_fp8(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_digits_fp8bal(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_digits_int8(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_digits_fp64(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_digits_fp16(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_exponents_big(const SplitArgs& g, cudaStream_t st);
cudaError_t launch_digits_big(const SplitArgs& g, cudaStream_t st);

static void init_exponents(const SplitArgs& g, cudaStream_t st) {
    int64_t mx = g.mp > g.np ? g.mp : g.np;
    if (mx == 0) mx = 1;
    k_init_exponents<<<(unsigned)((mx + 255) / 256), 256, 0, st>>>(g.E, g.mp, g.F, g.np, g.status);
}

// all_cols: reduce the column exponents here even where the one-pass column
// digit kernel would (the slice count is then chosen between the two passes)
template <typename T, int Q>
static cudaError_t exponents_impl(const SplitArgs& g, cudaStream_t st, bool all_cols) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    init_exponents(g, st);
    // short per-thread chains (16 elements a row chunk, k / split a column
    // part), so that many independent loads are in flight per SM
    if (g.m > 0 && g.k > 0) {
        int kchunk = 16;
        dim3 gr((unsigned)((g.m + 255) / 256), (unsigned)((g.k + kchunk - 1) / kchunk));
        k_exp_rows<T, Q><<<gr, 256, 0, st>>>(a, g.m, g.k, kchunk, g.E, g.status);
    }
    if (g.n > 0 && g.k > 0 && (all_cols || cols_fused_smem(g) == 0)) {   // else the column digit pass reduces them
        const int split = (int)((g.k + 1023) / 1024 < 8 ? (g.k + 1023) / 1024 : 8);
        k_exp_cols<T, Q><<<(unsigned)((g.n * split + 7) / 8), 256, 0, st>>>(b, g.k, g.n, g.F, g.status, split);
    }
    return cudaGetLastError();
}

static cudaError_t exponents(const SplitArgs& g, cudaStream_t st, bool all_cols) {
    if (g.big) {
        // more than 4 components or a window wider than the register splitter's (split_big.cu)
        init_exponents(g, st);
        return launch_exponents_big(g, st);
    }
    return g.is_f32     ? exponents_impl<float, 3>(g, st, all_cols)
           : g.q == 2   ? exponents_impl<double, 2>(g, st, all_cols)
           : g.q == 3   ? exponents_impl<double, 3>(g, st, all_cols)
                        : exponents_impl<double, 4>(g, st, all_cols);
}

cudaError_t launch_split_digits(const SplitArgs& g, cudaStream_t st) {
    // one operand at a time (parts) and the row norms (rowBf) only on the
    // 1-byte digit paths, whose launcher honours them
    const bool b1 = !g.big && (g.form == OZMP_FORM_FP8 || g.form == OZMP_FORM_FP8_MMA || g.form == OZMP_FORM_INT8);
    if ((g.parts != 0 || g.rowBf) && !b1) return cudaErrorInvalidValue;
    if (g.big) return launch_digits_big(g, st);
    if (g.form == OZMP_FORM_FP64) return launch_digits_fp64(g, st);
    if (g.form == OZMP_FORM_FP16) return launch_digits_fp16(g, st);
    if (g.form == OZMP_FORM_INT8) return launch_digits_int8(g, st);
    if (g.bal) return launch_digits_fp8bal(g, st);
    return launch_digits_fp8(g, st);   // FORM_FP8 and FORM_FP8_MMA share the e4m3 digits
}

cudaError_t launch_split_exponents(const SplitArgs& g, cudaStream_t st) { return exponents(g, st, true); }

template <typename T, int Q>
static cudaError_t exponents_norm_impl(const SplitArgs& g, double* colA, double* rowB, bool defer_cols,
                                       cudaStream_t st) {
    Operand<T> a = make_op<T>(g.A, g.q, g.lda);
    Operand<T> b = make_op<T>(g.B, g.q, g.ldb);
    init_exponents(g, st);
    if (g.m > 0 && g.k > 0) {
        dim3 gr((unsigned)((g.m + 255) / 256), (unsigned)((g.k + 15) / 16));
        k_exp_rows_norm<T, Q><<<gr, 256, 0, st>>>(a, g.m, g.k, g.E, g.status, colA);
    }
    if (g.n > 0 && g.k > 0 && !defer_cols) {
        dim3 gr((unsigned)((g.k + 255) / 256), (unsigned)((g.n + 63) / 64));
        k_exp_cols_norm<T, Q><<<gr, 256, 0, st>>>(b, g.k, g.n, g.F, g.status, rowB);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_exponents_norm(const SplitArgs& g, double* colA, double* rowB, bool* cols_deferred,
                                        cudaStream_t st) {
    if (g.big) return cudaErrorNotSupported;   // the caller takes the exponents and the norms separately
    // where the one-pass column digit kernel applies, it reduces B's exponents
    // and sums B's row norms itself (SplitArgs::rowBf), so B is read once
    const bool defer = cols_fused_smem(g) != 0 && g.n > 0 && g.k > 0;
    *cols_deferred = defer;
    return g.is_f32     ? exponents_norm_impl<float, 3>(g, colA, rowB, defer, st)
           : g.q == 2   ? exponents_norm_impl<double, 2>(g, colA, rowB, defer, st)
           : g.q == 3   ? exponents_norm_impl<double, 3>(g, colA, rowB, defer, st)
                        : exponents_norm_impl<double, 4>(g, colA, rowB, defer, st);
}

cudaError_t launch_split(const SplitArgs& g, cudaStream_t st) {
    cudaError_t e = exponents(g, st, false);
    if (e != cudaSuccess) return e;
    return launch_split_digits(g, st);
}

}  // namespace ozmp
