// Slice products, binary64 digits (DMMA), and the product dispatcher.
#include "gemm_impl.cuh"

namespace ozmp {
cudaError_t launch_gemm_fp8(const GemmArgs& g, cudaStream_t st);
cudaError_t launch_gemm_int8(const GemmArgs& g, cudaStream_t st);
cudaError_t launch_gemm_tc(const GemmArgs& g, cudaStream_t st);

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t st) {
    if (g.mp == 0 || g.np == 0) return cudaSuccess;
    if (g.form == OZMP_FORM_FP8 || g.form == OZMP_FORM_FP16)
        return launch_gemm_tc(g, st);   // records the timing pair itself
    if (g.tev_start) cudaEventRecord(g.tev_start, st);
    cudaError_t e;
    if (g.form == OZMP_FORM_INT8) {
        e = launch_gemm_int8(g, st);
    } else if (g.form == OZMP_FORM_FP8_MMA) {
        e = launch_gemm_fp8(g, st);
    } else {
        e = cudaFuncSetAttribute(k_gemm_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64::SMEM);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)(g.mp / f64::BM), (unsigned)(g.np / f64::BN));
        k_gemm_f64<<<grid, f64::NT, f64::SMEM, st>>>(g);
        e = cudaGetLastError();
    }
    if (g.tev_stop) cudaEventRecord(g.tev_stop, st);
    return e;
}
}  // namespace ozmp
