// Slice products, binary64 digits (DMMA), and the product dispatcher.
#include "gemm_impl.cuh"

namespace ozmp {
cudaError_t launch_gemm_fp8(const GemmArgs& g, cudaStream_t st);
cudaError_t launch_gemm_int8(const GemmArgs& g, cudaStream_t st);
cudaError_t launch_gemm_tc(const GemmArgs& g, cudaStream_t st);

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t st) {
    if (g.mp == 0 || g.np == 0) return cudaSuccess;
    if (g.form == OZMP_FORM_INT8) return launch_gemm_int8(g, st);
    if (g.form == OZMP_FORM_FP8) return launch_gemm_tc(g, st);
    if (g.form == OZMP_FORM_FP8_MMA) return launch_gemm_fp8(g, st);
    cudaError_t e = cudaFuncSetAttribute(k_gemm_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f64::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(g.mp / f64::BM), (unsigned)(g.np / f64::BN));
    k_gemm_f64<<<grid, f64::NT, f64::SMEM, st>>>(g);
    return cudaGetLastError();
}
}  // namespace ozmp
