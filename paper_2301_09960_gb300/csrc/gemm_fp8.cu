// Slice products, e4m3 digits (QMMA); kernel in gemm_impl.cuh.
#include "gemm_impl.cuh"

namespace ozmp {
cudaError_t launch_gemm_fp8(const GemmArgs& g, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_b1<OZMP_FORM_FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b1::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(g.mp / b1::BM), (unsigned)(g.np / b1::BN));
    k_gemm_b1<OZMP_FORM_FP8><<<grid, b1::NT, b1::SMEM, st>>>(g);
    return cudaGetLastError();
}
}  // namespace ozmp
