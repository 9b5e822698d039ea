// Digit split (K2) for the binary16-digit form; kernels in split_impl.cuh.
#include "split_impl.cuh"

namespace ozmp {
cudaError_t launch_digits_fp16(const SplitArgs& g, cudaStream_t st) {
    return g.is_f32 ? digits_impl<float, OZMP_FORM_FP16>(g, st) : digits_impl<double, OZMP_FORM_FP16>(g, st);
}
}  // namespace ozmp
