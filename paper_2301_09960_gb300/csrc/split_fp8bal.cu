// Digit split (K2) for the balanced radix-32 e4m3 digit form; kernels in split_impl.cuh.
#include "split_impl.cuh"

namespace ozmp {
cudaError_t launch_digits_fp8bal(const SplitArgs& g, cudaStream_t st) {
    return g.is_f32 ? digits_impl<float, OZMP_FORM_FP8_BAL>(g, st) : digits_impl<double, OZMP_FORM_FP8_BAL>(g, st);
}
}  // namespace ozmp
