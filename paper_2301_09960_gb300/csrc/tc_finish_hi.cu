// Rounding pass, accumulators of 9..16 words (see tc_finish.cuh).
#include "tc_finish.cuh"

namespace ozmp {

cudaError_t launch_tc_finish_hi(const GemmArgs& g, int nl, const int* ts, int rows, int slot_limbs, cudaStream_t st) {
    const dim3 fg = tc_finish_grid(g);
    switch (g.acc_words) {
        OZMP_TC_FIN_CASE(9) OZMP_TC_FIN_CASE(10) OZMP_TC_FIN_CASE(11) OZMP_TC_FIN_CASE(12)
        OZMP_TC_FIN_CASE(13) OZMP_TC_FIN_CASE(14) OZMP_TC_FIN_CASE(15) OZMP_TC_FIN_CASE(16)
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ozmp
