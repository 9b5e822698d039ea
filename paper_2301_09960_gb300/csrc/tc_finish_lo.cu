// Rounding pass, accumulators of 2..8 words (see tc_finish.cuh).
#include "tc_finish.cuh"

namespace ozmp {

cudaError_t launch_tc_finish_lo(const GemmArgs& g, int nl, const int* ts, int rows, int slot_limbs, cudaStream_t st) {
    const dim3 fg = tc_finish_grid(g);
    switch (g.acc_words) {
        OZMP_TC_FIN_CASE(2) OZMP_TC_FIN_CASE(3) OZMP_TC_FIN_CASE(4) OZMP_TC_FIN_CASE(5)
        OZMP_TC_FIN_CASE(6) OZMP_TC_FIN_CASE(7) OZMP_TC_FIN_CASE(8)
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ozmp
