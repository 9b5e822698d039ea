// The rounding pass of the single-problem tcgen05 path (kernel template),
// instantiated by tc_finish_lo.cu (2..8 accumulator words) and
// tc_finish_hi.cu (9..16) so that the two compile in parallel.
#pragma once
#include "gemm_tc_impl.cuh"

namespace ozmp {
namespace tc {

// Rounding pass of the single-problem path: one thread per element of C
// normalises the element's carry-save limbs 0 .. nl-1 (from its tile's split
// slot when the tile was split into chunks, else from acc) and rounds them
// canonically into the q components.  Bound by the limb reads.
template <int NW>
__global__ void __launch_bounds__(256) k_tc_finish(const GemmArgs g, int nl, const int* tile_slot, int tile_rows,
                                                   int slot_limbs) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= g.m) return;
    const size_t sstride = (size_t)BN * BM;
    for (int64_t j = blockIdx.y; j < g.n; j += gridDim.y) {
        const int slot =
            tile_slot ? tile_slot[(i / tile_rows) + (j / BN) * (g.mp / tile_rows)] : -1;
        if (slot < 0) {
            finish_element<NW>(g, nl, g.acc, (size_t)g.mp * g.np, (size_t)j * g.mp + i, i, j, 0, 0, false);
        } else {
            const int cta = slot * (tile_rows / BM) + (int)((i % tile_rows) / BM);
            finish_element<NW>(g, nl, g.sacc + (size_t)cta * slot_limbs * sstride, sstride,
                               (size_t)(j % BN) * BM + (size_t)(i % BM), i, j, 0, 0, false);
        }
    }
}

}  // namespace tc

#define OZMP_TC_FIN_CASE(NWV) \
    case NWV: tc::k_tc_finish<NWV><<<fg, 256, 0, st>>>(g, nl, ts, rows, slot_limbs); break;

inline dim3 tc_finish_grid(const GemmArgs& g) {
    return dim3((unsigned)((g.m + 255) / 256), (unsigned)(g.n < 65535 ? g.n : 65535));
}

}  // namespace ozmp
