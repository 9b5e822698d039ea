// The rounding pass of the single-problem tcgen05 path (kernel template),
// instantiated by tc_finish_lo.cu (2..8 accumulator words) and
// tc_finish_hi.cu (9..16) so that the two compile in parallel.
#pragma once
#include "gemm_tc_impl.cuh"

namespace ozmp {
namespace tc {

// Rounding pass of the single-problem path: one thread per row i of C and
// FIN_J consecutive columns j normalises each element's carry-save limbs
// 0 .. nl-1 (from its tile's split slot when the tile was split into chunks,
// else from acc) and rounds them canonically into the q components.  The
// row's tile coordinates are computed once per thread.  Bound by the limb
// reads and the rounding arithmetic.
constexpr int FIN_J = 8;

// With g.chk set the pass also sums the squared first components (scaled by
// 4^-(GE + GF)) for the a-posteriori bound check, whose last block decides.
template <int NW>
__global__ void __launch_bounds__(256) k_tc_finish(const GemmArgs g, int nl, const int* tile_slot, int tile_rows,
                                                   int slot_limbs) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    float sq = 0.f;
    int gsc = 0;
    if (g.chk) gsc = g.chk->GE + g.chk->GF;
    if (i < g.m) {
        const size_t sstride = (size_t)BN * BM;
        const int64_t trow = i / tile_rows, ntrow = g.mp / tile_rows;
        const int cta_in = (int)((i % tile_rows) / BM);
        const size_t irow = (size_t)(i % BM);
        for (int64_t j0 = (int64_t)blockIdx.y * FIN_J; j0 < g.n; j0 += (int64_t)gridDim.y * FIN_J) {
#pragma unroll 1
            for (int jj = 0; jj < FIN_J; ++jj) {
                const int64_t j = j0 + jj;
                if (j >= g.n) break;
                const int slot = tile_slot ? tile_slot[trow + (j / BN) * ntrow] : -1;
                double c0;
                if (slot < 0) {
                    c0 = finish_element<NW>(g, nl, g.acc, (size_t)g.mp * g.np, (size_t)j * g.mp + i, i, j, 0, 0,
                                            false);
                } else {
                    const int cta = slot * (tile_rows / BM) + cta_in;
                    c0 = finish_element<NW>(g, nl, g.sacc + (size_t)cta * slot_limbs * sstride, sstride,
                                            (size_t)(j % BN) * BM + irow, i, j, 0, 0, false);
                }
                if (g.chk) {
                    const float y = bound_abs_scaled_f32(c0, gsc);
                    sq += y * y;
                }
            }
        }
    }
    if (!g.chk) return;
    // block sum, then the check's per-block step
    __shared__ float sh[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += (double)sh[w];
        bound_finish_block(g.chk, b, gridDim.x * gridDim.y, g.chk_form, g.s, g.status, g.chk_flag);
    }
}

}  // namespace tc

#define OZMP_TC_FIN_CASE(NWV) \
    case NWV: tc::k_tc_finish<NWV><<<fg, 256, 0, st>>>(g, nl, ts, rows, slot_limbs); break;

inline dim3 tc_finish_grid(const GemmArgs& g) {
    const int64_t cy = (g.n + tc::FIN_J - 1) / tc::FIN_J;
    return dim3((unsigned)((g.m + 255) / 256), (unsigned)(cy < 65535 ? (cy > 0 ? cy : 1) : 65535));
}

}  // namespace ozmp
