// Host-side launch descriptors shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ozmp.h"

namespace ozmp {

struct SplitArgs {
    int form;
    int q;
    bool is_f32;
    int64_t m, n, k, mp, np, kp;
    const void* const* A;
    int64_t lda;
    const void* const* B;
    int64_t ldb;
    int32_t* E;
    int32_t* F;
    uint32_t* status;
    void* Adig;
    void* Bdig;
    int s, beta;
};

struct GemmArgs {
    int form;
    int q;
    int is_f32;
    int64_t m, n, k, mp, np, kp;
    const int32_t* E;
    const int32_t* F;
    const void* Adig;
    const void* Bdig;
    int s, beta;
    int ppd;               // slice pairs summed in the tensor-core accumulator before a drain
    uint64_t group_start;  // bit (d - 2): diagonal d opens a new group (diagonals run s+1 .. 2)
    int acc_words;         // 64-bit words of the per-element exact accumulator
    int ngroups;
    int64_t* acc;          // [acc_words][mp][np], used when ngroups > 1
    void* C[4];
    int64_t ldc;
    uint32_t* status;
    int d_only;            // diagnostic: only diagonal d_only, raw int64 T_d written to T
    int64_t* T;
};

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st);
cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t st);

}  // namespace ozmp
