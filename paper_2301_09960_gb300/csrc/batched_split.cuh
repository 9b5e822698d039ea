// Split (K1 exponents, K2 digits) of the batched products: the per-problem
// descriptor, the block-to-problem lookup, and the launch of one group of
// problems that share their component type and count.  Kernels in
// batched_split.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ozmp {

// per problem split descriptor (device memory)
struct BSplit {
    const void* A[4];
    const void* B[4];
    int64_t lda, ldb, m, n, k, mp, np, kp;
    int32_t* E;
    int32_t* F;
    uint8_t* Adig;
    uint8_t* Bdig;
    int q, s;
};

// columns of A per block of the row exponent kernel (one thread per row):
// short per-thread chains keep many independent loads in flight
constexpr int B_EXP_KCHUNK = 32;

// problem of batched block b: the last p with pre[p] <= b
__device__ __forceinline__ int find_prob(const int* pre, int count, int b) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// blocks of the five split launches of one problem: exponent init, row
// exponents, column exponents, row digits (32 x 64 tiles), column digits (quads)
inline void bsplit_blocks(int64_t m, int64_t n, int64_t k, int64_t mp, int64_t np, int (&nb)[5]) {
    nb[0] = (int)(((mp > np ? mp : np) + 255) / 256);
    nb[1] = (int)(((m + 255) / 256) * ((k + B_EXP_KCHUNK - 1) / B_EXP_KCHUNK));
    nb[2] = (int)((n + 7) / 8);
    nb[3] = (int)(((m + 31) / 32) * ((k + 63) / 64));
    nb[4] = (int)((((k + 3) / 4) * n + 255) / 256);
}

// one group's launches: problems of one component type and count
struct BSplitGroup {
    const BSplit* sp;      // descriptors (device)
    const int* pre[5];     // block prefix sums of the five launches (device)
    int blocks[5];         // block totals
    int count;             // problems
    int is_f32, q, nw;     // component type and count; digit window words (4 or 6)
    int bal;               // balanced radix-32 digits (else 4-bit e4m3)
    size_t smem;           // shared memory of the row digit kernel
    uint32_t* status;
};

// raise the row digit kernel's shared-memory limit (before a graph capture)
cudaError_t bsplit_set_smem(const BSplitGroup& g);
// the five launches of one group (capturable): the exponent init, then A's
// row exponents and digits on cs and B's column exponents and digits on cs_b,
// which waits for the init through ev_init (cs_b == cs: all on cs)
cudaError_t bsplit_launch(const BSplitGroup& g, cudaStream_t cs, cudaStream_t cs_b, cudaEvent_t ev_init);

}  // namespace ozmp
