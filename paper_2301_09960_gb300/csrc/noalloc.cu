// Double-double product that allocates no memory (ozmp_gemm_dd_noalloc).
//
// Who needs it: callers that must not call cudaMalloc.  A program whose
// device memory is all handed out by its own pool or caching allocator
// cannot have a library allocate behind the pool's back: the allocation can
// fail because the pool holds the memory, and cudaMalloc/cudaFree
// synchronise the device.  Plug-ins and real-time loops are often not
// allowed to allocate after start-up at all.  The regular entry points
// allocate their workspace on first use; this one instead uses a scratch
// area that is part of the library's device image.
//
// The scratch is a file-scope __device__ array of OZMP_NOALLOC_SCRATCH_BYTES
// (64 MiB).  Every GPU that loads the library holds it until the process
// exits.  Host code cannot use the array's name as a device address (on the
// host it is only a stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and every
// call passes that address to the kernels.  Make that first call before any
// stream capture.
//
// The scratch holds the plan layout of the whole-tile walk (exponents, digit
// slices of both operands, carry-save limbs): plan_init's workspace size,
// without the tile schedule and split-tile limbs that a regular plan appends.
// Larger problems are rejected.
//
// All calls share the one array and it keeps the last call's contents: the
// exponent vectors and the status word are reset by the first kernel of every
// call, the digit slices (padding included) are rewritten in full, and the
// exact accumulator is written before it is read.  Calls whose work overlaps
// on the GPU (different streams, different host threads) race on the array
// and must be serialised by the caller.
#include <mutex>
#include "kernels.h"
#include "ozmp_internal.cuh"
#include "plan.h"

using namespace ozmp;
using namespace ozmp_plan_detail;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[OZMP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once
// per device)
ozmp_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return OZMP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OZMP_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return OZMP_OK;
}

}  // namespace

extern "C" ozmp_status ozmp_gemm_dd_noalloc(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
                                            const double* const B[2], int64_t ldb, double* const C[2],
                                            int64_t ldc, int nslices, ozmp_stream stream) {
    ozmp_plan_s p;   // the plan lives on the stack
    ozmp_status st = plan_init(&p, OZMP_DD, m, n, k, OZMP_FORM_AUTO, nslices, stream);
    if (st != OZMP_OK) return st;
    if (p.ws_bytes > OZMP_NOALLOC_SCRATCH_BYTES) return OZMP_ERR_UNSUPPORTED;
    if (check_ld(&p, lda, ldb, ldc, true) != OZMP_OK) return OZMP_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return OZMP_OK;
    if (!ptrs_ok((void* const*)C, 2)) return OZMP_ERR_INVALID_ARG;
    if (k > 0 && (!ptrs_ok((const void* const*)A, 2) || !ptrs_ok((const void* const*)B, 2)))
        return OZMP_ERR_INVALID_ARG;
    void* base = nullptr;
    st = scratch_address(&base);
    if (st != OZMP_OK) return st;
    p.ws = base;
    p.ws_owned = false;
    if (k == 0) return zero_c(&p, (void* const*)C, ldc);
    SplitArgs sa = split_args(&p, (const void* const*)A, lda, (const void* const*)B, ldb);
    if (launch_split(sa, p.stream) != cudaSuccess) return OZMP_ERR_CUDA;
    GemmArgs g = gemm_args(&p);
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) g.C[c] = (c < 2) ? (void*)C[c] : nullptr;
    g.ldc = ldc;
    return launch_gemm(g, p.stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}
