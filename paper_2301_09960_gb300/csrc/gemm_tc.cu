// Slice-pair products on the 5th-generation tensor cores (tcgen05), e4m3
// digits, binary32 accumulation in tensor memory -- the GB300-native form of
// the e4m3 engine.
//
// Paper, Sec. 3, Algorithm 1: C_{alpha beta} := A_alpha B_beta over the pair
// triangle, then the L-bit sum.  One CTA owns a 128 x 256 tile of C and walks
// the triangle by anti-diagonal d = s+1 .. 2 exactly as the mma.sync kernels.
//
// Roles (192 threads):
//   warp 0      TMA producer: 128x128-byte A tile + 256x128-byte B tile per
//               stage (SWIZZLE_128B), 4 stages, mbarrier full/empty ring;
//   warp 1      TMEM owner (512 columns) and MMA issuer: per stage four
//               tcgen05.mma.kind::f8f6f4 (M=128, N=256, K=32) into one of two
//               256-column binary32 accumulators;
//   warps 2..5  epilogue: per drain, tcgen05.ld the accumulator (integers
//               below 2^24, exact), convert, and add v * 2^off into ONE int64
//               carry-save limb per element (limb l weighs 2^(16 l), off < 16,
//               so each limb stays below 2^48 for every k the form allows); the
//               last drain normalises the limbs to a two's complement integer
//               and rounds it canonically into the q output components.
// The two accumulator buffers let the MMAs of the next pairs run while the
// epilogue drains the previous ones.  Every wait is bounded: on timeout the
// kernel records OZMP_ERR_TIMEOUT in the status word, all roles leave their
// loops, and the TMEM is released before returning.
#include <cuda.h>
#include <cudaTypedefs.h>
#include "kernels.h"
#include "ozmp_internal.cuh"

namespace ozmp {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 128, NST = 4, NT = 192;
constexpr unsigned STAGE_A = BM * BK, STAGE_B = BN * BK;
constexpr unsigned TX_BYTES = STAGE_A + STAGE_B;
constexpr size_t SMEM = 1024 + (size_t)NST * (STAGE_A + STAGE_B) + 256;
constexpr long long WAIT_LIMIT = 1ll << 26;   // try_wait polls before giving up (seconds)

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of parity `parity`; false on timeout or abort
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
            saddr(dst)),
        "l"((uint64_t)map), "r"(saddr(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// shared memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), version bits 46-48 = 0b001
__device__ __forceinline__ uint64_t desc_sw128(uint32_t smem) {
    uint64_t d = 0;
    d |= (uint64_t)((smem & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;      // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// instruction descriptor, kind::f8f6f4: D = f32, A = B = e4m3, both K-major
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3_tc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// walk of the pair triangle shared by the three roles
struct Walk {
    int d, t;
    __device__ __forceinline__ bool next_pair() {   // advance; false when past the end
        if (++t == d) { --d; t = 1; }
        return true;
    }
};

// Limb accumulator of one element: NL int64 limbs, limb l weighs 2^(16 l),
// layout [l][np][mp] (consecutive rows contiguous).  `zero` skips the load
// (first and last drain of a tile coincide).
template <int NW>
__device__ __forceinline__ void finish_element(const GemmArgs& g, int nl, int64_t i, int64_t j, int64_t x, int li,
                                               bool zero) {
    const size_t plane = (size_t)g.mp * g.np;
    const size_t idx = (size_t)j * g.mp + i;
    constexpr int NLMAX = 4 * NW + 1;
    int64_t L[NLMAX];
#pragma unroll
    for (int l = 0; l < NLMAX; ++l) L[l] = (!zero && l < nl) ? g.acc[l * plane + idx] : 0;
#pragma unroll
    for (int l = 0; l < NLMAX; ++l)
        if (l == li) L[l] += x;
    // carry-save limbs -> two's complement words (the value fits 64 NW bits)
    uint64_t w[NW];
#pragma unroll
    for (int x2 = 0; x2 < NW; ++x2) w[x2] = 0;
    int64_t carry = 0;
#pragma unroll
    for (int l = 0; l < 4 * NW; ++l) {
        int64_t t = L[l] + carry;                 // |L| < 2^48, |carry| < 2^48
        w[l >> 2] |= ((uint64_t)t & 0xffffull) << (16 * (l & 3));
        carry = t >> 16;                           // arithmetic shift: floor division
    }
    if (i >= g.m || j >= g.n) return;
    if (g.d_only) {
        g.T[i + j * g.m] = (int64_t)w[0];
        return;
    }
    int Ei = g.E[i], Fj = g.F[j];
    bool ok = true;
    if (g.is_f32) {
        float out[4] = {0.f, 0.f, 0.f, 0.f};
        if (Ei != OZMP_EXP_ZERO && Fj != OZMP_EXP_ZERO)
            ok = canonical_round<NW, float>(w, Ei + Fj - g.beta * (g.s + 1), g.q, out);
        for (int c = 0; c < g.q; ++c) ((float*)g.C[c])[i + j * g.ldc] = out[c];
    } else {
        double out[4] = {0.0, 0.0, 0.0, 0.0};
        if (Ei != OZMP_EXP_ZERO && Fj != OZMP_EXP_ZERO)
            ok = canonical_round<NW, double>(w, Ei + Fj - g.beta * (g.s + 1), g.q, out);
        for (int c = 0; c < g.q; ++c) ((double*)g.C[c])[i + j * g.ldc] = out[c];
    }
    if (!ok) atomicOr(g.status, ST_RANGE);
}

__device__ __forceinline__ void finish_dispatch(const GemmArgs& g, int nl, int64_t i, int64_t j, int64_t x, int li,
                                                bool zero) {
    switch (g.acc_words) {
        case 2: finish_element<2>(g, nl, i, j, x, li, zero); break;
        case 3: finish_element<3>(g, nl, i, j, x, li, zero); break;
        case 4: finish_element<4>(g, nl, i, j, x, li, zero); break;
        case 5: finish_element<5>(g, nl, i, j, x, li, zero); break;
        case 6: finish_element<6>(g, nl, i, j, x, li, zero); break;
        default: finish_element<7>(g, nl, i, j, x, li, zero); break;
    }
}

__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const GemmArgs g, const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB) {
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + (size_t)NST * STAGE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)NST * STAGE_B);
    uint64_t* empty = full + NST;
    uint64_t* accf = empty + NST;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    const int KT = (int)(g.kp / BK);
    const int dhi = g.d_only ? g.d_only : g.s + 1;
    const int dlo = g.d_only ? g.d_only : 2;
    const int nl = 4 * g.acc_words + 1;

    if (threadIdx.x == 0) {
        for (int x = 0; x < NST; ++x) { mbar_init(&full[x], 1); mbar_init(&empty[x], 1); }
        for (int x = 0; x < 2; ++x) { mbar_init(&accf[x], 1); mbar_init(&acce[x], 4); }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(saddr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            Walk w{dhi, 1};
            long long n = 0;
            bool ok = true;
            while (ok && w.d >= dlo) {
                const int u = w.d - w.t;
                const int ya = (w.t - 1) * (int)g.mp + (int)i0;
                const int yb = (u - 1) * (int)g.np + (int)j0;
                for (int kc = 0; kc < KT; ++kc, ++n) {
                    const int st = (int)(n % NST);
                    const unsigned ph = (unsigned)((n / NST) & 1);
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(&full[st], TX_BYTES);
                    tma_load_2d(sA + (size_t)st * STAGE_A, &tmA, &full[st], kc * BK, ya);
                    tma_load_2d(sB + (size_t)st * STAGE_B, &tmB, &full[st], kc * BK, yb);
                }
                w.next_pair();
            }
            if (!ok) {
                *abort_flag = 1;
                atomicOr(g.status, ST_TIMEOUT);
                // let the copies already issued land before the CTA can exit
                volatile int never = 0;
                for (long long q = n - 1; q >= 0 && q >= n - NST; --q)
                    mbar_wait(&full[(int)(q % NST)], (unsigned)((q / NST) & 1), &never);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_e4m3(BM, BN);
            Walk w{dhi, 1};
            long long n = 0;
            int buf = 0, uses[2] = {0, 0}, since = 0;
            bool fresh = true, ok = true;
            ok = mbar_wait(&acce[0], 1u, abort_flag);     // first use of buffer 0
            while (ok && w.d >= dlo) {
                const uint32_t dcol = tmem + (uint32_t)(buf * BN);
                for (int kc = 0; kc < KT; ++kc, ++n) {
                    const int st = (int)(n % NST);
                    const unsigned ph = (unsigned)((n / NST) & 1);
                    if (!mbar_wait(&full[st], ph, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = desc_sw128(saddr(sA + (size_t)st * STAGE_A));
                    const uint64_t bd = desc_sw128(saddr(sB + (size_t)st * STAGE_B));
#pragma unroll
                    for (int kk = 0; kk < BK / 32; ++kk) {
                        mma_e4m3_tc(dcol, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), IDESC,
                                    (fresh && kk == 0) ? 0u : 1u);
                    }
                    fresh = false;
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                ++since;
                const bool diag_end = (w.t == w.d - 1);
                if (since == g.ppd || diag_end) {
                    mma_commit(&accf[buf]);
                    uses[buf]++;
                    buf ^= 1;
                    since = 0;
                    fresh = true;
                    // the k-th use of a buffer waits for the epilogue's (k-1)-th release
                    if (!mbar_wait(&acce[buf], (unsigned)((uses[buf] & 1) ^ 1), abort_flag)) { ok = false; break; }
                }
                w.next_pair();
            }
            if (!ok) { *abort_flag = 1; atomicOr(g.status, ST_TIMEOUT); }
            // every issued MMA has completed before the TMEM can be released
            mma_commit(done);
            volatile int never = 0;
            mbar_wait(done, 0u, &never);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int64_t i = i0 + quarter * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const size_t plane = (size_t)g.mp * g.np;
        Walk w{dhi, 1};
        int since = 0, ev = 0;
        bool first = true, ok = true;
        while (ok && w.d >= dlo) {
            ++since;
            const bool diag_end = (w.t == w.d - 1);
            if (since == g.ppd || diag_end) {
                since = 0;
                const bool last = diag_end && (w.d == dlo);
                const int buf = ev & 1;
                const unsigned par = (unsigned)((ev >> 1) & 1);
                ++ev;
                if (!mbar_wait(&accf[buf], par, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const int fsh = g.d_only ? 0 : g.beta * (g.s + 1 - w.d);
                const int li = fsh >> 4, off = fsh & 15;
#pragma unroll 1
                for (int c = 0; c < BN / 32; ++c) {
                    uint32_t r[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(buf * BN + c * 32), r);
                    if (c == BN / 32 - 1) {
                        // the accumulator buffer is free once its last columns are in registers
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acce[buf]);
                    }
                    const int64_t jb = j0 + c * 32;
                    if (last) {
#pragma unroll 1
                        for (int x = 0; x < 32; ++x) {
                            const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                            finish_dispatch(g, nl, i, jb + x, (int64_t)((uint64_t)v << off), li, first);
                        }
                    } else if (first) {
#pragma unroll 4
                        for (int x = 0; x < 32; ++x) {
                            const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                            const size_t idx = (size_t)(jb + x) * g.mp + i;
                            const int64_t val = (int64_t)((uint64_t)v << off);
                            for (int l = 0; l < nl; ++l) g.acc[l * plane + idx] = (l == li) ? val : 0;
                        }
                    } else {
                        int64_t cur[32];
#pragma unroll
                        for (int x = 0; x < 32; ++x) cur[x] = g.acc[li * plane + (size_t)(jb + x) * g.mp + i];
#pragma unroll
                        for (int x = 0; x < 32; ++x) {
                            const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                            g.acc[li * plane + (size_t)(jb + x) * g.mp + i] = cur[x] + (int64_t)((uint64_t)v << off);
                        }
                    }
                }
                first = false;
            }
            w.next_pair();
        }
        if (!ok) { *abort_flag = 1; atomicOr(g.status, ST_TIMEOUT); }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
    }
}

}  // namespace tc

// ----------------------------------------------------------------------------
// host: tensor maps and launch
// ----------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D byte tensor: rows x kp (row stride kp bytes), box 128 bytes x box_rows,
// 128-byte swizzle (the layout of the tcgen05 K-major descriptors)
static bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t kp, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp};
    cuuint32_t box[2] = {128u, box_rows};
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_gemm_tc(const GemmArgs& g, cudaStream_t st) {
    if (g.mp % tc::BM || g.np % tc::BN || g.kp % tc::BK) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.Adig, (uint64_t)g.s * g.mp, (uint64_t)g.kp, tc::BM)) return cudaErrorInvalidValue;
    if (!make_map(&mb, g.Bdig, (uint64_t)g.s * g.np, (uint64_t)g.kp, tc::BN)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(g.mp / tc::BM), (unsigned)(g.np / tc::BN));
    tc::k_gemm_tc<<<grid, tc::NT, tc::SMEM, st>>>(g, ma, mb);
    return cudaGetLastError();
}

}  // namespace ozmp
