// Slice-pair products with the fused exact accumulation (K3).
//
// Paper, Sec. 3, Algorithm 1: C_{alpha beta} := A_alpha B_beta for
// alpha + beta <= D + 1, then C := C + sum C_{alpha beta} in L-bit
// arithmetic.  One CTA owns one C tile and walks the pair triangle by
// anti-diagonal d = t + u from d = s+1 (smallest weight 2^-beta d) down to
// d = 2, so that every pair of a diagonal shares one scale 2^(E_i+F_j-beta d).
//
// Exactness chain for one C element:
//   tensor-core accumulator (int32 / binary32 integers < 2^24 / binary64
//   integers < 2^53; at most `ppd` pairs between drains, chosen on the host)
//   -> drain into an int64 Horner value H in shared memory,
//      H += T << beta*(d_group_first - d)  (|H| < 2^62, host-chosen groups)
//   -> fold H << beta*(s+1 - d_group_first) into a multiword two's
//      complement accumulator (global memory, one per element)
//   -> canonical rounding into the q output components.
// Nothing is rounded before the last step.
#pragma once
#include "ozmp_internal.cuh"
#include "kernels.h"
#include <type_traits>

namespace ozmp {

// ----------------------------------------------------------------------------
// PTX wrappers
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* smem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_e4m3(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_f64(double (&c)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                 : "+d"(c[0]), "+d"(c[1])
                 : "d"(a), "d"(b));
}

// ----------------------------------------------------------------------------
// schedule of the pair triangle
// ----------------------------------------------------------------------------
struct Cursor {
    int d, t, kc;
    __device__ __forceinline__ void advance(int KT) {
        if (++kc == KT) {
            kc = 0;
            if (++t == d) { --d; t = 1; }
        }
    }
};

__device__ __forceinline__ int64_t pairs_in(int dlo, int dhi) {
    // sum_{d=dlo}^{dhi} (d - 1)
    return (int64_t)(dhi - dlo + 1) * (dlo - 1 + dhi - 1) / 2;
}

// ----------------------------------------------------------------------------
// epilogue: one element's group value H into the exact accumulator
// ----------------------------------------------------------------------------
template <int NW>
__device__ __forceinline__ void fold_element(const GemmArgs& g, int64_t i, int64_t j, int64_t H, int fsh,
                                             bool first, bool last) {
    if (i >= g.mp || j >= g.np) return;
    uint64_t w[NW];
    const size_t plane = (size_t)g.mp * g.np;
    const size_t idx = (size_t)i * g.np + j;
    if (first) {
#pragma unroll
        for (int x = 0; x < NW; ++x) w[x] = 0;
    } else {
#pragma unroll
        for (int x = 0; x < NW; ++x) w[x] = (uint64_t)g.acc[x * plane + idx];
    }
    uint64_t p[NW];
    uint64_t mag = H < 0 ? (uint64_t)(-H) : (uint64_t)H;
    mw_place<NW>(p, mag, fsh);
    if (H < 0) mw_sub<NW>(w, p); else mw_add<NW>(w, p);
    if (!last) {
#pragma unroll
        for (int x = 0; x < NW; ++x) g.acc[x * plane + idx] = (int64_t)w[x];
        return;
    }
    if (i >= g.m || j >= g.n) return;
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

__device__ __forceinline__ void fold_dispatch(const GemmArgs& g, int64_t i, int64_t j, int64_t H, int fsh,
                                              bool first, bool last) {
    switch (g.acc_words) {
        case 2: fold_element<2>(g, i, j, H, fsh, first, last); break;
        case 3: fold_element<3>(g, i, j, H, fsh, first, last); break;
        case 4: fold_element<4>(g, i, j, H, fsh, first, last); break;
        case 5: fold_element<5>(g, i, j, H, fsh, first, last); break;
        case 6: fold_element<6>(g, i, j, H, fsh, first, last); break;
        default: fold_element<7>(g, i, j, H, fsh, first, last); break;
    }
}

// ----------------------------------------------------------------------------
// 1-byte digits: INT8 (IMMA s8 -> s32) and FP8 (QMMA e4m3 -> f32)
// ----------------------------------------------------------------------------
namespace b1 {
constexpr int BM = 128, BN = 128, BK = 64, ST = 4, NT = 256, NE = 64;
constexpr size_t SMEM = (size_t)ST * (BM + BN) * BK + (size_t)NE * NT * 8;
}

template <int FORM>
__global__ void __launch_bounds__(256, 1) k_gemm_b1(const GemmArgs g) {
    using namespace b1;
    typedef typename std::conditional<FORM == OZMP_FORM_INT8, int, float>::type AccT;
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sA = sm;
    unsigned char* sB = sm + (size_t)ST * BM * BK;
    int64_t* Hs = reinterpret_cast<int64_t*>(sm + (size_t)ST * (BM + BN) * BK);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    const int KT = (int)(g.kp / BK);
    const int dhi = g.d_only ? g.d_only : g.s + 1;
    const int dlo = g.d_only ? g.d_only : 2;
    const int64_t nsteps = pairs_in(dlo, dhi) * KT;
    const uint8_t* Ad = (const uint8_t*)g.Adig;
    const uint8_t* Bd = (const uint8_t*)g.Bdig;

    auto load_stage = [&](int stage, const Cursor& c) {
        const int u = c.d - c.t;
        const uint8_t* ga = Ad + ((size_t)(c.t - 1) * g.mp + i0) * g.kp + (size_t)c.kc * BK;
        const uint8_t* gb = Bd + ((size_t)(u - 1) * g.np + j0) * g.kp + (size_t)c.kc * BK;
        unsigned char* a_st = sA + (size_t)stage * BM * BK;
        unsigned char* b_st = sB + (size_t)stage * BN * BK;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int ci = tid + NT * r;
            int row = ci >> 2, c16 = ci & 3;
            int sw = c16 ^ ((row >> 1) & 3);
            cp_async16(a_st + row * BK + sw * 16, ga + (size_t)row * g.kp + c16 * 16);
            cp_async16(b_st + row * BK + sw * 16, gb + (size_t)row * g.kp + c16 * 16);
        }
    };

    Cursor lc{dhi, 1, 0};
    int64_t issued = 0;
#pragma unroll
    for (int s0 = 0; s0 < ST - 1; ++s0) {
        if (issued < nsteps) { load_stage(s0, lc); lc.advance(KT); }
        cp_async_commit();
        ++issued;
    }

    AccT acc[16][4];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e][0] = acc[e][1] = acc[e][2] = acc[e][3] = 0;

    Cursor cc{dhi, 1, 0};
    int since_drain = 0;
    bool fresh = true;
    int gfirst = dhi;      // first (largest) diagonal of the current group
    bool first_group = true;

    for (int64_t step = 0; step < nsteps; ++step) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        if (issued < nsteps) { load_stage((int)(issued % ST), lc); lc.advance(KT); }
        cp_async_commit();
        ++issued;

        const int stage = (int)(step % ST);
        const unsigned char* a_st = sA + (size_t)stage * BM * BK;
        const unsigned char* b_st = sB + (size_t)stage * BN * BK;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                int row = wm * 64 + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                int ch = kk * 2 + (lane >> 4);
                ldmatrix_x4(af[mt], a_st + row * BK + ((ch ^ ((row >> 1) & 3)) * 16));
            }
#pragma unroll
            for (int np2 = 0; np2 < 2; ++np2) {
                int mi = lane >> 3;
                int row = wn * 32 + np2 * 16 + (lane & 7) + (mi >> 1) * 8;
                int ch = kk * 2 + (mi & 1);
                uint32_t r[4];
                ldmatrix_x4(r, b_st + row * BK + ((ch ^ ((row >> 1) & 3)) * 16));
                bf[2 * np2][0] = r[0];
                bf[2 * np2][1] = r[1];
                bf[2 * np2 + 1][0] = r[2];
                bf[2 * np2 + 1][1] = r[3];
            }
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    if constexpr (FORM == OZMP_FORM_INT8) mma_s8(acc[mt * 4 + nt], af[mt], bf[nt]);
                    else mma_e4m3(acc[mt * 4 + nt], af[mt], bf[nt]);
                }
        }

        if (cc.kc == KT - 1) {
            ++since_drain;
            const bool diag_end = (cc.t == cc.d - 1);
            if (since_drain == g.ppd || diag_end) {
                const int dsh = g.beta * (gfirst - cc.d);
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                    int64_t v;
                    if constexpr (FORM == OZMP_FORM_INT8) v = (int64_t)acc[e >> 2][e & 3];
                    else v = (int64_t)__float2int_rn(acc[e >> 2][e & 3]);
                    int64_t add = (int64_t)((uint64_t)v << dsh);
                    int64_t* hp = &Hs[e * NT + tid];
                    *hp = fresh ? add : (*hp + add);
                    acc[e >> 2][e & 3] = 0;
                }
                fresh = false;
                since_drain = 0;
            }
            if (diag_end) {
                const int nd = cc.d - 1;
                const bool last = nd < dlo;
                const bool gend = last || ((g.group_start >> (nd - 2)) & 1ull);
                if (gend) {
                    const int fsh = g.beta * (g.s + 1 - gfirst);
#pragma unroll 1
                    for (int e = 0; e < NE; ++e) {
                        const int mt = e >> 4, nt = (e >> 2) & 3, v = e & 3;
                        const int64_t i = i0 + wm * 64 + mt * 16 + gq + (v >> 1) * 8;
                        const int64_t j = j0 + wn * 32 + nt * 8 + 2 * tq + (v & 1);
                        const int64_t H = Hs[e * NT + tid];
                        if (g.d_only) {
                            if (i < g.m && j < g.n) g.T[i + j * g.m] = H;
                        } else {
                            fold_dispatch(g, i, j, H, fsh, first_group, last);
                        }
                    }
                    fresh = true;
                    first_group = false;
                    gfirst = nd;
                }
            }
        }
        cc.advance(KT);
    }
    cp_async_wait<0>();
}

// ----------------------------------------------------------------------------
// binary64 digits: DMMA m8n8k4
// ----------------------------------------------------------------------------
namespace f64 {
constexpr int BM = 64, BN = 64, BK = 32, ST = 3, NT = 128, NE = 32;
constexpr int RS = BK * 8 + 16;   // padded row stride in bytes
constexpr size_t SMEM = (size_t)ST * (BM + BN) * RS + (size_t)NE * NT * 8;
}

static __global__ void __launch_bounds__(128, 1) k_gemm_f64(const GemmArgs g) {
    using namespace f64;
    extern __shared__ __align__(128) unsigned char sm[];
    unsigned char* sA = sm;
    unsigned char* sB = sm + (size_t)ST * BM * RS;
    int64_t* Hs = reinterpret_cast<int64_t*>(sm + (size_t)ST * (BM + BN) * RS);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const int gq = lane >> 2, tq = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
    const int KT = (int)(g.kp / BK);
    const int dhi = g.d_only ? g.d_only : g.s + 1;
    const int dlo = g.d_only ? g.d_only : 2;
    const int64_t nsteps = pairs_in(dlo, dhi) * KT;
    const double* Ad = (const double*)g.Adig;
    const double* Bd = (const double*)g.Bdig;

    auto load_stage = [&](int stage, const Cursor& c) {
        const int u = c.d - c.t;
        const double* ga = Ad + ((size_t)(c.t - 1) * g.mp + i0) * g.kp + (size_t)c.kc * BK;
        const double* gb = Bd + ((size_t)(u - 1) * g.np + j0) * g.kp + (size_t)c.kc * BK;
        unsigned char* a_st = sA + (size_t)stage * BM * RS;
        unsigned char* b_st = sB + (size_t)stage * BN * RS;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            int ci = tid + NT * r;          // 1024 chunks of 16 bytes per operand
            int row = ci >> 4, c16 = ci & 15;
            cp_async16(a_st + row * RS + c16 * 16, ga + (size_t)row * g.kp + c16 * 2);
            cp_async16(b_st + row * RS + c16 * 16, gb + (size_t)row * g.kp + c16 * 2);
        }
    };

    Cursor lc{dhi, 1, 0};
    int64_t issued = 0;
#pragma unroll
    for (int s0 = 0; s0 < ST - 1; ++s0) {
        if (issued < nsteps) { load_stage(s0, lc); lc.advance(KT); }
        cp_async_commit();
        ++issued;
    }

    double acc[16][2];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e][0] = acc[e][1] = 0.0;

    Cursor cc{dhi, 1, 0};
    int since_drain = 0;
    bool fresh = true;
    int gfirst = dhi;
    bool first_group = true;

    for (int64_t step = 0; step < nsteps; ++step) {
        cp_async_wait<ST - 2>();
        __syncthreads();
        if (issued < nsteps) { load_stage((int)(issued % ST), lc); lc.advance(KT); }
        cp_async_commit();
        ++issued;

        const int stage = (int)(step % ST);
        const double* a_st = reinterpret_cast<const double*>(sA + (size_t)stage * BM * RS);
        const double* b_st = reinterpret_cast<const double*>(sB + (size_t)stage * BN * RS);
        constexpr int RSD = RS / 8;
#pragma unroll
        for (int k4 = 0; k4 < BK / 4; ++k4) {
            double af[4], bfr[4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) af[mt] = a_st[(wm * 32 + mt * 8 + gq) * RSD + k4 * 4 + tq];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) bfr[nt] = b_st[(wn * 32 + nt * 8 + gq) * RSD + k4 * 4 + tq];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) mma_f64(acc[mt * 4 + nt], af[mt], bfr[nt]);
        }

        if (cc.kc == KT - 1) {
            ++since_drain;
            const bool diag_end = (cc.t == cc.d - 1);
            if (since_drain == g.ppd || diag_end) {
                const int dsh = g.beta * (gfirst - cc.d);
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                    int64_t v = __double2ll_rn(acc[e >> 1][e & 1]);
                    int64_t add = (int64_t)((uint64_t)v << dsh);
                    int64_t* hp = &Hs[e * NT + tid];
                    *hp = fresh ? add : (*hp + add);
                    acc[e >> 1][e & 1] = 0.0;
                }
                fresh = false;
                since_drain = 0;
            }
            if (diag_end) {
                const int nd = cc.d - 1;
                const bool last = nd < dlo;
                const bool gend = last || ((g.group_start >> (nd - 2)) & 1ull);
                if (gend) {
                    const int fsh = g.beta * (g.s + 1 - gfirst);
#pragma unroll 1
                    for (int e = 0; e < NE; ++e) {
                        const int mt = e >> 3, nt = (e >> 1) & 3, v = e & 1;
                        const int64_t i = i0 + wm * 32 + mt * 8 + gq;
                        const int64_t j = j0 + wn * 32 + nt * 8 + 2 * tq + v;
                        const int64_t H = Hs[e * NT + tid];
                        if (g.d_only) {
                            if (i < g.m && j < g.n) g.T[i + j * g.m] = H;
                        } else {
                            fold_dispatch(g, i, j, H, fsh, first_group, last);
                        }
                    }
                    fresh = true;
                    first_group = false;
                    gfirst = nd;
                }
            }
        }
        cc.advance(KT);
    }
    cp_async_wait<0>();
}

}  // namespace ozmp
