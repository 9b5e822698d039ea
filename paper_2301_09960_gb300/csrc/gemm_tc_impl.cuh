// Slice-pair products on the 5th-generation tensor cores (tcgen05), e4m3
// digits, binary32 accumulation in tensor memory -- the GB300-native form of
// the e4m3 engine.  Shared by the single-problem launch (gemm_tc.cu) and the
// persistent batched launch (batched.cu).
//
// Paper, Sec. 3, Algorithm 1: C_{alpha beta} := A_alpha B_beta over the pair
// triangle, then the L-bit sum.  One CTA owns a 128 x 256 tile of C and walks
// the triangle in the order of walk.h: where k >= 4096 two anti-diagonals
// interleaved so that consecutive pairs share an operand slice, else one
// anti-diagonal at a time, d = s+1 .. 2, as the mma.sync kernels.
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
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include "kernels.h"
#include "ozmp_internal.cuh"
#include "walk.h"

namespace ozmp {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 128, NST = 4, NT = 192;   // BN: widest tile
constexpr unsigned STAGE_A = BM * BK, STAGE_B = BN * BK;
constexpr unsigned TX_BYTES = STAGE_A + STAGE_B;
constexpr size_t SMEM = 1024 + (size_t)NST * (STAGE_A + STAGE_B) + 512;
// CTA-pair form (cta_group::2): a cluster of two CTAs owns a 256 x 256 tile;
// each CTA stages its 128 rows of A and its half (128 rows) of the B tile,
// so a stage is 32 KB per CTA and six stages fit
constexpr int NST2 = 6;
constexpr unsigned STAGE_B2 = (BN / 2) * BK;
constexpr size_t SMEM2 = 1024 + (size_t)NST2 * (STAGE_A + STAGE_B2) + 512;
constexpr long long WAIT_LIMIT = 1ll << 26;   // try_wait polls before giving up (seconds)
constexpr long long DRAIN_LIMIT = 1ll << 20;  // polls for copies / MMAs already in flight at the end

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
// the same with cluster-scope acquire (phases completed by the peer CTA of a pair)
__device__ __forceinline__ bool mbar_try_cl(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase of parity `parity`; false on timeout or abort
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, volatile int* abort_flag,
                                          long long limit = WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it) {
        if (CLUSTER ? mbar_try_cl(b, parity) : mbar_try(b, parity)) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

// ---- cluster helpers of the CTA-pair form
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;\n" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cl_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(cl_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cl_addr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;\n" ::"r"(cl_addr), "r"(v) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::"r"(
            saddr(dst)),
        "l"((uint64_t)map), "r"(saddr(bar)), "r"(x), "r"(y)
        : "memory");
}

// pair form: the copy lands in this CTA's shared memory and completes its
// bytes on the barrier at `bar_cl`, which may be the leader CTA's
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cl, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];\n" ::"r"(saddr(dst)),
        "l"((uint64_t)map), "r"(bar_cl), "r"(x), "r"(y)
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

// binary16 digits: one MMA of K = 16 reads the same 32 bytes of a row as an
// e4m3 MMA of K = 32, and the instruction descriptor has the same bits
// (D = f32, A = B = f16 are type code 0 of kind::f16)
__device__ __forceinline__ void mma_f16_tc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_f16_tc_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// pair form: M = 256 over the two CTAs (A rows 0..127 from the leader's
// shared memory, 128..255 from the peer's; B columns split the same way),
// each CTA's tensor memory holding its 128 rows of D
__device__ __forceinline__ void mma_e4m3_tc_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                 uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the barrier at the same offset in both CTAs of the pair once the
// issuing thread's earlier MMAs are complete
__device__ __forceinline__ void mma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n" ::"r"(
            saddr(bar)),
        "h"((unsigned short)3)
        : "memory");
}
__device__ __forceinline__ void mma_commit_local_pair(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
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

// Limb accumulator of one element: limbs 0 .. nl-1 of int64, limb l weighs
// 2^(16 l), limb l of the element at base[l * lstride + idx].  `x` is added
// to limb `li` (the last drain's contribution when it is fused here);
// `zero` skips the loads (first and last drain of a tile coincide), and only
// the limbs l < nl whose bit is set in `have` are loaded (the others hold no
// data yet: the fused last drain passes the limbs its tile has written).  The
// limbs are streamed through one carry chain into a two's complement value
// of 64 NW bits, rounded canonically into C(i, j) (or written to T in the
// diagnostic mode).  Returns the first component written (0 otherwise).
template <int NW>
__device__ __forceinline__ double finish_element(const GemmArgs& g, int nl, const int64_t* base, size_t lstride,
                                                 size_t idx, int64_t i, int64_t j, int64_t x, int li, bool zero,
                                                 uint64_t have = ~0ull) {
    uint64_t w[NW];
#pragma unroll
    for (int x2 = 0; x2 < NW; ++x2) w[x2] = 0;
    int64_t carry = 0;
#pragma unroll
    for (int l = 0; l < 4 * NW; ++l) {
        int64_t t = (!zero && l < nl && ((have >> l) & 1)) ? __ldcg(base + l * lstride + idx) : 0;   // |limb| < 2^48
        if (l == li) t += x;
        t += carry;                                // |carry| < 2^48
        w[l >> 2] |= ((uint64_t)t & 0xffffull) << (16 * (l & 3));
        carry = t >> 16;                           // arithmetic shift: floor division
    }
    if (i >= g.m || j >= g.n) return 0.0;
    if (g.d_only) {
        g.T[i + j * g.m] = (int64_t)w[0];
        return 0.0;
    }
    const int Ei = g.E[i], Fj = g.F[j];
    const bool nz = (Ei != OZMP_EXP_ZERO && Fj != OZMP_EXP_ZERO);
    const int U = nz ? Ei + Fj + g.eoff - g.beta * (g.s + 1) : 0;
    const size_t at = (size_t)(i + j * g.ldc);
    bool ok = true;
    double c0 = 0.0;
    if (g.is_f32) {
        if (nz) ok = canonical_round_put<NW, float>(w, U, g.q, [&](int c, float v) {
            ((float*)g.C[c])[at] = v;
            if (c == 0) c0 = (double)v;
        });
        else for (int c = 0; c < g.q; ++c) ((float*)g.C[c])[at] = 0.f;
    } else {
        if (nz) ok = canonical_round_put<NW, double>(w, U, g.q, [&](int c, double v) {
            ((double*)g.C[c])[at] = v;
            if (c == 0) c0 = v;
        });
        else for (int c = 0; c < g.q; ++c) ((double*)g.C[c])[at] = 0.0;
    }
    if (!ok) atomicOr(g.status, ST_RANGE);
    return c0;
}

__device__ __forceinline__ void finish_dispatch(const GemmArgs& g, int nl, const int64_t* base, size_t lstride,
                                                size_t idx, int64_t i, int64_t j, int64_t x, int li, bool zero,
                                                uint64_t have = ~0ull) {
    switch (g.acc_words) {
        case 2: finish_element<2>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
        case 3: finish_element<3>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
        case 4: finish_element<4>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
        case 5: finish_element<5>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
        case 6: finish_element<6>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
        default: finish_element<7>(g, nl, base, lstride, idx, i, j, x, li, zero, have); break;
    }
}


// One problem of a launch.  The tensor maps are those of the problem's digit
// arrays (box 128 x 128 bytes for A, bn x 128 bytes for B).
struct Prob {
    const int32_t* E;
    const int32_t* F;
    int64_t* acc;          // [nlimbs][np][mp] carry-save limbs
    void* C[OZMP_MAX_COMPONENTS];
    int64_t* T;            // diagnostic output (d_only)
    int64_t* sacc;         // split tiles: [slot][nlimbs][bn][BM] limbs, zeroed before the launch
    int* cnt;              // split tiles: chunks finished per slot, zeroed before the launch
    const int* tile_slot;  // batched mode: split-limb slot of each tile, or -1 (null: no split tile)
    int64_t m, n, mp, np, kp, ldc;
    int q, is_f32, s, beta, ppd, acc_words, bn, d_only;
    int eoff;              // exponent offset of the digit weights (2: balanced digits)
    int kind;              // 0: e4m3 digits (kind::f8f6f4); 1: binary16 digits (kind::f16); kp counts bytes
    int defer;             // 1: the limbs are rounded into C by a separate pass after the launch
};

// adapter: the fields of one problem the limb epilogue reads, in GemmArgs form
__device__ __forceinline__ GemmArgs as_gemm_args(const Prob& p, uint32_t* status) {
    GemmArgs g;
    g.form = OZMP_FORM_FP8;
    g.q = p.q;
    g.is_f32 = p.is_f32;
    g.m = p.m; g.n = p.n; g.k = 0; g.mp = p.mp; g.np = p.np; g.kp = p.kp;
    g.E = p.E; g.F = p.F; g.Adig = nullptr; g.Bdig = nullptr;
    g.s = p.s; g.beta = p.beta; g.eoff = p.eoff; g.ppd = p.ppd; g.group_start = 0; g.acc_words = p.acc_words;
    g.ngroups = 0;
    g.acc = p.acc;
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) g.C[c] = p.C[c];
    g.ldc = p.ldc;
    g.status = status;
    g.d_only = p.d_only;
    g.T = p.T;
    return g;
}

// Work of one CTA: items [off[cta], off[cta + 1]) of `items` (prob, tile);
// without an item list (single problem) tiles cta, cta + G, cta + 2G, ...
// One work item: pairs [pa, pb) (in the walk order) of one tile of one
// problem.  slot < 0: the item is the whole tile; else the tile is split into
// nchunks items that add into split-limb slot `slot`.
struct WorkItem {
    int prob, tile, pa, pb, slot, nchunks;
};

struct Sched {
    const Prob* probs;         // batched mode: one per problem (global memory); else null
    const CUtensorMap* maps;   // batched mode: A and B maps of problem p at 2p, 2p + 1
    const WorkItem* items;     // null: tiles cta, cta + G, ... of the one problem, whole
    const int* off;            // items [off[cta], off[cta + 1]) belong to CTA cta
    int ntiles;                // no item list: tiles of the one problem
    int* counter;              // non-null: items are taken in list order from this counter
    int nitems;                //   (zeroed before the launch) instead of the per-CTA lists
    long long wait_limit;      // polls before a wait gives up (0: WAIT_LIMIT)
    int inject_stall;          // test hook: never load the first stage of each CTA's first item
    int kind;                  // digit type of every problem of the launch (Prob::kind)
    int snake;                 // pair order (walk.h): 1 the snake, 0 one diagonal at a time
    // loose lockstep of the clusters' pair walks (null: off): step_done[P]
    // counts the clusters that issued their P-th whole-tile pair, retired the
    // clusters without whole tiles left; before pair P a leader waits a
    // bounded time until step_done[P - lock_w] + retired covers every cluster
    int* step_done;
    int* retired;
    int lock_w, lock_n;
};

// polls of one lockstep wait before the producer goes on regardless
constexpr int LOCK_POLLS = 160;

// Dynamic item feed: the leader's producer takes the next item index from the
// global counter and publishes it through a ring of RING slots (in both CTAs
// of a pair); every other role reads it from its own CTA's ring and releases
// the slot on the leader's `ring_empty` barrier.
constexpr int RING = 4;
// slot releases per ring entry: the leader's MMA issuer and 4 epilogue warps,
// plus the peer's producer and 4 epilogue warps in the pair form
__host__ __device__ constexpr unsigned ring_consumers(int cg) { return cg == 2 ? 10u : 5u; }

struct Item {
    const Prob* p;
    const CUtensorMap* ma;
    const CUtensorMap* mb;
    int64_t i0, j0;
    int KT, dhi, dlo, bn;
    int pa, pb, slot, nchunks;
};

// pairs of the walk d = dhi .. dlo, t = 1 .. d-1
__host__ __device__ __forceinline__ int walk_pairs(int dhi, int dlo) {
    return (dhi - dlo + 1) * (dlo - 1 + dhi - 1) / 2;
}

// CG = 2: the tile index counts 256-row tiles of the pair; this CTA (rank)
// owns rows rank * 128 .. + 127 of it
template <int CG = 1>
__device__ __forceinline__ bool item_at(const Sched& sc, const Prob* single, const CUtensorMap* ma,
                                        const CUtensorMap* mb, int idx, Item& it, uint32_t rank = 0) {
    int pi, tile;
    if (sc.items) {
        const WorkItem w = sc.items[idx];
        pi = w.prob;
        tile = w.tile;
        it.pa = w.pa;
        it.pb = w.pb;
        it.slot = w.slot;
        it.nchunks = w.nchunks;
        it.p = sc.probs ? &sc.probs[pi] : single;
        it.ma = sc.probs ? &sc.maps[2 * pi] : ma;
        it.mb = sc.probs ? &sc.maps[2 * pi + 1] : mb;
    } else {
        tile = idx;
        it.p = single;
        it.ma = ma;
        it.mb = mb;
        it.pa = 0;
        it.pb = -1;   // set below
        it.slot = -1;
        it.nchunks = 1;
    }
    const Prob& p = *it.p;
    const int tm = (int)(p.mp / (BM * CG));
    it.i0 = (int64_t)(tile % tm) * (BM * CG) + (int64_t)rank * BM;
    it.j0 = (int64_t)(tile / tm) * p.bn;
    it.KT = (int)(p.kp / BK);
    it.dhi = p.d_only ? p.d_only : p.s + 1;
    it.dlo = p.d_only ? p.d_only : 2;
    it.bn = p.bn;
    if (it.pb < 0) it.pb = walk_pairs(it.dhi, it.dlo);
    return true;
}

}  // namespace tc

// host helpers shared by the launches (gemm_tc.cu)
bool tc_make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t kp, uint32_t box_rows);
int tc_num_sms();
// launch of the tcgen05 product kernel: `grid` CTAs over the schedule; in
// single-problem mode (sc.items == nullptr) `single`, `ma`, `mb` describe it
cudaError_t tc_launch(const tc::Sched& sc, const tc::Prob& single, const CUtensorMap& ma, const CUtensorMap& mb,
                      uint32_t* status, int grid, cudaStream_t st);
cudaError_t tc_set_smem();
// the rounding pass over the limbs (tc_finish_lo.cu / tc_finish_hi.cu)
cudaError_t launch_tc_finish_lo(const GemmArgs& g, int nl, const int* ts, int rows, int slot_limbs, cudaStream_t st);
cudaError_t launch_tc_finish_hi(const GemmArgs& g, int nl, const int* ts, int rows, int slot_limbs, cudaStream_t st);
// the CTA-pair form: `clusters` clusters of two CTAs over the schedule
cudaError_t tc_launch_pair(const tc::Sched& sc, const tc::Prob& single, const CUtensorMap& ma,
                           const CUtensorMap& mb, uint32_t* status, int clusters, cudaStream_t st);

}  // namespace ozmp
