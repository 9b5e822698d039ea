// Single-problem launch of the tcgen05 e4m3 slice-product kernel (the
// kernel itself is in gemm_tc_impl.cuh) and the tensor-map helpers.
#include <type_traits>
#include <vector>
#include "gemm_tc_impl.cuh"

namespace ozmp {
namespace tc {

// Items come from the per-CTA lists of the schedule, from a fixed stride over
// the tiles, or (sc.counter set) from the dynamic feed, so that CTAs that run
// faster take more items.
// CG = 1: one CTA per 128 x bn tile.  CG = 2: a cluster of two CTAs per
// 256 x 256 tile, one tcgen05.mma.cta_group::2 (M = 256) issued by the leader
// (rank 0) reading both CTAs' shared memory; the leader's full barrier counts
// the bytes of both CTAs' copies, its MMA commits release the stage and the
// accumulator in both CTAs, and both CTAs' epilogues release the accumulator
// on the leader's barrier.
template <int CG>
__global__ void __launch_bounds__(NT, 1) k_gemm_tc(const Sched sc, const __grid_constant__ Prob single,
                                                    const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, uint32_t* status) {
    constexpr int NS = CG == 2 ? NST2 : NST;
    constexpr unsigned SB = CG == 2 ? STAGE_B2 : STAGE_B;   // bytes of B staged per CTA
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;
    unsigned char* sB = base + (size_t)NS * STAGE_A;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)NS * SB);
    uint64_t* empty = full + NS;
    uint64_t* accf = empty + NS;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint64_t* ring_full = done + 1;
    uint64_t* ring_empty = ring_full + RING;
    volatile int* ring = reinterpret_cast<volatile int*>(ring_empty + RING);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ring_empty + RING) + RING;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* fin_flag = reinterpret_cast<volatile int*>(tmem_slot + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = CG == 2 ? cluster_rank() : 0u;
    const long long WL = sc.wait_limit > 0 ? sc.wait_limit : WAIT_LIMIT;   // polls before a wait gives up
    const long long DL = WL < DRAIN_LIMIT ? WL : DRAIN_LIMIT;               // ... for work already in flight
    const int cid = CG == 2 ? (int)cluster_id_x() : (int)blockIdx.x;
    const int ncl = CG == 2 ? (int)cluster_count_x() : (int)gridDim.x;
    // the leader's full and acc-empty barriers, and the peer's abort flag
    const uint32_t full_cl = CG == 2 ? map_rank(saddr(full), 0) : saddr(full);
    const uint32_t acce_cl = CG == 2 ? map_rank(saddr(acce), 0) : saddr(acce);
    const uint32_t peer_abort = CG == 2 ? map_rank(saddr((const void*)abort_flag), rank ^ 1u) : 0u;
    auto raise_abort = [&]() {
        *abort_flag = 1;
        if (CG == 2) st_cluster_u32(peer_abort, 1u);
        atomicOr(status, ST_TIMEOUT);
    };

    // ---- item feed: the k-th item of this CTA; -1 past the end, -2 on timeout
    const bool dyn = sc.counter != nullptr;
    int it_begin, it_end, it_step;
    if (sc.items) { it_begin = dyn ? 0 : sc.off[cid]; it_end = dyn ? 0 : sc.off[cid + 1]; it_step = 1; }
    else { it_begin = cid; it_end = sc.ntiles; it_step = ncl; }
    const uint32_t ring_empty_cl = CG == 2 ? map_rank(saddr(ring_empty), 0) : saddr(ring_empty);
    const uint32_t peer_ring = CG == 2 ? map_rank(saddr((const void*)ring), 1) : 0u;
    const uint32_t peer_ring_full = CG == 2 ? map_rank(saddr(ring_full), 1) : 0u;
    auto take = [&](int k, bool publisher, bool warp_wide) -> int {
        if (!dyn) {
            const int idx = it_begin + k * it_step;
            return idx < it_end ? idx : -1;
        }
        const int r = k % RING;
        const unsigned ph = (unsigned)((k / RING) & 1);
        if (publisher) {
            if (!mbar_wait<CG == 2>(&ring_empty[r], ph ^ 1u, abort_flag, WL)) return -2;
            const int idx = atomicAdd(sc.counter, 1);
            ring[r] = idx;
            if (CG == 2) {
                st_cluster_u32(peer_ring + 4u * r, (uint32_t)idx);
                mbar_arrive_cluster(peer_ring_full + 8u * r);   // release: the store is visible first
            }
            mbar_arrive(&ring_full[r]);
            return idx < sc.nitems ? idx : -1;
        }
        // a warp-wide caller waits in lane 0 and broadcasts, so that the lanes
        // cannot part on a timeout
        int idx = -2;
        if (!warp_wide || lane == 0) {
            if (mbar_wait<CG == 2>(&ring_full[r], ph, abort_flag, WL)) {
                idx = ring[r];
                if (CG == 2) mbar_arrive_cluster(ring_empty_cl + 8u * r);
                else mbar_arrive(&ring_empty[r]);
            }
        }
        if (warp_wide) idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx == -2) return -2;
        return idx < sc.nitems ? idx : -1;
    };

    if (threadIdx.x == 0) {
        for (int x = 0; x < NS; ++x) { mbar_init(&full[x], 1); mbar_init(&empty[x], 1); }
        for (int x = 0; x < 2; ++x) { mbar_init(&accf[x], 1); mbar_init(&acce[x], 4 * CG); }
        mbar_init(done, 1);
        for (int x = 0; x < RING; ++x) { mbar_init(&ring_full[x], 1); mbar_init(&ring_empty[x], ring_consumers(CG)); }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 1) {
        if (CG == 2) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
                             saddr(tmem_slot))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
                             saddr(tmem_slot))
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CG == 2) cluster_sync();   // the peer's barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            long long n = 0;
            bool ok = true;
            // lockstep (the leader's producer of each cluster): whole-tile pairs issued so far
            const bool lock = sc.step_done != nullptr && rank == 0;
            long long P = 0;
            bool gone = false;
            for (int k = 0; ok; ++k) {
                const int idx = take(k, rank == 0, false);
                if (idx == -2) { ok = false; break; }
                if (idx < 0) break;
                Item it;
                item_at<CG>(sc, &single, &tmA, &tmB, idx, it, rank);
                const Prob p = *it.p;
                const unsigned tx = CG == 2 ? 2u * (STAGE_A + SB) : STAGE_A + (unsigned)it.bn * BK;
                const int jb = (int)it.j0 + (CG == 2 ? (int)rank * (BN / 2) : 0);
                const bool whole = it.pa == 0 && it.pb == p.s * (p.s + 1) / 2;
                if (lock && !whole && !gone) { atomicAdd(sc.retired, 1); gone = true; }
                PairWalk w;
                w.start(it.dhi, it.dlo, p.ppd, it.pa, it.pb, sc.snake, 0);   // (the accumulators do not matter here)
                for (int pi = it.pa; ok && pi < it.pb; ++pi) {
                    const PairStep ps = w.step();
                    if (lock && whole && P >= sc.lock_w && P - sc.lock_w < sc.lock_n) {
                        // soft: after LOCK_POLLS polls the walk goes on regardless
                        const volatile int* dp = sc.step_done + (P - sc.lock_w);
                        const volatile int* rp = sc.retired;
                        for (int x = 0; x < LOCK_POLLS && *dp + *rp < ncl; ++x) __nanosleep(128);
                    }
                    const int ya = (ps.t - 1) * (int)p.mp + (int)it.i0;
                    const int yb = (ps.u - 1) * (int)p.np + jb;
                    for (int kc = 0; kc < it.KT; ++kc, ++n) {
                        const int st = (int)(n % NS);
                        const unsigned ph = (unsigned)((n / NS) & 1);
                        if (!mbar_wait<CG == 2>(&empty[st], ph ^ 1u, abort_flag, WL)) { ok = false; break; }
                        // test hook: the first stage of this CTA's first item is never loaded
                        // (its full barrier is never completed), so the waits on it run out
                        if (sc.inject_stall && k == 0 && pi == it.pa && kc == 0) continue;
                        if (rank == 0) mbar_expect_tx(&full[st], tx);
                        if (CG == 2) {
                            tma_load_2d_pair(sA + (size_t)st * STAGE_A, it.ma, full_cl + 8u * st, kc * BK, ya);
                            tma_load_2d_pair(sB + (size_t)st * SB, it.mb, full_cl + 8u * st, kc * BK, yb);
                        } else {
                            tma_load_2d(sA + (size_t)st * STAGE_A, it.ma, &full[st], kc * BK, ya);
                            tma_load_2d(sB + (size_t)st * SB, it.mb, &full[st], kc * BK, yb);
                        }
                    }
                    if (lock && whole) {
                        if (P < sc.lock_n) atomicAdd(sc.step_done + P, 1);
                        ++P;
                    }
                }
            }
            if (lock && !gone) atomicAdd(sc.retired, 1);
            if (!ok) {
                raise_abort();
                // let the copies already issued land before the CTA can exit (the
                // leader's full barrier counts the copies of both CTAs)
                if (rank == 0) {
                    volatile int never = 0;
                    for (long long q = n - 1; q >= 0 && q >= n - NS; --q)
                        mbar_wait<CG == 2>(&full[(int)(q % NS)], (unsigned)((q / NS) & 1), &never, DL);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer (the leader's)
        if (lane == 0 && rank == 0) {
            // the digit type is the same for every item of a launch: one issue loop
            // per type, so that no MMA of the loop waits on a branch
            auto issue = [&](auto f16_tag) {
                constexpr bool F16 = decltype(f16_tag)::value;
                long long n = 0;
                int uses[2] = {0, 0};   // groups closed so far in each accumulator
                int nb = 0;             // accumulator of the next item's first pair
                bool ok = true;
                for (int k = 0; ok; ++k) {
                    const int idx = take(k, false, false);
                    if (idx == -2) { ok = false; break; }
                    if (idx < 0) break;
                    Item it;
                    item_at<CG>(sc, &single, &tmA, &tmB, idx, it, rank);
                    const Prob p = *it.p;
                    const uint32_t idesc = idesc_e4m3(BM * CG, it.bn);
                    PairWalk w;
                    w.start(it.dhi, it.dlo, p.ppd, it.pa, it.pb, sc.snake, nb);
                    for (int pi = it.pa; ok && pi < it.pb; ++pi) {
                        const PairStep ps = w.step();
                        const int buf = ps.buf;
                        nb = buf ^ 1;
                        // a group's first MMA waits until the epilogues have released the
                        // accumulator's previous group (the k-th use waits for the (k-1)-th release)
                        if (ps.open && !mbar_wait<CG == 2>(&acce[buf], (unsigned)((uses[buf] & 1) ^ 1), abort_flag, WL)) {
                            ok = false;
                            break;
                        }
                        bool fresh = ps.open;
                        const uint32_t dcol = tmem + (uint32_t)(buf * BN);
                        for (int kc = 0; kc < it.KT; ++kc, ++n) {
                            const int st = (int)(n % NS);
                            const unsigned ph = (unsigned)((n / NS) & 1);
                            if (!mbar_wait<CG == 2>(&full[st], ph, abort_flag, WL)) { ok = false; break; }
                            tc_fence_after();
                            const uint64_t ad = desc_sw128(saddr(sA + (size_t)st * STAGE_A));
                            const uint64_t bd = desc_sw128(saddr(sB + (size_t)st * SB));
#pragma unroll
                            for (int kk = 0; kk < BK / 32; ++kk) {
                                // 32 bytes of K per MMA: 32 e4m3 or 16 binary16 digits
                                const uint32_t acc = (fresh && kk == 0) ? 0u : 1u;
                                const uint64_t a2 = ad + (uint64_t)(2 * kk), b2 = bd + (uint64_t)(2 * kk);
                                if constexpr (F16) {
                                    if (CG == 2) mma_f16_tc_pair(dcol, a2, b2, idesc, acc);
                                    else mma_f16_tc(dcol, a2, b2, idesc, acc);
                                } else {
                                    if (CG == 2) mma_e4m3_tc_pair(dcol, a2, b2, idesc, acc);
                                    else mma_e4m3_tc(dcol, a2, b2, idesc, acc);
                                }
                            }
                            fresh = false;
                            if (CG == 2) mma_commit_pair(&empty[st]);
                            else mma_commit(&empty[st]);
                        }
                        if (!ok) break;
                        if (ps.close) {
                            if (CG == 2) mma_commit_pair(&accf[buf]);
                            else mma_commit(&accf[buf]);
                            uses[buf]++;
                        }
                    }
                }
                if (!ok) raise_abort();
                // every issued MMA (into both CTAs' tensor memory) has completed
                // before the pair passes the final cluster barrier
                if (CG == 2) mma_commit_local_pair(done);
                else mma_commit(done);
                volatile int never = 0;
                mbar_wait<CG == 2>(done, 0u, &never, DL);
            };
            if (sc.kind) issue(std::true_type{});
            else issue(std::false_type{});
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        int drains[2] = {0, 0};   // groups drained so far from each accumulator
        int nb = 0;               // accumulator of the next item's first pair
        bool ok = true;
        for (int k = 0; ok; ++k) {
            const int idx = take(k, false, true);
            if (idx == -2) { ok = false; break; }
            if (idx < 0) break;
            Item it;
            item_at<CG>(sc, &single, &tmA, &tmB, idx, it, rank);
            const Prob p = *it.p;
            const GemmArgs g = as_gemm_args(p, status);
            const int64_t i = it.i0 + quarter * 32 + lane;
            const int ii = quarter * 32 + lane;
            const size_t plane = (size_t)p.mp * p.np;
            const int nl = 4 * p.acc_words + 1;
            const bool split = it.slot >= 0;
            const int slot = it.slot * CG + (int)rank;   // split-limb slot of this CTA's rows
            // split tiles: limb l of tile column jj, row ii at sbase[l * sstride + jj * BM + ii]
            const size_t sstride = (size_t)it.bn * BM;
            int64_t* sbase = split ? p.sacc + (size_t)slot * nl * sstride : nullptr;
            PairWalk w;
            w.start(it.dhi, it.dlo, p.ppd, it.pa, it.pb, sc.snake, nb);
            // limbs of this tile written so far (whole tiles): bit l set once limb l has
            // been stored, so that a drain stores a limb's first value and adds to it after
            uint64_t touched = 0;
            for (int pi = it.pa; ok && pi < it.pb; ++pi) {
                const PairStep ps = w.step();
                nb = ps.buf ^ 1;
                if (ps.close) {
                    // the last drain rounds the tile into C unless a separate pass does
                    const bool last = (pi == it.pb - 1) && !p.defer;
                    const int buf = ps.buf;
                    const unsigned par = (unsigned)(drains[buf] & 1);
                    ++drains[buf];
                    int got = 0;
                    if (lane == 0) got = mbar_wait<CG == 2>(&accf[buf], par, abort_flag, WL) ? 1 : 0;
                    if (!__shfl_sync(0xffffffffu, got, 0)) { ok = false; break; }
                    __syncwarp();
                    tc_fence_after();
                    const int fsh = p.d_only ? 0 : p.beta * (p.s + 1 - ps.d);
                    const int li = fsh >> 4, off = fsh & 15;
                    const int nchunk = it.bn / 32;
#pragma unroll 1
                    for (int c = 0; c < nchunk; ++c) {
                        uint32_t r[32];
                        tmem_ld32(tmem + lane_base + (uint32_t)(buf * BN + c * 32), r);
                        if (c == nchunk - 1) {
                            // the accumulator buffer is free once its last columns are in registers
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) {
                                if (CG == 2) mbar_arrive_cluster(acce_cl + 8u * buf);
                                else mbar_arrive(&acce[buf]);
                            }
                        }
                        const int64_t jb = it.j0 + c * 32;
                        if (split) {
                            // exact, order-independent: add into the tile's shared limbs
                            unsigned long long* lp = (unsigned long long*)(sbase + li * sstride + (size_t)(c * 32) * BM + ii);
#pragma unroll
                            for (int x = 0; x < 32; ++x) {
                                const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                                atomicAdd(lp + (size_t)x * BM, (unsigned long long)((uint64_t)v << off));
                            }
                        } else if (last) {
                            // the limbs in `touched` hold data; this drain's adds into limb li
                            const int nlt = touched ? 64 - __clzll((long long)touched) : 0;
#pragma unroll 1
                            for (int x = 0; x < 32; ++x) {
                                const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                                finish_dispatch(g, nlt, p.acc, plane, (size_t)(jb + x) * p.mp + i, i, jb + x,
                                                (int64_t)((uint64_t)v << off), li, touched == 0, touched);
                            }
                        } else if (!((touched >> li) & 1)) {
                            // first touch of this limb: store (in the snake a drain may reach a
                            // limb before the drain of the diagonal above it does, so the
                            // written limbs are tracked one by one)
#pragma unroll
                            for (int x = 0; x < 32; ++x) {
                                const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                                p.acc[li * plane + (size_t)(jb + x) * p.mp + i] = (int64_t)((uint64_t)v << off);
                            }
                        } else {
                            int64_t cur[32];
#pragma unroll
                            for (int x = 0; x < 32; ++x) cur[x] = p.acc[li * plane + (size_t)(jb + x) * p.mp + i];
#pragma unroll
                            for (int x = 0; x < 32; ++x) {
                                const int64_t v = (int64_t)__float2int_rn(__uint_as_float(r[x]));
                                p.acc[li * plane + (size_t)(jb + x) * p.mp + i] = cur[x] + (int64_t)((uint64_t)v << off);
                            }
                        }
                    }
                    touched |= 1ull << li;
                    if (split && last) {
                        // the last chunk of the tile to finish rounds it: publish this chunk's
                        // additions, count it, and let the finisher read every chunk's
                        __threadfence();
                        asm volatile("bar.sync 1, 128;\n" ::: "memory");
                        if (warp == 2 && lane == 0) *fin_flag = atomicAdd(&p.cnt[slot], 1) == it.nchunks - 1;
                        asm volatile("bar.sync 1, 128;\n" ::: "memory");
                        if (*fin_flag) {
                            __threadfence();
#pragma unroll 1
                            for (int jj = 0; jj < it.bn; ++jj)
                                finish_dispatch(g, nl, sbase, sstride, (size_t)jj * BM + ii, i, it.j0 + jj, 0, 0,
                                                false);
                        }
                        asm volatile("bar.sync 1, 128;\n" ::: "memory");
                    }
                }
            }
        }
        if (!ok) raise_abort();
    }

    tc_fence_before();
    __syncthreads();
    if (CG == 2) cluster_sync();   // no MMA, copy or remote arrive of either CTA is outstanding
    tc_fence_after();
    if (warp == 1) {
        if (CG == 2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem) : "memory");
    }
    if (CG == 2) cluster_sync();
}

}  // namespace tc

cudaError_t tc_set_smem() {
    cudaError_t e = cudaFuncSetAttribute(tc::k_gemm_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tc::k_gemm_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM2);
}

cudaError_t tc_launch(const tc::Sched& sc, const tc::Prob& single, const CUtensorMap& ma, const CUtensorMap& mb,
                      uint32_t* status, int grid, cudaStream_t st) {
    if (grid <= 0) return cudaSuccess;
    tc::k_gemm_tc<1><<<grid, tc::NT, tc::SMEM, st>>>(sc, single, ma, mb, status);
    return cudaGetLastError();
}

cudaError_t tc_launch_pair(const tc::Sched& sc, const tc::Prob& single, const CUtensorMap& ma,
                           const CUtensorMap& mb, uint32_t* status, int clusters, cudaStream_t st) {
    if (clusters <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(2 * clusters), 1, 1);
    cfg.blockDim = dim3(tc::NT, 1, 1);
    cfg.dynamicSmemBytes = tc::SMEM2;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc::k_gemm_tc<2>, sc, single, ma, mb, status);
}

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
bool tc_make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t kp, uint32_t box_rows) {
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

int tc_schedule(int ntiles, int pairs, int sms, int* items, int* off, int* nitems, int* nslots, bool regroup,
                int tm, int group, int maxc) {
    if (maxc < 1 || maxc > TC_MAX_CHUNKS) maxc = TC_MAX_CHUNKS;
    if (sms < 1) sms = 1;
    // tile order: bands of `group` row tiles, column by column within a band
    // (group <= 0: plain column-major order of the tiles)
    std::vector<int> order(ntiles);
    if (group > 0 && tm > 0 && ntiles % tm == 0) {
        const int tn = ntiles / tm;
        int x = 0;
        for (int i0 = 0; i0 < tm; i0 += group)
            for (int j = 0; j < tn; ++j)
                for (int i = i0; i < i0 + group && i < tm; ++i) order[x++] = i + tm * j;
    } else {
        for (int t = 0; t < ntiles; ++t) order[t] = t;
    }
    const int waves = ntiles / sms, r = ntiles % sms;
    // chunks per tail tile: minimise waves + ceil(r c / sms) / c (+ a small per-chunk cost)
    int best_c = 1;
    double best = 1e30;
    for (int c = 1; c <= maxc && c <= pairs; ++c) {
        if (r == 0 && c > 1) break;
        const double span = waves + (r ? (double)((r * c + sms - 1) / sms) / c : 0.0) + 0.002 * c;
        if (span < best - 1e-9) { best = span; best_c = c; }
    }
    const int c = r ? best_c : 1;
    const int grid = waves > 0 ? sms : (r * c < sms ? r * c : sms);
    std::vector<std::vector<int>> per(grid);
    int n = 0, slots = 0;
    auto put = [&](int cta, int tile, int pa, int pb, int slot, int nch) {
        int* w = items + 6 * n;
        w[0] = 0; w[1] = tile; w[2] = pa; w[3] = pb; w[4] = slot; w[5] = nch;
        per[cta].push_back(n++);
    };
    for (int t = 0; t < waves * sms; ++t) put(t % sms, order[t], 0, pairs, -1, 1);
    int next = 0;
    for (int t = waves * sms; t < ntiles; ++t) {
        if (c == 1) { put(next, order[t], 0, pairs, -1, 1); next = (next + 1) % grid; continue; }
        const int slot = slots++;
        for (int x = 0; x < c; ++x) {
            const int pa = (int)((int64_t)pairs * x / c), pb = (int)((int64_t)pairs * (x + 1) / c);
            put(next, order[t], pa, pb, slot, c);
            next = (next + 1) % grid;
        }
    }
    if (!regroup) {
        // one list in creation order (whole tiles, then the chunks of the tail
        // tiles) for the dynamic feed; the CTA offsets are left unused
        for (int cta = 0; cta <= grid; ++cta) off[cta] = 0;
        *nitems = n;
        *nslots = slots;
        return grid;
    }
    // items regrouped per CTA
    std::vector<int> tmp(items, items + 6 * n);
    int pos = 0;
    for (int cta = 0; cta < grid; ++cta) {
        off[cta] = pos;
        for (int id : per[cta]) {
            for (int f = 0; f < 6; ++f) items[6 * pos + f] = tmp[6 * id + f];
            ++pos;
        }
    }
    off[grid] = pos;
    *nitems = n;
    *nslots = slots;
    return grid;
}

int tc_num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    }
    return sms;
}

// clusters of two CTAs of the pair form that can be resident at once (an SM
// left over in a GPC with an odd number of free SMs cannot host one)
int tc_num_pair_slots() {
    static int slots = 0;
    if (!slots) {
        int n = 0;
        if (tc_set_smem() == cudaSuccess) {
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3(2 * (unsigned)tc_num_sms(), 1, 1);
            cfg.blockDim = dim3(tc::NT, 1, 1);
            cfg.dynamicSmemBytes = tc::SMEM2;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&n, tc::k_gemm_tc<2>, &cfg) != cudaSuccess) n = 0;
        }
        cudaGetLastError();
        slots = n > 0 ? n : (tc_num_sms() / 2 > 0 ? tc_num_sms() / 2 : 1);
    }
    return slots;
}

cudaError_t launch_gemm_tc(const GemmArgs& g, cudaStream_t st) {
    // binary16 digits take two bytes: the maps and the K steps count bytes
    const int kind = g.form == OZMP_FORM_FP16 ? 1 : 0;
    const int64_t kpb = g.kp * (kind ? 2 : 1);
    if (g.mp % tc::BM || g.np % tc::BN || kpb % tc::BK) return cudaErrorInvalidValue;
    const int cg = (g.tc_cg == 2 && g.mp % (2 * tc::BM) == 0) ? 2 : 1;
    if (g.tc_cg == 2 && cg != 2) return cudaErrorInvalidValue;   // the schedule counts pair tiles
    CUtensorMap ma, mb;
    if (!tc_make_map(&ma, g.Adig, (uint64_t)g.s * g.mp, (uint64_t)kpb, tc::BM)) return cudaErrorInvalidValue;
    if (!tc_make_map(&mb, g.Bdig, (uint64_t)g.s * g.np, (uint64_t)kpb, tc::BN / cg)) return cudaErrorInvalidValue;
    cudaError_t e = tc_set_smem();
    if (e != cudaSuccess) return e;
    tc::Prob p;
    memset(&p, 0, sizeof(p));
    p.E = g.E; p.F = g.F; p.acc = g.acc;
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) p.C[c] = g.C[c];
    p.T = g.T;
    p.m = g.m; p.n = g.n; p.mp = g.mp; p.np = g.np; p.kp = kpb; p.ldc = g.ldc;
    p.kind = kind;
    p.q = g.q; p.is_f32 = g.is_f32; p.s = g.s; p.beta = g.beta; p.ppd = g.ppd; p.acc_words = g.acc_words;
    p.eoff = g.eoff;
    p.bn = tc::BN;
    p.d_only = g.d_only;
    p.sacc = g.sacc;
    p.cnt = g.cnt;
    p.defer = 1;
    tc::Sched sc;
    memset(&sc, 0, sizeof(sc));
    sc.probs = nullptr;
    sc.maps = nullptr;
    sc.items = (const tc::WorkItem*)g.sched_items;
    sc.off = g.sched_off;
    sc.ntiles = (int)((g.mp / (tc::BM * cg)) * (g.np / tc::BN));
    sc.counter = sc.items ? g.counter : nullptr;
    sc.nitems = g.sched_nitems;
    sc.wait_limit = g.wait_limit;
    sc.inject_stall = g.inject_stall;
    sc.kind = kind;
    sc.snake = g.tc_snake;
    sc.step_done = (sc.counter && g.lock_w > 0) ? g.step_done : nullptr;
    sc.retired = g.retired;
    sc.lock_w = g.lock_w;
    sc.lock_n = g.lock_n;
    if (sc.items && g.split_bytes) {
        // split limbs, chunk counters and the feed counter are one region
        e = cudaMemsetAsync(g.sacc ? (void*)g.sacc : (void*)g.cnt_region, 0, g.split_bytes, st);
        if (e != cudaSuccess) return e;
    }
    const int grid = sc.items ? g.sched_grid : sc.ntiles;
    if (g.tev_start) cudaEventRecord(g.tev_start, st);
    e = cg == 2 ? tc_launch_pair(sc, p, ma, mb, g.status, grid, st) : tc_launch(sc, p, ma, mb, g.status, grid, st);
    if (g.tev_stop) cudaEventRecord(g.tev_stop, st);
    if (e != cudaSuccess) return e;
    // the rounding pass: limbs 0 .. (beta (s - 1)) / 16 hold data (the last drain's shift)
    const int nl = g.d_only ? 1 : (g.beta * (g.s - 1)) / 16 + 1;
    const int slot_limbs = 4 * g.acc_words + 1;
    const int* ts = sc.items ? g.tile_slot : nullptr;
    const int rows = tc::BM * cg;
    if (g.acc_words < 2 || g.acc_words > 16) return cudaErrorInvalidValue;
    e = g.acc_words <= 8 ? launch_tc_finish_lo(g, nl, ts, rows, slot_limbs, st)
                         : launch_tc_finish_hi(g, nl, ts, rows, slot_limbs, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace ozmp
