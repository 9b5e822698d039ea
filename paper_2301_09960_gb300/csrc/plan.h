// Internal plan descriptor and its host-side scheduling helpers (not part
// of the C ABI): digit width, slice count, drain/group schedule, workspace
// layout and the launch descriptors built from a plan.
#pragma once
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include "bound.cuh"
#include "kernels.h"
#include "ozmp_internal.cuh"

struct ozmp_plan_s {
    int prec, q, is_f32, form;
    int64_t m, n, k, mp, np, kp;
    int s, beta, db;
    int ppd;
    uint64_t group_start;
    int ngroups, acc_words;
    int nlimbs;   // carry-save limbs of the tcgen05 epilogue (FORM_FP8)
    size_t ws_bytes, off_E, off_F, off_status, off_Adig, off_Bdig, off_acc;
    void* ws;
    bool ws_owned;
    cudaStream_t stream;
    void* batch;   // batched plan data (ozmp_gemm_batched), else null
    // tcgen05 tile schedule (plans made by ozmp_plan_create): host copy, sizes,
    // workspace regions, and the workspace it was last uploaded to
    int* sched_host;
    int sched_items, sched_slots, sched_grid;   // sched_slots: split-limb slots of single CTAs
    int tc_cg;                                   // 2: the schedule is over CTA-pair tiles
    int tc_dyn;                                  // items taken from a counter (else per-CTA lists)
    int big;                                     // the many-component splitter (q > 4 or wide windows)
    int bal;                                     // balanced radix-32 e4m3 digits (FORM_FP8_BAL, beta = 5)
    // tcgen05 form, for tests of the bounded waits (OZMP_TC_WAIT_LIMIT, OZMP_TC_INJECT_STALL)
    long long tc_wait_limit;
    int tc_inject_stall;
    // one-pass column splitter, the same test hooks (OZMP_SPLIT_WAIT_LIMIT, OZMP_SPLIT_INJECT_STALL)
    long long split_wait_limit;
    int split_inject_stall;
    // kernel timing ring (ozmp_plan_set_timing): tev[2 x] / tev[2 x + 1] around call x mod tev_n
    cudaEvent_t* tev;
    int tev_n;
    long long tev_calls;
    size_t off_items, off_soff, off_tslot, off_sacc, split_bytes;
    int sched_ntiles;
    void* sched_ws;
    // error bound (bound.cu): statistics region, per-column norms of A and
    // per-row norms of B (both k doubles), at offsets that depend on m, n, k only
    size_t off_stats, off_colA, off_rowB, off_rowBf;
    int target_bits;   // the precision's normwise target 2^-target_bits
    int adapt;         // s chosen from the data at every execution (nslices = 0 at creation)
    int check;         // a-posteriori bound check after every execution
    int s_lo, s_cap;   // adaptive plans: the slice counts the reserved workspace holds
    size_t ws_cap;     // bytes of the current workspace
    // schedule knobs, read from the environment once (OZMP_TC_PAIR, OZMP_TC_DYNAMIC,
    // OZMP_TC_GROUP, OZMP_TC_MAX_CHUNKS, OZMP_TC_LOCKSTEP, OZMP_TC_WALK) and kept
    // when the plan is re-made for another s
    int env_read, env_pair_off, env_static, env_group, env_maxc, env_lock, env_walk;
    // adaptive plans: pinned host word of the chosen s and the event after its copy
    int* host_s;
    cudaEvent_t ev_s;
};

namespace ozmp_batch {
void destroy(void* b);
}

namespace ozmp_plan_detail {
using namespace ozmp;

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int64_t roundup(int64_t x, int64_t r) { return (x + r - 1) / r * r; }

// components of a precision: q for q binary64 words (2 <= q <= 16), 3 for TS
inline int prec_q(int prec) {
    if (prec == OZMP_TS) return 3;
    if (prec >= 2 && prec <= OZMP_MAX_COMPONENTS) return prec;
    return 0;
}

// target error bits of each precision: 50 q for q binary64 words (2^-100 DD,
// 2^-150 TD, 2^-200 QD, ...), 66 for TS
inline int prec_target_bits(int prec) {
    if (prec == OZMP_TS) return 66;
    return 50 * prec_q(prec);
}

inline int ceil_log2(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Largest beta with k (2^beta - 1)^2 <= 2^53: every partial sum of one
// binary64 slice product is then an integer below 2^53 (Algorithm 1's
// requirement that C_{alpha beta} = A_alpha B_beta is error-free).
inline int beta_fp64(int64_t k) {
    if (k <= 0) k = 1;
    int b = 1;
    while (true) {
        unsigned __int128 d = ((unsigned __int128)1 << (b + 1)) - 1;
        if ((unsigned __int128)k * d * d <= ((unsigned __int128)1 << 53)) ++b;
        else break;
        if (b >= 26) break;
    }
    return b;
}

// Largest beta <= 11 with k (2^beta - 1)^2 <= 2^24: a binary32 sum of k
// digit products never rounds, and the digits are exact in binary16
// (integers up to 2048); 0 when even beta = 1 does not fit (k > 2^24).
inline int beta_fp16(int64_t k) {
    if (k <= 0) k = 1;
    int b = 0;
    while (b < 11) {
        const int64_t d = ((int64_t)1 << (b + 1)) - 1;
        if ((unsigned __int128)k * d * d <= ((unsigned __int128)1 << 24)) ++b;
        else break;
    }
    return b;
}

// the tcgen05 engine (carry-save limbs, tile schedule): e4m3 and binary16 digits
inline bool tc_engine(int form) { return form == OZMP_FORM_FP8 || form == OZMP_FORM_FP16; }

inline int bitlen128(unsigned __int128 x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

inline ozmp_status fill_schedule(ozmp_plan_s* p) {
    // largest digit magnitude and the exact-accumulation limit of the engine
    const bool e4m3 = (p->form == OZMP_FORM_FP8 || p->form == OZMP_FORM_FP8_MMA);
    uint64_t dmax = p->bal ? 16u : e4m3 ? 15u : ((1u << p->beta) - 1u);
    unsigned __int128 limit = (e4m3 || p->form == OZMP_FORM_FP16) ? ((unsigned __int128)1 << 24)
                            : (p->form == OZMP_FORM_INT8) ? (unsigned __int128)2147483647u
                            : ((unsigned __int128)1 << 53);
    int64_t kk = p->k > 0 ? p->k : 1;
    unsigned __int128 tpair = (unsigned __int128)kk * dmax * dmax;   // bound of one slice product entry
    if (tpair > limit) return OZMP_ERR_UNSUPPORTED;
    unsigned __int128 ppd = limit / tpair;
    p->ppd = ppd > (unsigned __int128)(1 << 20) ? (1 << 20) : (int)ppd;
    // diagonal groups: H = sum_{d in group} T_d 2^(beta (dfirst - d)) must stay below 2^62
    const unsigned __int128 HLIM = (unsigned __int128)1 << 62;
    p->group_start = 0;
    p->ngroups = 0;
    int dfirst = -1;
    unsigned __int128 hb = 0;
    // (the groups serve the mma.sync forms, whose bit mask holds s <= 64 diagonals;
    // the tcgen05 form keeps carry-save limbs and needs none)
    for (int d = p->s + 1; d >= 2 && p->s <= 64; --d) {
        unsigned __int128 tb = (unsigned __int128)(d - 1) * tpair;
        bool open = (dfirst < 0);
        if (!open) {
            int sh = p->beta * (dfirst - d);
            if (sh >= 62 || bitlen128(tb) + sh >= 126) open = true;
            else {
                unsigned __int128 nb = hb + (tb << sh);
                if (nb >= HLIM) open = true; else hb = nb;
            }
        }
        if (open) {
            if (tb >= HLIM) return OZMP_ERR_UNSUPPORTED;
            dfirst = d;
            hb = tb;
            p->group_start |= (uint64_t)1 << (d - 2);
            p->ngroups++;
        }
    }
    // exact accumulator width: |S| <= sum_d Tb_d 2^(beta (s + 1 - d))
    int maxbits = 0;
    for (int d = 2; d <= p->s + 1; ++d) {
        int b = bitlen128((unsigned __int128)(d - 1) * tpair) + p->beta * (p->s + 1 - d);
        if (b > maxbits) maxbits = b;
    }
    int bits = maxbits + ceil_log2(p->s + 1) + 2;   // sum of s terms, sign bit
    p->acc_words = (bits + 63) / 64;
    if (p->acc_words < 2) p->acc_words = 2;
    if (p->acc_words > (tc_engine(p->form) ? 16 : 7)) return OZMP_ERR_UNSUPPORTED;
    p->nlimbs = 4 * p->acc_words + 1;
    return OZMP_OK;
}

inline void fill_layout(ozmp_plan_s* p) {
    size_t off = 0;
    p->off_E = off; off = align256(off + (size_t)p->mp * 4);
    p->off_F = off; off = align256(off + (size_t)p->np * 4);
    p->off_status = off; off = align256(off + 16);
    const size_t kk = p->k > 0 ? (size_t)p->k : 1;
    p->off_stats = off; off = align256(off + 256);
    p->off_colA = off; off = align256(off + kk * 8);
    p->off_rowB = off; off = align256(off + kk * 8);
    p->off_rowBf = off; off = align256(off + kk * 4);
    p->off_Adig = off; off = align256(off + (size_t)p->s * p->mp * p->kp * p->db);
    p->off_Bdig = off; off = align256(off + (size_t)p->s * p->np * p->kp * p->db);
    p->off_acc = off;
    if (tc_engine(p->form)) off = align256(off + (size_t)p->nlimbs * p->mp * p->np * 8);
    else if (p->ngroups > 1) off = align256(off + (size_t)p->acc_words * p->mp * p->np * 8);
    p->ws_bytes = off;
}

inline ozmp_status ensure_ws(ozmp_plan_s* p) {
    if (p->ws) return OZMP_OK;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, p->ws_bytes ? p->ws_bytes : 256) != cudaSuccess) {
        cudaGetLastError();
        return OZMP_ERR_NOMEM;
    }
    p->ws = ptr;
    p->ws_owned = true;
    p->ws_cap = p->ws_bytes;
    return OZMP_OK;
}

// the digit form of the truncation bound (bound.cuh) of a plan
inline BoundForm bound_form(const ozmp_plan_s* p) {
    BoundForm f;
    f.beta = p->beta;
    f.eo = p->bal ? 1 : 0;
    const bool e4m3 = (p->form == OZMP_FORM_FP8 || p->form == OZMP_FORM_FP8_MMA);
    f.dmax = p->bal ? 16 : (e4m3 ? 15 : (1 << p->beta) - 1);
    f.target = p->target_bits;
    f.uq = ldexp(1.0, 1 - (p->is_f32 ? 24 : 53) * p->q);
    f.k = p->k;
    return f;
}

inline BoundStats* bound_stats(ozmp_plan_s* p) { return (BoundStats*)((char*)p->ws + p->off_stats); }

inline bool ptrs_ok(const void* const* v, int q) {
    if (!v) return false;
    for (int i = 0; i < q; ++i)
        if (!v[i]) return false;
    return true;
}

inline ozmp_status check_ld(const ozmp_plan_s* p, int64_t lda, int64_t ldb, int64_t ldc, bool need_c) {
    int64_t m1 = p->m > 1 ? p->m : 1, k1 = p->k > 1 ? p->k : 1;
    if (lda < m1 || ldb < k1) return OZMP_ERR_INVALID_ARG;
    if (need_c && ldc < m1) return OZMP_ERR_INVALID_ARG;
    return OZMP_OK;
}

inline SplitArgs split_args(ozmp_plan_s* p, const void* const* A, int64_t lda, const void* const* B, int64_t ldb) {
    SplitArgs a;
    memset(&a, 0, sizeof(a));
    a.form = p->form;
    a.q = p->q;
    a.is_f32 = p->is_f32 != 0;
    a.m = p->m; a.n = p->n; a.k = p->k;
    a.mp = p->mp; a.np = p->np; a.kp = p->kp;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
    char* w = (char*)p->ws;
    a.E = (int32_t*)(w + p->off_E);
    a.F = (int32_t*)(w + p->off_F);
    a.status = (uint32_t*)(w + p->off_status);
    a.wait_limit = p->split_wait_limit;
    a.inject_stall = p->split_inject_stall;
    a.Adig = w + p->off_Adig;
    a.Bdig = w + p->off_Bdig;
    a.s = p->s;
    a.beta = p->beta;
    a.big = p->big;
    a.bal = p->bal;
    return a;
}

inline GemmArgs gemm_args(ozmp_plan_s* p) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    char* w = (char*)p->ws;
    g.form = p->form; g.q = p->q; g.is_f32 = p->is_f32;
    g.m = p->m; g.n = p->n; g.k = p->k; g.mp = p->mp; g.np = p->np; g.kp = p->kp;
    g.E = (const int32_t*)(w + p->off_E);
    g.F = (const int32_t*)(w + p->off_F);
    g.Adig = w + p->off_Adig;
    g.Bdig = w + p->off_Bdig;
    g.s = p->s; g.beta = p->beta; g.ppd = p->ppd; g.group_start = p->group_start;
    g.eoff = p->bal ? 2 : 0;
    g.acc_words = p->acc_words; g.ngroups = p->ngroups;
    g.acc = (p->ngroups > 1 || tc_engine(p->form)) ? (int64_t*)(w + p->off_acc) : nullptr;
    g.status = (uint32_t*)(w + p->off_status);
    if (p->sched_host) {
        g.sched_items = w + p->off_items;
        g.sched_off = (const int*)(w + p->off_soff);
        g.sched_grid = p->sched_grid;
        g.sacc = p->sched_slots ? (int64_t*)(w + p->off_sacc) : nullptr;
        int* cnt = (int*)(w + p->off_sacc + (size_t)p->sched_slots * p->nlimbs * 256 * 128 * 8);
        g.cnt = p->sched_slots ? cnt : nullptr;
        g.counter = p->tc_dyn ? cnt + p->sched_slots : nullptr;
        if (p->env_lock > 0 && p->tc_dyn) {
            g.retired = cnt + p->sched_slots + 1;
            g.step_done = g.retired + 1;
            g.lock_w = p->env_lock;
            g.lock_n = p->sched_ntiles * (p->s * (p->s + 1) / 2);
        }
        g.tc_snake = p->env_walk >= 0 ? p->env_walk : (p->k >= TC_SNAKE_K ? 1 : 0);
        g.cnt_region = cnt;
        g.tile_slot = (const int*)(w + p->off_tslot);
        g.sched_nitems = p->sched_items;
        g.split_bytes = p->split_bytes;
        g.tc_cg = p->tc_cg;
    }
    g.wait_limit = p->tc_wait_limit;
    g.inject_stall = p->tc_inject_stall;
    return g;
}

// the timing pair of the next product launch (none without a timing ring)
inline void take_timing(ozmp_plan_s* p, GemmArgs& g) {
    if (!p->tev_n) return;
    const int x = (int)(p->tev_calls % p->tev_n);
    g.tev_start = p->tev[2 * x];
    g.tev_stop = p->tev[2 * x + 1];
    p->tev_calls++;
}

// tcgen05 form: build the tile schedule and append its workspace regions
// (items, CTA offsets, split-tile limbs + counters).  Tiles are 256 x 256 over
// a CTA pair when the padded row count allows it (OZMP_TC_PAIR=0 in the
// environment keeps one 128 x 256 tile per CTA), the schedule then running
// over clusters (half the SMs) and every split slot holding two CTAs' rows.
// The items are taken from a counter in list order (OZMP_TC_DYNAMIC=0: fixed
// per-CTA lists).
inline ozmp_status plan_schedule(ozmp_plan_s* p) {
    if (!tc_engine(p->form) || p->m == 0 || p->n == 0 || p->k == 0) return OZMP_OK;
    if (!p->env_read) {
        const char* env = getenv("OZMP_TC_PAIR");
        p->env_pair_off = (env && env[0] == '0') ? 1 : 0;
        const char* dyn = getenv("OZMP_TC_DYNAMIC");
        p->env_static = (dyn && dyn[0] == '0') ? 1 : 0;
        // defaults: bands of 8 row tiles, walked in a loose lockstep of one pair
        // (at QD 8192^2 x 16384, where the operand panels no longer stay in L2,
        // 945 -> 831 ms; DD 4096^3 unchanged)
        const char* grp = getenv("OZMP_TC_GROUP");
        p->env_group = grp ? atoi(grp) : 8;
        const char* mxc = getenv("OZMP_TC_MAX_CHUNKS");
        p->env_maxc = mxc ? atoi(mxc) : 0;
        const char* lk = getenv("OZMP_TC_LOCKSTEP");
        p->env_lock = lk ? atoi(lk) : 1;
        // pair order (walk.h): 0 one diagonal at a time, 1 the snake; unset: the
        // snake where k >= TC_SNAKE_K
        const char* wk = getenv("OZMP_TC_WALK");
        p->env_walk = wk ? (wk[0] == '1' ? 1 : 0) : -1;
        // test hooks of the bounded waits: a smaller poll limit, and a stage
        // whose copies are never issued so that the waits on it run out
        const char* wl = getenv("OZMP_TC_WAIT_LIMIT");
        p->tc_wait_limit = wl ? atoll(wl) : 0;
        const char* inj = getenv("OZMP_TC_INJECT_STALL");
        p->tc_inject_stall = (inj && inj[0] == '1') ? 1 : 0;
        p->env_read = 1;
    }
    p->tc_cg = (p->mp % 256 == 0 && !p->env_pair_off) ? 2 : 1;
    const int ntiles = (int)((p->mp / (128 * p->tc_cg)) * (p->np / 256));
    const int pairs = p->s * (p->s + 1) / 2;
    const int sms = p->tc_cg == 2 ? tc_num_pair_slots() : tc_num_sms();
    p->sched_host = new (std::nothrow) int[(size_t)6 * ntiles * TC_MAX_CHUNKS + sms + 1 + ntiles];
    p->sched_ntiles = ntiles;
    if (!p->sched_host) return OZMP_ERR_NOMEM;
    int* items = p->sched_host;
    int* off = p->sched_host + (size_t)6 * ntiles * TC_MAX_CHUNKS;
    p->tc_dyn = !p->env_static;
    const int tm = (int)(p->mp / (128 * p->tc_cg));
    p->sched_grid = tc_schedule(ntiles, pairs, sms, items, off, &p->sched_items, &p->sched_slots, !p->tc_dyn, tm,
                                p->env_group, p->env_maxc);
    p->sched_slots *= p->tc_cg;
    // CTA offsets right after the items in the host copy
    int* off2 = items + 6 * p->sched_items;
    for (int c = 0; c <= p->sched_grid; ++c) off2[c] = off[c];
    // then the split-limb slot of every tile (-1: whole)
    int* tslot = off2 + p->sched_grid + 1;
    for (int t = 0; t < ntiles; ++t) tslot[t] = -1;
    for (int x = 0; x < p->sched_items; ++x)
        if (items[6 * x + 4] >= 0) tslot[items[6 * x + 1]] = items[6 * x + 4];
    size_t o = p->ws_bytes;
    p->off_items = o; o = align256(o + (size_t)p->sched_items * 24);
    p->off_soff = o; o = align256(o + (size_t)(p->sched_grid + 1) * 4);
    p->off_tslot = o; o = align256(o + (size_t)ntiles * 4);
    p->off_sacc = o;
    // split limbs, their chunk counters, the item-feed counter and (lockstep)
    // the retired count and one step counter per whole-tile pair a cluster can
    // walk, zeroed before each launch
    const size_t lock_n = (p->env_lock > 0 && p->tc_dyn) ? (size_t)ntiles * pairs : 0;
    p->split_bytes = (size_t)p->sched_slots * p->nlimbs * 256 * 128 * 8 + (size_t)p->sched_slots * 4 + 4 +
                     (lock_n ? 4 + 4 * lock_n : 0);
    o = align256(o + p->split_bytes);
    p->ws_bytes = o;
    return OZMP_OK;
}

// copy the schedule into the current workspace (once per workspace)
inline ozmp_status plan_upload_schedule(ozmp_plan_s* p) {
    if (!p->sched_host || p->sched_ws == p->ws) return OZMP_OK;
    const size_t bytes = (size_t)p->sched_items * 24;
    if (cudaMemcpyAsync((char*)p->ws + p->off_items, p->sched_host, bytes, cudaMemcpyHostToDevice, p->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync((char*)p->ws + p->off_soff, p->sched_host + 6 * p->sched_items,
                        (size_t)(p->sched_grid + 1) * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess ||
        cudaMemcpyAsync((char*)p->ws + p->off_tslot, p->sched_host + 6 * p->sched_items + p->sched_grid + 1,
                        (size_t)p->sched_ntiles * 4, cudaMemcpyHostToDevice, p->stream) != cudaSuccess)
        return OZMP_ERR_CUDA;
    p->sched_ws = p->ws;
    return OZMP_OK;
}

inline ozmp_status zero_c(ozmp_plan_s* p, void* const* C, int64_t ldc) {
    size_t wb = p->is_f32 ? 4 : 8;
    for (int c = 0; c < p->q; ++c)
        if (cudaMemset2DAsync(C[c], (size_t)ldc * wb, 0, (size_t)p->m * wb, (size_t)p->n, p->stream) != cudaSuccess)
            return OZMP_ERR_CUDA;
    if (cudaMemsetAsync((char*)p->ws + p->off_status, 0, 16, p->stream) != cudaSuccess) return OZMP_ERR_CUDA;
    return OZMP_OK;
}

// Fill a plan descriptor: argument checks, digit width, slice count
// (automatic: target bits + log2 k + 16 guard bits), padded sizes, the
// drain/group schedule and the workspace layout.  No memory is allocated.
inline ozmp_status plan_init(ozmp_plan_s* p, int prec, int64_t m, int64_t n, int64_t k, int form, int nslices,
                             ozmp_stream stream) {
    memset(p, 0, sizeof(*p));
    {
        // test hooks of the splitter's bounded wait: a smaller poll limit, and
        // columns whose copies are never issued so that the wait runs out
        const char* wl = getenv("OZMP_SPLIT_WAIT_LIMIT");
        p->split_wait_limit = wl ? atoll(wl) : 0;
        const char* inj = getenv("OZMP_SPLIT_INJECT_STALL");
        p->split_inject_stall = (inj && inj[0] == '1') ? 1 : 0;
    }
    int q = prec_q(prec);
    if (!q || m < 0 || n < 0 || k < 0 || nslices < 0 || nslices > OZMP_MAX_SLICES) return OZMP_ERR_INVALID_ARG;
    if (form < OZMP_FORM_AUTO || form > OZMP_FORM_FP16) return OZMP_ERR_INVALID_ARG;
    p->prec = prec;
    p->q = q;
    p->is_f32 = (prec == OZMP_TS);
    // balanced digits run on the tcgen05 engine of the e4m3 form, beta = 5;
    // the automatic form takes them up to their largest slice count (191),
    // and the 4-bit digits beyond it
    p->bal = (form == OZMP_FORM_FP8_BAL || (form == OZMP_FORM_AUTO && nslices <= (1024 - 65) / 5)) ? 1 : 0;
    p->form = (form == OZMP_FORM_AUTO || p->bal) ? OZMP_FORM_FP8 : form;
    p->m = m; p->n = n; p->k = k;
    p->beta = (p->form == OZMP_FORM_FP64) ? beta_fp64(k)
            : (p->form == OZMP_FORM_FP16) ? beta_fp16(k)
            : (p->form == OZMP_FORM_INT8 ? 7 : (p->bal ? 5 : 4));
    if (p->beta < 1) return OZMP_ERR_UNSUPPORTED;
    p->db = (p->form == OZMP_FORM_FP64) ? 8 : (p->form == OZMP_FORM_FP16 ? 2 : 1);
    // slice limits: the register-resident splitters hold 4 components,
    // windows of beta s + 65 bits in 7 words (binary64 digits: beta s <= 376)
    // or 6 words (1-byte digits), and write at most 64 e4m3 slices (63
    // balanced ones); the tcgen05 form goes on with the many-component
    // splitter up to beta s + 65 <= 1024 (16-word windows)
    const bool tc = (p->form == OZMP_FORM_FP8);
    if (q > 4 && !tc) return OZMP_ERR_UNSUPPORTED;
    const int maxs = tc ? (1024 - 65) / p->beta : (p->form == OZMP_FORM_INT8 ? 36 : 64);
    const int maxbits = tc ? 1024 - 65 : 376;
    if (nslices == 0) {
        int bits = prec_target_bits(prec) + ceil_log2(k > 0 ? k : 1) + 16;
        // balanced digits keep 5 s - 1 bits below 2^E (the top digit is at most 16)
        nslices = p->bal ? (bits + 1 + 4) / 5 : (bits + p->beta - 1) / p->beta;
        if (nslices > maxs) nslices = maxs;
        while (nslices > 1 && nslices * p->beta > maxbits) --nslices;
    }
    if (nslices > maxs || nslices * p->beta > maxbits) return OZMP_ERR_UNSUPPORTED;
    p->s = nslices;
    p->target_bits = prec_target_bits(prec);
    p->big = (q > 4 || nslices > (p->bal ? 63 : 64)) ? 1 : 0;
    if (p->big && p->is_f32) return OZMP_ERR_UNSUPPORTED;   // the many-component splitter reads binary64
    p->mp = roundup(m, 128);
    p->np = roundup(n, tc_engine(p->form) ? 256 : 128);
    p->kp = roundup(k, 128);
    ozmp_status st = fill_schedule(p);
    if (st != OZMP_OK) return st;
    fill_layout(p);
    p->stream = (cudaStream_t)stream;
    return OZMP_OK;
}

}  // namespace ozmp_plan_detail

// plan creation with the data-dependent slice count (adapt, nslices = 0) and
// the a-posteriori bound check (check) switched on or off; ozmp_plan_create
// has both on (api.cu)
ozmp_status plan_create_internal(ozmp_plan* plan, ozmp_prec prec, int64_t m, int64_t n, int64_t k, ozmp_form form,
                                 int nslices, ozmp_stream stream, bool adapt, bool check);
