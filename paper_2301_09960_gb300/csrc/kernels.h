// Host-side launch descriptors shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ozmp.h"
#include "bound.cuh"

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
    int big;               // the many-component / wide-window splitter (split_big.cu)
    int bal;               // balanced radix-32 e4m3 digits (beta = 5)
    long long wait_limit;  // one-pass column kernel: polls before its wait gives up (0: the default)
    int inject_stall;      // one-pass column kernel, test hook: copies never issued
    int parts;             // digits of 1: A's rows only, 2: B's columns only (0: both)
    float* rowBf;          // one-pass column kernel: also add each element's squared
                           // magnitude estimate into rowBf[p] (null: no norms)
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
    int eoff;              // digit t of a row weighs 2^(E + eoff/2 - beta t): 0, or 2 for balanced digits
    int ppd;               // slice pairs summed in the tensor-core accumulator before a drain
    uint64_t group_start;  // bit (d - 2): diagonal d opens a new group (diagonals run s+1 .. 2)
    int acc_words;         // 64-bit words of the per-element exact accumulator
    int ngroups;
    int64_t* acc;          // [acc_words][mp][np], used when ngroups > 1
    void* C[OZMP_MAX_COMPONENTS];
    int64_t ldc;
    uint32_t* status;
    int d_only;            // diagnostic: only diagonal d_only, raw int64 T_d written to T
    int64_t* T;
    // tcgen05 form: precomputed tile schedule (null: one whole tile per CTA)
    const void* sched_items;   // tc::WorkItem[]
    const int* sched_off;      // items of CTA c: [off[c], off[c + 1])
    int sched_grid;
    int64_t* sacc;             // split-tile limbs, zeroed before every launch
    int* cnt;                  // split-tile chunk counters (follow sacc)
    int* counter;              // dynamic item feed counter (follows cnt); null: per-CTA lists
    int* cnt_region;           // start of the counters (cnt, then the feed counter)
    const int* tile_slot;      // per tile of the schedule: its split-limb slot, or -1 (whole tile)
    cudaEvent_t tev_start, tev_stop;   // recorded around the product kernel when non-null
    long long wait_limit;      // tcgen05 form: polls before a wait gives up (0: the default)
    int inject_stall;          // tcgen05 form, test hook: a stage that is never loaded
    int sched_nitems;
    size_t split_bytes;        // bytes of sacc + cnt + counter
    int tc_cg;                 // 2: CTA-pair tiles (256 x 256, cta_group::2); else one CTA per tile
    int tc_snake;              // tcgen05 pair order (walk.h): 1 two diagonals interleaved, 0 one at a time
    // loose lockstep of the clusters' pair walks (lock_w > 0, dynamic feed):
    // step counters and the retired count, zeroed with the split region
    int* step_done;
    int* retired;
    int lock_w, lock_n;
    // the a-posteriori bound check run by the tcgen05 rounding pass (null: none)
    BoundStats* chk;
    BoundForm chk_form;
    uint32_t chk_flag;
};

// Tile schedule of one tcgen05 problem (host): whole tiles in full waves over
// `sms` CTAs; the tiles of a partial last wave (or of a problem with fewer
// tiles than CTAs) split into pair-range chunks.  Writes items (6 ints each:
// prob, tile, pa, pb, slot, nchunks), regrouped per CTA with CTA offsets when
// `regroup` (else in creation order for the dynamic feed); returns the grid.
// Tiles are taken in bands of `group` of the tm row tiles (0: column-major).
// maxc: pair-range chunks of one tail tile at most (0: TC_MAX_CHUNKS).
constexpr int TC_MAX_CHUNKS = 32;
// The snake pair order (walk.h) overlaps each drain with one pair's MMAs
// only, so it is the default where a pair takes long against a drain and the
// operand panels are large: k >= TC_SNAKE_K.
constexpr int64_t TC_SNAKE_K = 4096;
int tc_schedule(int ntiles, int pairs, int sms, int* items, int* off, int* nitems, int* nslots, bool regroup,
                int tm, int group, int maxc = 0);
int tc_num_sms();
int tc_num_pair_slots();   // co-resident clusters of two CTAs of the tcgen05 pair form

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st);
// the two passes of launch_split: exponents E, F (all column exponents
// included), then the digits for the plan's slice count
cudaError_t launch_split_exponents(const SplitArgs& a, cudaStream_t st);
// the exponent pass together with the unscaled squared norms, colA[p] =
// sum_i a_ip^2 and rowB[p] = sum_j b_pj^2 (each element's magnitude estimated
// from its exponent and leading component, in binary32; both zeroed by the
// caller); cudaErrorNotSupported for the many-component splitter.  Where the
// one-pass column digit kernel applies, B is left to it: *cols_deferred is
// set, and F and the row norms (into SplitArgs::rowBf) come from that
// kernel's launch (launch_split_digits with parts = 2)
cudaError_t launch_split_exponents_norm(const SplitArgs& a, double* colA, double* rowB, bool* cols_deferred,
                                        cudaStream_t st);
// the digits for the plan's slice count (SplitArgs::parts: one operand only,
// on the 1-byte digit forms)
cudaError_t launch_split_digits(const SplitArgs& a, cudaStream_t st);
cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t st);

}  // namespace ozmp
