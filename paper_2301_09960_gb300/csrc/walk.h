// Order of the slice-pair walk over one tile, and its accumulator groups:
// one definition for the three roles of the tcgen05 product kernel (the TMA
// producer, the MMA issuer and the epilogue), compilable on the host so that
// its invariants are checked on the CPU.
//
// Sec. 3, Algorithm 1: the products A_t B_u of the pair triangle
// t + u <= s + 1 are summed; the products on one anti-diagonal d = t + u
// carry the same weight 2^(-beta d).  A binary32 accumulator in tensor memory
// sums at most `ppd` of them exactly (every sum below 2^24) before the
// epilogue drains it into the integer limbs; two accumulators take turns so
// that the MMAs of one group run while the other is drained.
//
// Two orders of the pairs:
//  - one diagonal at a time (the default where k < 4096): d = dhi .. dlo,
//    t = 1 .. d - 1; a group is a run of at most ppd pairs of one diagonal
//    and the accumulators alternate group by group.  Consecutive pairs
//    share no operand slice.
//  - the snake (the default where k >= 4096): diagonals in twos, d and
//    d - 1, their pairs interleaved,
//    (1, d-1) (1, d-2) (2, d-2) (2, d-3) ... (d-2, 1) (d-1, 1),
//    so that each pair shares one operand slice with the pair before it: A_t
//    when it steps from diagonal d to d - 1, B_u when it steps back.  The next
//    snake (d - 2, d - 3) runs the other way, starting at (d-3, 1), so the
//    walk keeps sharing B_1 or A_1 across the seam; with an odd number of
//    diagonals the last one is walked alone.  The pairs alternate between
//    the two accumulators, every diagonal of a snake in one of them, and a
//    group ends where its diagonal ends in that accumulator, after ppd pairs,
//    or with the work item; so the drain of a group closed after pair p
//    overlaps the MMAs of pair p + 1, which go to the other accumulator.
// In the snake half of the operand panels a step reads were read by the
// same clusters one step before and are still in L2: at DD 4096^3 (s = 25)
// the product kernel reads 18.9 instead of 32.2 GB from DRAM, draws less
// power under the cap and runs 3.7 % faster.  Its drains overlap one pair
// each, so for short pairs (small k) the order of one diagonal at a time,
// whose drains overlap many pairs, stays.
#pragma once

#if defined(__CUDACC__)
#define OZMP_HD __host__ __device__ __forceinline__
#else
#define OZMP_HD inline
#endif

namespace ozmp {

struct PairStep {
    int t, u;    // slice indices, 1-based: the product A_t B_u
    int d;       // its diagonal t + u
    int buf;     // accumulator (0 or 1)
    bool open;   // first pair of a group: the accumulator starts from zero
    bool close;  // last pair of a group: the accumulator is drained after it
};

struct PairWalk {
    int dhi, dlo, ppd, pa, pb, snake;
    int pi;          // index of the next pair in the walk of the whole tile
    int k, j;        // stretch k of the walk, position j in it
    int L, dA, two;  // the stretch: diagonal dA (and dA - 1 when two), L pairs
    int buf0;        // snake: accumulator of pair pa
    int cur;         // one diagonal at a time: accumulator of the open group
    int since0, since1;   // pairs in the open group of accumulator 0 / 1 (0: none)

    OZMP_HD void stretch() {
        if (snake) {
            dA = dhi - 2 * k;
            two = (dA - 1 >= dlo) ? 1 : 0;
            L = two ? 2 * dA - 3 : dA - 1;
        } else {
            dA = dhi - k;
            two = 0;
            L = dA - 1;
        }
    }

    // pairs [pa_, pb_) of the walk over diagonals dhi_ .. dlo_ (dhi_ >= dlo_ >= 2),
    // the first of them in accumulator first_buf
    OZMP_HD void start(int dhi_, int dlo_, int ppd_, int pa_, int pb_, int snake_, int first_buf) {
        dhi = dhi_; dlo = dlo_; ppd = ppd_; pa = pa_; pb = pb_; snake = snake_ ? 1 : 0;
        pi = pa;
        k = 0;
        stretch();
        int idx = pa;
        while (idx >= L && L > 0) { idx -= L; ++k; stretch(); }   // (L > 0: ends past the last diagonal too)
        j = idx;
        buf0 = first_buf & 1;
        cur = buf0;
        since0 = since1 = 0;
    }

    // the pair at index pi, then advance
    OZMP_HD PairStep step() {
        PairStep s;
        const int f = (snake && (k & 1)) ? L - 1 - j : j;   // odd snakes run backwards
        if (two && (f & 1)) { s.d = dA - 1; s.t = (f + 1) >> 1; }
        else { s.d = dA; s.t = two ? (f >> 1) + 1 : f + 1; }
        s.u = s.d - s.t;
        s.buf = snake ? ((buf0 + (pi - pa)) & 1) : cur;
        const int n = (s.buf ? since1 : since0) + 1;   // (no indexed array: registers only)
        s.open = n == 1;
        // the next pair of this accumulator: two ahead (snake) or the next one
        const int ahead = snake ? 2 : 1;
        s.close = n >= ppd || j + ahead >= L || pi + ahead >= pb;
        const int keep = s.close ? 0 : n;
        if (s.buf) since1 = keep;
        else since0 = keep;
        if (s.close && !snake) cur ^= 1;
        ++pi;
        if (++j == L && pi < pb) { j = 0; ++k; stretch(); }
        return s;
    }
};

}  // namespace ozmp
