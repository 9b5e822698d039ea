// Host check of the pair walk of the tcgen05 product kernel (csrc/walk.h):
// every pair of the triangle t + u <= s + 1 (Sec. 3, Algorithm 1) is visited
// once, every accumulator group holds pairs of one diagonal, at most ppd of
// them, in one accumulator, opened and closed within its work item; in the
// snake order consecutive pairs of different diagonals share an operand
// slice, and an accumulator is never reused before one pair of the other
// accumulator has run.
// Prints "ok <walks checked>" or the first violation; exit status 1 on one.
#include <cstdio>
#include <vector>
#include "../paper_2301_09960_gb300/csrc/walk.h"

using ozmp::PairStep;
using ozmp::PairWalk;

static int fail(const char* what, int dhi, int dlo, int ppd, int snake, int pa, int pb, int pi) {
    std::printf("FAIL %s: dhi=%d dlo=%d ppd=%d snake=%d item=[%d,%d) pair=%d\n", what, dhi, dlo, ppd, snake, pa, pb,
                pi);
    return 1;
}

// one work item [pa, pb); seen[t][u] counts visits
static int check_item(int dhi, int dlo, int ppd, int snake, int pa, int pb, int first_buf,
                      std::vector<std::vector<int>>& seen, int& last_buf, int& prev_t, int& prev_u) {
    PairWalk w;
    w.start(dhi, dlo, ppd, pa, pb, snake, first_buf);
    int open_d[2] = {0, 0}, open_n[2] = {0, 0};
    int closed_at[2] = {-10, -10};
    for (int pi = pa; pi < pb; ++pi) {
        const PairStep s = w.step();
        if (s.t < 1 || s.u < 1 || s.t + s.u != s.d || s.d > dhi || s.d < dlo)
            return fail("pair outside the walked diagonals", dhi, dlo, ppd, snake, pa, pb, pi);
        seen[s.t][s.u]++;
        const int b = s.buf;
        if (b != 0 && b != 1) return fail("accumulator index", dhi, dlo, ppd, snake, pa, pb, pi);
        if (pi == pa && b != (first_buf & 1)) return fail("first accumulator", dhi, dlo, ppd, snake, pa, pb, pi);
        if (s.open) {
            if (open_n[b]) return fail("group opened twice", dhi, dlo, ppd, snake, pa, pb, pi);
            if (snake && pi - closed_at[b] < 2) return fail("no pair between drain and reuse", dhi, dlo, ppd, snake, pa, pb, pi);
            open_d[b] = s.d;
        } else {
            if (!open_n[b]) return fail("pair outside any group", dhi, dlo, ppd, snake, pa, pb, pi);
            if (open_d[b] != s.d) return fail("two diagonals in one group", dhi, dlo, ppd, snake, pa, pb, pi);
        }
        if (++open_n[b] > ppd) return fail("group above ppd pairs", dhi, dlo, ppd, snake, pa, pb, pi);
        if (snake && pi > pa && b == last_buf) return fail("accumulators do not alternate", dhi, dlo, ppd, snake, pa, pb, pi);
        // (a diagonal walked alone shares nothing between its own pairs)
        if (snake && prev_t > 0 && prev_t + prev_u != s.d && s.t != prev_t && s.u != prev_u)
            return fail("consecutive pairs share no slice", dhi, dlo, ppd, snake, pa, pb, pi);
        if (!snake && open_n[b ^ 1]) return fail("two groups open at once", dhi, dlo, ppd, snake, pa, pb, pi);
        if (s.close) {
            open_n[b] = 0;
            closed_at[b] = pi;
        }
        last_buf = b;
        prev_t = s.t;
        prev_u = s.u;
    }
    if (open_n[0] || open_n[1]) return fail("group left open at the item's end", dhi, dlo, ppd, snake, pa, pb, pb);
    return 0;
}

int main() {
    long walks = 0;
    const int ppds[] = {1, 2, 3, 5, 16, 1 << 20};
    const int chunks[] = {1, 2, 3, 4, 7};
    std::vector<int> svals;
    for (int s = 1; s <= 64; ++s) svals.push_back(s);
    svals.push_back(191);
    svals.push_back(239);
    for (int s : svals) {
        for (int ppd : ppds) {
            for (int snake = 0; snake < 2; ++snake) {
                // the whole triangle (dhi = s + 1, dlo = 2) in 1..7 chunks, and
                // the single diagonals of the diagnostic mode
                const int npairs = s * (s + 1) / 2;
                for (int c : chunks) {
                    if (c > npairs) continue;
                    std::vector<std::vector<int>> seen(s + 2, std::vector<int>(s + 2, 0));
                    int last_buf = 1, prev_t = 0, prev_u = 0;
                    for (int x = 0; x < c; ++x) {
                        const int pa = (int)((long)npairs * x / c), pb = (int)((long)npairs * (x + 1) / c);
                        if (x > 0) prev_t = prev_u = 0;   // sharing is checked within an item
                        if (check_item(s + 1, 2, ppd, snake, pa, pb, last_buf ^ 1, seen, last_buf, prev_t, prev_u))
                            return 1;
                        ++walks;
                    }
                    for (int t = 1; t <= s; ++t)
                        for (int u = 1; u <= s; ++u)
                            if (seen[t][u] != (t + u <= s + 1 ? 1 : 0))
                                return fail("pair not visited exactly once", s + 1, 2, ppd, snake, 0, npairs, t * 1000 + u);
                }
                if (s <= 64) {
                    for (int d = 2; d <= s + 1; ++d) {
                        std::vector<std::vector<int>> seen(s + 2, std::vector<int>(s + 2, 0));
                        int last_buf = 1, prev_t = 0, prev_u = 0;
                        if (check_item(d, d, ppd, snake, 0, d - 1, 0, seen, last_buf, prev_t, prev_u)) return 1;
                        for (int t = 1; t < d; ++t)
                            if (seen[t][d - t] != 1) return fail("diagonal pair not visited once", d, d, ppd, snake, 0, d - 1, t);
                        ++walks;
                    }
                }
            }
        }
    }
    std::printf("ok %ld\n", walks);
    return 0;
}
