/*
 * Oracle (test infrastructure only): exact and 512-bit reference products.
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code with the CUDA path.
 *
 * What it computes: the product C = A*B of the paper's problem statement
 * (Sec. 1: C := AB; Sec. 3, Algorithm 1 input/output) for multi-component
 * operands, whose value is the exact sum of their components.
 *
 *  1. exact mode: every term a^(c)_ip * b^(c')_pj is a dyadic rational; the
 *     whole dot product is summed exactly in a fixed-point (Kulisch) integer
 *     accumulator covering the full range of products of two doubles, and the
 *     exact result is rounded once to a 512-bit binary float (round to
 *     nearest, ties to even).
 *  2. naive mode: the plain triple loop in 512-bit floating point; every
 *     component sum, product and accumulation is rounded to 512 bits.
 *
 * The 512-bit float (mp512) is written here from the definition of binary
 * floating point: value = (-1)^sign * M * 2^e with a 512-bit integer M whose
 * top bit is set (or M = 0).
 */
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* exact fixed-point accumulator                                        */
/* ------------------------------------------------------------------ */
/* bit 0 of limb 0 has weight 2^KBASE.  The product of two finite doubles has
 * its least significant bit at >= 2^-2148 and its value below 2^2048; KW
 * limbs leave > 128 bits of headroom above for carries of long sums. */
#define KBASE (-2240)
#define KW 72

typedef struct { uint64_t w[KW]; } kacc;

static void kacc_clear(kacc* a) { memset(a->w, 0, sizeof(a->w)); }

/* decode a finite double: value = (-1)^s * M * 2^e, returns 0 on non-finite */
static int dec_double(double x, int* s, uint64_t* M, int* e) {
    uint64_t b; memcpy(&b, &x, 8);
    int ex = (int)((b >> 52) & 0x7ff);
    uint64_t fr = b & ((1ULL << 52) - 1);
    *s = (int)(b >> 63);
    if (ex == 0x7ff) { *M = 0; *e = 0; return 0; }
    if (ex == 0) { *M = fr; *e = -1074; }
    else { *M = fr | (1ULL << 52); *e = ex - 1075; }
    return 1;
}

/* add (neg=0) or subtract (neg=1) the unsigned value v * 2^(KBASE+pos) */
static void kacc_addu(kacc* a, u128 v, int pos, int neg) {
    if (v == 0) return;
    int li = pos >> 6, sh = pos & 63;
    uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    uint64_t p[3];
    p[0] = lo << sh;
    p[1] = sh ? ((hi << sh) | (lo >> (64 - sh))) : hi;
    p[2] = sh ? (hi >> (64 - sh)) : 0;
    int i;
    if (!neg) {
        uint64_t c = 0;
        for (i = 0; i < 3; i++) {
            u128 t = (u128)a->w[li + i] + p[i] + c;
            a->w[li + i] = (uint64_t)t; c = (uint64_t)(t >> 64);
        }
        for (i = li + 3; c && i < KW; i++) { a->w[i] += 1; c = (a->w[i] == 0); }
    } else {
        uint64_t bw = 0;
        for (i = 0; i < 3; i++) {
            uint64_t x = a->w[li + i];
            uint64_t d = x - p[i] - bw;
            bw = (x < p[i]) || (x - p[i] < bw);
            a->w[li + i] = d;
        }
        for (i = li + 3; bw && i < KW; i++) { bw = (a->w[i] == 0); a->w[i] -= 1; }
    }
}

static void kacc_add_prod(kacc* a, double x, double y) {
    int sx, sy, ex, ey; uint64_t mx, my;
    dec_double(x, &sx, &mx, &ex);
    dec_double(y, &sy, &my, &ey);
    if (mx == 0 || my == 0) return;
    kacc_addu(a, (u128)mx * my, ex + ey - KBASE, sx ^ sy);
}

/* ------------------------------------------------------------------ */
/* 512-bit float                                                        */
/* ------------------------------------------------------------------ */
typedef struct { int sign; int zero; int64_t e; uint64_t m[8]; } mp512;

static int bit_of(const uint64_t* w, int nw, int64_t b) {
    if (b < 0 || b >= 64LL * nw) return 0;
    return (int)((w[b >> 6] >> (b & 63)) & 1);
}
static int any_below(const uint64_t* w, int nw, int64_t b) {   /* any bit < b set */
    if (b <= 0) return 0;
    if (b > 64LL * nw) b = 64LL * nw;
    int64_t full = b >> 6;
    for (int64_t i = 0; i < full; i++) if (w[i]) return 1;
    int r = (int)(b & 63);
    if (r && (w[full] & ((1ULL << r) - 1))) return 1;
    return 0;
}
/* extract 64 bits starting at bit position b (may be negative) */
static uint64_t limb_at(const uint64_t* w, int nw, int64_t i) {
    return (i >= 0 && i < nw) ? w[i] : 0;
}
static uint64_t bits64(const uint64_t* w, int nw, int64_t b) {
    int64_t li = b >> 6;                 /* arithmetic shift: floor division */
    int sh = (int)(b - li * 64);
    uint64_t lo = limb_at(w, nw, li), hi = limb_at(w, nw, li + 1);
    return sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
}
static int top_bit(const uint64_t* w, int nw) {           /* -1 if zero */
    for (int i = nw - 1; i >= 0; i--)
        if (w[i]) return 64 * i + 63 - __builtin_clzll(w[i]);
    return -1;
}

/* round the unsigned integer w (nw limbs) times 2^base to 512 bits, RNE */
static void round_to_mp(const uint64_t* w, int nw, int64_t base, int sign, mp512* r) {
    int t = top_bit(w, nw);
    r->sign = sign;
    if (t < 0) { r->zero = 1; r->e = 0; memset(r->m, 0, sizeof(r->m)); return; }
    r->zero = 0;
    int64_t lo = (int64_t)t - 511;               /* bit index of the new LSB */
    for (int i = 0; i < 8; i++) r->m[i] = bits64(w, nw, lo + 64 * i);
    r->e = base + lo;
    if (lo > 0) {
        int rb = bit_of(w, nw, lo - 1);
        int st = any_below(w, nw, lo - 1);
        if (rb && (st || (r->m[0] & 1))) {
            int c = 1;
            for (int i = 0; i < 8 && c; i++) { r->m[i] += 1; c = (r->m[i] == 0); }
            if (c) {                               /* overflow to 2^512 */
                memset(r->m, 0, sizeof(r->m)); r->m[7] = 1ULL << 63; r->e += 1;
            }
        }
    }
}

static void kacc_to_mp(const kacc* a, mp512* r) {
    uint64_t mag[KW];
    int neg = (int)(a->w[KW - 1] >> 63);
    if (neg) {
        uint64_t c = 1;
        for (int i = 0; i < KW; i++) { uint64_t x = ~a->w[i]; mag[i] = x + c; c = c && (mag[i] == 0); }
    } else memcpy(mag, a->w, sizeof(mag));
    round_to_mp(mag, KW, KBASE, neg, r);
}

static void mp_from_double(double x, mp512* r) {
    int s, e; uint64_t M;
    dec_double(x, &s, &M, &e);
    uint64_t w[1] = {M};
    round_to_mp(w, 1, e, s, r);
}

/* r = RN512(a * b) */
static void mp_mul(const mp512* a, const mp512* b, mp512* r) {
    if (a->zero || b->zero) { memset(r, 0, sizeof(*r)); r->zero = 1; return; }
    uint64_t p[16]; memset(p, 0, sizeof(p));
    for (int i = 0; i < 8; i++) {
        uint64_t c = 0;
        for (int j = 0; j < 8; j++) {
            u128 t = (u128)a->m[i] * b->m[j] + p[i + j] + c;
            p[i + j] = (uint64_t)t; c = (uint64_t)(t >> 64);
        }
        p[i + 8] = c;
    }
    round_to_mp(p, 16, a->e + b->e, a->sign ^ b->sign, r);
}

/* r = RN512(a + b) */
static void mp_add(const mp512* a, const mp512* b, mp512* r) {
    if (a->zero) { *r = *b; return; }
    if (b->zero) { *r = *a; return; }
    const mp512 *x = a, *y = b;                /* x: larger exponent */
    if (y->e > x->e) { x = b; y = a; }
    int64_t d = x->e - y->e;
    if (d > 1100) {
        /* |y| < 2^-588 |x|: the exact sum rounds to x (its distance from x
         * is far below half an ulp of x, also at a binade boundary). */
        *r = *x; return;
    }
    /* exact sum in a wide buffer: x shifted left by d */
    enum { NB = 8 + 18 + 2 };
    uint64_t bx[NB], by[NB], s[NB];
    memset(bx, 0, sizeof(bx)); memset(by, 0, sizeof(by));
    int wsh = (int)(d >> 6), bsh = (int)(d & 63);
    for (int i = 0; i < 8; i++) {
        bx[i + wsh] |= x->m[i] << bsh;
        if (bsh) bx[i + wsh + 1] |= x->m[i] >> (64 - bsh);
    }
    memcpy(by, y->m, sizeof(y->m));
    int sign;
    if (x->sign == y->sign) {
        uint64_t c = 0;
        for (int i = 0; i < NB; i++) { u128 t = (u128)bx[i] + by[i] + c; s[i] = (uint64_t)t; c = (uint64_t)(t >> 64); }
        sign = x->sign;
    } else {
        int cmp = 0;
        for (int i = NB - 1; i >= 0 && !cmp; i--) cmp = (bx[i] > by[i]) - (bx[i] < by[i]);
        const uint64_t *p = bx, *q = by;
        sign = x->sign;
        if (cmp < 0) { p = by; q = bx; sign = y->sign; }
        if (cmp == 0) { memset(r, 0, sizeof(*r)); r->zero = 1; return; }
        uint64_t bw = 0;
        for (int i = 0; i < NB; i++) {
            uint64_t t = p[i] - q[i] - bw;
            bw = (p[i] < q[i]) || (p[i] - q[i] < bw);
            s[i] = t;
        }
    }
    round_to_mp(s, NB, y->e, sign, r);
}

/* ------------------------------------------------------------------ */
/* exported entry points                                                */
/* ------------------------------------------------------------------ */
static double load_comp(const void* base, int is_float, int64_t idx) {
    return is_float ? (double)((const float*)base)[idx] : ((const double*)base)[idx];
}

static void store_mp(const mp512* r, int64_t o, int8_t* sgn, int64_t* ex, uint64_t* limbs) {
    sgn[o] = r->zero ? 0 : (r->sign ? -1 : 1);
    ex[o] = r->e;
    memcpy(limbs + 8 * o, r->m, 64);
}

/*
 * Exact product rounded once to 512 bits, for the sampled block rows x cols.
 * A: qa component arrays, column-major m x k with leading dimension lda.
 * B: qb component arrays, column-major k x n with leading dimension ldb.
 * Output element (r, c) of the block goes to index r + c*nrows.
 */
void oz_exact_block(int qa, int qb, int is_float, int64_t k,
                    const void* const* A, int64_t lda, const void* const* B, int64_t ldb,
                    const int64_t* rows, int64_t nrows, const int64_t* cols, int64_t ncols,
                    int8_t* sgn, int64_t* ex, uint64_t* limbs) {
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t cj = 0; cj < ncols; cj++) {
        for (int64_t ri = 0; ri < nrows; ri++) {
            kacc acc; kacc_clear(&acc);
            int64_t i = rows[ri], j = cols[cj];
            for (int64_t p = 0; p < k; p++) {
                for (int ca = 0; ca < qa; ca++) {
                    double a = load_comp(A[ca], is_float, i + p * lda);
                    if (a == 0.0) continue;
                    for (int cb = 0; cb < qb; cb++) {
                        double b = load_comp(B[cb], is_float, p + j * ldb);
                        kacc_add_prod(&acc, a, b);
                    }
                }
            }
            mp512 r; kacc_to_mp(&acc, &r);
            store_mp(&r, ri + cj * nrows, sgn, ex, limbs);
        }
    }
}

/* The plain triple loop in 512-bit floating point: each operand element is
 * summed from its components, then acc := RN512(acc + RN512(a*b)). */
void oz_naive512_block(int qa, int qb, int is_float, int64_t k,
                       const void* const* A, int64_t lda, const void* const* B, int64_t ldb,
                       const int64_t* rows, int64_t nrows, const int64_t* cols, int64_t ncols,
                       int8_t* sgn, int64_t* ex, uint64_t* limbs) {
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t cj = 0; cj < ncols; cj++) {
        for (int64_t ri = 0; ri < nrows; ri++) {
            mp512 acc; memset(&acc, 0, sizeof(acc)); acc.zero = 1;
            int64_t i = rows[ri], j = cols[cj];
            for (int64_t p = 0; p < k; p++) {
                mp512 a, b, t, u;
                memset(&a, 0, sizeof(a)); a.zero = 1;
                memset(&b, 0, sizeof(b)); b.zero = 1;
                for (int ca = 0; ca < qa; ca++) {
                    mp_from_double(load_comp(A[ca], is_float, i + p * lda), &t);
                    mp_add(&a, &t, &u); a = u;
                }
                for (int cb = 0; cb < qb; cb++) {
                    mp_from_double(load_comp(B[cb], is_float, p + j * ldb), &t);
                    mp_add(&b, &t, &u); b = u;
                }
                mp_mul(&a, &b, &t);
                mp_add(&acc, &t, &u); acc = u;
            }
            store_mp(&acc, ri + cj * nrows, sgn, ex, limbs);
        }
    }
}

/* Elementwise 512-bit operations, exposed so the tests can pin the
 * arithmetic against exact rationals.  op: 0 = add, 1 = mul.  Operands are
 * given as (sign, exponent, 8 limbs) like the outputs above. */
void oz_mp_binop(int op, int64_t count,
                 const int8_t* s1, const int64_t* e1, const uint64_t* m1,
                 const int8_t* s2, const int64_t* e2, const uint64_t* m2,
                 int8_t* so, int64_t* eo, uint64_t* mo) {
    for (int64_t i = 0; i < count; i++) {
        mp512 a, b, r;
        a.zero = (s1[i] == 0); a.sign = s1[i] < 0; a.e = e1[i]; memcpy(a.m, m1 + 8 * i, 64);
        b.zero = (s2[i] == 0); b.sign = s2[i] < 0; b.e = e2[i]; memcpy(b.m, m2 + 8 * i, 64);
        uint64_t tmp[8];
        if (!a.zero) { memcpy(tmp, a.m, 64); round_to_mp(tmp, 8, a.e, a.sign, &a); }
        if (!b.zero) { memcpy(tmp, b.m, 64); round_to_mp(tmp, 8, b.e, b.sign, &b); }
        if (op == 0) mp_add(&a, &b, &r); else mp_mul(&a, &b, &r);
        store_mp(&r, i, so, eo, mo);
    }
}

/* Exact integer slice products used by the CPU Ozaki product:
 * T[i + j*m] = sum_p X[i*k + p] * Y[j*k + p]   (digits K-contiguous, int64
 * accumulation; callers keep |T| < 2^63). */
void oz_int_gemm_tn(int64_t m, int64_t n, int64_t k, const int64_t* X, const int64_t* Y, int64_t* T) {
    #pragma omp parallel for schedule(static) collapse(2)
    for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++) {
            int64_t s = 0;
            const int64_t* x = X + i * k; const int64_t* y = Y + j * k;
            for (int64_t p = 0; p < k; p++) s += x[p] * y[p];
            T[i + j * m] = s;
        }
}
