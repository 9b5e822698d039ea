/*
 * ozmp -- Ozaki-scheme multiple-precision matrix product on GB300 (sm_103a).
 *
 * C ABI of the library.  It computes C := A * B (paper, Sec. 1 problem
 * statement; Sec. 3, Algorithm 1) for multi-component operands: every
 * element is the exact sum of q components, DD/TD/QD = 2/3/4 binary64
 * words, TS = 3 binary32 words (Sec. 1), and more generally any q from 2
 * to OZMP_MAX_COMPONENTS binary64 words (about 53 q bits; Sec. 5 compares
 * the scheme with arbitrary-precision arithmetic of 212 to 742 bits).
 *
 * Layout and ownership (every entry point):
 *   - Matrices are column-major (BLAS convention of the problem C := AB).
 *     A is m x k with leading dimension lda >= max(1, m), B is k x n with
 *     ldb >= max(1, k), C is m x n with ldc >= max(1, m).
 *   - Each component is a separate device array; all components of one
 *     operand share its leading dimension.  A[c], B[c], C[c] are device
 *     pointers owned by the caller.  C's components must not alias A's or
 *     B's.  Inputs may be unnormalised and sign-mixed: the value is the exact
 *     component sum.
 *   - Output: C's components are the canonical expansion of the computed
 *     Ozaki sum S: c_0 = RN(S), c_t = RN(S - c_0 - ... - c_{t-1}).
 *
 * Method (Algorithm 1 with exact truncating digit slices):
 *   1. exponent reduce: E_i = max_p E(a_ip), F_j = max_p E(b_pj) with
 *      E(x) = floor(log2|x|) + 1 of the exact value (the power of two of the
 *      tau vectors of Algorithm 1); all-zero rows/columns get OZMP_EXP_ZERO.
 *   2. digit split: |x| * 2^(beta*s - E) truncated toward zero to beta*s
 *      bits, cut into s signed digits of beta bits (sign of x); the digits
 *      plus a remainder below 2^(E - beta*s) sum to x exactly.
 *   3. slice products over the pairs t + u <= s + 1 (Algorithm 1's pair
 *      triangle), exact on the tensor cores: binary64 digits (DMMA),
 *      int8 digits (IMMA, int32 accumulation) or e4m3 digits |d| <= 15
 *      (QMMA, binary32 accumulation of integers below 2^24).
 *   4. the slice products are summed exactly in integer arithmetic and
 *      rounded once into the output components (the "L-bit computation" of
 *      Algorithm 1), fused into the product kernel.
 *
 * Errors: argument errors return synchronously; data errors (NaN/Inf input,
 * exponents outside the representable window) are written to a device
 * status word, readable with ozmp_plan_get_status / ozmp_last_status after
 * the stream has been synchronised.  C is unspecified after a data error.
 * Every product of a plan is followed by an a-posteriori check of its error
 * bound (OZMP_ERR_ACCURACY when the bound does not certify the target).
 * Calls are stream-ordered and asynchronous, except that a plan with a
 * data-dependent slice count (nslices = 0) waits for the passes that reduce
 * its exponents.
 */
#ifndef OZMP_H
#define OZMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OZMP_OK = 0,
    OZMP_ERR_INVALID_ARG = 1,  /* null pointer, ld too small, bad enum, s out of range */
    OZMP_ERR_NONFINITE = 2,    /* device status: an input component is NaN or Inf */
    OZMP_ERR_RANGE = 3,        /* device status: a scale or output exponent leaves the normal range */
    OZMP_ERR_NOMEM = 4,        /* workspace allocation failed or supplied workspace too small */
    OZMP_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    OZMP_ERR_UNSUPPORTED = 6,  /* shape/precision/form combination not provided */
    OZMP_ERR_TIMEOUT = 7,      /* device status: a bounded wait in the batched scheduler gave up */
    OZMP_ERR_ACCURACY = 8      /* device status: the result's error bound does not certify the
                                  precision's target (more slices are needed); C holds the result */
} ozmp_status;

/* precision of the operands (component count and word type).  A value q
 * with 2 <= q <= OZMP_MAX_COMPONENTS is q binary64 components (OZMP_DD,
 * OZMP_TD and OZMP_QD are q = 2, 3, 4; OZMP_PREC_Q(q) names the others);
 * OZMP_TS is 3 binary32 components.  The automatic slice count targets a
 * normwise error of 2^(-50 q) for q binary64 components and 2^-66 for TS.
 * More than 4 components are provided by the FP8 (tcgen05) form only. */
typedef enum { OZMP_DD = 2, OZMP_TD = 3, OZMP_QD = 4, OZMP_TS = 103 } ozmp_prec;
#define OZMP_MAX_COMPONENTS 16
#define OZMP_PREC_Q(q) ((ozmp_prec)(q))

/* digit form of the slice products */
typedef enum {
    OZMP_FORM_AUTO = 0,     /* fastest exact form on this GPU: FP8_BAL up to 191 slices, else FP8 */
    OZMP_FORM_FP64 = 1,     /* binary64 digits, beta = max{b: k (2^b - 1)^2 <= 2^53}, DMMA */
    OZMP_FORM_INT8 = 2,     /* int8 digits, beta = 7, IMMA int32 accumulation */
    OZMP_FORM_FP8  = 3,     /* e4m3 digits, beta = 4, tcgen05 kind::f8f6f4, binary32 accumulation in TMEM */
    OZMP_FORM_FP8_MMA = 4,  /* the same e4m3 digits on the legacy mma.sync QMMA path */
    OZMP_FORM_FP8_BAL = 5,  /* e4m3 digits, beta = 5: the truncated value floor(|x| 2^(5s-1-E)) in
                               balanced radix-32 digits (|d| <= 16, signed like x), tcgen05
                               kind::f8f6f4; a third fewer slices than FORM_FP8 for one bound */
    OZMP_FORM_FP16 = 6      /* the binary32-slice form (the paper's SGEMM slices, S = 24): digits
                               of beta = max{b <= 11: k (2^b - 1)^2 <= 2^24} bits held exactly in
                               binary16, tcgen05 kind::f16 with binary32 accumulation in TMEM;
                               at most 4 components */
} ozmp_form;

/* all-zero row/column exponent */
#define OZMP_EXP_ZERO ((int32_t)(-2147483647 - 1))
/* largest slice count accepted as an argument; each form provides fewer:
 * FP8 (tcgen05) up to 239 and FP8_BAL up to 191 (beta s + 65 <= 1024 window
 * bits; TS: 64 and 63), FP8_MMA 64, INT8 36, FP64 up to beta s <= 376; above
 * the form's limit plan creation returns OZMP_ERR_UNSUPPORTED */
#define OZMP_MAX_SLICES 256

/* cudaStream_t, passed as an opaque pointer (NULL = the legacy default stream) */
typedef void* ozmp_stream;
typedef struct ozmp_plan_s* ozmp_plan;

/* Read-only description of a plan. */
typedef struct {
    int prec;            /* ozmp_prec */
    int form;            /* ozmp_form actually used */
    int beta;            /* bits per digit */
    int nslices;         /* s */
    int64_t npairs;      /* s (s + 1) / 2 */
    int64_t m, n, k;
    int64_t mp, np, kp;  /* padded sizes of the digit workspace */
    int digit_bytes;     /* 1 (int8 / e4m3) or 8 (binary64) */
    int acc_words;       /* 64-bit words of the exact per-element accumulator */
    int ngroups;         /* diagonal groups, one accumulator update each */
    int pairs_per_drain; /* slice pairs summed in the tensor-core accumulator */
    size_t workspace_bytes;
    /* byte offsets of the workspace regions (device layout) */
    size_t off_E, off_F, off_status, off_Adig, off_Bdig, off_acc;
} ozmp_plan_info;

/*
 * ozmp_plan_create -- fix precision, shape, digit form and slice count.
 * Sec. 3, Algorithm 1 (the choice of D, here nslices) and Sec. 3's remark
 * that the needed slice count depends on the data.
 *   Truncation bound: with s slices the computed sum S satisfies
 *   |S_ij - C*_ij| <= k c(s) 2^(E_i + F_j - W(s)) (W(s) = beta s, or 5 s - 1
 *   for balanced digits; c(s) about s), so
 *   ||S - C*||_F <= k c(s) 2^-W(s) ||2^E||_2 ||2^F||_2.
 *   nslices = 0: s is chosen from the data at every execution (split): after
 *   the exponent reduce, the smallest s whose bound is half of 2^-target
 *   times an estimate of ||C||_F (from the column norms of A and the row
 *   norms of B) -- target 2^-100 DD, 2^-150 TD, 2^-200 QD, 2^(-50 q) for q
 *   binary64 components, 2^-66 TS.  That choice is read back to the host, so
 *   the execution waits for the passes that reduce the exponents (for 1-byte
 *   e4m3 digits whose columns of B are 16-byte aligned and at most 112 KB,
 *   B's pass also writes B's digits for the previous count; A's digits are
 *   queued before the wait).  The plan reserves the
 *   workspace of the slice counts within about 50 bits of the count
 *   ceil((target + log2 k + 16) / beta) (for s outside, the nearest end is
 *   used); ozmp_plan_get_info reports the count of the last execution.
 *   1..OZMP_MAX_SLICES forces s (see the form limits).
 *   Every execution then checks the result: with N a lower bound of
 *   ||S||_F, the device status becomes OZMP_ERR_ACCURACY when
 *   (bound + u_q N) / (N - bound) exceeds 2^-target (u_q: the rounding into
 *   q components), e.g. for a forced s that is too small.
 *   stream: stream used by later executions through this plan.
 * The plan allocates its workspace lazily on first execution unless one is
 * supplied with ozmp_plan_set_workspace.  Returns INVALID_ARG for bad
 * arguments, UNSUPPORTED when k exceeds the form's exact-accumulation limit.
 */
ozmp_status ozmp_plan_create(ozmp_plan* plan, ozmp_prec prec, int64_t m, int64_t n, int64_t k,
                             ozmp_form form, int nslices, ozmp_stream stream);

/* Release the plan and any workspace it allocated (not a supplied one). */
ozmp_status ozmp_plan_destroy(ozmp_plan plan);

/* Describe the plan (sizes, digit width, workspace layout). */
ozmp_status ozmp_plan_get_info(ozmp_plan plan, ozmp_plan_info* info);

/* Use caller-owned device memory of at least info.workspace_bytes bytes
 * (256-byte aligned) as the workspace; the caller keeps ownership. */
ozmp_status ozmp_plan_set_workspace(ozmp_plan plan, void* dev_ptr, size_t bytes);

/* Change the stream of later executions. */
ozmp_status ozmp_plan_set_stream(ozmp_plan plan, ozmp_stream stream);

/*
 * Execute the whole product through a plan: exponent reduce, digit split,
 * fused slice products + exact accumulation.  A, B, C are arrays of q
 * component pointers (double* for DD/TD/QD, float* for TS).
 */
ozmp_status ozmp_plan_execute(ozmp_plan plan, const void* const* A, int64_t lda,
                              const void* const* B, int64_t ldb, void* const* C, int64_t ldc);

/* Device status word of the plan's last execution (synchronises the plan's
 * stream first). */
ozmp_status ozmp_plan_get_status(ozmp_plan plan, ozmp_status* device_status);

/*
 * Plain entry points (Sec. 1 problem statement, C := AB), one per precision.
 * They use a per-thread cached plan on the stream set with ozmp_set_stream
 * (default: legacy stream), the form set with ozmp_set_form (default
 * FORM_AUTO), and nslices as for ozmp_plan_create (0: chosen from the data).
 */
ozmp_status ozmp_gemm_dd(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
                         const double* const B[2], int64_t ldb, double* const C[2], int64_t ldc,
                         int nslices);
ozmp_status ozmp_gemm_td(int64_t m, int64_t n, int64_t k, const double* const A[3], int64_t lda,
                         const double* const B[3], int64_t ldb, double* const C[3], int64_t ldc,
                         int nslices);
ozmp_status ozmp_gemm_qd(int64_t m, int64_t n, int64_t k, const double* const A[4], int64_t lda,
                         const double* const B[4], int64_t ldb, double* const C[4], int64_t ldc,
                         int nslices);
ozmp_status ozmp_gemm_ts(int64_t m, int64_t n, int64_t k, const float* const A[3], int64_t lda,
                         const float* const B[3], int64_t ldb, float* const C[3], int64_t ldc,
                         int nslices);
/* q binary64 components, 2 <= q <= OZMP_MAX_COMPONENTS (A, B, C: arrays of q
 * device pointers); INVALID_ARG for q out of range.  Sec. 5's multiple
 * precision beyond QD. */
ozmp_status ozmp_gemm_md(int q, int64_t m, int64_t n, int64_t k, const double* const* A, int64_t lda,
                         const double* const* B, int64_t ldb, double* const* C, int64_t ldc, int nslices);

/*
 * ozmp_gemm_dd_noalloc -- the double-double product (as ozmp_gemm_dd, form
 * AUTO) without any memory allocation, on `stream`.  The paper has no
 * counterpart.  It serves callers that cannot call cudaMalloc: programs
 * whose device memory is all handed out by their own pool or caching
 * allocator (an allocation behind the pool's back can fail when the pool
 * holds the memory, and cudaMalloc/cudaFree synchronise the device), and
 * plug-ins or real-time loops that are not allowed to allocate after start-up.
 * Scratch: a file-scope device array of OZMP_NOALLOC_SCRATCH_BYTES (64 MiB)
 * inside the library, held by every GPU that loads the library until the
 * process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.
 * Limit: the scratch holds the exponents, both operands' digits and the
 * exact accumulator of the whole-tile walk, off_acc + (4 acc_words + 1)
 * mp np 8 bytes of a DD FORM_AUTO plan of the same m, n, k, nslices
 * (ozmp_plan_get_info; rounded up to 256).  That is less than the plan's
 * workspace_bytes, which adds a tile schedule and split-tile buffers that
 * this entry point does not use.  Larger problems are rejected with
 * OZMP_ERR_UNSUPPORTED: m = n = k = 512 fits, 1024^3 does not.
 * nslices = 0 is the automatic count ceil((100 + log2 k + 16) / 5) (no
 * data-dependent choice and no a-posteriori check: both would need more).
 * All calls share the scratch and it keeps the last call's contents: calls
 * whose work overlaps on the GPU race and must be serialised by the caller.
 * The device status word is not reported; C is unspecified for NaN/Inf input.
 */
#define OZMP_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
ozmp_status ozmp_gemm_dd_noalloc(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
                                 const double* const B[2], int64_t ldb, double* const C[2], int64_t ldc,
                                 int nslices, ozmp_stream stream);

/*
 * Batched products (the paper computes one product at a time, Sec. 3;
 * batching is this library's addition): count independent problems
 * C_i := A_i B_i, each with its own precision, shape, leading dimensions and
 * slice count (0 = the precision's automatic count ceil((target + log2 k +
 * 16) / beta): a graph holds no read-back, so there is no data-dependent
 * choice and no a-posteriori check in a batch), run as one captured CUDA graph.  For
 * FORM_FP8 / FORM_FP8_BAL / FORM_AUTO the graph holds one batched exponent launch, one
 * batched digit launch per operand and ONE persistent tcgen05 product launch
 * whose CTAs walk a load-balanced list of (problem, tile) items; the tile
 * width of each problem (128 or 256 columns) comes from an autotuner that
 * times both widths once per process (cached in the file named by the
 * environment variable OZMP_AUTOTUNE_CACHE, if set).  Other forms run the
 * problems one after another inside the graph.
 *   *plan == NULL: build a batched plan (workspace, schedule, graph), store it
 *   in *plan and run it.  *plan from an earlier call with the same count,
 *   precisions and shapes: run it again; the A/B/C pointers may change
 *   between calls.  Destroy with ozmp_plan_destroy; status with
 *   ozmp_plan_get_status (one word for the whole batch).
 * The problem array and the component-pointer arrays it points to are read
 * during the call only.  Batched problems hold at most 4 components,
 * 64 four-bit or 63 balanced slices and m n < 2^31 elements of C (else
 * OZMP_ERR_UNSUPPORTED); larger ones go through single-problem plans, and
 * so does FORM_FP16 (UNSUPPORTED in a batch).  form FP8_BAL runs every problem in balanced
 * radix-32 digits; a plan is reused only with the form it was made for.
 */
typedef struct {
    ozmp_prec prec;
    int64_t m, n, k, lda, ldb, ldc;
    const void* const* A;   /* q component pointers (double* or float* for TS) */
    const void* const* B;
    void* const* C;
    int nslices;            /* 0 = automatic */
} ozmp_problem;
ozmp_status ozmp_gemm_batched(const ozmp_problem* problems, int count, ozmp_form form, ozmp_stream stream,
                              ozmp_plan* plan);

/*
 * ozmp_gemm_naive -- the paper's "simple matrix multiplication" baseline
 * (Sec. 4; its GPU form with shared memory, Sec. 4.4): the triple loop in
 * multi-component arithmetic (TwoProd / TwoSum per word product, the q-word
 * accumulator renormalised after every multiply-add), 16 x 16 shared-memory
 * tiles.  Not an Ozaki-scheme product and not exact; it is the yardstick the
 * paper compares the scheme with.  Arguments as ozmp_plan_execute, on
 * `stream`.
 */
ozmp_status ozmp_gemm_naive(ozmp_prec prec, int64_t m, int64_t n, int64_t k, const void* const* A, int64_t lda,
                            const void* const* B, int64_t ldb, void* const* C, int64_t ldc, ozmp_stream stream);

/* Stream and digit form used by the plain entry points of this thread. */
ozmp_status ozmp_set_stream(ozmp_stream stream);
ozmp_status ozmp_set_form(ozmp_form form);
/* Device status of this thread's last plain call (synchronises its stream). */
ozmp_status ozmp_last_status(ozmp_status* device_status);

/*
 * Diagnostics (parity checks of the individual stages).
 * ozmp_plan_split: run only the exponent reduce and the digit split into the
 *   workspace (read E, F and the digits through ozmp_plan_get_info's
 *   offsets).  Digit t of row i of A sits at
 *   Adig[((t * mp) + i) * kp + p], of column j of B at Bdig[((t * np) + j) * kp + p].
 * ozmp_plan_diagonal: after a split, write T_d = sum_{t+u=d} A_t B_u^T as
 *   int64 to the device array T (column-major m x n, leading dimension m),
 *   computed by the same tensor-core main loop as the product.
 */
ozmp_status ozmp_plan_split(ozmp_plan plan, const void* const* A, int64_t lda,
                            const void* const* B, int64_t ldb);
/* ozmp_plan_multiply: the fused slice products + exact accumulation alone,
 *   on the digits and exponents left in the workspace by ozmp_plan_split
 *   (ozmp_plan_execute = ozmp_plan_split + ozmp_plan_multiply).  C as for
 *   ozmp_plan_execute. */
ozmp_status ozmp_plan_multiply(ozmp_plan plan, void* const* C, int64_t ldc);
ozmp_status ozmp_plan_diagonal(ozmp_plan plan, int d, int64_t* T);

/*
 * LU factorisation without pivoting (Sec. 4.6, "LU decomposition using
 * matrix multiplication"): A = L U in place, L unit lower (its diagonal not
 * stored), U upper, for q binary64 components, 2 <= q <= 4 (DD, TD, QD).
 * A: q device pointers, n x n column-major, leading dimension lda >= n.
 * The factorisation recurses on halves down to 32 x 32 blocks; the trailing
 * updates A22 - L21 U12 and the off-diagonal updates of the triangular
 * solves are Ozaki-scheme products (tcgen05 e4m3 form, slice count for the
 * precision's target); every other operation is evaluated exactly and
 * rounded once into q components (pivot reciprocals by a fixed Newton
 * sequence of such operations).  Synchronous: returns after the stream has
 * finished, with the device status (RANGE for a zero pivot or an exponent
 * outside the accumulator, NONFINITE, ...).  Errors: INVALID_ARG, NOMEM,
 * CUDA.  Workspace and product plans are kept per calling thread.
 */
ozmp_status ozmp_lu(int q, int64_t n, double* const* A, int64_t lda, ozmp_stream stream);
/* Solve A X = B with the factors of ozmp_lu (L Y = B, then U X = Y), in
 * place in B (n x nrhs, ldb >= n, q components); synchronous as ozmp_lu. */
ozmp_status ozmp_lu_solve(int q, int64_t n, int64_t nrhs, const double* const* LU, int64_t lda,
                          double* const* B, int64_t ldb, ozmp_stream stream);

/*
 * Algorithm 1 as printed (Sec. 3), kept beside the truncating-digit form for
 * comparisons of accuracy and slice count: for alpha = 1 .. D-1 the slice
 * A_alpha = (V_s + tau) - tau in binary64 round-to-nearest, V_s = RN64 of the
 * exact remainder, tau = 2^(ceil(log2 mu) + ceil((53 + log2 k) / 2)) per row
 * (per column for B) with mu the largest |V_s| of the row; the last slice is
 * RN64 of the remainder.  The D (D + 1) / 2 products A_alpha B_beta with
 * alpha + beta <= D + 1 are binary64 GEMMs (cuBLAS DGEMM, as the paper's GPU
 * path); they are summed exactly and rounded canonically into C.
 * q binary64 components (2 <= q <= OZMP_MAX_COMPONENTS), 1 <= D <= 32.
 * Optional device outputs (NULL: internal): slices_A (D x m x k, slice
 * alpha at (alpha-1) m k, column-major, ld m), slices_B (D x k x n, ld k),
 * products (D (D+1)/2 x m x n, ld m, pairs alpha-major).  Synchronous;
 * returns the device status (NONFINITE, RANGE).  Errors: INVALID_ARG,
 * NOMEM, CUDA.
 */
ozmp_status ozmp_gemm_literal(int q, int D, int64_t m, int64_t n, int64_t k, const double* const* A, int64_t lda,
                              const double* const* B, int64_t ldb, double* const* C, int64_t ldc,
                              double* slices_A, double* slices_B, double* products, ozmp_stream stream);

/* Kernel timing (instrumentation; the paper has no counterpart).
 * ozmp_plan_set_timing: with nslots > 0 the plan owns a ring of nslots CUDA
 *   event pairs and, at every ozmp_plan_execute / ozmp_plan_multiply, records
 *   one pair on its stream immediately around the slice-product kernel (the
 *   tcgen05 / mma.sync / DMMA main loop, without the rounding pass or the
 *   split).  nslots = 0 frees the events.  Errors: INVALID_ARG (null or
 *   batched plan, nslots < 0 or > 4096), NOMEM, CUDA (event creation failed).
 * ozmp_plan_read_timing: waits for and writes the durations in milliseconds
 *   of the last min(n, calls recorded, nslots) product kernels, oldest first,
 *   into ms[0 .. *count - 1] (host memory, caller-owned). */
ozmp_status ozmp_plan_set_timing(ozmp_plan plan, int nslots);
ozmp_status ozmp_plan_read_timing(ozmp_plan plan, float* ms, int n, int* count);

/* Version string of the library build. */
const char* ozmp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OZMP_H */
