// C ABI of the ozmp library: plans, argument checks, launches, status.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include "kernels.h"
#include "ozmp_internal.cuh"
#include "plan.h"

using namespace ozmp;

#define OZMP_VERSION_STR "ozmp 0.1 (sm_103a)"

using namespace ozmp_plan_detail;

// ---------------------------------------------------------------------------
// plan creation and the data-dependent slice count
// ---------------------------------------------------------------------------
// A plan descriptor for a forced slice count s, made like p (same precision,
// shape, digit form, stream and environment knobs); no memory is allocated.
static ozmp_status plan_make_like(const ozmp_plan_s* p, int s, ozmp_plan_s* t) {
    const int form = p->bal ? (int)OZMP_FORM_FP8_BAL : p->form;
    ozmp_status st = plan_init(t, p->prec, p->m, p->n, p->k, form, s, p->stream);
    if (st != OZMP_OK) return st;
    t->split_wait_limit = p->split_wait_limit;
    t->split_inject_stall = p->split_inject_stall;
    if (p->env_read) {
        t->env_read = 1;
        t->env_pair_off = p->env_pair_off;
        t->env_static = p->env_static;
        t->env_group = p->env_group;
        t->env_maxc = p->env_maxc;
        t->env_lock = p->env_lock;
        t->env_walk = p->env_walk;
        t->tc_wait_limit = p->tc_wait_limit;
        t->tc_inject_stall = p->tc_inject_stall;
    }
    st = plan_schedule(t);
    if (st != OZMP_OK) { delete[] t->sched_host; t->sched_host = nullptr; }
    return st;
}

// Re-make p for s slices inside its workspace (every s in [s_lo, s_cap] fits
// the workspace reserved at creation; E, F and the statistics keep their
// offsets, which depend on m, n, k only).
static ozmp_status plan_set_slices(ozmp_plan_s* p, int s) {
    if (s == p->s) return OZMP_OK;
    ozmp_plan_s t;
    ozmp_status st = plan_make_like(p, s, &t);
    if (st != OZMP_OK) return st;
    if (t.ws_bytes > p->ws_bytes || t.off_stats != p->off_stats || t.off_E != p->off_E || t.off_F != p->off_F) {
        delete[] t.sched_host;
        return OZMP_ERR_UNSUPPORTED;
    }
    t.ws = p->ws;
    t.ws_owned = p->ws_owned;
    t.ws_cap = p->ws_cap;
    t.ws_bytes = p->ws_bytes;
    t.tev = p->tev;
    t.tev_n = p->tev_n;
    t.tev_calls = p->tev_calls;
    t.adapt = p->adapt;
    t.check = p->check;
    t.s_lo = p->s_lo;
    t.s_cap = p->s_cap;
    t.host_s = p->host_s;
    t.ev_s = p->ev_s;
    t.sched_ws = nullptr;   // the new schedule is uploaded before the next product
    delete[] p->sched_host;
    *p = t;
    return OZMP_OK;
}

// adapt: nslices = 0 chooses s from the data at every execution, within
// s0 -/+ about 50 bits of the automatic count s0 (the workspace holds the
// largest of those layouts); check: the a-posteriori bound check runs after
// every execution.
ozmp_status plan_create_internal(ozmp_plan* plan, ozmp_prec prec, int64_t m, int64_t n, int64_t k, ozmp_form form,
                                 int nslices, ozmp_stream stream, bool adapt, bool check) {
    if (!plan) return OZMP_ERR_INVALID_ARG;
    *plan = nullptr;
    ozmp_plan_s* p = new (std::nothrow) ozmp_plan_s();   // zeroed: a rejected plan frees nothing it has not set
    if (!p) return OZMP_ERR_NOMEM;
    ozmp_status st = plan_init(p, prec, m, n, k, form, nslices, stream);
    if (st == OZMP_OK) st = plan_schedule(p);
    if (st != OZMP_OK) { delete[] p->sched_host; delete p; return st; }
    p->check = check ? 1 : 0;
    p->s_lo = p->s_cap = p->s;
    if (adapt && nslices == 0 && m > 0 && n > 0 && k > 0) {
        p->adapt = 1;
        const int span = (50 + p->beta - 1) / p->beta;
        const int s0 = p->s;
        size_t most = p->ws_bytes;
        for (int s = s0 + 1; s <= s0 + span; ++s) {
            ozmp_plan_s t;
            if (plan_make_like(p, s, &t) != OZMP_OK) break;
            delete[] t.sched_host;
            if (t.ws_bytes > most) most = t.ws_bytes;
            p->s_cap = s;
        }
        for (int s = s0 - 1; s >= 1 && s >= s0 - span; --s) {
            ozmp_plan_s t;
            if (plan_make_like(p, s, &t) != OZMP_OK) break;
            delete[] t.sched_host;
            if (t.ws_bytes > most) most = t.ws_bytes;
            p->s_lo = s;
        }
        p->ws_bytes = most;
    }
    *plan = p;
    return OZMP_OK;
}

extern "C" {

const char* ozmp_version(void) { return OZMP_VERSION_STR; }

ozmp_status ozmp_plan_create(ozmp_plan* plan, ozmp_prec prec, int64_t m, int64_t n, int64_t k,
                             ozmp_form form, int nslices, ozmp_stream stream) {
    return plan_create_internal(plan, prec, m, n, k, form, nslices, stream, true, true);
}

static void free_timing(ozmp_plan p) {
    for (int x = 0; x < 2 * p->tev_n; ++x) cudaEventDestroy(p->tev[x]);
    delete[] p->tev;
    p->tev = nullptr;
    p->tev_n = 0;
    p->tev_calls = 0;
}

ozmp_status ozmp_plan_destroy(ozmp_plan p) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    if (p->batch) {
        cudaStreamSynchronize(p->stream);
        ozmp_batch::destroy(p->batch);
        delete p;
        return OZMP_OK;
    }
    if (p->ws && p->ws_owned) {
        cudaStreamSynchronize(p->stream);
        cudaFree(p->ws);
    }
    free_timing(p);
    if (p->host_s) {
        cudaStreamSynchronize(p->stream);
        cudaFreeHost(p->host_s);
        cudaEventDestroy(p->ev_s);
    }
    delete[] p->sched_host;
    delete p;
    return OZMP_OK;
}

ozmp_status ozmp_plan_get_info(ozmp_plan p, ozmp_plan_info* info) {
    if (!p || !info) return OZMP_ERR_INVALID_ARG;
    info->prec = p->prec;
    info->form = p->bal ? OZMP_FORM_FP8_BAL : p->form;
    info->beta = p->beta;
    info->nslices = p->s;
    info->npairs = (int64_t)p->s * (p->s + 1) / 2;
    info->m = p->m; info->n = p->n; info->k = p->k;
    info->mp = p->mp; info->np = p->np; info->kp = p->kp;
    info->digit_bytes = p->db;
    info->acc_words = p->acc_words;
    info->ngroups = p->ngroups;
    info->pairs_per_drain = p->ppd;
    info->workspace_bytes = p->ws_bytes;
    info->off_E = p->off_E; info->off_F = p->off_F; info->off_status = p->off_status;
    info->off_Adig = p->off_Adig; info->off_Bdig = p->off_Bdig; info->off_acc = p->off_acc;
    return OZMP_OK;
}

ozmp_status ozmp_plan_set_workspace(ozmp_plan p, void* dev_ptr, size_t bytes) {
    if (!p || !dev_ptr || bytes < p->ws_bytes || ((uintptr_t)dev_ptr & 255)) return OZMP_ERR_INVALID_ARG;
    if (p->ws && p->ws_owned) { cudaStreamSynchronize(p->stream); cudaFree(p->ws); }
    p->ws = dev_ptr;
    p->ws_owned = false;
    p->ws_cap = bytes;
    p->sched_ws = nullptr;
    return OZMP_OK;
}

ozmp_status ozmp_plan_set_stream(ozmp_plan p, ozmp_stream stream) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    p->stream = (cudaStream_t)stream;
    return OZMP_OK;
}

// Exponents and digits.  An adaptive plan reduces the exponents, chooses s
// from the data (one 4-byte read-back: the call waits for that pass; the
// digits for the previous count are already queued behind it), re-makes
// itself for a new s and writes its digits; other plans split in one go and
// take the exponent statistics of the a-posteriori check.
static ozmp_status do_split(ozmp_plan p, const void* const* A, int64_t lda, const void* const* B, int64_t ldb) {
    SplitArgs a = split_args(p, A, lda, B, ldb);
    char* w = (char*)p->ws;
    if (p->adapt) {
        // the read-back of the chosen s: a pinned word and an event after its
        // copy, made at the plan's first split (like its workspace)
        if (!p->host_s) {
            if (cudaMallocHost((void**)&p->host_s, sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                p->host_s = nullptr;
                return OZMP_ERR_NOMEM;
            }
            if (cudaEventCreateWithFlags(&p->ev_s, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                cudaFreeHost(p->host_s);
                p->host_s = nullptr;
                return OZMP_ERR_CUDA;
            }
        }
        BoundStats* bs = bound_stats(p);
        double* colA = (double*)(w + p->off_colA);
        double* rowB = (double*)(w + p->off_rowB);
        auto copy_s = [&]() {   // the chosen s into the pinned word, then the event
            return cudaMemcpyAsync(p->host_s, &bs->s_needed, sizeof(int), cudaMemcpyDeviceToHost, p->stream) ==
                       cudaSuccess &&
                   cudaEventRecord(p->ev_s, p->stream) == cudaSuccess;
        };
        auto read_s = [&](int* s) {
            if (!copy_s() || cudaEventSynchronize(p->ev_s) != cudaSuccess) return false;
            *s = *p->host_s;
            return true;
        };
        auto scaled_choice = [&]() {   // norms scaled by the largest exponents (any exponent range)
            return launch_bound_scale(a.E, p->m, a.F, p->n, bs, rowB, p->k, true, p->stream) == cudaSuccess &&
                   launch_bound_choose(A, lda, B, ldb, p->q, p->is_f32 != 0, p->m, p->n, p->k, bs, colA, rowB,
                                       bound_form(p), p->s_lo, p->s_cap, p->stream) == cudaSuccess;
        };
        // the exponent pass with the unscaled norms folded in, and the choice
        // in one launch; the scaled norms when the exponents leave their range
        // (and for the many-component splitter).  Where the one-pass column
        // digit kernel applies, it takes B's exponents and row norms itself:
        // B's digits for the count of the last execution are then written
        // before the choice, and B is read once.
        float* rowBf = (float*)(w + p->off_rowBf);
        if (cudaMemsetAsync(colA, 0, p->off_rowBf - p->off_colA + (size_t)p->k * 4, p->stream) != cudaSuccess)
            return OZMP_ERR_CUDA;
        bool deferred = false;
        const cudaError_t en = launch_split_exponents_norm(a, colA, rowB, &deferred, p->stream);
        bool ok;
        if (en == cudaErrorNotSupported) {
            cudaGetLastError();
            ok = launch_split_exponents(a, p->stream) == cudaSuccess && scaled_choice();
        } else {
            ok = en == cudaSuccess;
            if (ok && deferred) {
                SplitArgs b = a;
                b.parts = 2;
                b.rowBf = rowBf;
                ok = launch_split_digits(b, p->stream) == cudaSuccess;
            }
            ok = ok && launch_bound_choose_raw(a.E, p->m, a.F, p->n, colA, rowB, deferred ? rowBf : nullptr, p->k,
                                               bs, bound_form(p), p->s_lo, p->s_cap, p->stream) == cudaSuccess;
        }
        if (!ok || !copy_s()) return OZMP_ERR_CUDA;
        // the digits for the count of the last execution (those of A alone
        // when B's are written) go into the stream before the host waits for
        // the new choice, so that the GPU splits while the host reads; a
        // different choice splits again
        SplitArgs ra = a;
        if (deferred) ra.parts = 1;
        if (launch_split_digits(ra, p->stream) != cudaSuccess || cudaEventSynchronize(p->ev_s) != cudaSuccess)
            return OZMP_ERR_CUDA;
        int s = *p->host_s;
        if (s < 0 && (!scaled_choice() || !read_s(&s))) return OZMP_ERR_CUDA;
        if (s < p->s_lo) s = p->s_lo;
        if (s > p->s_cap) s = p->s_cap;
        if (s == p->s) return OZMP_OK;
        ozmp_status st = plan_set_slices(p, s);
        if (st != OZMP_OK) return st;
        a = split_args(p, A, lda, B, ldb);
        return launch_split_digits(a, p->stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
    }
    if (launch_split(a, p->stream) != cudaSuccess) return OZMP_ERR_CUDA;
    if (p->check && launch_bound_scale(a.E, p->m, a.F, p->n, bound_stats(p), nullptr, p->k, false, p->stream) !=
                        cudaSuccess)
        return OZMP_ERR_CUDA;
    return OZMP_OK;
}

// Slice products, exact accumulation and rounding into C; then the
// a-posteriori check of the result.
static ozmp_status do_multiply(ozmp_plan p, void* const* C, int64_t ldc) {
    if (plan_upload_schedule(p) != OZMP_OK) return OZMP_ERR_CUDA;
    GemmArgs g = gemm_args(p);
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) g.C[c] = (c < p->q) ? C[c] : nullptr;
    g.ldc = ldc;
    take_timing(p, g);
    // the tcgen05 rounding pass runs the check as it writes C; the other
    // engines take a pass over C's first component
    const bool in_pass = p->check && tc_engine(p->form);
    if (in_pass) {
        g.chk = bound_stats(p);
        g.chk_form = bound_form(p);
        g.chk_flag = ST_ACCURACY;
    }
    if (launch_gemm(g, p->stream) != cudaSuccess) return OZMP_ERR_CUDA;
    if (p->check && !in_pass &&
        launch_bound_check(C[0], p->is_f32 != 0, p->m, p->n, ldc, bound_stats(p), bound_form(p), p->s,
                           (uint32_t*)((char*)p->ws + p->off_status), ST_ACCURACY, p->stream) != cudaSuccess)
        return OZMP_ERR_CUDA;
    return OZMP_OK;
}

ozmp_status ozmp_plan_split(ozmp_plan p, const void* const* A, int64_t lda, const void* const* B, int64_t ldb) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    if (check_ld(p, lda, ldb, 0, false) != OZMP_OK) return OZMP_ERR_INVALID_ARG;
    if ((p->m > 0 && p->k > 0 && !ptrs_ok(A, p->q)) || (p->n > 0 && p->k > 0 && !ptrs_ok(B, p->q)))
        return OZMP_ERR_INVALID_ARG;
    ozmp_status st = ensure_ws(p);
    if (st != OZMP_OK) return st;
    return do_split(p, A, lda, B, ldb);
}

ozmp_status ozmp_plan_execute(ozmp_plan p, const void* const* A, int64_t lda, const void* const* B, int64_t ldb,
                              void* const* C, int64_t ldc) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    if (check_ld(p, lda, ldb, ldc, true) != OZMP_OK) return OZMP_ERR_INVALID_ARG;
    if (p->m == 0 || p->n == 0) return OZMP_OK;
    if (!ptrs_ok(C, p->q)) return OZMP_ERR_INVALID_ARG;
    if (p->k > 0 && (!ptrs_ok(A, p->q) || !ptrs_ok(B, p->q))) return OZMP_ERR_INVALID_ARG;
    ozmp_status st = ensure_ws(p);
    if (st != OZMP_OK) return st;
    if (p->k == 0) return zero_c(p, C, ldc);
    st = do_split(p, A, lda, B, ldb);
    if (st != OZMP_OK) return st;
    return do_multiply(p, C, ldc);
}

ozmp_status ozmp_plan_multiply(ozmp_plan p, void* const* C, int64_t ldc) {
    if (!p || !p->ws) return OZMP_ERR_INVALID_ARG;
    int64_t m1 = p->m > 1 ? p->m : 1;
    if (ldc < m1) return OZMP_ERR_INVALID_ARG;
    if (p->m == 0 || p->n == 0) return OZMP_OK;
    if (!ptrs_ok(C, p->q)) return OZMP_ERR_INVALID_ARG;
    if (p->k == 0) return zero_c(p, C, ldc);
    return do_multiply(p, C, ldc);
}

ozmp_status ozmp_plan_diagonal(ozmp_plan p, int d, int64_t* T) {
    if (!p || !T || d < 2 || d > p->s + 1 || !p->ws) return OZMP_ERR_INVALID_ARG;
    if (p->m == 0 || p->n == 0) return OZMP_OK;
    GemmArgs g = gemm_args(p);
    g.d_only = d;
    g.T = T;
    g.sched_items = nullptr;   // the diagnostic walks one diagonal, one whole tile per CTA
    return launch_gemm(g, p->stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}


ozmp_status ozmp_plan_set_timing(ozmp_plan p, int nslots) {
    if (!p || p->batch || nslots < 0 || nslots > 4096) return OZMP_ERR_INVALID_ARG;
    free_timing(p);
    if (!nslots) return OZMP_OK;
    p->tev = new (std::nothrow) cudaEvent_t[2 * (size_t)nslots];
    if (!p->tev) return OZMP_ERR_NOMEM;
    for (int x = 0; x < 2 * nslots; ++x) {
        if (cudaEventCreate(&p->tev[x]) != cudaSuccess) {
            for (int y = 0; y < x; ++y) cudaEventDestroy(p->tev[y]);
            delete[] p->tev;
            p->tev = nullptr;
            return OZMP_ERR_CUDA;
        }
    }
    p->tev_n = nslots;
    return OZMP_OK;
}

ozmp_status ozmp_plan_read_timing(ozmp_plan p, float* ms, int n, int* count) {
    if (!p || !count || n < 0 || (n > 0 && !ms)) return OZMP_ERR_INVALID_ARG;
    const long long have = p->tev_calls < p->tev_n ? p->tev_calls : p->tev_n;
    const int got = (int)(have < n ? have : n);
    for (int x = 0; x < got; ++x) {
        const int slot = (int)((p->tev_calls - got + x) % p->tev_n);
        if (cudaEventSynchronize(p->tev[2 * slot + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms[x], p->tev[2 * slot], p->tev[2 * slot + 1]) != cudaSuccess)
            return OZMP_ERR_CUDA;
    }
    *count = got;
    return OZMP_OK;
}

ozmp_status ozmp_plan_get_status(ozmp_plan p, ozmp_status* device_status) {
    if (!p || !device_status) return OZMP_ERR_INVALID_ARG;
    *device_status = OZMP_OK;
    if (!p->ws) return OZMP_OK;
    uint32_t w = 0;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return OZMP_ERR_CUDA;
    if (cudaMemcpy(&w, (char*)p->ws + p->off_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return OZMP_ERR_CUDA;
    if (w & ST_NONFINITE) *device_status = OZMP_ERR_NONFINITE;
    else if (w & ST_RANGE) *device_status = OZMP_ERR_RANGE;
    else if (w & ST_TIMEOUT) *device_status = OZMP_ERR_TIMEOUT;
    else if (w & ST_ACCURACY) *device_status = OZMP_ERR_ACCURACY;
    return OZMP_OK;
}

// ---------------------------------------------------------------------------
// plain entry points: a per-thread cached plan
// ---------------------------------------------------------------------------
static thread_local ozmp_plan tl_plan = nullptr;
static thread_local cudaStream_t tl_stream = nullptr;
static thread_local int tl_form = OZMP_FORM_AUTO;
static thread_local int tl_nslices = -1;
static thread_local int tl_plan_form = -1;   // the form tl_plan was created for (as requested)

ozmp_status ozmp_set_stream(ozmp_stream stream) {
    tl_stream = (cudaStream_t)stream;
    if (tl_plan) tl_plan->stream = tl_stream;
    return OZMP_OK;
}

ozmp_status ozmp_set_form(ozmp_form form) {
    if (form < OZMP_FORM_AUTO || form > OZMP_FORM_FP16) return OZMP_ERR_INVALID_ARG;
    tl_form = form;
    return OZMP_OK;
}

ozmp_status ozmp_last_status(ozmp_status* device_status) {
    if (!device_status) return OZMP_ERR_INVALID_ARG;
    if (!tl_plan) { *device_status = OZMP_OK; return OZMP_OK; }
    return ozmp_plan_get_status(tl_plan, device_status);
}

static ozmp_status plain_gemm(ozmp_prec prec, int64_t m, int64_t n, int64_t k, const void* const* A, int64_t lda,
                              const void* const* B, int64_t ldb, void* const* C, int64_t ldc, int nslices) {
    // the cached plan is reused only for the form it was requested with: the
    // plan's own form field is the engine (FP8 for both e4m3 digit forms)
    ozmp_plan p = tl_plan;
    if (!p || p->prec != prec || p->m != m || p->n != n || p->k != k || tl_plan_form != tl_form ||
        tl_nslices != nslices) {
        if (p) { ozmp_plan_destroy(p); tl_plan = nullptr; tl_plan_form = -1; }
        ozmp_status st = ozmp_plan_create(&p, prec, m, n, k, (ozmp_form)tl_form, nslices, tl_stream);
        if (st != OZMP_OK) return st;
        tl_plan = p;
        tl_plan_form = tl_form;
        tl_nslices = nslices;
    }
    p->stream = tl_stream;
    return ozmp_plan_execute(p, A, lda, B, ldb, C, ldc);
}

ozmp_status ozmp_gemm_dd(int64_t m, int64_t n, int64_t k, const double* const A[2], int64_t lda,
                         const double* const B[2], int64_t ldb, double* const C[2], int64_t ldc, int nslices) {
    return plain_gemm(OZMP_DD, m, n, k, (const void* const*)A, lda, (const void* const*)B, ldb, (void* const*)C, ldc, nslices);
}
ozmp_status ozmp_gemm_td(int64_t m, int64_t n, int64_t k, const double* const A[3], int64_t lda,
                         const double* const B[3], int64_t ldb, double* const C[3], int64_t ldc, int nslices) {
    return plain_gemm(OZMP_TD, m, n, k, (const void* const*)A, lda, (const void* const*)B, ldb, (void* const*)C, ldc, nslices);
}
ozmp_status ozmp_gemm_qd(int64_t m, int64_t n, int64_t k, const double* const A[4], int64_t lda,
                         const double* const B[4], int64_t ldb, double* const C[4], int64_t ldc, int nslices) {
    return plain_gemm(OZMP_QD, m, n, k, (const void* const*)A, lda, (const void* const*)B, ldb, (void* const*)C, ldc, nslices);
}
ozmp_status ozmp_gemm_ts(int64_t m, int64_t n, int64_t k, const float* const A[3], int64_t lda,
                         const float* const B[3], int64_t ldb, float* const C[3], int64_t ldc, int nslices) {
    return plain_gemm(OZMP_TS, m, n, k, (const void* const*)A, lda, (const void* const*)B, ldb, (void* const*)C, ldc, nslices);
}
ozmp_status ozmp_gemm_md(int q, int64_t m, int64_t n, int64_t k, const double* const* A, int64_t lda,
                         const double* const* B, int64_t ldb, double* const* C, int64_t ldc, int nslices) {
    if (q < 2 || q > OZMP_MAX_COMPONENTS) return OZMP_ERR_INVALID_ARG;
    return plain_gemm(OZMP_PREC_Q(q), m, n, k, (const void* const*)A, lda, (const void* const*)B, ldb,
                      (void* const*)C, ldc, nslices);
}

}  // extern "C"
