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

extern "C" {

const char* ozmp_version(void) { return OZMP_VERSION_STR; }

ozmp_status ozmp_plan_create(ozmp_plan* plan, ozmp_prec prec, int64_t m, int64_t n, int64_t k,
                             ozmp_form form, int nslices, ozmp_stream stream) {
    if (!plan) return OZMP_ERR_INVALID_ARG;
    *plan = nullptr;
    ozmp_plan_s* p = new (std::nothrow) ozmp_plan_s();   // zeroed: a rejected plan frees nothing it has not set
    if (!p) return OZMP_ERR_NOMEM;
    ozmp_status st = plan_init(p, prec, m, n, k, form, nslices, stream);
    if (st == OZMP_OK) st = plan_schedule(p);
    if (st != OZMP_OK) { delete[] p->sched_host; delete p; return st; }
    *plan = p;
    return OZMP_OK;
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
    return OZMP_OK;
}

ozmp_status ozmp_plan_set_stream(ozmp_plan p, ozmp_stream stream) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    p->stream = (cudaStream_t)stream;
    return OZMP_OK;
}

ozmp_status ozmp_plan_split(ozmp_plan p, const void* const* A, int64_t lda, const void* const* B, int64_t ldb) {
    if (!p) return OZMP_ERR_INVALID_ARG;
    if (check_ld(p, lda, ldb, 0, false) != OZMP_OK) return OZMP_ERR_INVALID_ARG;
    if ((p->m > 0 && p->k > 0 && !ptrs_ok(A, p->q)) || (p->n > 0 && p->k > 0 && !ptrs_ok(B, p->q)))
        return OZMP_ERR_INVALID_ARG;
    ozmp_status st = ensure_ws(p);
    if (st != OZMP_OK) return st;
    SplitArgs a = split_args(p, A, lda, B, ldb);
    return launch_split(a, p->stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
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
    SplitArgs a = split_args(p, A, lda, B, ldb);
    if (launch_split(a, p->stream) != cudaSuccess) return OZMP_ERR_CUDA;
    if (plan_upload_schedule(p) != OZMP_OK) return OZMP_ERR_CUDA;
    GemmArgs g = gemm_args(p);
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) g.C[c] = (c < p->q) ? C[c] : nullptr;
    g.ldc = ldc;
    take_timing(p, g);
    return launch_gemm(g, p->stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
}

ozmp_status ozmp_plan_multiply(ozmp_plan p, void* const* C, int64_t ldc) {
    if (!p || !p->ws) return OZMP_ERR_INVALID_ARG;
    int64_t m1 = p->m > 1 ? p->m : 1;
    if (ldc < m1) return OZMP_ERR_INVALID_ARG;
    if (p->m == 0 || p->n == 0) return OZMP_OK;
    if (!ptrs_ok(C, p->q)) return OZMP_ERR_INVALID_ARG;
    if (p->k == 0) return zero_c(p, C, ldc);
    if (plan_upload_schedule(p) != OZMP_OK) return OZMP_ERR_CUDA;
    GemmArgs g = gemm_args(p);
    for (int c = 0; c < OZMP_MAX_COMPONENTS; ++c) g.C[c] = (c < p->q) ? C[c] : nullptr;
    g.ldc = ldc;
    take_timing(p, g);
    return launch_gemm(g, p->stream) == cudaSuccess ? OZMP_OK : OZMP_ERR_CUDA;
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
    if (form < OZMP_FORM_AUTO || form > OZMP_FORM_FP8_BAL) return OZMP_ERR_INVALID_ARG;
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
