// C ABI of the SQD library (include/sqd.h): context, validation, string
// filtering, table construction, sigma, Davidson and RDM orchestration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sqd_internal.cuh"

int build_ab_schedule(sqd_ctx *ctx, sqd_tables *t);

static thread_local std::string g_err;

static int fail_noctx(int code, const char *msg) {
    g_err = msg;
    return code;
}

template <typename T>
static int dalloc(sqd_ctx *ctx, T **p, int64_t count, int64_t *bytes = nullptr) {
    size_t b = sizeof(T) * (size_t)(count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void **)p, b);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return sqd_fail(ctx, e == cudaErrorMemoryAllocation ? SQD_ENOMEM : SQD_ECUDA,
                        "cudaMalloc(%zu) failed: %s", b, cudaGetErrorString(e));
    }
    if (bytes) *bytes += (int64_t)b;
    return SQD_OK;
}

static int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ---------------------------------------------------------- profiling ----

static cudaEvent_t pool_event(sqd_ctx *ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(sqd_ctx *ctx, int cls) {
    if (!ctx->prof) return;
    if (ctx->open_cls >= 0) {  // a region left open by an error return: drop it
        ctx->pool.push_back(ctx->recs.back().a);
        ctx->pool.push_back(ctx->recs.back().b);
        ctx->recs.pop_back();
        ctx->open_cls = -1;
    }
    prof_rec r;
    r.cls = cls;
    r.a = pool_event(ctx);
    r.b = pool_event(ctx);
    cudaEventRecord(r.a, ctx->stream);
    ctx->recs.push_back(r);
    ctx->open_cls = cls;
}

void prof_end(sqd_ctx *ctx, double flops, double bytes) {
    if (!ctx->prof || ctx->open_cls < 0) return;
    prof_rec &r = ctx->recs.back();
    cudaEventRecord(r.b, ctx->stream);
    ctx->cls_launches[r.cls]++;
    ctx->cls_flops[r.cls] += flops;
    ctx->cls_bytes[r.cls] += bytes;
    ctx->open_cls = -1;
}

// fold finished event pairs into the per-class times
static int prof_collect(sqd_ctx *ctx) {
    if (ctx->recs.empty()) return SQD_OK;
    if (ctx->open_cls >= 0) {
        ctx->pool.push_back(ctx->recs.back().a);
        ctx->pool.push_back(ctx->recs.back().b);
        ctx->recs.pop_back();
        ctx->open_cls = -1;
    }
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (prof_rec &r : ctx->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->cls_ms[r.cls] += ms;
        else cudaGetLastError();
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    return SQD_OK;
}

static int use_device(sqd_ctx *ctx) {
    SQD_CUDA(ctx, cudaSetDevice(ctx->device));
    return SQD_OK;
}

extern "C" {

const char *sqd_version(void) { return "sqd-gb300 0.1"; }

int sqd_create(sqd_ctx **out, int device, void *stream) {
    if (!out) return fail_noctx(SQD_EINVAL, "sqd_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail_noctx(SQD_ECUDA, "sqd_create: no CUDA device available");
    if (device < 0 || device >= ndev) return fail_noctx(SQD_EINVAL, "sqd_create: bad device");
    sqd_ctx *ctx = new sqd_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess) {
        delete ctx;
        return fail_noctx(SQD_ECUDA, "sqd_create: cannot use device");
    }
    *out = ctx;
    return SQD_OK;
}

int sqd_set_stream(sqd_ctx *ctx, void *stream) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_set_stream: ctx is NULL");
    ctx->stream = (cudaStream_t)stream;
    return SQD_OK;
}

void sqd_destroy(sqd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (!ctx->recs.empty()) cudaStreamSynchronize(ctx->stream);
    for (prof_rec &r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    delete ctx;
}

static const char *k_prof_names[PROF_NCLASS] = {
    "same_spin_alpha", "same_spin_beta", "alpha_beta", "transpose",
    "tables",          "strings",        "davidson",   "rdm", "stored",
    "ortho",           "eigh",           "batched",    "batched_sigma", "batched_vector",
    "batched_eigh",    "gcols",          "ortho_block", "batched_sigma_ab"};

int sqd_profile_enable(sqd_ctx *ctx, int enable) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_profile_enable: ctx is NULL");
    SQD_TRY(use_device(ctx));
    SQD_TRY(prof_collect(ctx));
    for (int c = 0; c < PROF_NCLASS; c++) {
        ctx->cls_launches[c] = 0;
        ctx->cls_flops[c] = ctx->cls_bytes[c] = ctx->cls_ms[c] = 0.0;
    }
    ctx->launches = 0;
    ctx->prof = enable != 0;
    return SQD_OK;
}

int sqd_profile_read(sqd_ctx *ctx, int cls, const char **name, int64_t *regions, double *ms,
                     double *flops, double *bytes) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_profile_read: ctx is NULL");
    if (cls < 0 || cls >= PROF_NCLASS) return sqd_fail(ctx, SQD_EINVAL, "bad profile class");
    SQD_TRY(use_device(ctx));
    SQD_TRY(prof_collect(ctx));
    if (name) *name = k_prof_names[cls];
    if (regions) *regions = ctx->cls_launches[cls];
    if (ms) *ms = ctx->cls_ms[cls];
    if (flops) *flops = ctx->cls_flops[cls];
    if (bytes) *bytes = ctx->cls_bytes[cls];
    return SQD_OK;
}

int sqd_launch_count(const sqd_ctx *ctx, int64_t *launches) {
    if (!ctx || !launches) return fail_noctx(SQD_EINVAL, "sqd_launch_count: NULL argument");
    *launches = ctx->launches;
    return SQD_OK;
}

int sqd_measure_fp64_peaks(sqd_ctx *ctx, double *dfma_tflops, double *dmma_tflops) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_measure_fp64_peaks: ctx is NULL");
    SQD_TRY(use_device(ctx));
    return measure_fp64_peaks(ctx, dfma_tflops, dmma_tflops);
}

const char *sqd_last_error(const sqd_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

// --------------------------------------------------------- a1: strings --

int sqd_build_strings(sqd_ctx *ctx, const uint64_t *d_raw, int64_t n_raw, int norb, int nelec,
                      uint64_t *d_out, int64_t *n_out) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_build_strings: ctx is NULL");
    if (!n_out) return sqd_fail(ctx, SQD_EINVAL, "sqd_build_strings: n_out is NULL");
    *n_out = 0;
    if (norb < 1 || norb > 64) return sqd_fail(ctx, SQD_EINVAL, "norb must be in [1, 64]");
    if (nelec < 0 || nelec > norb) return sqd_fail(ctx, SQD_EINVAL, "nelec must be in [0, norb]");
    if (n_raw < 0) return sqd_fail(ctx, SQD_EINVAL, "n_raw < 0");
    if (n_raw == 0) return SQD_OK;
    if (!d_raw || !d_out) return sqd_fail(ctx, SQD_EINVAL, "NULL string buffer");
    SQD_TRY(use_device(ctx));
    prof_begin(ctx, PROF_STRINGS);
    cudaStream_t st = ctx->stream;
    int64_t *flags = nullptr, *pos = nullptr, *tot = nullptr;
    uint64_t *keys = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&flags, sizeof(int64_t) * n_raw, st));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&pos, sizeof(int64_t) * n_raw, st));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&tot, sizeof(int64_t), st));
    SQD_TRY(launch_filter_flags(ctx, d_raw, n_raw, norb, nelec, flags));
    SQD_TRY(launch_exclusive_scan(ctx, flags, pos, n_raw, tot));
    int64_t m = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t P = next_pow2(m > 0 ? m : 1);
    SQD_CUDA(ctx, cudaMallocAsync((void **)&keys, sizeof(uint64_t) * P, st));
    SQD_TRY(launch_fill_u64(ctx, keys, P, ~0ull));
    SQD_TRY(launch_scatter_flagged(ctx, d_raw, flags, pos, n_raw, keys));
    SQD_TRY(launch_bitonic_sort_u64(ctx, keys, P));
    // keys[0..m) sorted; mark first occurrences and compact into d_out
    SQD_TRY(launch_unique_flags(ctx, keys, m, flags));
    SQD_TRY(launch_exclusive_scan(ctx, flags, pos, m, tot));
    SQD_TRY(launch_scatter_flagged(ctx, keys, flags, pos, m, d_out));
    int64_t u = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&u, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SQD_CUDA(ctx, cudaFreeAsync(flags, st));
    SQD_CUDA(ctx, cudaFreeAsync(pos, st));
    SQD_CUDA(ctx, cudaFreeAsync(tot, st));
    SQD_CUDA(ctx, cudaFreeAsync(keys, st));
    prof_end(ctx, 0.0, 8.0 * n_raw);
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    *n_out = m > 0 ? u : 0;
    return SQD_OK;
}

// ----------------------------------------------------------- a2-a4 ------

static void free_spin(spin_tables *s) {
    void *ptrs[] = {s->str,  s->off1, s->tgt1,   s->pq1, s->sgn1, s->val1,  s->src1, s->off2,
                    s->tgt2, s->orb2, s->sgn2,   s->val2, s->energy, s->W, s->u,
                    s->val1f, s->val2f, s->Wf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    *s = spin_tables();
}

static int build_kind(sqd_ctx *ctx, sqd_tables *t, spin_tables *s, int kind) {
    cudaStream_t st = ctx->stream;
    const int64_t n = s->n;
    int64_t *counts = nullptr, *cursor = nullptr, *tot = nullptr, *off = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&counts, sizeof(int64_t) * n, st));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&cursor, sizeof(int64_t) * n, st));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&tot, sizeof(int64_t), st));
    SQD_TRY(dalloc(ctx, &off, n + 1, &t->bytes));
    SQD_TRY(launch_count_excitations(ctx, s->str, n, t->norb, kind, counts));
    SQD_TRY(launch_exclusive_scan(ctx, counts, off, n, off + n));
    int64_t nnz = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&nnz, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t P = next_pow2(nnz > 0 ? nnz : 1);
    uint64_t *keys = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&keys, sizeof(uint64_t) * P, st));
    SQD_TRY(launch_fill_u64(ctx, keys, P, ~0ull));
    SQD_TRY(launch_fill_excitations(ctx, s->str, n, t->norb, kind, off, cursor, keys));
    SQD_TRY(launch_bitonic_sort_u64(ctx, keys, P));
    std::vector<int64_t> hoff(n + 1);
    SQD_CUDA(ctx, cudaMemcpyAsync(hoff.data(), off, sizeof(int64_t) * (n + 1),
                                  cudaMemcpyDeviceToHost, st));
    if (kind == 1) {
        s->nnz1 = nnz;
        s->off1 = off;
        SQD_TRY(dalloc(ctx, &s->tgt1, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->pq1, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->sgn1, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->val1, nnz, &t->bytes));
        SQD_TRY(launch_finalize_singles(ctx, s->str, t->norb, keys, nnz, t->h, t->V, s->tgt1,
                                        s->pq1, s->sgn1, s->val1));
    } else {
        s->nnz2 = nnz;
        s->off2 = off;
        SQD_TRY(dalloc(ctx, &s->tgt2, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->orb2, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->sgn2, nnz, &t->bytes));
        SQD_TRY(dalloc(ctx, &s->val2, nnz, &t->bytes));
        SQD_TRY(launch_finalize_doubles(ctx, s->str, t->norb, keys, nnz, t->V, s->tgt2, s->orb2,
                                        s->sgn2, s->val2));
    }
    SQD_CUDA(ctx, cudaFreeAsync(keys, st));
    SQD_CUDA(ctx, cudaFreeAsync(counts, st));
    SQD_CUDA(ctx, cudaFreeAsync(cursor, st));
    SQD_CUDA(ctx, cudaFreeAsync(tot, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t mx = 0;
    for (int64_t i = 0; i < n; i++) mx = std::max(mx, hoff[i + 1] - hoff[i]);
    if (kind == 1) {
        s->max1 = mx;
        s->h_off1 = std::move(hoff);
    } else {
        s->max2 = mx;
    }
    return SQD_OK;
}

static int build_spin(sqd_ctx *ctx, sqd_tables *t, spin_tables *s, const uint64_t *d_str,
                      int64_t n, int ne) {
    s->n = n;
    s->ne = ne;
    SQD_TRY(dalloc(ctx, &s->str, n, &t->bytes));
    SQD_CUDA(ctx, cudaMemcpyAsync(s->str, d_str, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SQD_TRY(build_kind(ctx, t, s, 1));
    SQD_TRY(build_kind(ctx, t, s, 2));
    const int64_t n2 = (int64_t)t->norb * t->norb;
    SQD_TRY(dalloc(ctx, &s->energy, n, &t->bytes));
    SQD_TRY(dalloc(ctx, &s->W, n2 * n, &t->bytes));
    SQD_TRY(launch_string_terms(ctx, s->str, n, t->norb, t->h, t->V, s->energy, s->W, nullptr));
    return SQD_OK;
}

static int check_set(sqd_ctx *ctx, const uint64_t *d, int64_t n, int norb, int ne,
                     const char *name) {
    int *bad = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&bad, sizeof(int), ctx->stream));
    SQD_CUDA(ctx, cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    SQD_TRY(launch_check_sorted_unique(ctx, d, n, norb, ne, bad));
    int hb = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(bad, ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hb & 1) return sqd_fail(ctx, SQD_EINVAL, "%s strings: wrong electron count", name);
    if (hb & 2) return sqd_fail(ctx, SQD_EINVAL, "%s strings: orbital index >= norb", name);
    if (hb & 4) return sqd_fail(ctx, SQD_EINVAL, "%s strings: not sorted ascending/unique", name);
    return SQD_OK;
}

static int tables_impl(sqd_ctx *ctx, sqd_tables *t, int norb, const uint64_t *d_alpha,
                       int64_t n_alpha, int nalpha_e, const uint64_t *d_beta, int64_t n_beta,
                       int nbeta_e, const double *d_h, const double *d_V, double ecore) {
    const int64_t n2 = (int64_t)norb * norb, n4 = n2 * n2;
    SQD_TRY(check_set(ctx, d_alpha, n_alpha, norb, nalpha_e, "alpha"));
    SQD_TRY(check_set(ctx, d_beta, n_beta, norb, nbeta_e, "beta"));
    double *res = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&res, sizeof(double) * 3, ctx->stream));
    SQD_CUDA(ctx, cudaMemsetAsync(res, 0, sizeof(double) * 3, ctx->stream));
    SQD_TRY(launch_check_integrals(ctx, d_h, d_V, norb, res));
    double hres[3];
    SQD_CUDA(ctx, cudaMemcpyAsync(hres, res, sizeof(hres), cudaMemcpyDeviceToHost, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(res, ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hres[2] != 0.0) return sqd_fail(ctx, SQD_EINVAL, "integrals contain NaN or Inf");
    if (hres[0] > 1e-10 * std::max(1.0, hres[1]))
        return sqd_fail(ctx, SQD_EINVAL,
                        "integrals are not symmetric (max deviation %.3e): h must be symmetric "
                        "and V 8-fold symmetric",
                        hres[0]);
    t->norb = norb;
    t->ecore = ecore;
    SQD_TRY(dalloc(ctx, &t->h, n2, &t->bytes));
    SQD_TRY(dalloc(ctx, &t->V, n4, &t->bytes));
    SQD_CUDA(ctx, cudaMemcpyAsync(t->h, d_h, sizeof(double) * n2, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SQD_CUDA(ctx, cudaMemcpyAsync(t->V, d_V, sizeof(double) * n4, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    SQD_TRY(build_spin(ctx, t, &t->a, d_alpha, n_alpha, nalpha_e));
    t->shared = (d_alpha == d_beta && n_alpha == n_beta && nalpha_e == nbeta_e);
    if (t->shared) {
        t->b = &t->a;
    } else {
        SQD_TRY(build_spin(ctx, t, &t->b_own, d_beta, n_beta, nbeta_e));
        t->b = &t->b_own;
    }
    SQD_TRY(dalloc(ctx, &t->diag, n_alpha * n_beta, &t->bytes));
    SQD_TRY(launch_diagonal(ctx, &t->a, t->b, norb, ecore, t->a.str, t->diag));
    SQD_TRY(build_ab_schedule(ctx, t));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return SQD_OK;
}

int sqd_excitation_tables(sqd_ctx *ctx, int norb, const uint64_t *d_alpha, int64_t n_alpha,
                          int nalpha_e, const uint64_t *d_beta, int64_t n_beta, int nbeta_e,
                          const double *d_h, const double *d_V, double ecore,
                          sqd_tables **tables) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_excitation_tables: ctx is NULL");
    if (!tables) return sqd_fail(ctx, SQD_EINVAL, "tables is NULL");
    *tables = nullptr;
    if (norb < 1 || norb > 64) return sqd_fail(ctx, SQD_EINVAL, "norb must be in [1, 64]");
    if (nalpha_e < 0 || nalpha_e > norb || nbeta_e < 0 || nbeta_e > norb)
        return sqd_fail(ctx, SQD_EINVAL, "electron count must be in [0, norb]");
    if (n_alpha < 1 || n_beta < 1) return sqd_fail(ctx, SQD_EINVAL, "empty string set");
    if (n_alpha >= (1LL << 31) || n_beta >= (1LL << 31))
        return sqd_fail(ctx, SQD_EINVAL, "string set too large (>= 2^31)");
    if ((double)n_alpha * (double)n_beta >= 1099511627776.0)
        return sqd_fail(ctx, SQD_EINVAL, "subspace too large (>= 2^40 determinants)");
    if (!d_alpha || !d_beta || !d_h || !d_V) return sqd_fail(ctx, SQD_EINVAL, "NULL input");
    if (!std::isfinite(ecore)) return sqd_fail(ctx, SQD_EINVAL, "ecore is not finite");
    SQD_TRY(use_device(ctx));
    sqd_tables *t = new sqd_tables();
    t->ctx = ctx;
    prof_begin(ctx, PROF_TABLES);
    int r = tables_impl(ctx, t, norb, d_alpha, n_alpha, nalpha_e, d_beta, n_beta, nbeta_e, d_h,
                        d_V, ecore);
    prof_end(ctx, 0.0, 0.0);
    if (r != SQD_OK) {
        cudaStreamSynchronize(ctx->stream);
        sqd_free_tables(t);
        return r;
    }
    *tables = t;
    return SQD_OK;
}

void sqd_free_tables(sqd_tables *t) {
    if (!t) return;
    if (t->ctx) cudaSetDevice(t->ctx->device);
    cudaDeviceSynchronize();
    free_spin(&t->a);
    if (!t->shared) free_spin(&t->b_own);
    void *ptrs[] = {t->h,         t->V,          t->diag,       t->ab.chunk_e, t->ab.chunk_y,
                    t->ab.chunk_e_wide, t->ab.chunk_y_wide,
                    t->ab.group_rows, t->scratch_t, t->scratch_s, t->rdm_iket,
                    t->rdm_ibra,  t->rdm_ipq,    t->rdm_chunks, t->rdm_groups,
                    t->st_rowptr, t->st_col,     t->st_val,  t->Vf,
                    t->diagf,     t->scratch_c, t->scratch_h};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete t;
}

int sqd_tables_set_sigma_mode(sqd_tables *t, int mode) {
    if (!t) return fail_noctx(SQD_EINVAL, "sqd_tables_set_sigma_mode: tables is NULL");
    if (mode != 0 && mode != 1) return fail_noctx(SQD_EINVAL, "sigma mode must be 0 or 1");
    t->sigma_mode = mode;
    return SQD_OK;
}

int sqd_tables_set_spin_flip(sqd_tables *t, int sector) {
    if (!t) return fail_noctx(SQD_EINVAL, "sqd_tables_set_spin_flip: tables is NULL");
    if (sector < -1 || sector > 1)
        return fail_noctx(SQD_EINVAL, "spin-flip sector must be -1, 0 or +1");
    if (sector && !t->shared)
        return fail_noctx(SQD_EINVAL,
                          "spin flip needs one string set shared by both spins (the same "
                          "device array and electron count)");
    t->spin_flip = sector;
    return SQD_OK;
}

int sqd_tables_info(const sqd_tables *t, int64_t *info) {
    if (!t || !info) return fail_noctx(SQD_EINVAL, "sqd_tables_info: NULL argument");
    info[0] = t->norb;
    info[1] = t->a.n;
    info[2] = t->b->n;
    info[3] = t->a.nnz1;
    info[4] = t->a.nnz2;
    info[5] = t->b->nnz1;
    info[6] = t->b->nnz2;
    info[7] = t->shared ? 1 : 0;
    info[8] = t->bytes;
    info[9] = std::max(t->a.max1, t->b->max1);
    info[10] = std::max(t->a.max2, t->b->max2);
    info[11] = t->ab.ngroups;
    return SQD_OK;
}

int sqd_tables_export(sqd_ctx *ctx, const sqd_tables *t, int spin, int kind, int64_t *h_off,
                      int32_t *h_tgt, uint8_t *h_orb, int8_t *h_sign, double *h_val) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_tables_export: NULL argument");
    if ((spin != 0 && spin != 1) || (kind != 1 && kind != 2))
        return sqd_fail(ctx, SQD_EINVAL, "spin must be 0/1 and kind 1/2");
    SQD_TRY(use_device(ctx));
    const spin_tables *s = spin ? t->b : &t->a;
    int64_t n = s->n, nnz = kind == 1 ? s->nnz1 : s->nnz2;
    cudaStream_t st = ctx->stream;
    if (h_off)
        SQD_CUDA(ctx, cudaMemcpyAsync(h_off, kind == 1 ? s->off1 : s->off2,
                                      sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st));
    if (nnz > 0) {
        if (h_tgt)
            SQD_CUDA(ctx, cudaMemcpyAsync(h_tgt, kind == 1 ? s->tgt1 : s->tgt2,
                                          sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st));
        if (h_sign)
            SQD_CUDA(ctx, cudaMemcpyAsync(h_sign, kind == 1 ? s->sgn1 : s->sgn2, nnz,
                                          cudaMemcpyDeviceToHost, st));
        if (h_val)
            SQD_CUDA(ctx, cudaMemcpyAsync(h_val, kind == 1 ? s->val1 : s->val2,
                                          sizeof(double) * nnz, cudaMemcpyDeviceToHost, st));
    }
    std::vector<uint16_t> pq;
    if (h_orb && nnz > 0) {
        if (kind == 2) {
            SQD_CUDA(ctx, cudaMemcpyAsync(h_orb, s->orb2, sizeof(uint32_t) * nnz,
                                          cudaMemcpyDeviceToHost, st));
        } else {
            pq.resize(nnz);
            SQD_CUDA(ctx, cudaMemcpyAsync(pq.data(), s->pq1, sizeof(uint16_t) * nnz,
                                          cudaMemcpyDeviceToHost, st));
        }
    }
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    if (!pq.empty()) {
        for (int64_t e = 0; e < nnz; e++) {
            h_orb[2 * e] = (uint8_t)(pq[e] / t->norb);
            h_orb[2 * e + 1] = (uint8_t)(pq[e] % t->norb);
        }
    }
    return SQD_OK;
}

int sqd_diagonal(sqd_ctx *ctx, const sqd_tables *t, double *d_diag) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_diagonal: NULL argument");
    if (!d_diag) return sqd_fail(ctx, SQD_EINVAL, "d_diag is NULL");
    SQD_TRY(use_device(ctx));
    SQD_CUDA(ctx, cudaMemcpyAsync(d_diag, t->diag, sizeof(double) * t->a.n * t->b->n,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    return SQD_OK;
}

// ------------------------------------------------------------ a5-a7 -----

static int ensure_scratch(sqd_ctx *ctx, sqd_tables *t) {
    const int64_t N = t->a.n * t->b->n;
    if (!t->scratch_t) SQD_TRY(dalloc(ctx, &t->scratch_t, N, &t->bytes));
    if (!t->scratch_s) SQD_TRY(dalloc(ctx, &t->scratch_s, N, &t->bytes));
    return SQD_OK;
}

// Algorithmic FP64 flops of the sigma terms (2 per multiply-add):
//  alpha side: N (diagonal) + nb*(2*nnz1_a + nnz2_a)   [single: value + W coupling]
//  beta side : na*(2*nnz1_b + nnz2_b)
//  alpha-beta: nnz1_a * nnz1_b
// and their compulsory HBM bytes (read C, read/write sigma, the diagonal).
extern "C++" void sigma_work(const sqd_tables *t, double *f_a, double *f_b, double *f_ab) {
    const double na = (double)t->a.n, nb = (double)t->b->n;
    *f_a = 2.0 * (na * nb + nb * (2.0 * t->a.nnz1 + t->a.nnz2));
    *f_b = 2.0 * na * (2.0 * t->b->nnz1 + t->b->nnz2);
    *f_ab = 2.0 * (double)t->a.nnz1 * (double)t->b->nnz1;
}

static int ab_launch_fp64(sqd_ctx *ctx, sqd_tables *t, const void *C, double *S) {
    return launch_alpha_beta(ctx, t, (const double *)C, S);
}

static int sigma_impl(sqd_ctx *ctx, sqd_tables *t, const double *C, double *S, int nvec) {
    const int64_t na = t->a.n, nb = t->b->n, N = na * nb;
    const double vb = 8.0 * (double)N;
    double f_a, f_b, f_ab;
    sigma_work(t, &f_a, &f_b, &f_ab);
    SQD_TRY(ensure_scratch(ctx, t));
    if (t->sigma_mode == 1) {
        SQD_TRY(df_prepare(ctx, t));
        for (int v = 0; v < nvec; v++)
            SQD_TRY(sigma_df_one(ctx, t, C + (int64_t)v * N, S + (int64_t)v * N, f_a, f_b, f_ab));
        return SQD_OK;
    }
    SQD_TRY(tune_ab_groups(ctx, t, 0, ab_launch_fp64, C));
    if (t->spin_flip) {
        // C^T = s C: sigma = (T + s T^T) + H_II C + (Y + s Y^T) with T the
        // alpha side and Y the paired singles of the upper triangle Ch
        const int s = t->spin_flip;
        if (!t->scratch_h) SQD_TRY(dalloc(ctx, &t->scratch_h, N, &t->bytes));
        double fu = 0.0;
        SQD_TRY(alpha_beta_upper_work(ctx, t, &fu));
        for (int v = 0; v < nvec; v++) {
            const double *Cv = C + (int64_t)v * N;
            double *Sv = S + (int64_t)v * N;
            prof_begin(ctx, PROF_SAME_ALPHA);
            SQD_TRY(launch_same_spin(ctx, &t->a, t->b, na, nb, Cv, t->scratch_s, nullptr));
            prof_end(ctx, f_a - 2.0 * (double)N, 2 * vb);
            prof_begin(ctx, PROF_TRANSPOSE);
            SQD_TRY(launch_upper_half(ctx, s, Cv, t->scratch_h, na));
            SQD_CUDA(ctx, cudaMemsetAsync(t->scratch_t, 0, sizeof(double) * N, ctx->stream));
            prof_end(ctx, 0.0, 3 * vb);
            prof_begin(ctx, PROF_ALPHA_BETA);
            SQD_TRY(launch_alpha_beta_upper(ctx, t, t->scratch_h, t->scratch_t));
            prof_end(ctx, 2.0 * fu, 3 * vb);
            prof_begin(ctx, PROF_TRANSPOSE);
            SQD_TRY(launch_sym_combine(ctx, s, t->scratch_s, t->scratch_t, t->diag, Cv, Sv, na));
            prof_end(ctx, 2.0 * (double)N, 6 * vb);
        }
        return SQD_OK;
    }
    for (int v = 0; v < nvec; v++) {
        const double *Cv = C + (int64_t)v * N;
        double *Sv = S + (int64_t)v * N;
        // alpha side (+ diagonal): writes sigma
        prof_begin(ctx, PROF_SAME_ALPHA);
        SQD_TRY(launch_same_spin(ctx, &t->a, t->b, na, nb, Cv, Sv, t->diag));
        prof_end(ctx, f_a, 3 * vb);
        // alpha-beta paired singles: adds into sigma
        prof_begin(ctx, PROF_ALPHA_BETA);
        SQD_TRY(launch_alpha_beta(ctx, t, Cv, Sv));
        prof_end(ctx, f_ab, 3 * vb);
        // beta side on C^T, added back transposed
        prof_begin(ctx, PROF_TRANSPOSE);
        SQD_TRY(launch_transpose(ctx, Cv, t->scratch_t, na, nb, false));
        prof_end(ctx, 0.0, 2 * vb);
        prof_begin(ctx, PROF_SAME_BETA);
        SQD_TRY(launch_same_spin(ctx, t->b, &t->a, nb, na, t->scratch_t, t->scratch_s, nullptr));
        prof_end(ctx, f_b, 2 * vb);
        prof_begin(ctx, PROF_TRANSPOSE);
        SQD_TRY(launch_transpose(ctx, t->scratch_s, Sv, nb, na, true));
        prof_end(ctx, 0.0, 3 * vb);
    }
    return SQD_OK;
}

int sqd_sigma(sqd_ctx *ctx, sqd_tables *t, const double *d_C, double *d_sigma, int nvec) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_sigma: NULL argument");
    if (nvec < 1) return sqd_fail(ctx, SQD_EINVAL, "nvec must be >= 1");
    if (!d_C || !d_sigma) return sqd_fail(ctx, SQD_EINVAL, "NULL vector");
    if (d_C == d_sigma) return sqd_fail(ctx, SQD_EINVAL, "d_C and d_sigma must differ");
    SQD_TRY(use_device(ctx));
    return sigma_impl(ctx, t, d_C, d_sigma, nvec);
}

// --------------------------------------------------------- a8: Davidson --

struct dav_work {
    double *Vb = nullptr, *Wb = nullptr, *X = nullptr, *R = nullptr, *Tmp = nullptr;
    double *G = nullptr, *evals = nullptr, *evecs = nullptr, *dots = nullptr, *partial = nullptr;
    double *phase = nullptr, *Yprev = nullptr, *Z = nullptr, *P = nullptr, *GZ = nullptr;
    double *tn2 = nullptr, *Eold = nullptr, *thold = nullptr;
    int64_t *idx = nullptr;
    int *rdev = nullptr, *sel = nullptr;
    ~dav_work() {
        void *p[] = {Vb, Wb, X, R, Tmp, G, evals, evecs, dots, partial, phase, idx, Yprev, Z, P,
                     GZ, tn2, Eold, thold, rdev, sel};
        for (void *q : p)
            if (q) cudaFree(q);
    }
};

// Block Davidson with GD+k restart.  Per iteration: Rayleigh-Ritz on the
// projected matrix G = V^T H V (one-block Jacobi), Ritz vectors and residuals
// of the nroots lowest pairs in one pass over V and W, convergence test, the
// preconditioned residuals of the unconverged roots as one new block,
// Gram-Schmidt of that block against V (block classical Gram-Schmidt, two
// passes when the first lost more than half a vector's squared norm), then
// within the block (CGS twice per vector, dropping vectors below 1e-12; from
// the block's Gram matrix where that is resolved), H applied to the block and
// the new columns of G.  In exact
// arithmetic this is the same basis as vector-by-vector CGS2 of the
// preconditioned residuals in root order.
//
// Second block Gram-Schmidt pass when a vector lost more than this fraction
// of its squared norm in the first (Daniel-Gragg-Kaufman-Stewart test with
// eta^2 = 1 - SQD_REORTH_LOSS), decided on the device.
#ifndef SQD_REORTH_LOSS
#define SQD_REORTH_LOSS 0.5
#endif

// One root (block width one, m <= 16, Davidson correction): the fused passes
// of k_davidson.cu form the correction and its first projections in the pass
// that reads V and W for the Ritz pair (the Ritz vector is formed only on
// exit), fuse the first update with the second projections, and the second
// update with the normalisation, whose norm follows from Pythagoras
// (|t''|^2 = |t'|^2 - |V^T t'|^2 for orthonormal V).  Where that difference
// is not safely resolved (the second pass removed more than half of |t'|^2,
// or |t''| < 1e-10) the norm is taken explicitly, as in the general path.

static int davidson_impl(sqd_ctx *ctx, sqd_tables *t, const sqd_options *o, double *h_energies,
                         double *d_C, int *h_iters, double *h_res) {
    cudaStream_t st = ctx->stream;
    const int64_t N = t->a.n * t->b->n;
    const int k = o->nroots;
    int M = o->max_subspace > 0 ? o->max_subspace : std::max(6 * k, 16);
    if (M > SQD_MAX_SUBSPACE) M = SQD_MAX_SUBSPACE;
    if ((int64_t)M > N) M = (int)N;
    if (M < std::min<int64_t>(4 * k, N))
        return sqd_fail(ctx, SQD_EINVAL, "max_subspace must be >= 4*nroots (or the dimension)");
    const int nblk = multidot_blocks(N);
    const int nbd = block_dot_blocks(ctx, N);
    const int nbr = 4 * ctx->sm_count;
    const int k2 = std::min(2 * k, M);
    const int kr = std::min(3 * k, M);  // restart basis: 2k Ritz + k previous Ritz
    // one-root fused passes (register-resident projections need m <= MDf)
    const int MDf = (k == 1 && o->correction == 0) ? fused_md(M) : 0;
    dav_work w;
    // partial sums: multidot (M x nblk), block dot (nbd x M x k), Ritz (nbr x k),
    // preconditioner with Olsen's dots (2 x nbr + 2), fused passes (nbr x (MDf + 2))
    // packed Gram of a block of up to 8 (nbr x 36)
    const int64_t npart = std::max<int64_t>(
        std::max<int64_t>(std::max<int64_t>((int64_t)M * nblk, (int64_t)nbd * M * k),
                          std::max<int64_t>((int64_t)nbr * std::max(k, 1), 2LL * nbr + 2)),
        std::max<int64_t>((int64_t)nbr * (MDf + 2), (int64_t)nbr * 36));
    SQD_TRY(dalloc(ctx, &w.Vb, (int64_t)M * N));
    SQD_TRY(dalloc(ctx, &w.Wb, (int64_t)M * N));
    SQD_TRY(dalloc(ctx, &w.X, (int64_t)k * N));
    SQD_TRY(dalloc(ctx, &w.R, (int64_t)k * N));
    if (!MDf) SQD_TRY(dalloc(ctx, &w.Tmp, (int64_t)kr * N));
    SQD_TRY(dalloc(ctx, &w.Yprev, (int64_t)M * k));
    SQD_TRY(dalloc(ctx, &w.Z, (int64_t)M * kr));
    SQD_TRY(dalloc(ctx, &w.P, (int64_t)M * k + 3 * (MDf + 2)));
    SQD_TRY(dalloc(ctx, &w.GZ, (int64_t)M * kr));
    SQD_TRY(dalloc(ctx, &w.tn2, k));
    SQD_TRY(dalloc(ctx, &w.rdev, 2));  // [0] restart size, [1] second-pass gate
    SQD_TRY(dalloc(ctx, &w.sel, k));
    SQD_TRY(dalloc(ctx, &w.G, (int64_t)M * M));
    SQD_TRY(dalloc(ctx, &w.evals, M));
    SQD_TRY(dalloc(ctx, &w.evecs, (int64_t)M * M));
    SQD_TRY(dalloc(ctx, &w.Eold, (int64_t)M * M));
    SQD_TRY(dalloc(ctx, &w.thold, M));
    SQD_TRY(dalloc(ctx, &w.dots, M));
    SQD_TRY(dalloc(ctx, &w.partial, npart));
    SQD_TRY(dalloc(ctx, &w.phase, 3 * 4 * ctx->sm_count + 8));
    SQD_TRY(dalloc(ctx, &w.idx, k));
    SQD_TRY(ensure_scratch(ctx, t));
    const double dN = (double)N;
    // fused-pass sums: s1 = (V^T t, |r|^2, |t|^2), s2 = (V^T t', |t'|^2), s3 = restarted V^T t
    double *s1 = w.P + (int64_t)M * k, *s2 = s1 + (MDf + 2), *s3 = s2 + (MDf + 2);

    // G[0..m, m0..m0+b) = V[0..m)^T W[m0..m0+b) (one new vector of a one-root
    // solve: the register-resident dot pass)
    auto g_cols = [&](int m, int m0, int b) -> int {
        prof_begin(ctx, PROF_GCOLS);
        if (b == 1 && MDf && m <= MDf)
            SQD_TRY(launch_dots_one(ctx, MDf, w.Vb, N, m, w.Wb + (int64_t)m0 * N, N, w.partial,
                                    nbr, w.G + (int64_t)m0 * M));
        else
            SQD_TRY(launch_block_dot(ctx, w.Vb, N, m, w.Wb + (int64_t)m0 * N, N, b, N, w.partial,
                                     nbd, w.G + (int64_t)m0 * M, M));
        prof_end(ctx, 2.0 * m * b * dN, 8.0 * (m + b) * dN);
        return SQD_OK;
    };
    // Within-block Gram-Schmidt of the vectors V[m0..m0+b) (already
    // orthogonal to V[0..m0)): CGS twice per vector against the accepted
    // ones, drop below 1e-12, normalise; accepted vectors are packed to
    // V[m0..m0+*nacc).
    auto within_block = [&](int m0, int b, int *nacc) -> int {
        double *T = w.Vb + (int64_t)m0 * N;
        int acc = 0;
        for (int j = 0; j < b; j++) {
            double *dst = T + (int64_t)acc * N;
            if (acc != j)
                SQD_CUDA(ctx, cudaMemcpyAsync(dst, T + (int64_t)j * N, sizeof(double) * N,
                                              cudaMemcpyDeviceToDevice, st));
            prof_begin(ctx, PROF_ORTHO_BLOCK);
            for (int pass = 0; pass < 2 && acc > 0; pass++) {
                SQD_TRY(launch_multidot(ctx, T, N, acc, dst, N, w.partial, nblk, w.dots));
                SQD_TRY(launch_gemv_sub(ctx, T, N, acc, w.dots, dst, N));
            }
            SQD_TRY(launch_multidot(ctx, dst, N, 1, dst, N, w.partial, nblk, w.dots));
            prof_end(ctx, (8.0 * acc + 2.0) * dN, 8.0 * (4.0 * acc + 5.0) * dN);
            double n2 = 0.0;
            SQD_CUDA(ctx, cudaMemcpyAsync(&n2, w.dots, sizeof(double), cudaMemcpyDeviceToHost, st));
            SQD_CUDA(ctx, cudaStreamSynchronize(st));
            if (!(std::sqrt(n2) >= 1e-12)) continue;  // dropped
            SQD_TRY(launch_scale(ctx, dst, N, w.dots, 1));
            acc++;
        }
        *nacc = acc;
        return SQD_OK;
    };
    // Within-block Gram-Schmidt of b >= 2 vectors from their Gram matrix
    // (one block-dot pass instead of a chain of per-vector passes and host
    // round trips): CGS twice on the b x b Gram matrix in order gives the
    // coefficients Z (upper triangular) of the same orthonormal vectors,
    // Q = T Z, which are formed in one pass; a second round on the Gram
    // matrix of Q removes the rounding the first left (Cholesky QR twice,
    // Fukaya et al. 2014).  Used only while every vector keeps at least
    // 1e-8 of its squared norm (|t| > 1e-10 too), where the Gram matrix
    // resolves the result; otherwise *ok = false and nothing was changed.
    std::vector<double> hG, hZ;
    // work of the last gated second pass, booked when its flag is read
    double pend_f = 0.0, pend_b = 0.0;
    int gate_h = 0;
    auto book_gated = [&]() {
        if (ctx->prof && gate_h && pend_f > 0.0) {
            ctx->cls_flops[PROF_ORTHO] += pend_f;
            ctx->cls_bytes[PROF_ORTHO] += pend_b;
        }
        pend_f = pend_b = 0.0;
    };
    auto within_block_gram = [&](int m0, int b, int *nacc, bool *ok) -> int {
        double *T = w.Vb + (int64_t)m0 * N;
        double *Zd = w.GZ;
        *ok = false;
        hG.assign((size_t)b * b, 0.0);
        hZ.assign((size_t)b * b, 0.0);
        for (int round = 0; round < 2; round++) {
            prof_begin(ctx, PROF_ORTHO_BLOCK);
            if (b <= 8) {  // upper triangle only, unpacked on the host
                SQD_TRY(launch_gram_tri(ctx, T, N, b, N, w.partial, nbr, w.P));
                prof_end(ctx, 1.0 * b * (b + 1) * dN, 8.0 * b * dN);
                double packed[36];
                SQD_CUDA(ctx, cudaMemcpyAsync(packed, w.P, sizeof(double) * b * (b + 1) / 2,
                                              cudaMemcpyDeviceToHost, st));
                SQD_CUDA(ctx, cudaStreamSynchronize(st));
                for (int j = 0; j < b; j++)
                    for (int i = 0; i <= j; i++)
                        hG[i + (size_t)j * b] = hG[j + (size_t)i * b] = packed[j * (j + 1) / 2 + i];
            } else {
                SQD_TRY(launch_block_dot(ctx, T, N, b, T, N, b, N, w.partial, nbd, w.P, b));
                prof_end(ctx, 2.0 * b * b * dN, 16.0 * b * dN);
                SQD_CUDA(ctx, cudaMemcpyAsync(hG.data(), w.P, sizeof(double) * b * b,
                                              cudaMemcpyDeviceToHost, st));
                SQD_CUDA(ctx, cudaStreamSynchronize(st));
            }
            std::fill(hZ.begin(), hZ.end(), 0.0);
            std::vector<double> z(b), gz(b);
            for (int j = 0; j < b; j++) {
                std::fill(z.begin(), z.end(), 0.0);
                z[j] = 1.0;
                for (int pass = 0; pass < 2; pass++) {
                    for (int l = 0; l < b; l++) {  // gz = G z
                        double a = 0.0;
                        for (int q = 0; q < b; q++) a += hG[l + (size_t)q * b] * z[q];
                        gz[l] = a;
                    }
                    std::vector<double> c(j, 0.0);
                    for (int i = 0; i < j; i++)  // c_i = Q_i . (T z) = Z_i^T G z
                        for (int l = 0; l < b; l++) c[i] += hZ[l + (size_t)i * b] * gz[l];
                    for (int i = 0; i < j; i++)
                        for (int l = 0; l < b; l++) z[l] -= c[i] * hZ[l + (size_t)i * b];
                }
                double n2 = 0.0;
                for (int l = 0; l < b; l++) {
                    double a = 0.0;
                    for (int q = 0; q < b; q++) a += hG[l + (size_t)q * b] * z[q];
                    n2 += z[l] * a;
                }
                const double d = hG[j + (size_t)j * b];
                if (!(n2 >= 1e-8 * d) || !(n2 >= 1e-20)) {
                    if (round == 0) return SQD_OK;  // not resolved: explicit path
                    return sqd_fail(ctx, SQD_EBREAKDOWN, "block lost orthogonality");
                }
                const double inv = 1.0 / std::sqrt(n2);
                for (int l = 0; l < b; l++) hZ[l + (size_t)j * b] = z[l] * inv;
            }
            SQD_CUDA(ctx, cudaMemcpyAsync(Zd, hZ.data(), sizeof(double) * b * b,
                                          cudaMemcpyHostToDevice, st));
            prof_begin(ctx, PROF_ORTHO_BLOCK);
            if (b <= 8) {  // Z is upper triangular
                SQD_TRY(launch_combine_tri(ctx, T, N, b, Zd, b, N));
            } else {
                SQD_TRY(launch_combine(ctx, T, N, b, Zd, b, b, w.Tmp, N, N));
                SQD_CUDA(ctx, cudaMemcpyAsync(T, w.Tmp, sizeof(double) * b * N,
                                              cudaMemcpyDeviceToDevice, st));
            }
            prof_end(ctx, 1.0 * b * (b + 1) * dN, 8.0 * 2.0 * b * dN);
        }
        *nacc = b;
        *ok = true;
        return SQD_OK;
    };
    // Orthonormalise the block T = V[m0..m0+b) against V[0..m0) (block CGS)
    // and within itself.  The second block pass runs when some vector lost
    // more than half its squared norm in the first (Daniel-Gragg-Kaufman-
    // Stewart test), decided on the device: its kernels read the flag and
    // exit, so no host round trip sits between the passes.  tn2 (device) holds
    // the squared norms before the first pass; without it both passes run.
    auto orthonormalize_block = [&](int m0, int b, bool have_tn2, int *nacc) -> int {
        double *T = w.Vb + (int64_t)m0 * N;
        if (m0 > 0) {
            for (int pass = 0; pass < 2; pass++) {
                const int *gate = (pass == 1 && have_tn2) ? w.rdev + 1 : nullptr;
                prof_begin(ctx, PROF_ORTHO);
                SQD_TRY(launch_block_dot(ctx, w.Vb, N, m0, T, N, b, N, w.partial, nbd, w.P, m0,
                                         gate));
                if (pass == 0 && have_tn2)
                    SQD_TRY(launch_dgks_flag(ctx, w.P, m0, m0, b, w.tn2, SQD_REORTH_LOSS,
                                             w.rdev + 1));
                SQD_TRY(launch_combine_sub(ctx, w.Vb, N, m0, w.P, m0, b, T, N, N, gate));
                const double f = 4.0 * m0 * b * dN, by = 8.0 * (m0 + 2.0 * b) * dN + 8.0 * m0 * dN;
                if (gate) {
                    // a gated pass is booked once the host learns whether it ran
                    prof_end(ctx, 0.0, 0.0);
                    pend_f = f;
                    pend_b = by;
                } else {
                    prof_end(ctx, f, by);
                }
            }
        }
        if (b >= 2 && w.Tmp && b <= kr) {
            bool ok = false;
            SQD_TRY(within_block_gram(m0, b, nacc, &ok));
            if (ok) return SQD_OK;
        }
        return within_block(m0, b, nacc);
    };

    // spin flip: every basis vector is kept exactly in the sector
    // (C^T = s C), so the solve stays there whatever the rounding
    const int sflip = t->spin_flip;
    const int64_t nsym = sflip ? t->a.n : 0;
    auto symmetrize = [&](double *X, int cnt) -> int {
        if (!nsym) return SQD_OK;
        prof_begin(ctx, PROF_DAVIDSON);
        for (int q = 0; q < cnt; q++)
            SQD_TRY(launch_symmetrize(ctx, sflip, X + (int64_t)q * N, nsym));
        prof_end(ctx, 1.0 * cnt * dN, 32.0 * cnt * dN);
        return SQD_OK;
    };
    int m = 0;
    if (o->use_guess) {
        SQD_CUDA(ctx, cudaMemcpyAsync(w.Vb, d_C, sizeof(double) * k * N, cudaMemcpyDeviceToDevice,
                                      st));
        SQD_TRY(symmetrize(w.Vb, k));
        SQD_TRY(orthonormalize_block(0, k, false, &m));
        if (m < k) return sqd_fail(ctx, SQD_EINVAL, "initial guess vectors are linearly dependent");
    } else {
        SQD_CUDA(ctx, cudaMemsetAsync(w.Vb, 0, sizeof(double) * k * N, st));
        SQD_TRY(launch_argmin_k(ctx, t->diag, N, k, w.idx, sflip < 0 ? -nsym : nsym));
        if (nsym)
            SQD_TRY(launch_set_unit_sym(ctx, w.Vb, N, k, w.idx, nsym, sflip));
        else
            SQD_TRY(launch_set_unit(ctx, w.Vb, N, k, w.idx));
        m = k;
    }
    auto apply_h = [&](const double *Cin, double *Sout, int nv) -> int {
        if (o->use_stored_h) return stored_sigma(ctx, t, Cin, Sout, nv);
        return sigma_impl(ctx, t, Cin, Sout, nv);
    };
    if (o->use_stored_h && !t->st_rowptr)
        return sqd_fail(ctx, SQD_EINVAL, "use_stored_h set but sqd_stored_h_build was not called");
    SQD_TRY(apply_h(w.Vb, w.Wb, m));
    SQD_TRY(g_cols(m, 0, m));

    // Soft locking: a root that met both tests is locked and its Ritz vector
    // and residual are no longer formed; once every root is locked, one
    // iteration forms all of them and the solve ends only if every root
    // passes there (failing roots are unlocked and the solve goes on).
    // Energy test: the change of theta_j across the last growth of the basis.
    std::vector<double> theta(M), theta_old(k, INFINITY), dth(k, INFINITY), rn2(k), rn(k, INFINITY);
    std::vector<char> locked(k, 0);
    std::vector<int> sel;
    int it = 0;
    int mprev = 0;  // rows of Yprev (0: no previous Ritz vectors yet)
    int m_warm = 0;  // basis size of the previous eigensolve if the basis only grew since
    bool grown = true;  // basis changed since the previous eigensolve
    int status = SQD_OK;
    // Ritz vectors and residual norms of every root from the current eigensolve
    auto ritz_all = [&]() -> int {
        sel.clear();
        for (int j = 0; j < k; j++) sel.push_back(j);
        SQD_CUDA(ctx, cudaMemcpyAsync(w.sel, sel.data(), sizeof(int) * k, cudaMemcpyHostToDevice,
                                      st));
        SQD_TRY(launch_ritz_block(ctx, w.Vb, w.Wb, N, m, w.evecs, w.evals, w.sel, k, w.X, w.R, N,
                                  w.partial, nbr, w.dots));
        SQD_CUDA(ctx, cudaMemcpyAsync(rn2.data(), w.dots, sizeof(double) * k,
                                      cudaMemcpyDeviceToHost, st));
        SQD_CUDA(ctx, cudaMemcpyAsync(theta.data(), w.evals, sizeof(double) * m,
                                      cudaMemcpyDeviceToHost, st));
        SQD_CUDA(ctx, cudaStreamSynchronize(st));
        for (int j = 0; j < k; j++) rn[j] = std::sqrt(std::max(rn2[j], 0.0));
        return SQD_OK;
    };
    // GD+k restart basis Z (m x r) of the current eigensolve; returns r
    auto restart_basis = [&](int *r) -> int {
        const int m2 = std::min(k2, m);
        SQD_TRY(launch_gdk_basis(ctx, w.evecs, m, m2, mprev ? w.Yprev : nullptr, mprev, k, M,
                                 w.Z, M, w.rdev));
        *r = m2;
        SQD_CUDA(ctx, cudaMemcpyAsync(r, w.rdev, sizeof(int), cudaMemcpyDeviceToHost, st));
        SQD_CUDA(ctx, cudaStreamSynchronize(st));
        return SQD_OK;
    };
    // the basis only grew: keep the Ritz coefficients and seed the next eigensolve
    auto keep_coefficients = [&]() -> int {
        SQD_CUDA(ctx, cudaMemcpy2DAsync(w.Yprev, sizeof(double) * M, w.evecs, sizeof(double) * m,
                                        sizeof(double) * m, k, cudaMemcpyDeviceToDevice, st));
        mprev = m;
        SQD_CUDA(ctx, cudaMemcpyAsync(w.Eold, w.evecs, sizeof(double) * m * m,
                                      cudaMemcpyDeviceToDevice, st));
        SQD_CUDA(ctx, cudaMemcpyAsync(w.thold, w.evals, sizeof(double) * m,
                                      cudaMemcpyDeviceToDevice, st));
        m_warm = m;
        return SQD_OK;
    };

    if (MDf) {
        // ------------------------------------------ one root, fused passes --
        double hs[36];
        bool x_ready = false;
        for (;;) {
            prof_begin(ctx, PROF_EIGH);
            SQD_TRY(launch_jacobi_eigh(ctx, w.G, M, m, w.evals, w.evecs, m_warm, w.Eold,
                                       w.thold));
            prof_end(ctx, 0.0, 0.0);
            const bool restart = m + 1 > M;
            double *T = restart ? w.R : w.Vb + (int64_t)m * N;
            prof_begin(ctx, PROF_DAVIDSON);
            SQD_TRY(launch_ritz_prec_dot(ctx, MDf, w.Vb, w.Wb, N, m, w.evecs, w.evals, t->diag,
                                         o->precond_floor, N, T, w.partial, nbr, s1));
            prof_end(ctx, (6.0 * m + 7.0) * dN, 8.0 * (2.0 * m + 3.0) * dN);
            // (V^T t is unchanged by the symmetrisation: V is symmetric)
            SQD_TRY(symmetrize(T, 1));
            SQD_CUDA(ctx, cudaMemcpyAsync(hs, s1 + m, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                                          st));
            SQD_CUDA(ctx, cudaMemcpyAsync(theta.data(), w.evals, sizeof(double),
                                          cudaMemcpyDeviceToHost, st));
            SQD_CUDA(ctx, cudaStreamSynchronize(st));
            if (grown) dth[0] = std::fabs(theta[0] - theta_old[0]);
            theta_old[0] = theta[0];
            rn[0] = std::sqrt(std::max(hs[0], 0.0));
            if (rn[0] <= o->tol_residual && dth[0] <= o->tol_energy) break;
            if (it >= o->max_iter) {
                status = SQD_ENOTCONVERGED;
                break;
            }
            it++;
            const double *P1 = s1;
            if (restart && (int64_t)m >= N) {
                // the basis spans the whole space: the Ritz pair is exact
                if (!(rn[0] <= o->tol_residual)) status = SQD_EBREAKDOWN;
                break;
            }
            if (restart) {
                int r = 0;
                SQD_TRY(restart_basis(&r));
                if (r >= M) return sqd_fail(ctx, SQD_EINVAL, "restart basis fills the subspace");
                prof_begin(ctx, PROF_DAVIDSON);
                SQD_TRY(launch_combine_inplace(ctx, w.Vb, N, m, w.Z, M, r, N));
                SQD_TRY(launch_combine_inplace(ctx, w.Wb, N, m, w.Z, M, r, N));
                // projected matrix and projections of t on the new basis
                SQD_TRY(launch_project_g(ctx, w.G, M, m, w.Z, M, r, w.GZ));
                SQD_TRY(launch_project_coeffs(ctx, w.Z, M, m, r, s1, s3));
                SQD_CUDA(ctx, cudaMemcpyAsync(w.Vb + (int64_t)r * N, T, sizeof(double) * N,
                                              cudaMemcpyDeviceToDevice, st));
                prof_end(ctx, 4.0 * m * r * dN, 8.0 * (2.0 * m + 2.0 * r + 2.0) * dN);
                P1 = s3;
                m = r;
                SQD_TRY(launch_identity_cols(ctx, w.Yprev, m, k, M));
                mprev = m;
                m_warm = 0;
                T = w.Vb + (int64_t)m * N;
            } else {
                SQD_TRY(keep_coefficients());
            }
            grown = true;
            // first update (with the second projections), then the second
            prof_begin(ctx, PROF_ORTHO);
            SQD_TRY(launch_gs_update_dot(ctx, MDf, w.Vb, N, m, P1, T, N, w.partial, nbr, s2));
            prof_end(ctx, (4.0 * m + 3.0) * dN, 8.0 * (m + 2.0) * dN);
            SQD_CUDA(ctx, cudaMemcpyAsync(hs, s2, sizeof(double) * (m + 1), cudaMemcpyDeviceToHost,
                                          st));
            SQD_CUDA(ctx, cudaStreamSynchronize(st));
            const double n2a = hs[m];  // |t'|^2
            double p2 = 0.0;
            for (int i = 0; i < m; i++) p2 += hs[i] * hs[i];
            const double n2b = n2a - p2;  // |t''|^2 by Pythagoras
            int nacc = 1;
            if (p2 <= 0.5 * n2a && n2b >= 1e-20) {
                prof_begin(ctx, PROF_ORTHO);
                SQD_TRY(launch_gs_update_scale(ctx, MDf, w.Vb, N, m, s2, 1.0 / std::sqrt(n2b), T, N,
                                               nbr));
                prof_end(ctx, (2.0 * m + 2.0) * dN, 8.0 * (m + 2.0) * dN);
            } else {
                // not safely resolved: second update, then the explicit norm
                prof_begin(ctx, PROF_ORTHO);
                SQD_TRY(launch_gemv_sub(ctx, w.Vb, N, m, s2, T, N));
                prof_end(ctx, 2.0 * m * dN, 8.0 * (m + 2.0) * dN);
                SQD_TRY(within_block(m, 1, &nacc));
            }
            if (nacc == 0) {
                // the correction lies in the basis: the Ritz pair of the
                // current basis is final (converged unless its residual is
                // above the tolerance)
                SQD_TRY(launch_jacobi_eigh(ctx, w.G, M, m, w.evals, w.evecs));
                SQD_TRY(ritz_all());
                x_ready = true;
                if (!(rn[0] <= o->tol_residual)) status = SQD_EBREAKDOWN;
                break;
            }
            m += 1;
            SQD_TRY(apply_h(w.Vb + (int64_t)(m - 1) * N, w.Wb + (int64_t)(m - 1) * N, 1));
            SQD_TRY(g_cols(m, m - 1, 1));
        }
        // the Ritz vector of the final eigensolve
        if (!x_ready) {
            prof_begin(ctx, PROF_DAVIDSON);
            SQD_TRY(launch_combine(ctx, w.Vb, N, m, w.evecs, m, 1, w.X, N, N));
            prof_end(ctx, 2.0 * m * dN, 8.0 * (m + 1.0) * dN);
        }
    } else {
        for (;;) {
            prof_begin(ctx, PROF_EIGH);
            SQD_TRY(launch_jacobi_eigh(ctx, w.G, M, m, w.evals, w.evecs, m_warm, w.Eold,
                                       w.thold));
            prof_end(ctx, 0.0, 0.0);
            sel.clear();
            for (int j = 0; j < k; j++)
                if (!locked[j]) sel.push_back(j);
            const bool full = sel.empty();
            if (full)
                for (int j = 0; j < k; j++) sel.push_back(j);
            const int ks = (int)sel.size();
            SQD_CUDA(ctx, cudaMemcpyAsync(w.sel, sel.data(), sizeof(int) * ks,
                                          cudaMemcpyHostToDevice, st));
            prof_begin(ctx, PROF_DAVIDSON);
            SQD_TRY(launch_ritz_block(ctx, w.Vb, w.Wb, N, m, w.evecs, w.evals, w.sel, ks, w.X, w.R,
                                      N, w.partial, nbr, w.dots));
            prof_end(ctx, 4.0 * m * ks * dN + 2.0 * ks * dN, 8.0 * (2.0 * m + 2.0 * ks) * dN);
            SQD_CUDA(ctx, cudaMemcpyAsync(theta.data(), w.evals, sizeof(double) * m,
                                          cudaMemcpyDeviceToHost, st));
            SQD_CUDA(ctx, cudaMemcpyAsync(rn2.data(), w.dots, sizeof(double) * ks,
                                          cudaMemcpyDeviceToHost, st));
            if (pend_f > 0.0)
                SQD_CUDA(ctx, cudaMemcpyAsync(&gate_h, w.rdev + 1, sizeof(int),
                                              cudaMemcpyDeviceToHost, st));
            SQD_CUDA(ctx, cudaStreamSynchronize(st));
            book_gated();
            if (grown)
                for (int j = 0; j < k; j++) dth[j] = std::fabs(theta[j] - theta_old[j]);
            for (int j = 0; j < k; j++) theta_old[j] = theta[j];
            bool all = true;
            std::vector<int> todo;
            for (int q = 0; q < ks; q++) {
                const int j = sel[q];
                rn[j] = std::sqrt(std::max(rn2[q], 0.0));
                const bool c = rn[j] <= o->tol_residual && dth[j] <= o->tol_energy;
                locked[j] = c ? 1 : 0;
                if (!c) {
                    all = false;
                    todo.push_back(j);
                }
            }
            if (full && all) break;
            if (it >= o->max_iter) {
                status = SQD_ENOTCONVERGED;
                if (!full) SQD_TRY(ritz_all());
                break;
            }
            it++;
            grown = !todo.empty();
            if (todo.empty()) continue;  // every root locked: check them all next
            if (m + (int)todo.size() > M && (int64_t)m >= N) {
                // the basis spans the whole space: the Ritz pairs are exact
                SQD_TRY(ritz_all());
                bool res_ok = true;
                for (int j = 0; j < k; j++) res_ok = res_ok && rn[j] <= o->tol_residual;
                if (!res_ok) status = SQD_EBREAKDOWN;
                break;
            }
            if (m + (int)todo.size() > M) {
                // restart (GD+k): the 2k lowest Ritz vectors plus the k Ritz
                // vectors of the previous iteration, orthonormalised against them
                int r = 0;
                SQD_TRY(restart_basis(&r));
                prof_begin(ctx, PROF_DAVIDSON);
                if (r <= 8) {  // one pass, in place
                    SQD_TRY(launch_combine_inplace(ctx, w.Vb, N, m, w.Z, M, r, N));
                    SQD_TRY(launch_combine_inplace(ctx, w.Wb, N, m, w.Z, M, r, N));
                } else {
                    SQD_TRY(launch_combine(ctx, w.Vb, N, m, w.Z, M, r, w.Tmp, N, N));
                    SQD_CUDA(ctx, cudaMemcpyAsync(w.Vb, w.Tmp, sizeof(double) * r * N,
                                                  cudaMemcpyDeviceToDevice, st));
                    SQD_TRY(launch_combine(ctx, w.Wb, N, m, w.Z, M, r, w.Tmp, N, N));
                    SQD_CUDA(ctx, cudaMemcpyAsync(w.Wb, w.Tmp, sizeof(double) * r * N,
                                                  cudaMemcpyDeviceToDevice, st));
                }
                // projected matrix of the new basis: G' = Z^T G Z
                SQD_TRY(launch_project_g(ctx, w.G, M, m, w.Z, M, r, w.GZ));
                prof_end(ctx, 4.0 * m * r * dN, 8.0 * (2.0 * m + 4.0 * r) * dN);
                m = r;
                // the current Ritz vectors are the first k basis vectors now
                SQD_TRY(launch_identity_cols(ctx, w.Yprev, m, k, M));
                mprev = m;
                m_warm = 0;
            } else {
                SQD_TRY(keep_coefficients());
            }
            // room for the block (a restart of a space smaller than 4 nroots
            // may leave less): the remaining roots are corrected next time
            const int m_old = m, b = std::min((int)todo.size(), M - m);
            if (b <= 0) return sqd_fail(ctx, SQD_EINVAL, "no room for a new block");
            prof_begin(ctx, PROF_DAVIDSON);
            for (int q = 0; q < b; q++) {
                const int j = todo[q];
                if (o->correction == 1)
                    SQD_TRY(launch_precondition_olsen(ctx, w.R + (int64_t)j * N,
                                                      w.X + (int64_t)j * N, t->diag, theta[j],
                                                      o->precond_floor, N,
                                                      w.Vb + (int64_t)(m_old + q) * N, w.partial,
                                                      w.tn2 + q));
                else
                    SQD_TRY(launch_precondition_norm(ctx, w.R + (int64_t)j * N, t->diag, theta[j],
                                                     o->precond_floor, N,
                                                     w.Vb + (int64_t)(m_old + q) * N, w.partial,
                                                     w.tn2 + q));
            }
            prof_end(ctx, 2.0 * b * dN, 24.0 * b * dN);
            SQD_TRY(symmetrize(w.Vb + (int64_t)m_old * N, b));
            int nacc = 0;
            SQD_TRY(orthonormalize_block(m_old, b, true, &nacc));
            m = m_old + nacc;
            if (nacc == 0) {
                SQD_TRY(launch_jacobi_eigh(ctx, w.G, M, m, w.evals, w.evecs));
                SQD_TRY(ritz_all());
                bool res_ok = true;
                for (int j = 0; j < k; j++) res_ok = res_ok && rn[j] <= o->tol_residual;
                if (!res_ok) status = SQD_EBREAKDOWN;
                break;
            }
            SQD_TRY(apply_h(w.Vb + (int64_t)m_old * N, w.Wb + (int64_t)m_old * N, nacc));
            SQD_TRY(g_cols(m, m_old, nacc));
        }
    }
    // outputs: Ritz vectors with the phase fixed, energies, residuals
    SQD_CUDA(ctx, cudaMemcpyAsync(d_C, w.X, sizeof(double) * k * N, cudaMemcpyDeviceToDevice, st));
    SQD_TRY(launch_fix_phase(ctx, d_C, N, k, N, w.phase));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    for (int j = 0; j < k; j++) {
        h_energies[j] = theta[j];
        if (h_res) h_res[j] = rn[j];
    }
    if (h_iters) *h_iters = it;
    if (status == SQD_ENOTCONVERGED)
        return sqd_fail(ctx, status, "Davidson did not converge in %d iterations", it);
    if (status == SQD_EBREAKDOWN)
        return sqd_fail(ctx, status, "Davidson basis could not be extended");
    return SQD_OK;
}

int sqd_davidson(sqd_ctx *ctx, sqd_tables *t, const sqd_options *o, double *h_energies,
                 double *d_C, int *h_iters, double *h_res) {
    if (!ctx || !t || !o) return fail_noctx(SQD_EINVAL, "sqd_davidson: NULL argument");
    if (!h_energies || !d_C) return sqd_fail(ctx, SQD_EINVAL, "NULL output");
    const int64_t N = t->a.n * t->b->n;
    if (o->nroots < 1 || o->nroots > SQD_MAX_ROOTS || o->nroots > N)
        return sqd_fail(ctx, SQD_EINVAL,
                        "nroots must be in [1, min(%d, dimension)] (the subspace is limited to "
                        "%d vectors and a restart keeps 4 per root)",
                        SQD_MAX_ROOTS, SQD_MAX_SUBSPACE);
    if (o->max_iter < 0 || !(o->tol_energy >= 0) || !(o->tol_residual >= 0) ||
        !(o->precond_floor > 0) || o->max_subspace < 0 || o->correction < 0 ||
        o->correction > 1)
        return sqd_fail(ctx, SQD_EINVAL, "invalid Davidson options");
    SQD_TRY(use_device(ctx));
    return davidson_impl(ctx, t, o, h_energies, d_C, h_iters, h_res);
}

int sqd_string_weights(sqd_ctx *ctx, const sqd_tables *t, const double *d_C, double *d_wa,
                       double *d_wb) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_string_weights: NULL argument");
    if (!d_C || (!d_wa && !d_wb)) return sqd_fail(ctx, SQD_EINVAL, "NULL buffer");
    SQD_TRY(use_device(ctx));
    return launch_string_weights(ctx, d_C, t->a.n, t->b->n, d_wa, d_wb);
}

int sqd_select_strings(sqd_ctx *ctx, const uint64_t *d_str, const double *d_w, int64_t n,
                       double threshold, uint64_t *d_out, int64_t *n_out) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_select_strings: NULL context");
    if (!n_out || n < 0 || (n > 0 && (!d_str || !d_w || !d_out)))
        return sqd_fail(ctx, SQD_EINVAL, "bad arguments");
    if (!std::isfinite(threshold)) return sqd_fail(ctx, SQD_EINVAL, "threshold not finite");
    SQD_TRY(use_device(ctx));
    return launch_select_strings(ctx, d_str, d_w, n, threshold, d_out, n_out);
}

int sqd_map_vector(sqd_ctx *ctx, const uint64_t *d_old_a, int64_t n_old_a,
                   const uint64_t *d_old_b, int64_t n_old_b, const double *d_old_C,
                   const uint64_t *d_new_a, int64_t n_new_a, const uint64_t *d_new_b,
                   int64_t n_new_b, double *d_new_C, double *h_norm) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_map_vector: NULL context");
    if (n_old_a < 1 || n_old_b < 1 || n_new_a < 1 || n_new_b < 1 || !d_old_a || !d_old_b ||
        !d_old_C || !d_new_a || !d_new_b || !d_new_C || !h_norm)
        return sqd_fail(ctx, SQD_EINVAL, "bad arguments");
    SQD_TRY(use_device(ctx));
    return launch_map_vector(ctx, d_old_a, n_old_a, d_old_b, n_old_b, d_old_C, d_new_a, n_new_a,
                             d_new_b, n_new_b, d_new_C, h_norm);
}

int sqd_stored_h_build(sqd_ctx *ctx, sqd_tables *t, int64_t max_bytes, int64_t *nnz) {
    if (!ctx || !t || !nnz) return fail_noctx(SQD_EINVAL, "sqd_stored_h_build: NULL argument");
    SQD_TRY(use_device(ctx));
    return stored_build(ctx, t, max_bytes, nnz);
}

int sqd_sigma_stored(sqd_ctx *ctx, sqd_tables *t, const double *d_C, double *d_sigma,
                     int nvec) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_sigma_stored: NULL argument");
    if (!t->st_rowptr) return sqd_fail(ctx, SQD_EINVAL, "sqd_stored_h_build was not called");
    if (nvec < 1 || !d_C || !d_sigma || d_C == d_sigma)
        return sqd_fail(ctx, SQD_EINVAL, "bad vectors");
    SQD_TRY(use_device(ctx));
    return stored_sigma(ctx, t, d_C, d_sigma, nvec);
}

int sqd_davidson_batched(sqd_ctx *ctx, int nbatch, sqd_tables *const *tables,
                         const sqd_options *o, double *h_energies, double *const *d_C,
                         int *h_iters, int *h_status) {
    if (!ctx || !o) return fail_noctx(SQD_EINVAL, "sqd_davidson_batched: NULL argument");
    if (nbatch < 1 || !tables || !h_energies)
        return sqd_fail(ctx, SQD_EINVAL, "nbatch >= 1, tables and h_energies are required");
    if (o->nroots != 1) return sqd_fail(ctx, SQD_EINVAL, "the batched solver finds one root");
    if (o->max_iter < 0 || !(o->tol_energy >= 0) || !(o->tol_residual >= 0) ||
        !(o->precond_floor > 0) || o->max_subspace < 0 || o->correction < 0 ||
        o->correction > 1)
        return sqd_fail(ctx, SQD_EINVAL, "invalid Davidson options");
    for (int b = 0; b < nbatch; b++)
        if (!tables[b]) return sqd_fail(ctx, SQD_EINVAL, "tables[%d] is NULL", b);
    SQD_TRY(use_device(ctx));
    return davidson_batched_impl(ctx, nbatch, tables, o, h_energies, d_C, h_iters, h_status);
}

int sqd_batched_set_tile(sqd_ctx *ctx, int entries_per_thread, double group_scale) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_batched_set_tile: NULL context");
    if (entries_per_thread == 0) {
        ctx->batched_force_ept = 0;
        ctx->batched_force_scale = 0.0;
        return SQD_OK;
    }
    if ((entries_per_thread != 8 && entries_per_thread != 16) ||
        (group_scale != 0.5 && group_scale != 1.0 && group_scale != 2.0 && group_scale != 4.0))
        return sqd_fail(ctx, SQD_EINVAL,
                        "tile must be 8 or 16 entries per thread with scale 0.5, 1, 2 or 4");
    ctx->batched_force_ept = entries_per_thread;
    ctx->batched_force_scale = group_scale;
    return SQD_OK;
}

int sqd_batched_tuning_buckets(const sqd_ctx *ctx, int max_buckets, int *nbuckets,
                               int64_t *h_max_det, double *h_scale, int *h_entries) {
    if (!ctx || !nbuckets) return fail_noctx(SQD_EINVAL, "sqd_batched_tuning_buckets: NULL argument");
    const int nb = (int)ctx->batched_buckets.size();
    *nbuckets = nb;
    for (int q = 0; q < nb && q < max_buckets; q++) {
        if (h_max_det) h_max_det[q] = ctx->batched_buckets[q].max_det;
        if (h_scale) h_scale[q] = ctx->batched_buckets[q].scale;
        if (h_entries) h_entries[q] = ctx->batched_buckets[q].entries_per_thread;
    }
    return SQD_OK;
}

int sqd_batched_tuning(const sqd_ctx *ctx, double *group_scale, int *device_loop) {
    if (!ctx) return fail_noctx(SQD_EINVAL, "sqd_batched_tuning: NULL argument");
    if (group_scale) *group_scale = ctx->batched_group_scale;
    if (device_loop) *device_loop = ctx->batched_device_loop;
    return SQD_OK;
}

// ----------------------------------------------------------------- RDMs --

int sqd_rdm(sqd_ctx *ctx, sqd_tables *t, const double *d_C, double *d_rdm1, double *d_rdm2) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_rdm: NULL argument");
    if (!d_C || !d_rdm1) return sqd_fail(ctx, SQD_EINVAL, "NULL buffer");
    SQD_TRY(use_device(ctx));
    return launch_rdm(ctx, t, d_C, d_rdm1, d_rdm2);
}

int sqd_orbital_gradient(sqd_ctx *ctx, sqd_tables *t, const double *d_rdm1,
                         const double *d_rdm2, double *d_grad) {
    if (!ctx || !t) return fail_noctx(SQD_EINVAL, "sqd_orbital_gradient: NULL argument");
    if (!d_rdm1 || !d_rdm2 || !d_grad) return sqd_fail(ctx, SQD_EINVAL, "NULL buffer");
    SQD_TRY(use_device(ctx));
    return launch_orbital_gradient(ctx, t, d_rdm1, d_rdm2, d_grad);
}

}  // extern "C"
