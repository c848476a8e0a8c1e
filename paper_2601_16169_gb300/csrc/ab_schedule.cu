// Work split of the paired-singles kernel (k_alpha_beta and its
// double-float and batched variants): beta chunks of AB_ECAP single entries,
// alpha row groups sized to whole waves of AB_MINB blocks per SM, the owning
// row of each alpha single, and the per-table tuning of the group count.
// Host code and one helper kernel; the sigma kernels themselves are in
// k_sigma.cu and sigma_body.cuh.
#include <cmath>
#include <vector>

#include "sigma_body.cuh"

// Schedule for k_alpha_beta: beta chunks of at most AB_YW rows and AB_ECAP
// entries; alpha groups of roughly equal single counts, about scale * 8
// waves of AB_MINB blocks per SM in all (scale is tuned on the first sigma).
int set_ab_groups(sqd_ctx *ctx, sqd_tables *t, double scale) {
    const spin_tables *A = &t->a;
    const int64_t target_blocks = (int64_t)(scale * 8.0 * AB_MINB * ctx->sm_count + 0.5);
    const int64_t nch = std::max(1, t->ab.nchunks);
    // round down: target_blocks is a whole number of waves,
    // and one block over it would cost a nearly empty extra wave
    int64_t G = target_blocks / nch;
    if (G > A->n) G = A->n;
    if (G < 1) G = 1;
    if (G > 65535) G = 65535;
    const std::vector<int64_t> &ao = A->h_off1;
    const int64_t total = ao[A->n];
    std::vector<int64_t> groups{0};
    int64_t r = 0;
    for (int64_t g = 1; g < G; g++) {
        const int64_t want = total * g / G;
        while (r < A->n && ao[r] < want) r++;
        if (r > groups.back()) groups.push_back(r);
    }
    groups.push_back(A->n);
    if (t->ab.group_rows) {
        SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // no launch still reads it
        cudaFree(t->ab.group_rows);
        t->ab.group_rows = nullptr;
        t->bytes -= sizeof(int64_t) * (t->ab.ngroups + 1);
    }
    t->ab.ngroups = (int)groups.size() - 1;
    SQD_CUDA(ctx, cudaMalloc((void **)&t->ab.group_rows, sizeof(int64_t) * groups.size()));
    SQD_CUDA(ctx, cudaMemcpy(t->ab.group_rows, groups.data(), sizeof(int64_t) * groups.size(),
                             cudaMemcpyHostToDevice));
    t->bytes += sizeof(int64_t) * groups.size();
    t->ab.scale = scale;
    return SQD_OK;
}

// out[e] = row of entry e of a CSR with offsets off (one warp per row)
__global__ void k_row_index(const int64_t *__restrict__ off, int64_t n, int32_t *__restrict__ out) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    for (int64_t e = off[r] + (threadIdx.x & 31); e < off[r + 1]; e += 32) out[e] = (int32_t)r;
}

// beta chunks of `cap` consecutive single entries (a row may be split between
// chunks), cut earlier where they would span more than AB_YW rows; device
// arrays of the entry bounds (n+1) and of the [first, end) rows (2n)
static int build_chunks(sqd_ctx *ctx, sqd_tables *t, int64_t cap, int *n_out, int64_t **ce_out,
                        int64_t **cy_out) {
    const std::vector<int64_t> &bo = t->b->h_off1;
    const int64_t nb = t->b->n, nnz = bo[nb];
    std::vector<int64_t> ce{0}, cy;
    int64_t e = 0, r = 0;
    while (e < nnz) {
        while (bo[r + 1] <= e) r++;  // row of entry e
        int64_t end = std::min<int64_t>(e + cap, nnz);
        if (r + AB_YW < nb && bo[r + AB_YW] < end) end = bo[r + AB_YW];
        int64_t r2 = r;
        while (bo[r2 + 1] < end) r2++;  // row of entry end-1
        cy.push_back(r);
        cy.push_back(r2 + 1);
        ce.push_back(end);
        e = end;
    }
    *n_out = (int)cy.size() / 2;
    SQD_CUDA(ctx, cudaMalloc((void **)ce_out, sizeof(int64_t) * ce.size()));
    SQD_CUDA(ctx, cudaMalloc((void **)cy_out, sizeof(int64_t) * (cy.size() + 2)));
    SQD_CUDA(ctx, cudaMemcpy(*ce_out, ce.data(), sizeof(int64_t) * ce.size(),
                             cudaMemcpyHostToDevice));
    if (!cy.empty())
        SQD_CUDA(ctx, cudaMemcpy(*cy_out, cy.data(), sizeof(int64_t) * cy.size(),
                                 cudaMemcpyHostToDevice));
    t->bytes += sizeof(int64_t) * (ce.size() + cy.size() + 2);
    return SQD_OK;
}

int build_ab_schedule(sqd_ctx *ctx, sqd_tables *t) {
    spin_tables *A = &t->a;
    if (!A->src1) {
        SQD_CUDA(ctx, cudaMalloc((void **)&A->src1, sizeof(int32_t) * (A->nnz1 + 1)));
        t->bytes += sizeof(int32_t) * (A->nnz1 + 1);
        if (A->n > 0) {
            k_row_index<<<grid_1d(A->n * 32, 256), 256, 0, ctx->stream>>>(A->off1, A->n, A->src1);
            SQD_LAUNCHED(ctx);
        }
    }
    SQD_TRY(build_chunks(ctx, t, AB_ECAP, &t->ab.nchunks, &t->ab.chunk_e, &t->ab.chunk_y));
    SQD_TRY(build_chunks(ctx, t, AB_ECAP_WIDE, &t->ab.nchunks_wide, &t->ab.chunk_e_wide,
                         &t->ab.chunk_y_wide));
    return set_ab_groups(ctx, t, 1.0);
}

// Pick the alpha-group scale of sigma mode `mode` by timing paired-singles
// launches on the caller's vector (output to scratch), once per table and
// mode; afterwards only re-applies the chosen schedule.  One untimed launch
// first, then the best of two launches per candidate (one launch each when a
// launch takes 20 ms or more); the default split (scale 1) is kept unless a
// candidate beats it by more than 3% (1% for launches of 20 ms or more,
// whose timing noise is far below that: at 4e8 determinants 75 groups ran
// 2.8% faster than the default 18, which a 3% bar threw away).
int tune_ab_groups(sqd_ctx *ctx, sqd_tables *t, int mode,
                   int (*launch)(sqd_ctx *, sqd_tables *, const void *, double *),
                   const void *C) {
    if (t->a.nnz1 == 0 || t->b->nnz1 == 0) return SQD_OK;
    if (t->ab.best[mode] > 0.0) {
        if (t->ab.scale != t->ab.best[mode]) SQD_TRY(set_ab_groups(ctx, t, t->ab.best[mode]));
        return SQD_OK;
    }
    const double cand[] = {1.0, 0.125, 0.25, 0.5, 2.0, 4.0, 8.0};  // the default first
    const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    const int64_t N = t->a.n * t->b->n;
    cudaEvent_t e0, e1;
    SQD_CUDA(ctx, cudaEventCreate(&e0));
    SQD_CUDA(ctx, cudaEventCreate(&e1));
    double best = 1.0;
    float best_ms = INFINITY, default_ms = INFINITY;
    int rc = SQD_OK;
    // one timed launch of the current split into scratch
    auto time_one = [&](float *ms) -> int {
        cudaEventRecord(e0, ctx->stream);
        SQD_TRY(launch(ctx, t, C, t->scratch_s));
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess)
            return sqd_fail(ctx, SQD_ECUDA, "paired-singles tuning launch failed: %s",
                            cudaGetErrorString(cudaGetLastError()));
        cudaEventElapsedTime(ms, e0, e1);
        return SQD_OK;
    };
    // launches of 20 ms or more are timed once each, the first one counting
    // for the default split (its start-up costs are negligible at that length)
    int reps = 2;
    for (int c = 0; c < ncand && rc == SQD_OK; c++) {
        if ((rc = set_ab_groups(ctx, t, cand[c])) != SQD_OK) break;
        if (cudaMemsetAsync(t->scratch_s, 0, sizeof(double) * N, ctx->stream) != cudaSuccess) {
            rc = sqd_fail(ctx, SQD_ECUDA, "memset failed");
            break;
        }
        float ms_c = INFINITY;
        int r0 = 0;
        if (c == 0) {  // warm-up, or the default's timing for long launches
            float ms = 0.f;
            if ((rc = time_one(&ms)) != SQD_OK) break;
            if (ms >= 20.f) {
                reps = 1;
                ms_c = ms;
                r0 = 1;
            }
        }
        for (int rep = r0; rep < reps; rep++) {
            float ms = 0.f;
            if ((rc = time_one(&ms)) != SQD_OK) break;
            ms_c = fminf(ms_c, ms);
        }
        if (c == 0) default_ms = ms_c;
        if (ms_c < best_ms) {
            best_ms = ms_c;
            best = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SQD_OK) return rc;
    if (!(best_ms < (reps == 1 ? 0.99f : 0.97f) * default_ms)) best = 1.0;
    t->ab.best[mode] = best;
    return set_ab_groups(ctx, t, best);
}

