// sigma = (P H P) C on the alpha x beta product space, C stored as an
// n_alpha x n_beta row-major matrix.
//
// The Slater-Condon rules split the bra/ket pairs into three kinds
// (Section IV): one or two alpha excitations (beta equal), one or two beta
// excitations (alpha equal), one alpha and one beta excitation.  With the
// alpha-block-first determinant ordering an alpha operator never picks up a
// sign from the beta string and vice versa, so
//
//   sigma(Ia,Ib) = H_II C(Ia,Ib)
//     + sum_{Ja in S1(Ia)+S2(Ia)} [Ha(Ia,Ja) + s_a W_b[pq_a][Ib]] C(Ja,Ib)       (alpha side)
//     + sum_{Jb in S1(Ib)+S2(Ib)} [Hb(Ib,Jb) + s_b W_a[rs_b][Ia]] C(Ia,Jb)       (beta side)
//     + sum_{Ja in S1(Ia)} sum_{Jb in S1(Ib)} s_a s_b (pq_a|rs_b) C(Ja,Jb)        (alpha-beta)
//
// where S1/S2 are the in-set single/double excitations, Ha/Hb the one-spin
// elements (h plus same-spin two-electron part), and the W terms the
// Coulomb coupling of a single of one spin with the occupied orbitals of the
// other spin ((pq|ll) summed over l in the other string).  Every term uses
// only strings of the sets, so the product is exactly P H P.
//
// Kernels (all FP64, owner-computes except the alpha-beta scatter):
//  k_same_spin   one block per (row, 256-column tile): every thread walks
//                the same CSR row (uniform trip count, broadcast loads) and
//                reads C rows coalesced along the column.  Runs once on C
//                with the alpha tables (diagonal included) and once on C^T
//                with the beta tables.
//  k_alpha_beta  paired singles.  A block owns AB_ECAP consecutive beta
//                single entries, whose rows form a contiguous range Y (each
//                entry of row Jb in Y points to a neighbour Ib).  For every alpha row Ia of its
//                group it stages the slabs C(Ja, Y) of all alpha singles of
//                Ia in shared memory (contiguous, coalesced), accumulates
//                acc_e = sum_a s_a s_e V[pq_a][pq_e] C(Ja, Jb_e) in
//                registers and adds acc_e into sigma(Ia, Ib_e) atomically.
//                The symmetric singles relation (entry Jb -> Ib exists iff
//                Ib -> Jb does, with the same sign, and (pq|rs) = (pq|sr))
//                is what lets the slab be contiguous.
#include "sigma_body.cuh"


// ------------------------------------------------------------ same spin --

template <bool DIAG>
__global__ void __launch_bounds__(256) k_same_spin(ss_args a) {
    same_spin_tile<DIAG>(a, blockIdx.x, blockIdx.y);
}

ss_args make_ss_args(const spin_tables *R, const spin_tables *Cc, int64_t nrows, int64_t ncols,
                     const double *C, double *S, const double *diag) {
    ss_args a;
    a.nrows = nrows;
    a.ncols = ncols;
    a.C = C;
    a.S = S;
    a.off1 = R->off1;
    a.tgt1 = R->tgt1;
    a.pq1 = R->pq1;
    a.sgn1 = R->sgn1;
    a.val1 = R->val1;
    a.off2 = R->off2;
    a.tgt2 = R->tgt2;
    a.val2 = R->val2;
    a.W = Cc->W;
    a.diag = diag;
    return a;
}

int launch_same_spin(sqd_ctx *ctx, const spin_tables *R, const spin_tables *Cc, int64_t nrows,
                     int64_t ncols, const double *C, double *S, const double *diag) {
    if (nrows == 0 || ncols == 0) return SQD_OK;
    int64_t tiles = (ncols + 255) / 256;
    if (tiles > 65535 || nrows > 2147483647LL)
        return sqd_fail(ctx, SQD_EINVAL, "string set too large for the sigma grid");
    dim3 g((unsigned)nrows, (unsigned)tiles);
    ss_args a = make_ss_args(R, Cc, nrows, ncols, C, S, diag);
    if (diag) k_same_spin<true><<<g, 256, 0, ctx->stream>>>(a);
    else k_same_spin<false><<<g, 256, 0, ctx->stream>>>(a);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ---------------------------------------------------------- alpha-beta ---

__global__ void __launch_bounds__(AB_THREADS, AB_MINB) k_alpha_beta(ab_args a) {
    alpha_beta_block(a, blockIdx.x, blockIdx.y);
}

ab_args make_ab_args(const sqd_tables *t, const double *C, double *S) {
    const spin_tables *A = &t->a, *B = t->b;
    ab_args a;
    a.nb = B->n;
    a.norb2 = t->norb * t->norb;
    a.a_off = A->off1;
    a.a_src = A->src1;
    a.a_tgt = A->tgt1;
    a.a_pq = A->pq1;
    a.a_sgn = A->sgn1;
    a.b_off = B->off1;
    a.b_tgt = B->tgt1;
    a.b_pq = B->pq1;
    a.b_sgn = B->sgn1;
    a.chunk_e = t->ab.chunk_e;
    a.chunk_y = t->ab.chunk_y;
    a.group_rows = t->ab.group_rows;
    a.C = C;
    a.S = S;
    a.V = t->V;
    return a;
}

int launch_alpha_beta(sqd_ctx *ctx, const sqd_tables *t, const double *C, double *S) {
    const spin_tables *A = &t->a, *B = t->b;
    if (A->nnz1 == 0 || B->nnz1 == 0) return SQD_OK;
    dim3 g((unsigned)t->ab.nchunks, (unsigned)t->ab.ngroups);
    const size_t shm = sizeof(double) * 2 * AB_NA * AB_YW;
    SQD_CUDA(ctx, cudaFuncSetAttribute(k_alpha_beta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm));
    k_alpha_beta<<<g, AB_THREADS, shm, ctx->stream>>>(make_ab_args(t, C, S));
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

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

int build_ab_schedule(sqd_ctx *ctx, sqd_tables *t) {
    const spin_tables *B = t->b;
    spin_tables *A = &t->a;
    if (!A->src1) {
        SQD_CUDA(ctx, cudaMalloc((void **)&A->src1, sizeof(int32_t) * (A->nnz1 + 1)));
        t->bytes += sizeof(int32_t) * (A->nnz1 + 1);
        if (A->n > 0) {
            k_row_index<<<grid_1d(A->n * 32, 256), 256, 0, ctx->stream>>>(A->off1, A->n, A->src1);
            SQD_LAUNCHED(ctx);
        }
    }
    // beta chunks: AB_ECAP consecutive single entries (a row may be split
    // between chunks), cut earlier where they would span more than AB_YW rows
    const std::vector<int64_t> &bo = B->h_off1;
    const int64_t nb = B->n, nnz = bo[nb];
    std::vector<int64_t> ce{0}, cy;
    int64_t e = 0, r = 0;
    while (e < nnz) {
        while (bo[r + 1] <= e) r++;  // row of entry e
        int64_t end = std::min<int64_t>(e + AB_ECAP, nnz);
        if (r + AB_YW < nb && bo[r + AB_YW] < end) end = bo[r + AB_YW];
        int64_t r2 = r;
        while (bo[r2 + 1] < end) r2++;  // row of entry end-1
        cy.push_back(r);
        cy.push_back(r2 + 1);
        ce.push_back(end);
        e = end;
    }
    t->ab.nchunks = (int)cy.size() / 2;
    SQD_CUDA(ctx, cudaMalloc((void **)&t->ab.chunk_e, sizeof(int64_t) * ce.size()));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->ab.chunk_y, sizeof(int64_t) * (cy.size() + 2)));
    SQD_CUDA(ctx, cudaMemcpy(t->ab.chunk_e, ce.data(), sizeof(int64_t) * ce.size(),
                             cudaMemcpyHostToDevice));
    if (!cy.empty())
        SQD_CUDA(ctx, cudaMemcpy(t->ab.chunk_y, cy.data(), sizeof(int64_t) * cy.size(),
                                 cudaMemcpyHostToDevice));
    t->bytes += sizeof(int64_t) * (ce.size() + cy.size() + 2);
    return set_ab_groups(ctx, t, 1.0);
}

// Pick the alpha-group scale of sigma mode `mode` by timing paired-singles
// launches on the caller's vector (output to scratch), once per table and
// mode; afterwards only re-applies the chosen schedule.  One untimed launch
// first, then the best of two launches per candidate; the default split
// (scale 1) is kept unless a candidate beats it by more than 3%.
int tune_ab_groups(sqd_ctx *ctx, sqd_tables *t, int mode,
                   int (*launch)(sqd_ctx *, sqd_tables *, const void *, double *),
                   const void *C) {
    if (t->a.nnz1 == 0 || t->b->nnz1 == 0) return SQD_OK;
    if (t->ab.best[mode] > 0.0) {
        if (t->ab.scale != t->ab.best[mode]) SQD_TRY(set_ab_groups(ctx, t, t->ab.best[mode]));
        return SQD_OK;
    }
    const double cand[] = {1.0, 0.125, 0.25, 0.5, 2.0, 4.0};  // the default first
    const int64_t N = t->a.n * t->b->n;
    cudaEvent_t e0, e1;
    SQD_CUDA(ctx, cudaEventCreate(&e0));
    SQD_CUDA(ctx, cudaEventCreate(&e1));
    double best = 1.0;
    float best_ms = INFINITY, default_ms = INFINITY;
    int rc = SQD_OK;
    for (int c = 0; c < 6 && rc == SQD_OK; c++) {
        if ((rc = set_ab_groups(ctx, t, cand[c])) != SQD_OK) break;
        if (cudaMemsetAsync(t->scratch_s, 0, sizeof(double) * N, ctx->stream) != cudaSuccess) {
            rc = sqd_fail(ctx, SQD_ECUDA, "memset failed");
            break;
        }
        if (c == 0 && (rc = launch(ctx, t, C, t->scratch_s)) != SQD_OK) break;  // warm-up
        float ms_c = INFINITY;
        for (int rep = 0; rep < 2; rep++) {
            cudaEventRecord(e0, ctx->stream);
            if ((rc = launch(ctx, t, C, t->scratch_s)) != SQD_OK) break;
            cudaEventRecord(e1, ctx->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = sqd_fail(ctx, SQD_ECUDA, "paired-singles tuning launch failed: %s",
                              cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
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
    if (!(best_ms < 0.97f * default_ms)) best = 1.0;
    t->ab.best[mode] = best;
    return set_ab_groups(ctx, t, best);
}

// ------------------------------------------------------------ transpose --

template <bool ADD>
__global__ void k_transpose(const double *__restrict__ in, double *__restrict__ out,
                            int64_t rows, int64_t cols) {
    for (int64_t rr = (int64_t)blockIdx.y * 32; rr < rows; rr += (int64_t)gridDim.y * 32)
        transpose_tile<ADD>(in, out, rows, cols, (int64_t)blockIdx.x * 32, rr);
}

int launch_transpose(sqd_ctx *ctx, const double *in, double *out, int64_t rows, int64_t cols,
                     bool add) {
    if (rows == 0 || cols == 0) return SQD_OK;
    int64_t gx = (cols + 31) / 32, gy = (rows + 31) / 32;
    if (gx > 2147483647LL) return sqd_fail(ctx, SQD_EINVAL, "transpose too large");
    dim3 g((unsigned)gx, (unsigned)(gy < 65535 ? gy : 65535));
    dim3 b(32, 8);
    if (add) k_transpose<true><<<g, b, 0, ctx->stream>>>(in, out, rows, cols);
    else k_transpose<false><<<g, b, 0, ctx->stream>>>(in, out, rows, cols);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}
