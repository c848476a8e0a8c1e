// Stored-H variant: P H P assembled once as a CSR matrix and applied as a
// sparse matrix-vector product.  This is the paper's second CPU method
// (Section II: the Hamiltonian is computed once and stored, the stored
// values re-used in every Davidson iteration), worth it while the matrix
// fits in memory; the product is then bound by HBM bandwidth instead of the
// FP64 ALUs.
//
// Row (ia, ib) holds, in this order: the diagonal; alpha singles and
// doubles (beta unchanged); beta singles and doubles (alpha unchanged);
// alpha single x beta single pairs.  Its length is
//   1 + nnzH_a(ia) + nnzH_b(ib) + k1_a(ia) k1_b(ib)
// and every value is the same Slater-Condon element the matrix-free sigma
// uses.  Column indices are int32 (N < 2^31), values FP64: 12 B per entry.
#include <vector>

#include "sqd_internal.cuh"

__device__ __forceinline__ int64_t row_len(const int64_t *__restrict__ a1, const int64_t *__restrict__ a2,
                                           const int64_t *__restrict__ b1, const int64_t *__restrict__ b2,
                                           int64_t ia, int64_t ib) {
    const int64_t k1a = a1[ia + 1] - a1[ia], k2a = a2[ia + 1] - a2[ia];
    const int64_t k1b = b1[ib + 1] - b1[ib], k2b = b2[ib + 1] - b2[ib];
    return 1 + k1a + k2a + k1b + k2b + k1a * k1b;
}

__global__ void k_stored_count(int64_t na, int64_t nb, const int64_t *__restrict__ a1,
                               const int64_t *__restrict__ a2, const int64_t *__restrict__ b1,
                               const int64_t *__restrict__ b2, int64_t *__restrict__ len) {
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= na * nb) return;
    len[I] = row_len(a1, a2, b1, b2, I / nb, I % nb);
}

struct stored_args {
    int64_t na, nb, norb2;
    const int64_t *a_off1, *a_off2, *b_off1, *b_off2;
    const int32_t *a_tgt1, *a_tgt2, *b_tgt1, *b_tgt2;
    const uint16_t *a_pq1, *b_pq1;
    const int8_t *a_sgn1, *b_sgn1;
    const double *a_val1, *a_val2, *b_val1, *b_val2;
    const double *a_W, *b_W, *diag, *V;
    const int64_t *rowptr;
    int32_t *col;
    double *val;
};

// one warp per row; lanes fill consecutive entries (coalesced stores)
__global__ void k_stored_fill(stored_args s) {
    const int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= s.na * s.nb) return;
    const int64_t ia = I / s.nb, ib = I % s.nb;
    const int64_t a1s = s.a_off1[ia], k1a = s.a_off1[ia + 1] - a1s;
    const int64_t a2s = s.a_off2[ia], k2a = s.a_off2[ia + 1] - a2s;
    const int64_t b1s = s.b_off1[ib], k1b = s.b_off1[ib + 1] - b1s;
    const int64_t b2s = s.b_off2[ib], k2b = s.b_off2[ib + 1] - b2s;
    const int64_t len = 1 + k1a + k2a + k1b + k2b + k1a * k1b;
    const int64_t base = s.rowptr[I];
    for (int64_t e = lane; e < len; e += 32) {
        int64_t J;
        double v;
        int64_t t = e;
        if (t == 0) {
            J = I;
            v = s.diag[I];
        } else if ((t -= 1) < k1a) {
            const int64_t x = a1s + t;
            J = (int64_t)s.a_tgt1[x] * s.nb + ib;
            double w = s.b_W[(int64_t)s.a_pq1[x] * s.nb + ib];
            v = s.a_val1[x] + ((s.a_sgn1[x] < 0) ? -w : w);
        } else if ((t -= k1a) < k2a) {
            const int64_t x = a2s + t;
            J = (int64_t)s.a_tgt2[x] * s.nb + ib;
            v = s.a_val2[x];
        } else if ((t -= k2a) < k1b) {
            const int64_t x = b1s + t;
            J = ia * s.nb + s.b_tgt1[x];
            double w = s.a_W[(int64_t)s.b_pq1[x] * s.na + ia];
            v = s.b_val1[x] + ((s.b_sgn1[x] < 0) ? -w : w);
        } else if ((t -= k1b) < k2b) {
            const int64_t x = b2s + t;
            J = ia * s.nb + s.b_tgt2[x];
            v = s.b_val2[x];
        } else {
            t -= k2b;
            const int64_t xa = a1s + t / k1b, xb = b1s + t % k1b;
            J = (int64_t)s.a_tgt1[xa] * s.nb + s.b_tgt1[xb];
            v = s.V[(int64_t)s.a_pq1[xa] * s.norb2 + s.b_pq1[xb]];
            if ((s.a_sgn1[xa] < 0) != (s.b_sgn1[xb] < 0)) v = -v;
        }
        s.col[base + e] = (int32_t)J;
        s.val[base + e] = v;
    }
}

// sigma = H C with the stored matrix: one warp per row
__global__ void __launch_bounds__(256) k_stored_spmv(int64_t N, const int64_t *__restrict__ rowptr,
                                                     const int32_t *__restrict__ col,
                                                     const double *__restrict__ val,
                                                     const double *__restrict__ C,
                                                     double *__restrict__ S) {
    const int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (I >= N) return;
    const int64_t e0 = rowptr[I], e1 = rowptr[I + 1];
    double acc = 0.0;
    for (int64_t e = e0 + lane; e < e1; e += 32) acc = fma(__ldcs(val + e), __ldg(C + __ldcs(col + e)), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) S[I] = acc;
}

int stored_build(sqd_ctx *ctx, sqd_tables *t, int64_t max_bytes, int64_t *nnz_out) {
    const spin_tables *A = &t->a, *B = t->b;
    const int64_t na = A->n, nb = B->n, N = na * nb;
    if (N >= (1LL << 31)) return sqd_fail(ctx, SQD_EINVAL, "stored H needs fewer than 2^31 determinants");
    // exact size from the host copies of the offsets
    std::vector<int64_t> ho2a(na + 1), ho2b(nb + 1);
    SQD_CUDA(ctx, cudaMemcpy(ho2a.data(), A->off2, sizeof(int64_t) * (na + 1), cudaMemcpyDeviceToHost));
    SQD_CUDA(ctx, cudaMemcpy(ho2b.data(), B->off2, sizeof(int64_t) * (nb + 1), cudaMemcpyDeviceToHost));
    const std::vector<int64_t> &ho1a = A->h_off1, &ho1b = B->h_off1;
    double sa = 0, sb = 0, k1sa = 0, k1sb = 0;
    sa = (double)(ho1a[na] + ho2a[na]);
    sb = (double)(ho1b[nb] + ho2b[nb]);
    k1sa = (double)ho1a[na];
    k1sb = (double)ho1b[nb];
    const double nnz = (double)N + sa * nb + sb * na + k1sa * k1sb;
    const double bytes = 12.0 * nnz + 8.0 * (N + 1);
    size_t fre = 0, tot = 0;
    cudaMemGetInfo(&fre, &tot);
    if ((max_bytes > 0 && bytes > (double)max_bytes) || bytes > 0.9 * (double)fre)
        return sqd_fail(ctx, SQD_ENOMEM,
                        "stored H would need %.3g GB (%.3g nonzeros); limit %.3g GB, free %.3g GB",
                        bytes / 1e9, nnz, max_bytes > 0 ? max_bytes / 1e9 : 0.0, fre / 1e9);
    if (t->st_rowptr) {
        cudaFree(t->st_rowptr);
        cudaFree(t->st_col);
        cudaFree(t->st_val);
        t->st_rowptr = nullptr;
        t->st_col = nullptr;
        t->st_val = nullptr;
    }
    const int64_t nz = (int64_t)nnz;
    int64_t *len = nullptr;
    SQD_CUDA(ctx, cudaMalloc((void **)&t->st_rowptr, sizeof(int64_t) * (N + 1)));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->st_col, sizeof(int32_t) * nz));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->st_val, sizeof(double) * nz));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&len, sizeof(int64_t) * N, ctx->stream));
    k_stored_count<<<grid_1d(N, 256), 256, 0, ctx->stream>>>(na, nb, A->off1, A->off2, B->off1,
                                                              B->off2, len);
    SQD_LAUNCHED(ctx);
    SQD_TRY(launch_exclusive_scan(ctx, len, t->st_rowptr, N, t->st_rowptr + N));
    stored_args s;
    s.na = na;
    s.nb = nb;
    s.norb2 = (int64_t)t->norb * t->norb;
    s.a_off1 = A->off1;
    s.a_off2 = A->off2;
    s.b_off1 = B->off1;
    s.b_off2 = B->off2;
    s.a_tgt1 = A->tgt1;
    s.a_tgt2 = A->tgt2;
    s.b_tgt1 = B->tgt1;
    s.b_tgt2 = B->tgt2;
    s.a_pq1 = A->pq1;
    s.b_pq1 = B->pq1;
    s.a_sgn1 = A->sgn1;
    s.b_sgn1 = B->sgn1;
    s.a_val1 = A->val1;
    s.a_val2 = A->val2;
    s.b_val1 = B->val1;
    s.b_val2 = B->val2;
    s.a_W = A->W;
    s.b_W = B->W;
    s.diag = t->diag;
    s.V = t->V;
    s.rowptr = t->st_rowptr;
    s.col = t->st_col;
    s.val = t->st_val;
    k_stored_fill<<<grid_1d(N * 32, 256), 256, 0, ctx->stream>>>(s);
    SQD_LAUNCHED(ctx);
    SQD_CUDA(ctx, cudaFreeAsync(len, ctx->stream));
    int64_t last = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&last, t->st_rowptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (last != nz) return sqd_fail(ctx, SQD_ECUDA, "stored H size mismatch");
    t->st_nnz = nz;
    t->bytes += (int64_t)bytes;
    *nnz_out = nz;
    return SQD_OK;
}

int stored_sigma(sqd_ctx *ctx, const sqd_tables *t, const double *C, double *S, int nvec) {
    const int64_t N = t->a.n * t->b->n;
    for (int v = 0; v < nvec; v++) {
        prof_begin(ctx, PROF_STORED);
        k_stored_spmv<<<grid_1d(N * 32, 256), 256, 0, ctx->stream>>>(
            N, t->st_rowptr, t->st_col, t->st_val, C + (int64_t)v * N, S + (int64_t)v * N);
        SQD_LAUNCHED(ctx);
        prof_end(ctx, 2.0 * t->st_nnz, 12.0 * t->st_nnz + 8.0 * (N + 1) + 16.0 * N);
    }
    return SQD_OK;
}
