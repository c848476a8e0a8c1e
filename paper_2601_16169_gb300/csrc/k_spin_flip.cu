// Spin-flip sectors of a shared string set (sqd_tables_set_spin_flip); not
// in the paper, which forms the three parts of sigma (Section IV) on every
// vector.
//
// With one string set for both spins the exchange (Ia, Ib) -> (Ib, Ia)
// commutes with the spin-free H of Section II: the two same-spin tables, the
// couplings W and the diagonal are the same for both spins, and
// (pq|rs) = (rs|pq).  On a vector
// of one sector, C^T = s C with s = +1 or -1:
//  - the beta side of sigma is s times the transposed alpha side;
//  - the paired-singles part commutes with the transposition too,
//    sigma_ab(X^T) = sigma_ab(X)^T, so with C = Ch + s Ch^T, where Ch keeps
//    the upper triangle of C (half the diagonal for s = +1, none for s = -1),
//    sigma_ab(C) = Y + s Y^T with Y = sigma_ab(Ch).  Ch is zero in every row
//    below the diagonal, so a beta chunk of rows [y0, y1) meets only the
//    alpha singles whose target lies below y1: about half the pairs.
// Hence
//   sigma = (T + s T^T) + H_II C + (Y + s Y^T),   T = sigma_aa(C) without
// the diagonal: one same-spin pass and about half of the paired singles.
#include <algorithm>
#include <vector>

#include "sigma_body.cuh"

// Ch[r][c] = C[r][c] above the diagonal, C[r][r] / 2 (s = +1) or 0 (s = -1)
// on it, 0 below; one row per blockIdx.y step, 256 columns per block
template <int SGN>
__global__ void k_upper_half(const double *__restrict__ C, double *__restrict__ Ch, int64_t n) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int64_t r = blockIdx.y; r < n; r += gridDim.y) {
        const int64_t p = r * n + c;
        Ch[p] = r < c ? C[p] : (r == c && SGN > 0 ? 0.5 * C[p] : 0.0);
    }
}

int launch_upper_half(sqd_ctx *ctx, int sgn, const double *C, double *Ch, int64_t n) {
    if (n == 0) return SQD_OK;
    if (sgn != 1 && sgn != -1) return sqd_fail(ctx, SQD_EINVAL, "sector must be +1 or -1");
    dim3 grid((unsigned)((n + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
    if (sgn > 0) k_upper_half<1><<<grid, 256, 0, ctx->stream>>>(C, Ch, n);
    else k_upper_half<-1><<<grid, 256, 0, ctx->stream>>>(C, Ch, n);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// S[r][c] = (T[r][c] + s T[c][r]) + D[r][c] C[r][c] + (Y[r][c] + s Y[c][r])
// for one 32 x 32 tile of n x n matrices (the mirrored tiles of T and Y
// staged transposed in shared memory)
template <int SGN>
__global__ void k_sym_combine(const double *__restrict__ T, const double *__restrict__ Y,
                              const double *__restrict__ D, const double *__restrict__ C,
                              double *__restrict__ S, int64_t n) {
    __shared__ double tt[32][33], ty[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    for (int64_t r0 = (int64_t)blockIdx.y * 32; r0 < n; r0 += (int64_t)gridDim.y * 32) {
        // tt[i][x] = T[c0 + i][r0 + x] (rows of the mirrored tile, coalesced)
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int64_t c = c0 + i, r = r0 + threadIdx.x;
            if (c < n && r < n) {
                tt[i][threadIdx.x] = T[c * n + r];
                ty[i][threadIdx.x] = Y[c * n + r];
            }
        }
        __syncthreads();
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int64_t r = r0 + i, c = c0 + threadIdx.x;
            if (r < n && c < n) {
                const int64_t p = r * n + c;
                const double mt = tt[threadIdx.x][i], my = ty[threadIdx.x][i];
                const double same = SGN > 0 ? T[p] + mt : T[p] - mt;
                const double ab = SGN > 0 ? Y[p] + my : Y[p] - my;
                S[p] = (same + D[p] * C[p]) + ab;
            }
        }
        __syncthreads();
    }
}

int launch_sym_combine(sqd_ctx *ctx, int sgn, const double *T, const double *Y, const double *D,
                       const double *C, double *S, int64_t n) {
    if (n == 0) return SQD_OK;
    if (sgn != 1 && sgn != -1) return sqd_fail(ctx, SQD_EINVAL, "sector must be +1 or -1");
    const int64_t g = (n + 31) / 32;
    if (g > 2147483647LL) return sqd_fail(ctx, SQD_EINVAL, "symmetric combine too large");
    dim3 grid((unsigned)g, (unsigned)(g < 65535 ? g : 65535));
    if (sgn > 0) k_sym_combine<1><<<grid, dim3(32, 8), 0, ctx->stream>>>(T, Y, D, C, S, n);
    else k_sym_combine<-1><<<grid, dim3(32, 8), 0, ctx->stream>>>(T, Y, D, C, S, n);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// X <- (X + s X^T) / 2 in place for an n x n matrix: the block of tile pair
// (bi, bj), bi <= bj, reads both tiles and writes the result and its mirror
// (blocks with bi > bj have nothing to do).  Mirrored elements get the same
// rounded sum (s = +1) or exactly opposite differences (s = -1, zero on the
// diagonal), so the result lies exactly in the sector.
template <int SGN>
__global__ void k_symmetrize(double *X, int64_t n) {
    __shared__ double a[32][33], b[32][33];
    const int64_t bj = blockIdx.x;
    for (int64_t bi = blockIdx.y; bi <= bj; bi += gridDim.y) {
        const int64_t r0 = bi * 32, c0 = bj * 32;
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int64_t r = r0 + i, c = c0 + threadIdx.x;  // tile (bi, bj)
            if (r < n && c < n) a[i][threadIdx.x] = X[r * n + c];
            const int64_t r2 = c0 + i, c2 = r0 + threadIdx.x;  // tile (bj, bi)
            if (r2 < n && c2 < n) b[i][threadIdx.x] = X[r2 * n + c2];
        }
        __syncthreads();
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            const int64_t r = r0 + i, c = c0 + threadIdx.x;
            const double x = a[i][threadIdx.x], xm = b[threadIdx.x][i];
            if (r < n && c < n) X[r * n + c] = 0.5 * (SGN > 0 ? x + xm : x - xm);
            const int64_t r2 = c0 + i, c2 = r0 + threadIdx.x;
            const double y = b[i][threadIdx.x], ym = a[threadIdx.x][i];
            if (r2 < n && c2 < n) X[r2 * n + c2] = 0.5 * (SGN > 0 ? y + ym : y - ym);
        }
        __syncthreads();
    }
}

int launch_symmetrize(sqd_ctx *ctx, int sgn, double *X, int64_t n) {
    if (n == 0) return SQD_OK;
    if (sgn != 1 && sgn != -1) return sqd_fail(ctx, SQD_EINVAL, "sector must be +1 or -1");
    const int64_t g = (n + 31) / 32;
    if (g > 2147483647LL) return sqd_fail(ctx, SQD_EINVAL, "symmetrisation too large");
    dim3 grid((unsigned)g, (unsigned)(g < 65535 ? g : 65535));
    if (sgn > 0) k_symmetrize<1><<<grid, dim3(32, 8), 0, ctx->stream>>>(X, n);
    else k_symmetrize<-1><<<grid, dim3(32, 8), 0, ctx->stream>>>(X, n);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// The paired singles on the upper-triangle input Ch (Y = sigma_ab(Ch), added
// into Y with atomics; Y zeroed by the caller): the k_alpha_beta tile with
// the alpha singles whose target lies at or above the chunk's rows skipped.
__global__ void __launch_bounds__(AB_THREADS, AB_MINB) k_alpha_beta_upper(ab_args a) {
    alpha_beta_block_t<AB_EPT, true>(a, blockIdx.x, blockIdx.y);
}

int launch_alpha_beta_upper(sqd_ctx *ctx, const sqd_tables *t, const double *Ch, double *Y) {
    const spin_tables *A = &t->a, *B = t->b;
    if (A->nnz1 == 0 || B->nnz1 == 0) return SQD_OK;
    dim3 g((unsigned)t->ab.nchunks, (unsigned)t->ab.ngroups);
    const size_t shm = sizeof(double) * 2 * AB_NA * AB_YW;
    SQD_CUDA(ctx, cudaFuncSetAttribute(k_alpha_beta_upper,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_alpha_beta_upper<<<g, AB_THREADS, shm, ctx->stream>>>(make_ab_args(t, Ch, Y));
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// Multiply-adds of k_alpha_beta_upper, counted once per table: for every
// beta chunk, its entries times the alpha singles whose target lies below
// the chunk's last row.
int alpha_beta_upper_work(sqd_ctx *ctx, sqd_tables *t, double *fmas) {
    if (t->ab_upper_fmas >= 0.0) {
        *fmas = t->ab_upper_fmas;
        return SQD_OK;
    }
    const spin_tables *A = &t->a;
    const int nch = t->ab.nchunks;
    std::vector<int32_t> tgt(A->nnz1);
    std::vector<int64_t> ce(nch + 1), cy(2 * (size_t)nch);
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the tables are complete
    if (A->nnz1 > 0)
        SQD_CUDA(ctx, cudaMemcpy(tgt.data(), A->tgt1, sizeof(int32_t) * A->nnz1,
                                 cudaMemcpyDeviceToHost));
    if (nch > 0) {
        SQD_CUDA(ctx, cudaMemcpy(ce.data(), t->ab.chunk_e, sizeof(int64_t) * (nch + 1),
                                 cudaMemcpyDeviceToHost));
        SQD_CUDA(ctx, cudaMemcpy(cy.data(), t->ab.chunk_y, sizeof(int64_t) * 2 * nch,
                                 cudaMemcpyDeviceToHost));
    }
    std::sort(tgt.begin(), tgt.end());
    double total = 0.0;
    for (int c = 0; c < nch; c++) {
        const int64_t below =
            std::lower_bound(tgt.begin(), tgt.end(), (int64_t)cy[2 * c + 1]) - tgt.begin();
        total += (double)(ce[c + 1] - ce[c]) * (double)below;
    }
    t->ab_upper_fmas = total;
    *fmas = total;
    return SQD_OK;
}
