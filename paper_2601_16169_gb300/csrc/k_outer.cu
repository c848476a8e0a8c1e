// SQD outer-loop support: after a diagonalisation, the configurations to
// carry into the next sampling round are identified from the wavefunction
// (Section I: the diagonalisation determines which configurations are
// carried over in the iterative process), and the converged vector seeds the
// next round's Davidson guess.
//
//  - string weights: w_a(I) = sum_b C(I,b)^2, w_b(J) = sum_a C(a,J)^2 (the
//    probability of finding the alpha / beta string in the state);
//  - selection: the strings of a set whose weight reaches a threshold;
//  - vector mapping: C'(I', J') = C(I', J') where both strings belong to the
//    old sets, 0 elsewhere, then normalised.
#include "sqd_internal.cuh"

__global__ void k_row_weights(const double *__restrict__ C, int64_t na, int64_t nb,
                              double *__restrict__ wa) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= na) return;
    double s = 0.0;
    for (int64_t c = lane; c < nb; c += 32) {
        const double v = C[r * nb + c];
        s = fma(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) wa[r] = s;
}

__global__ void k_col_weights(const double *__restrict__ C, int64_t na, int64_t nb,
                              double *__restrict__ wb) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nb) return;
    double s = 0.0;
    for (int64_t r = 0; r < na; r++) {
        const double v = C[r * nb + c];
        s = fma(v, v, s);
    }
    wb[c] = s;
}

int launch_string_weights(sqd_ctx *ctx, const double *C, int64_t na, int64_t nb, double *wa,
                          double *wb) {
    if (wa) {
        k_row_weights<<<grid_1d(na * 32, 256), 256, 0, ctx->stream>>>(C, na, nb, wa);
        SQD_LAUNCHED(ctx);
    }
    if (wb) {
        k_col_weights<<<grid_1d(nb, 128), 128, 0, ctx->stream>>>(C, na, nb, wb);
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

__global__ void k_weight_flags(const double *__restrict__ w, int64_t n, double thr,
                               int64_t *__restrict__ flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = (w[i] >= thr) ? 1 : 0;
}

int launch_select_strings(sqd_ctx *ctx, const uint64_t *s, const double *w, int64_t n,
                          double thr, uint64_t *out, int64_t *n_out) {
    *n_out = 0;
    if (n == 0) return SQD_OK;
    int64_t *flags = nullptr, *pos = nullptr, *tot = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&flags, sizeof(int64_t) * n, ctx->stream));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&pos, sizeof(int64_t) * n, ctx->stream));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&tot, sizeof(int64_t), ctx->stream));
    k_weight_flags<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(w, n, thr, flags);
    SQD_LAUNCHED(ctx);
    SQD_TRY(launch_exclusive_scan(ctx, flags, pos, n, tot));
    SQD_TRY(launch_scatter_flagged(ctx, s, flags, pos, n, out));
    int64_t m = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(flags, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(pos, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(tot, ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *n_out = m;
    return SQD_OK;
}

__device__ __forceinline__ int64_t find_sorted(const uint64_t *__restrict__ s, int64_t n,
                                               uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (s[mid] < x) lo = mid + 1; else hi = mid;
    }
    return (lo < n && s[lo] == x) ? lo : -1;
}

// Cnew(i, j) = Cold(ia, ib) for new strings found in the old sets, else 0;
// partial sums of squares per block for the normalisation
__global__ void __launch_bounds__(256) k_map_vector(
    const uint64_t *__restrict__ oa, int64_t noa, const uint64_t *__restrict__ ob, int64_t nob,
    const double *__restrict__ Cold, const uint64_t *__restrict__ na_s, int64_t nna,
    const uint64_t *__restrict__ nb_s, int64_t nnb, double *__restrict__ Cnew,
    double *__restrict__ partial) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nna * nnb;
         I += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = I / nnb, j = I % nnb;
        const int64_t ia = find_sorted(oa, noa, na_s[i]);
        const int64_t ib = ia >= 0 ? find_sorted(ob, nob, nb_s[j]) : -1;
        const double v = (ia >= 0 && ib >= 0) ? Cold[ia * nob + ib] : 0.0;
        Cnew[I] = v;
        s = fma(v, v, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(const double *partial, int n, double *out) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += partial[i];
    *out = s;
}

int launch_map_vector(sqd_ctx *ctx, const uint64_t *oa, int64_t noa, const uint64_t *ob,
                      int64_t nob, const double *Cold, const uint64_t *nas, int64_t nna,
                      const uint64_t *nbs, int64_t nnb, double *Cnew, double *norm_out) {
    const int nblk = 4 * ctx->sm_count;
    double *partial = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&partial, sizeof(double) * (nblk + 1), ctx->stream));
    k_map_vector<<<nblk, 256, 0, ctx->stream>>>(oa, noa, ob, nob, Cold, nas, nna, nbs, nnb, Cnew,
                                                partial);
    SQD_LAUNCHED(ctx);
    k_sum_partials<<<1, 1, 0, ctx->stream>>>(partial, nblk, partial + nblk);
    SQD_LAUNCHED(ctx);
    double n2 = 0.0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&n2, partial + nblk, sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (n2 > 0.0) SQD_TRY(launch_scale(ctx, Cnew, nna * nnb, partial + nblk, 1));
    SQD_CUDA(ctx, cudaFreeAsync(partial, ctx->stream));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *norm_out = sqrt(n2);
    return SQD_OK;
}
