// sigma = H C with the multiply-adds in double-float arithmetic on the FP32
// pipe ("df32" mode), an opt-in alternative to the native FP64 kernels.
//
// Why: GB300 executes FP32 at 128 lanes/clk/SM and FP64 at 2 DFMA/clk/SM;
// the sigma terms are FP64-ALU bound (k_sigma.cu), so emulating each
// multiply-add with ~11 FP32 operations is several times faster.
//
// Representation: every FP64 operand x is stored as a float pair
// (hi, lo) = (rn(x), rn(x - hi)), which keeps 48 of its 53 bits (|x - hi -
// lo| <= 2^-48 |x|) in the same 8 bytes.  One multiply-add of a = (ah, al)
// and b = (bh, bl) into the accumulator (s, e):
//   p  = ah*bh,  pe = fma(ah, bh, -p)              (exact product, Dekker)
//   t  = fma(ah, bl, pe) + al*bh                    (cross terms)
//   (s, err) = TwoSum(s, p)                          (Knuth, error-free)
//   e += err + t
// so the result (double)s + (double)e carries a relative error of a few
// units of 2^-48 per term (al*bl is dropped, 2^-48 relative), far inside the
// 1e-12 sigma tolerance.  All intrinsics are the explicitly rounded ones so
// that the compiler cannot contract the error-free steps.
// Storage of C, sigma and the tables stays FP64 for the caller; the float
// pairs are made once per table (coefficients) and once per sigma (C).
#include "sigma_body.cuh"

__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &s,
                                       float &e) {
    const float p = __fmul_rn(ah, bh);
    const float pe = __fmaf_rn(ah, bh, -p);
    float t = __fmaf_rn(ah, bl, pe);
    t = __fmaf_rn(al, bh, t);
    const float s2 = __fadd_rn(s, p);
    const float bb = __fsub_rn(s2, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb)), __fsub_rn(p, bb));
    s = s2;
    e = __fadd_rn(e, __fadd_rn(err, t));
}

__device__ __forceinline__ float2 df_neg_if(float2 v, bool neg) {
    if (neg) {
        v.x = -v.x;
        v.y = -v.y;
    }
    return v;
}

__device__ __forceinline__ double df_value(float s, float e) {
    return (double)s + (double)e;
}

__global__ void k_split_df(const double *__restrict__ x, float2 *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        const float hi = __double2float_rn(v);
        y[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

int launch_split_df(sqd_ctx *ctx, const double *x, float2 *y, int64_t n) {
    if (n == 0) return SQD_OK;
    unsigned g = grid_1d(n, 256);
    if (g > 16u * (unsigned)ctx->sm_count * 8u) g = 16u * (unsigned)ctx->sm_count * 8u;
    k_split_df<<<g, 256, 0, ctx->stream>>>(x, y, n);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------------------------ same spin --

struct ss_df_args {
    int64_t nrows, ncols;
    const float2 *C;
    double *S;
    const int64_t *off1;
    const int32_t *tgt1;
    const uint16_t *pq1;
    const int8_t *sgn1;
    const float2 *val1;
    const int64_t *off2;
    const int32_t *tgt2;
    const float2 *val2;
    const float2 *W;
    const float2 *diag;
};

template <bool DIAG>
__global__ void __launch_bounds__(256) k_same_spin_df(ss_df_args a) {
    const int64_t row = blockIdx.x, ncols = a.ncols;
    const int64_t col = (int64_t)blockIdx.y * 256 + threadIdx.x;
    if (col >= ncols) return;
    const float2 *__restrict__ C = a.C;
    float s = 0.f, e = 0.f;
    if (DIAG) {
        const float2 d = a.diag[row * ncols + col], c = C[row * ncols + col];
        df_mac(d.x, d.y, c.x, c.y, s, e);
    }
    const int64_t s1 = a.off1[row], e1 = a.off1[row + 1];
    for (int64_t k = s1; k < e1; k++) {
        const float2 c = C[(int64_t)a.tgt1[k] * ncols + col];
        const float2 v = a.val1[k];
        df_mac(v.x, v.y, c.x, c.y, s, e);
        const float2 w = df_neg_if(a.W[(int64_t)a.pq1[k] * ncols + col], a.sgn1[k] < 0);
        df_mac(w.x, w.y, c.x, c.y, s, e);
    }
    const int64_t s2 = a.off2[row], e2 = a.off2[row + 1];
    for (int64_t k = s2; k < e2; k++) {
        const float2 c = C[(int64_t)a.tgt2[k] * ncols + col];
        const float2 v = a.val2[k];
        df_mac(v.x, v.y, c.x, c.y, s, e);
    }
    a.S[row * ncols + col] = df_value(s, e);
}

// ----------------------------------------------------------- alpha-beta --
// Same work decomposition as k_alpha_beta (beta chunk x alpha row group,
// slabs of C staged by cp.async, AB_EPT entries per thread); float-pair data.

// the float-pair operands need more registers than the FP64 kernel: 3 blocks
// per SM keep them without spills
#ifndef AB_DF_MINB
#define AB_DF_MINB 3
#endif
__global__ void __launch_bounds__(AB_THREADS, AB_DF_MINB)
    k_alpha_beta_df(int64_t nb, int norb2, const int64_t *__restrict__ a_off,
                    const int32_t *__restrict__ a_src, const int32_t *__restrict__ a_tgt, const uint16_t *__restrict__ a_pq,
                    const int8_t *__restrict__ a_sgn, const int64_t *__restrict__ b_off,
                    const int32_t *__restrict__ b_tgt, const uint16_t *__restrict__ b_pq,
                    const int8_t *__restrict__ b_sgn, const int64_t *__restrict__ chunk_e,
                    const int64_t *__restrict__ chunk_y, const int64_t *__restrict__ group_rows,
                    const float2 *__restrict__ C,
                    double *__restrict__ S, const float2 *__restrict__ V) {
    extern __shared__ float2 abdf_dyn[];
    float2(*slab)[AB_NA][AB_YW] = reinterpret_cast<float2(*)[AB_NA][AB_YW]>(abdf_dyn);
    __shared__ int64_t sh_vrow[2][AB_NA];
    __shared__ uint32_t sh_sa[2][AB_NA];
    __shared__ int64_t sh_row[2][AB_NA];
    __shared__ int64_t sh_off[AB_YW + 1];

    const int tid = threadIdx.x;
    const int64_t e0 = chunk_e[blockIdx.x], e1 = chunk_e[blockIdx.x + 1];
    const int64_t y0 = chunk_y[2 * blockIdx.x], y1 = chunk_y[2 * blockIdx.x + 1];
    const int width = (int)(y1 - y0);
    for (int t = tid; t <= width; t += AB_THREADS) sh_off[t] = b_off[y0 + t];
    __syncthreads();
    const int nk = (int)((e1 - e0 + AB_THREADS - 1) / AB_THREADS);  // entry slots in use

    int32_t ib[AB_EPT];
    uint32_t info[AB_EPT];
    float as[AB_EPT], ae[AB_EPT];
#pragma unroll
    for (int k = 0; k < AB_EPT; k++) {
        const int64_t e = e0 + tid + (int64_t)k * AB_THREADS;
        ib[k] = -1;
        info[k] = 0;
        if (e < e1) {
            int lo = 0, hi = width;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (sh_off[mid] <= e) lo = mid; else hi = mid;
            }
            ib[k] = b_tgt[e];
            info[k] = (uint32_t)b_pq[e] | ((uint32_t)lo << 12) | ((b_sgn[e] < 0) ? 0x80000000u : 0u);
        }
        as[k] = 0.f;
        ae[k] = 0.f;
    }

    const int64_t g0 = group_rows[blockIdx.y], g1 = group_rows[blockIdx.y + 1];
    const int64_t xs = a_off[g0], xe = a_off[g1];
    auto stage = [&](int64_t x0, int buf) {
        const int nbat = (int)min((int64_t)AB_NA, xe - x0);
        if (tid < nbat) {
            const int64_t x = x0 + tid;
            sh_vrow[buf][tid] = (int64_t)a_pq[x] * norb2;
            sh_sa[buf][tid] = (a_sgn[x] < 0) ? 1u : 0u;
            sh_row[buf][tid] = a_src[x];
        }
        for (int idx = tid; idx < nbat * width; idx += AB_THREADS) {
            const int aa = idx / width, j = idx - aa * width;
            cp_async8(&slab[buf][aa][j], C + (int64_t)a_tgt[x0 + aa] * nb + y0 + j);
        }
        cp_async_commit();
    };
    auto flush = [&](int64_t row) {
#pragma unroll
        for (int k = 0; k < AB_EPT; k++) {
            if (ib[k] >= 0) atomicAdd(&S[row * nb + ib[k]], df_value(as[k], ae[k]));
            as[k] = 0.f;
            ae[k] = 0.f;
        }
    };

    if (xs < xe) stage(xs, 0);
    int buf = 0;
    int64_t row_cur = -1;  // alpha row of the sums held (uniform across the block)
    for (int64_t xb = xs; xb < xe; xb += AB_NA) {
        if (xb + AB_NA < xe) stage(xb + AB_NA, buf ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int nbat = (int)min((int64_t)AB_NA, xe - xb);
        auto pairs = [&](auto km) {
            constexpr int KM = decltype(km)::value;
            for (int ai = 0; ai < nbat; ai++) {
                const int64_t row = sh_row[buf][ai];
                if (row != row_cur) {
                    if (row_cur >= 0) flush(row_cur);
                    row_cur = row;
                }
                const float2 *vr = V + sh_vrow[buf][ai];
                const uint32_t sa = sh_sa[buf][ai] << 31;
                const float2 *sl = slab[buf][ai];
#pragma unroll
                for (int k = 0; k < KM; k++) {
                    const uint32_t inf = info[k];
                    const float2 v =
                        df_neg_if(__ldg(vr + (inf & 0xfffu)), ((inf ^ sa) & 0x80000000u) != 0);
                    const float2 c = sl[(inf >> 12) & 0x1ffu];
                    df_mac(v.x, v.y, c.x, c.y, as[k], ae[k]);
                }
            }
        };
        AB_DISPATCH(nk, pairs, AB_EPT);
        __syncthreads();
        buf ^= 1;
    }
    if (row_cur >= 0) flush(row_cur);
    cp_async_wait<0>();
}

// ------------------------------------------------------------- driver ---

// float-pair copies of one spin's coefficient tables
static int split_spin(sqd_ctx *ctx, const sqd_tables *t, spin_tables *s) {
    const int64_t n2 = (int64_t)t->norb * t->norb;
    if (!s->val1f) {
        SQD_CUDA(ctx, cudaMalloc((void **)&s->val1f, sizeof(float2) * (s->nnz1 + 1)));
        SQD_CUDA(ctx, cudaMalloc((void **)&s->val2f, sizeof(float2) * (s->nnz2 + 1)));
        SQD_CUDA(ctx, cudaMalloc((void **)&s->Wf, sizeof(float2) * n2 * s->n));
        SQD_TRY(launch_split_df(ctx, s->val1, s->val1f, s->nnz1));
        SQD_TRY(launch_split_df(ctx, s->val2, s->val2f, s->nnz2));
        SQD_TRY(launch_split_df(ctx, s->W, s->Wf, n2 * s->n));
    }
    return SQD_OK;
}

int df_prepare(sqd_ctx *ctx, sqd_tables *t) {
    if (t->df_ready) return SQD_OK;
    const int64_t N = t->a.n * t->b->n, n4 = (int64_t)t->norb * t->norb * t->norb * t->norb;
    SQD_TRY(split_spin(ctx, t, &t->a));
    if (!t->shared) SQD_TRY(split_spin(ctx, t, t->b));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->Vf, sizeof(float2) * n4));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->diagf, sizeof(float2) * N));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->scratch_c, sizeof(float2) * N));
    SQD_TRY(launch_split_df(ctx, t->V, t->Vf, n4));
    SQD_TRY(launch_split_df(ctx, t->diag, t->diagf, N));
    SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    t->df_ready = true;
    return SQD_OK;
}

static ss_df_args make_df_args(const spin_tables *R, const spin_tables *Cc, int64_t nrows,
                               int64_t ncols, const float2 *C, double *S, const float2 *diag) {
    ss_df_args a;
    a.nrows = nrows;
    a.ncols = ncols;
    a.C = C;
    a.S = S;
    a.off1 = R->off1;
    a.tgt1 = R->tgt1;
    a.pq1 = R->pq1;
    a.sgn1 = R->sgn1;
    a.val1 = R->val1f;
    a.off2 = R->off2;
    a.tgt2 = R->tgt2;
    a.val2 = R->val2f;
    a.W = Cc->Wf;
    a.diag = diag;
    return a;
}

// the paired-singles term on float-pair C, added into S
static int launch_alpha_beta_df(sqd_ctx *ctx, sqd_tables *t, const void *Cv, double *S) {
    const spin_tables *A = &t->a, *B = t->b;
    if (A->nnz1 == 0 || B->nnz1 == 0) return SQD_OK;
    const size_t shm = sizeof(float2) * 2 * AB_NA * AB_YW;
    SQD_CUDA(ctx, cudaFuncSetAttribute(k_alpha_beta_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm));
    k_alpha_beta_df<<<dim3((unsigned)t->ab.nchunks, (unsigned)t->ab.ngroups), AB_THREADS, shm,
                      ctx->stream>>>(B->n, t->norb * t->norb, A->off1, A->src1, A->tgt1, A->pq1,
                                     A->sgn1,
                                     B->off1, B->tgt1, B->pq1, B->sgn1, t->ab.chunk_e,
                                     t->ab.chunk_y, t->ab.group_rows, (const float2 *)Cv, S, t->Vf);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// one vector: split, alpha side + diagonal, alpha-beta, beta side on C^T
int sigma_df_one(sqd_ctx *ctx, sqd_tables *t, const double *Cv, double *Sv, double f_a,
                 double f_b, double f_ab) {
    const spin_tables *A = &t->a, *B = t->b;
    const int64_t na = A->n, nb = B->n, N = na * nb;
    const double vb = 8.0 * (double)N;
    float2 *Cf = (float2 *)t->scratch_c;
    float2 *Tf = (float2 *)t->scratch_t;  // C^T as float pairs (same 8 bytes)
    SQD_TRY(launch_split_df(ctx, Cv, Cf, N));
    if ((nb + 255) / 256 > 65535 || na > 2147483647LL || (na + 255) / 256 > 65535)
        return sqd_fail(ctx, SQD_EINVAL, "string set too large for the sigma grid");
    prof_begin(ctx, PROF_SAME_ALPHA);
    k_same_spin_df<true><<<dim3((unsigned)na, (unsigned)((nb + 255) / 256)), 256, 0, ctx->stream>>>(
        make_df_args(A, B, na, nb, Cf, Sv, t->diagf));
    SQD_LAUNCHED(ctx);
    prof_end(ctx, f_a, 3 * vb);
    if (A->nnz1 > 0 && B->nnz1 > 0) {
        SQD_TRY(tune_ab_groups(ctx, t, 1, launch_alpha_beta_df, Cf));
        prof_begin(ctx, PROF_ALPHA_BETA);
        SQD_TRY(launch_alpha_beta_df(ctx, t, Cf, Sv));
        prof_end(ctx, f_ab, 3 * vb);
    }
    // C^T of the float pairs (moved as 8-byte words), beta side, add back
    prof_begin(ctx, PROF_TRANSPOSE);
    SQD_TRY(launch_transpose(ctx, (const double *)Cf, (double *)Tf, na, nb, false));
    prof_end(ctx, 0.0, 2 * vb);
    prof_begin(ctx, PROF_SAME_BETA);
    k_same_spin_df<false><<<dim3((unsigned)nb, (unsigned)((na + 255) / 256)), 256, 0, ctx->stream>>>(
        make_df_args(B, A, nb, na, Tf, t->scratch_s, nullptr));
    SQD_LAUNCHED(ctx);
    prof_end(ctx, f_b, 2 * vb);
    prof_begin(ctx, PROF_TRANSPOSE);
    SQD_TRY(launch_transpose(ctx, t->scratch_s, Sv, nb, na, true));
    prof_end(ctx, 0.0, 3 * vb);
    return SQD_OK;
}
