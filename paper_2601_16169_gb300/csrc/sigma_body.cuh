// Device bodies of the sigma kernels, shared by the single-problem kernels
// (k_sigma.cu) and the persistent batched kernels (k_batched.cu).
#pragma once

#include "sqd_internal.cuh"

// same-spin product over one table set (rows) and the other spin (columns)
struct ss_args {
    int64_t nrows, ncols;
    const double *C;
    double *S;
    const int64_t *off1;
    const int32_t *tgt1;
    const uint16_t *pq1;
    const int8_t *sgn1;
    const double *val1;
    const int64_t *off2;
    const int32_t *tgt2;
    const double *val2;
    const double *W;     // [norb^2][ncols] coupling of the column spin
    const double *diag;  // [nrows][ncols] or null
};

// paired alpha x beta singles
struct ab_args {
    int64_t nb;
    int norb2;
    const int64_t *a_off;
    const int32_t *a_src;
    const int32_t *a_tgt;
    const uint16_t *a_pq;
    const int8_t *a_sgn;
    const int64_t *b_off;
    const int32_t *b_tgt;
    const uint16_t *b_pq;
    const int8_t *b_sgn;
    const int64_t *chunk_e;  // entry range [chunk_e[c], chunk_e[c+1]) of beta chunk c
    const int64_t *chunk_y;  // its beta rows [chunk_y[2c], chunk_y[2c+1])
    const int64_t *group_rows;
    const double *C;
    double *S;
    const double *V;
};

ss_args make_ss_args(const spin_tables *R, const spin_tables *Cc, int64_t nrows, int64_t ncols,
                     const double *C, double *S, const double *diag);
ab_args make_ab_args(const sqd_tables *t, const double *C, double *S);

// compile-time integer for templated lambdas
template <int N>
struct ab_int {
    static constexpr int value = N;
};
// call f(ab_int<n>{}) for n in [1, M] (uniform across the block), M <= 16
#define AB_CASE(N, f, M)                                     \
    case N:                                                  \
        f(ab_int<((N) <= (M) ? (N) : (M))>{});               \
        break;
#define AB_DISPATCH(n, f, M)                                                                   \
    switch (n) {                                                                               \
        AB_CASE(1, f, M) AB_CASE(2, f, M) AB_CASE(3, f, M) AB_CASE(4, f, M) AB_CASE(5, f, M)   \
        AB_CASE(6, f, M) AB_CASE(7, f, M) AB_CASE(8, f, M) AB_CASE(9, f, M) AB_CASE(10, f, M)  \
        AB_CASE(11, f, M) AB_CASE(12, f, M) AB_CASE(13, f, M) AB_CASE(14, f, M)                \
        AB_CASE(15, f, M)                                                                      \
        default: f(ab_int<(M)>{}); break;                                                      \
    }

// 8 entries per thread in 64 registers and batches of 12 alpha singles (48 KB
// of double-buffered slabs) let 4 blocks (32 warps) share an SM and hide the
// gather latency of V and the slabs.  Measured fractions of the FP64 peak:
//   16 entries, 2 blocks/SM, 16-single batches: 0.84 h2o29, 0.90 scale36;
//    8 entries, 3 blocks/SM, 16-single batches: 0.89 h2o29, 0.92 adjoint29,
//                                                 0.90 scale36;
//    8 entries, 4 blocks/SM, 12-single batches: 0.91 h2o29, 0.93 adjoint29,
//                                                 0.94 scale36;
//    (4 blocks with 8-single batches: 0.91 scale36; 6 entries at 4 blocks:
//    0.94 scale36, 0.945 adjoint29; 5 blocks spill.)
#define AB_THREADS 256
#ifndef AB_EPT
#define AB_EPT 8                           // beta entries per thread
#endif
#ifndef AB_MINB
#define AB_MINB 4                          // resident blocks per SM (launch bounds)
#endif
#define AB_ECAP (AB_THREADS * AB_EPT)      // beta entries per block
#define AB_YW 256                          // beta rows (slab width) per block
#ifndef AB_NA
#define AB_NA 12                           // alpha singles staged per batch
#endif
static_assert(AB_EPT >= 1 && AB_EPT <= 16, "AB_DISPATCH covers 1..16 entry slots");
#define AB_EPT_WIDE 16                     // entries per thread of the batched kernel
#define AB_ECAP_WIDE (AB_THREADS * AB_EPT_WIDE)

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// The work of a block is the alpha singles of its row group, the contiguous
// range [a_off[g0], a_off[g1]) of the singles table, in batches of AB_NA
// consecutive singles; a batch may span alpha rows.  The slabs of batch i+1
// are copied (cp.async) while batch i is computed, and the entry sums are
// flushed to sigma whenever the alpha row changes.


// One (row, 256-column tile) of the same-spin product; blockDim.x == 256.
template <bool DIAG>
__device__ __forceinline__ void same_spin_tile(const ss_args &a, int64_t row, int64_t tile) {
    const int64_t ncols = a.ncols;
    const int64_t col = tile * 256 + threadIdx.x;
    if (col >= ncols) return;
    const double *__restrict__ C = a.C;
    double acc = 0.0;
    if (DIAG) acc = a.diag[row * ncols + col] * C[row * ncols + col];
    const int64_t s1 = a.off1[row], e1 = a.off1[row + 1];
    for (int64_t e = s1; e < e1; e++) {
        int64_t J = a.tgt1[e];
        double c = C[J * ncols + col];
        double w = a.W[(int64_t)a.pq1[e] * ncols + col];
        // sign of the coupling as an integer flip of the sign bit: a
        // negation would cost an FP64 add, the pipe every term is bound by
        w = __longlong_as_double(__double_as_longlong(w) ^
                                 ((long long)(a.sgn1[e] < 0) << 63));
        acc = fma(a.val1[e], c, acc);
        acc = fma(w, c, acc);
    }
    const int64_t s2 = a.off2[row], e2 = a.off2[row + 1];
    for (int64_t e = s2; e < e2; e++) acc = fma(a.val2[e], C[(int64_t)a.tgt2[e] * ncols + col], acc);
    a.S[row * ncols + col] = acc;
}

// One block's work of the paired-singles product: beta chunk `chunk`,
// alpha row group `group` (dynamic shared memory: 2*AB_NA*AB_YW doubles).
// SKIP_HI: the caller's C is zero in every row Ja at or above the chunk's
// last beta row (the upper-triangle input of the spin-flip product), so the
// alpha singles with such targets are neither staged nor multiplied.
template <int EPT, bool SKIP_HI = false>
__device__ __forceinline__ void alpha_beta_block_t(const ab_args &a, int64_t chunk, int64_t group) {
    // double-buffered slabs in dynamic shared memory: [2][AB_NA][AB_YW] doubles
    extern __shared__ double ab_dyn[];
    double(*slab)[AB_NA][AB_YW] = reinterpret_cast<double(*)[AB_NA][AB_YW]>(ab_dyn);
    __shared__ int64_t sh_vrow[2][AB_NA];
    __shared__ uint32_t sh_sa[2][AB_NA];
    __shared__ int64_t sh_row[2][AB_NA];
    __shared__ int64_t sh_off[AB_YW + 1];
    __shared__ int sh_live[2][AB_NA];

    const int tid = threadIdx.x;
    const int64_t e0 = a.chunk_e[chunk], e1 = a.chunk_e[chunk + 1];
    const int64_t y0 = a.chunk_y[2 * chunk], y1 = a.chunk_y[2 * chunk + 1];
    const int width = (int)(y1 - y0);
    for (int t = tid; t <= width; t += AB_THREADS) sh_off[t] = a.b_off[y0 + t];
    __syncthreads();
    // entry slots in use: the pair loop runs over these only (a predicated-off
    // FP64 instruction still takes its issue slot)
    const int nk = (int)((e1 - e0 + AB_THREADS - 1) / AB_THREADS);

    // this thread's beta entries: neighbour Ib and packed
    // (V column | slab column << 12 | sign << 31)
    int32_t ib[EPT];
    uint32_t info[EPT];
    double acc[EPT];
#pragma unroll
    for (int k = 0; k < EPT; k++) {
        int64_t e = e0 + tid + (int64_t)k * AB_THREADS;
        ib[k] = -1;
        info[k] = 0;
        if (e < e1) {
            int lo = 0, hi = width;  // sh_off[lo] <= e < sh_off[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (sh_off[mid] <= e) lo = mid; else hi = mid;
            }
            ib[k] = a.b_tgt[e];
            info[k] = (uint32_t)a.b_pq[e] | ((uint32_t)lo << 12) | ((a.b_sgn[e] < 0) ? 0x80000000u : 0u);
        }
        acc[k] = 0.0;
    }

    const int64_t g0 = a.group_rows[group], g1 = a.group_rows[group + 1];
    const int64_t xs = a.a_off[g0], xe = a.a_off[g1];
    // stage the slabs and alpha data of the batch starting at single x0
    auto stage = [&](int64_t x0, int buf) {
        const int nbat = (int)min((int64_t)AB_NA, xe - x0);
        if (tid < nbat) {
            const int64_t x = x0 + tid;
            sh_vrow[buf][tid] = (int64_t)a.a_pq[x] * a.norb2;
            sh_sa[buf][tid] = (a.a_sgn[x] < 0) ? 1u : 0u;
            sh_row[buf][tid] = a.a_src[x];
            if (SKIP_HI) sh_live[buf][tid] = a.a_tgt[x] < y1;
        }
        for (int idx = tid; idx < nbat * width; idx += AB_THREADS) {
            int aa = idx / width, j = idx - aa * width;
            const int64_t ja = a.a_tgt[x0 + aa];
            if (!SKIP_HI || ja < y1) cp_async8(&slab[buf][aa][j], a.C + ja * a.nb + y0 + j);
        }
        cp_async_commit();
    };
    auto flush = [&](int64_t row) {
#pragma unroll
        for (int k = 0; k < EPT; k++) {
            if (ib[k] >= 0) atomicAdd(&a.S[row * a.nb + ib[k]], acc[k]);
            acc[k] = 0.0;
        }
    };

    if (xs < xe) stage(xs, 0);
    int buf = 0;
    int64_t row_cur = -1;  // alpha row of the sums in acc (uniform across the block)
    for (int64_t xb = xs; xb < xe; xb += AB_NA) {
        if (xb + AB_NA < xe) stage(xb + AB_NA, buf ^ 1);
        else cp_async_commit();  // keep the group count uniform
        cp_async_wait<1>();
        __syncthreads();  // slabs of this batch visible to all threads
        const int nbat = (int)min((int64_t)AB_NA, xe - xb);
        auto pairs = [&](auto km) {
            constexpr int KM = decltype(km)::value;
            for (int ai = 0; ai < nbat; ai++) {
                if (SKIP_HI && !sh_live[buf][ai]) continue;  // a zero slab row
                const int64_t row = sh_row[buf][ai];
                if (row != row_cur) {
                    if (row_cur >= 0) flush(row_cur);
                    row_cur = row;
                }
                const double *vr = a.V + sh_vrow[buf][ai];
                const uint32_t sa = sh_sa[buf][ai] << 31;
                const double *sl = slab[buf][ai];
#pragma unroll
                for (int k = 0; k < KM; k++) {
                    const uint32_t inf = info[k];
                    double v = __ldg(vr + (inf & 0xfffu));
                    unsigned long long bits = (unsigned long long)__double_as_longlong(v) ^
                                              ((unsigned long long)((inf ^ sa) & 0x80000000u) << 32);
                    acc[k] = fma(__longlong_as_double((long long)bits), sl[(inf >> 12) & 0x1ffu], acc[k]);
                }
            }
        };
        AB_DISPATCH(nk, pairs, EPT);
        __syncthreads();  // buffer `buf` is reused by the batch after next
        buf ^= 1;
    }
    if (row_cur >= 0) flush(row_cur);
    cp_async_wait<0>();
}

// the sigma kernel's block: AB_EPT entries per thread, chunks of AB_ECAP entries
__device__ __forceinline__ void alpha_beta_block(const ab_args &a, int64_t chunk, int64_t group) {
    alpha_beta_block_t<AB_EPT>(a, chunk, group);
}

// out[c][r] (+)= in[r][c] for one 32 x 32 tile at (row r0, column c0); in is
// rows x cols; blockDim = (32, 8).
template <bool ADD>
__device__ __forceinline__ void transpose_tile(const double *__restrict__ in,
                                               double *__restrict__ out, int64_t rows,
                                               int64_t cols, int64_t c0, int64_t r0) {
    __shared__ double tile[32][33];
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) {
            if (ADD) out[c * rows + r] += tile[threadIdx.x][i];
            else out[c * rows + r] = tile[threadIdx.x][i];
        }
    }
    __syncthreads();
}
