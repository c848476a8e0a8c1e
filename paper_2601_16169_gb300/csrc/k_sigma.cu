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
//  k_alpha_beta  paired singles.  A block owns a contiguous range Y of beta
//                rows and their single entries (each entry of row Jb in Y
//                points to a neighbour Ib).  For every alpha row Ia of its
//                group it stages the slabs C(Ja, Y) of all alpha singles of
//                Ia in shared memory (contiguous, coalesced), accumulates
//                acc_e = sum_a s_a s_e V[pq_a][pq_e] C(Ja, Jb_e) in
//                registers and adds acc_e into sigma(Ia, Ib_e) atomically.
//                The symmetric singles relation (entry Jb -> Ib exists iff
//                Ib -> Jb does, with the same sign, and (pq|rs) = (pq|sr))
//                is what lets the slab be contiguous.
#include "sqd_internal.cuh"

// ------------------------------------------------------------ same spin --

template <bool DIAG>
__global__ void __launch_bounds__(256)
    k_same_spin(int64_t nrows, int64_t ncols, const double *__restrict__ C,
                double *__restrict__ S, const int64_t *__restrict__ off1,
                const int32_t *__restrict__ tgt1, const uint16_t *__restrict__ pq1,
                const int8_t *__restrict__ sgn1, const double *__restrict__ val1,
                const int64_t *__restrict__ off2, const int32_t *__restrict__ tgt2,
                const double *__restrict__ val2, const double *__restrict__ W,
                const double *__restrict__ diag) {
    int64_t row = blockIdx.x;
    int64_t col = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    double acc = 0.0;
    if (DIAG) acc = diag[row * ncols + col] * C[row * ncols + col];
    const int64_t s1 = off1[row], e1 = off1[row + 1];
    for (int64_t e = s1; e < e1; e++) {
        int64_t J = tgt1[e];
        double c = C[J * ncols + col];
        double w = W[(int64_t)pq1[e] * ncols + col];
        w = (sgn1[e] < 0) ? -w : w;
        acc = fma(val1[e], c, acc);
        acc = fma(w, c, acc);
    }
    const int64_t s2 = off2[row], e2 = off2[row + 1];
    for (int64_t e = s2; e < e2; e++) acc = fma(val2[e], C[(int64_t)tgt2[e] * ncols + col], acc);
    S[row * ncols + col] = acc;
}

int launch_same_spin(sqd_ctx *ctx, const spin_tables *R, const spin_tables *Cc, int64_t nrows,
                     int64_t ncols, const double *C, double *S, const double *diag) {
    if (nrows == 0 || ncols == 0) return SQD_OK;
    int64_t tiles = (ncols + 255) / 256;
    if (tiles > 65535 || nrows > 2147483647LL)
        return sqd_fail(ctx, SQD_EINVAL, "string set too large for the sigma grid");
    dim3 g((unsigned)nrows, (unsigned)tiles);
    if (diag)
        k_same_spin<true><<<g, 256, 0, ctx->stream>>>(nrows, ncols, C, S, R->off1, R->tgt1,
                                                      R->pq1, R->sgn1, R->val1, R->off2,
                                                      R->tgt2, R->val2, Cc->W, diag);
    else
        k_same_spin<false><<<g, 256, 0, ctx->stream>>>(nrows, ncols, C, S, R->off1, R->tgt1,
                                                       R->pq1, R->sgn1, R->val1, R->off2,
                                                       R->tgt2, R->val2, Cc->W, nullptr);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ---------------------------------------------------------- alpha-beta ---

#define AB_THREADS 256
#define AB_EPT 16                          // beta entries per thread
#define AB_ECAP (AB_THREADS * AB_EPT)      // beta entries per block
#define AB_YW 256                          // beta rows (slab width) per block
#define AB_NA 16                           // alpha singles staged per batch

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Work items of a block are (alpha row, batch of AB_NA alpha singles) pairs
// over the rows of its group that have singles, in order.  The slabs of
// item i+1 are copied (cp.async) while item i is computed.
struct ab_item {
    int64_t ia, ab, a1;  // row, first single of the batch, end of the row's singles
};

__device__ __forceinline__ bool ab_next(const int64_t *__restrict__ a_off, int64_t g1,
                                        ab_item &it) {
    it.ab += AB_NA;
    if (it.ab < it.a1) return true;
    for (int64_t ia = it.ia + 1; ia < g1; ia++) {
        int64_t a0 = a_off[ia], a1 = a_off[ia + 1];
        if (a1 > a0) {
            it.ia = ia;
            it.ab = a0;
            it.a1 = a1;
            return true;
        }
    }
    it.ia = g1;
    return false;
}

__global__ void __launch_bounds__(AB_THREADS, 2)
    k_alpha_beta(int64_t nb, int norb2, const int64_t *__restrict__ a_off,
                 const int32_t *__restrict__ a_tgt, const uint16_t *__restrict__ a_pq,
                 const int8_t *__restrict__ a_sgn, const int64_t *__restrict__ b_off,
                 const int32_t *__restrict__ b_tgt, const uint16_t *__restrict__ b_pq,
                 const int8_t *__restrict__ b_sgn, const int64_t *__restrict__ chunk_rows,
                 const int64_t *__restrict__ group_rows, const double *__restrict__ C,
                 double *__restrict__ S, const double *__restrict__ V) {
    // double-buffered slabs in dynamic shared memory: [2][AB_NA][AB_YW] doubles
    extern __shared__ double ab_dyn[];
    double(*slab)[AB_NA][AB_YW] = reinterpret_cast<double(*)[AB_NA][AB_YW]>(ab_dyn);
    __shared__ int64_t sh_vrow[2][AB_NA];
    __shared__ uint32_t sh_sa[2][AB_NA];
    __shared__ int64_t sh_off[AB_YW + 1];

    const int tid = threadIdx.x;
    const int64_t y0 = chunk_rows[blockIdx.x], y1 = chunk_rows[blockIdx.x + 1];
    const int width = (int)(y1 - y0);
    for (int t = tid; t <= width; t += AB_THREADS) sh_off[t] = b_off[y0 + t];
    __syncthreads();
    const int64_t e0 = sh_off[0], e1 = sh_off[width];

    // this thread's beta entries: neighbour Ib and packed
    // (V column | slab column << 12 | sign << 31)
    int32_t ib[AB_EPT];
    uint32_t info[AB_EPT];
    double acc[AB_EPT];
#pragma unroll
    for (int k = 0; k < AB_EPT; k++) {
        int64_t e = e0 + tid + (int64_t)k * AB_THREADS;
        ib[k] = -1;
        info[k] = 0;
        if (e < e1) {
            int lo = 0, hi = width;  // sh_off[lo] <= e < sh_off[hi]
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (sh_off[mid] <= e) lo = mid; else hi = mid;
            }
            ib[k] = b_tgt[e];
            info[k] = (uint32_t)b_pq[e] | ((uint32_t)lo << 12) | ((b_sgn[e] < 0) ? 0x80000000u : 0u);
        }
        acc[k] = 0.0;
    }

    const int64_t g0 = group_rows[blockIdx.y], g1 = group_rows[blockIdx.y + 1];
    // stage the slabs and alpha data of one item into buffer `buf`
    auto stage = [&](const ab_item &it, int buf) {
        const int nbat = (int)min((int64_t)AB_NA, it.a1 - it.ab);
        if (tid < nbat) {
            sh_vrow[buf][tid] = (int64_t)a_pq[it.ab + tid] * norb2;
            sh_sa[buf][tid] = (a_sgn[it.ab + tid] < 0) ? 1u : 0u;
        }
        for (int idx = tid; idx < nbat * width; idx += AB_THREADS) {
            int a = idx / width, j = idx - a * width;
            cp_async8(&slab[buf][a][j], C + (int64_t)a_tgt[it.ab + a] * nb + y0 + j);
        }
        cp_async_commit();
    };

    ab_item cur;
    cur.ia = g0 - 1;
    cur.ab = 0;
    cur.a1 = 0;
    bool have = ab_next(a_off, g1, cur);
    if (have) stage(cur, 0);
    int buf = 0;
    while (have) {
        ab_item nxt = cur;
        bool more = ab_next(a_off, g1, nxt);
        if (more) stage(nxt, buf ^ 1);
        else cp_async_commit();  // keep the group count uniform
        cp_async_wait<1>();
        __syncthreads();  // slabs of `cur` visible to all threads
        const int nbat = (int)min((int64_t)AB_NA, cur.a1 - cur.ab);
        for (int a = 0; a < nbat; a++) {
            const double *vr = V + sh_vrow[buf][a];
            const uint32_t sa = sh_sa[buf][a] << 31;
            const double *sl = slab[buf][a];
#pragma unroll
            for (int k = 0; k < AB_EPT; k++) {
                const uint32_t inf = info[k];
                double v = __ldg(vr + (inf & 0xfffu));
                unsigned long long bits = (unsigned long long)__double_as_longlong(v) ^
                                          ((unsigned long long)((inf ^ sa) & 0x80000000u) << 32);
                acc[k] = fma(__longlong_as_double((long long)bits), sl[(inf >> 12) & 0x1ffu], acc[k]);
            }
        }
        if (cur.ab + AB_NA >= cur.a1) {  // last batch of this alpha row: flush
#pragma unroll
            for (int k = 0; k < AB_EPT; k++) {
                if (ib[k] >= 0) atomicAdd(&S[cur.ia * nb + ib[k]], acc[k]);
                acc[k] = 0.0;
            }
        }
        __syncthreads();  // buffer `buf` is reused by the item after next
        cur = nxt;
        have = more;
        buf ^= 1;
    }
    cp_async_wait<0>();
}

int launch_alpha_beta(sqd_ctx *ctx, const sqd_tables *t, const double *C, double *S) {
    const spin_tables *A = &t->a, *B = t->b;
    if (A->nnz1 == 0 || B->nnz1 == 0) return SQD_OK;
    dim3 g((unsigned)t->ab.nchunks, (unsigned)t->ab.ngroups);
    const size_t shm = sizeof(double) * 2 * AB_NA * AB_YW;
    SQD_CUDA(ctx, cudaFuncSetAttribute(k_alpha_beta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)shm));
    k_alpha_beta<<<g, AB_THREADS, shm, ctx->stream>>>(
        B->n, t->norb * t->norb, A->off1, A->tgt1, A->pq1, A->sgn1, B->off1, B->tgt1, B->pq1,
        B->sgn1, t->ab.chunk_rows, t->ab.group_rows, C, S, t->V);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// Schedule for k_alpha_beta: beta chunks of at most AB_YW rows and AB_ECAP
// entries; alpha groups of roughly equal single counts, enough of them to
// give every SM several blocks.
int build_ab_schedule(sqd_ctx *ctx, sqd_tables *t) {
    const spin_tables *A = &t->a, *B = t->b;
    std::vector<int64_t> chunks{0};
    const std::vector<int64_t> &bo = B->h_off1;
    int64_t y = 0;
    while (y < B->n) {
        int64_t y_end = y;
        while (y_end < B->n && y_end - y < AB_YW && bo[y_end + 1] - bo[y] <= AB_ECAP) y_end++;
        if (y_end == y) y_end = y + 1;  // cannot happen: a row has <= 1024 singles
        chunks.push_back(y_end);
        y = y_end;
    }
    int nchunks = (int)chunks.size() - 1;
    int64_t target_blocks = 8LL * ctx->sm_count * 2;
    int64_t G = (target_blocks + nchunks - 1) / nchunks;
    if (G > A->n) G = A->n;
    if (G < 1) G = 1;
    if (G > 65535) G = 65535;
    const std::vector<int64_t> &ao = A->h_off1;
    int64_t total = ao[A->n];
    std::vector<int64_t> groups{0};
    int64_t r = 0;
    for (int64_t g = 1; g < G; g++) {
        int64_t want = total * g / G;
        while (r < A->n && ao[r] < want) r++;
        if (r > groups.back()) groups.push_back(r);
    }
    groups.push_back(A->n);
    t->ab.nchunks = nchunks;
    t->ab.ngroups = (int)groups.size() - 1;
    SQD_CUDA(ctx, cudaMalloc((void **)&t->ab.chunk_rows, sizeof(int64_t) * chunks.size()));
    SQD_CUDA(ctx, cudaMalloc((void **)&t->ab.group_rows, sizeof(int64_t) * groups.size()));
    SQD_CUDA(ctx, cudaMemcpy(t->ab.chunk_rows, chunks.data(), sizeof(int64_t) * chunks.size(),
                             cudaMemcpyHostToDevice));
    SQD_CUDA(ctx, cudaMemcpy(t->ab.group_rows, groups.data(), sizeof(int64_t) * groups.size(),
                             cudaMemcpyHostToDevice));
    t->bytes += sizeof(int64_t) * (chunks.size() + groups.size());
    return SQD_OK;
}

// ------------------------------------------------------------ transpose --

// out[c][r] (+)= in[r][c]; in is rows x cols
template <bool ADD>
__global__ void k_transpose(const double *__restrict__ in, double *__restrict__ out,
                            int64_t rows, int64_t cols) {
    __shared__ double tile[32][33];
    int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int64_t rr = r0; rr < rows; rr += (int64_t)gridDim.y * 32) {
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            int64_t r = rr + i, c = c0 + threadIdx.x;
            if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
        }
        __syncthreads();
        for (int i = threadIdx.y; i < 32; i += blockDim.y) {
            int64_t c = c0 + i, r = rr + threadIdx.x;
            if (r < rows && c < cols) {
                if (ADD) out[c * rows + r] += tile[threadIdx.x][i];
                else out[c * rows + r] = tile[threadIdx.x][i];
            }
        }
        __syncthreads();
    }
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
