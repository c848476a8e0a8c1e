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
