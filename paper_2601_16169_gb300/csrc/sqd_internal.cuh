// Internal declarations of the sm_103a SQD library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sqd.h"

// Kernel classes for the measurement counters (sqd_profile_*).
// largest Davidson subspace (the one-block Jacobi eigensolver's limit);
// nroots is limited to a quarter of it (the restart needs 4 nroots vectors)
#define SQD_MAX_SUBSPACE 112
#define SQD_MAX_ROOTS (SQD_MAX_SUBSPACE / 4)

enum prof_class {
    PROF_SAME_ALPHA = 0,  // k_same_spin on C with the alpha tables (+ diagonal)
    PROF_SAME_BETA,       // k_same_spin on C^T with the beta tables
    PROF_ALPHA_BETA,      // k_alpha_beta (paired singles)
    PROF_TRANSPOSE,       // C -> C^T and the transposed add-back
    PROF_TABLES,          // excitation tables, string terms, diagonal
    PROF_STRINGS,         // string filtering, sort, scan
    PROF_DAVIDSON,        // Davidson Ritz vectors, residuals, preconditioner, restart
    PROF_RDM,             // density matrices
    PROF_STORED,          // stored-H sparse matrix-vector product
    PROF_ORTHO,           // Davidson Gram-Schmidt of the new block against the basis
    PROF_EIGH,            // Davidson Rayleigh-Ritz eigensolver
    PROF_BATCHED,         // a whole batched solve (setup, tuning, loop, outputs)
    PROF_B_SIGMA,         // batched loop: sigma stages (device-timed per iteration)
    PROF_B_VECTOR,        // batched loop: Ritz, restart, correction, Gram-Schmidt, G columns
    PROF_B_EIGH,          // batched loop: the per-subspace Jacobi eigensolves
    PROF_GCOLS,           // Davidson: new columns of the projected matrix G = V^T W
    PROF_ORTHO_BLOCK,     // Davidson: orthonormalisation within the new block
    PROF_B_SIGMA_AB,      // batched loop: the paired-singles part of the sigma stage
    PROF_NCLASS
};

struct prof_rec {
    int cls;
    cudaEvent_t a, b;
};

struct sqd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    // measurement counters
    int64_t launches = 0;                // kernel launches since the last reset
    bool prof = false;                   // event timing enabled
    int open_cls = -1;
    std::vector<prof_rec> recs;          // timed regions (event pairs)
    std::vector<cudaEvent_t> pool;       // free events
    int64_t cls_launches[PROF_NCLASS] = {0};
    double cls_flops[PROF_NCLASS] = {0};
    double cls_bytes[PROF_NCLASS] = {0};
    double cls_ms[PROF_NCLASS] = {0};
    double batched_group_scale = 0.0;    // last autotuned alpha-group scale (largest bucket)
    struct bucket_choice {
        int64_t max_det;         // largest subspace (determinants) of the bucket
        double scale;            // alpha-row group scale
        int entries_per_thread;  // paired-singles tile: 16 (wide, persistent) or 8 (grid)
    };
    std::vector<bucket_choice> batched_buckets;  // last batched solve's per-bucket tiles
    int batched_force_ept = 0;       // fixed paired-singles tile (8 or 16), 0 = autotune
    double batched_force_scale = 0;  // fixed alpha-group scale with it
    int batched_device_loop = 0;         // 1: last batched solve looped inside one graph
};

// Time the launches between prof_begin/prof_end as one region of class cls
// (no-op unless profiling is enabled) and book its algorithmic work.
void prof_begin(sqd_ctx *ctx, int cls);
void prof_end(sqd_ctx *ctx, double flops, double bytes);

// Excitation tables of one string set (one spin).
struct spin_tables {
    int64_t n = 0;   // strings
    int ne = 0;      // electrons
    uint64_t *str = nullptr;  // sorted strings, device

    // singles CSR (entries of a row sorted by target)
    int64_t nnz1 = 0;
    int64_t *off1 = nullptr;   // n+1
    int32_t *tgt1 = nullptr;   // target string index
    uint16_t *pq1 = nullptr;   // p*norb+q (p created, q annihilated)
    int8_t *sgn1 = nullptr;    // <J|a+_p a_q|I>
    double *val1 = nullptr;    // <I|H_s|J>
    int32_t *src1 = nullptr;   // owning row of each entry (paired-singles batches)

    // doubles CSR
    int64_t nnz2 = 0;
    int64_t *off2 = nullptr;
    int32_t *tgt2 = nullptr;
    uint32_t *orb2 = nullptr;  // i | j<<8 | a<<16 | b<<24
    int8_t *sgn2 = nullptr;
    double *val2 = nullptr;

    double *energy = nullptr;  // E_s(I) = <I|H_s|I>
    double *W = nullptr;       // [norb*norb][n]: sum_{l in I} (pq|ll)
    double *u = nullptr;       // [n][norb]: sum_{l in I} (kk|ll)

    std::vector<int64_t> h_off1;  // host copy of off1 (scheduling)
    int64_t max1 = 0, max2 = 0;

    // float-pair copies for the double-float sigma mode (made on first use)
    float2 *val1f = nullptr, *val2f = nullptr, *Wf = nullptr;
};

// Work decomposition of the alpha-beta (paired singles) kernel.
struct ab_schedule {
    // beta chunks: rows [rows[c], rows[c+1]) of the beta singles table
    int nchunks = 0;
    int64_t *chunk_e = nullptr;  // device, nchunks+1: entry ranges of the beta singles
    int64_t *chunk_y = nullptr;  // device, 2*nchunks: [first, end) beta rows of each chunk
    // the same for the wider chunks of the batched kernel (AB_ECAP_WIDE entries)
    int nchunks_wide = 0;
    int64_t *chunk_e_wide = nullptr;
    int64_t *chunk_y_wide = nullptr;
    // alpha row groups: [grp[g], grp[g+1])
    int ngroups = 0;
    int64_t *group_rows = nullptr;  // device, ngroups+1
    double scale = 0.0;             // blocks = scale * 16 per SM (current groups)
    double best[2] = {0.0, 0.0};    // tuned scale per sigma mode (0: not yet)
};

struct sqd_tables {
    sqd_ctx *ctx = nullptr;
    int norb = 0;
    double ecore = 0.0;
    double *h = nullptr;  // device copy
    double *V = nullptr;  // device copy
    spin_tables a, b_own;
    spin_tables *b = nullptr;  // == &a when shared
    bool shared = false;
    double *diag = nullptr;    // [na][nb]
    ab_schedule ab;
    // sigma scratch
    double *scratch_t = nullptr;  // C^T
    double *scratch_s = nullptr;  // (sigma_bb)^T
    // RDM: extended alpha items sorted by pq, beta chunks, item groups
    bool rdm_ready = false;
    int64_t rdm_items = 0;
    int32_t *rdm_iket = nullptr, *rdm_ibra = nullptr;
    uint32_t *rdm_ipq = nullptr;
    int rdm_nchunks = 0, rdm_ngroups = 0;
    int64_t *rdm_chunks = nullptr, *rdm_groups = nullptr;
    // double-float sigma mode (0: FP64, 1: df32)
    int sigma_mode = 0;
    // +1 / -1: C^T = spin_flip * C asserted by the caller (shared string
    // set): the beta side of sigma is the alpha side transposed times the
    // sign; Davidson searches that sector.  0: general vectors.
    int spin_flip = 0;
    double *scratch_h = nullptr;   // upper-triangle copy of C (spin flip)
    double ab_upper_fmas = -1.0;   // multiply-adds of the upper-input paired singles
    bool df_ready = false;
    float2 *Vf = nullptr, *diagf = nullptr;
    double *scratch_c = nullptr;  // C as float pairs (8 bytes per element)
    // stored-H CSR (built on request)
    int64_t st_nnz = 0;
    int64_t *st_rowptr = nullptr;
    int32_t *st_col = nullptr;
    double *st_val = nullptr;
    int64_t bytes = 0;
};

// ---- error helpers -----------------------------------------------------
int sqd_fail(sqd_ctx *ctx, int code, const char *fmt, ...);
#define SQD_CUDA(ctx, call)                                                   \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess)                                                \
            return sqd_fail((ctx), e_ == cudaErrorMemoryAllocation ? SQD_ENOMEM \
                                                                    : SQD_ECUDA, \
                            "%s failed: %s (%s:%d)", #call,                   \
                            cudaGetErrorString(e_), __FILE__, __LINE__);      \
    } while (0)
// after every kernel launch: count it and surface launch errors
#define SQD_LAUNCHED(ctx)                                                     \
    do {                                                                      \
        (ctx)->launches++;                                                    \
        SQD_CUDA((ctx), cudaGetLastError());                                  \
    } while (0)
#define SQD_TRY(call)          \
    do {                       \
        int r_ = (call);       \
        if (r_ != SQD_OK)      \
            return r_;         \
    } while (0)

static inline unsigned grid_1d(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g < 1 ? 1 : g);
}

// ---- launchers (implemented in the k_*.cu files) ------------------------
// strings / sort / scan
int launch_filter_flags(sqd_ctx *, const uint64_t *raw, int64_t n, int norb, int nelec,
                        int64_t *flags);
int launch_exclusive_scan(sqd_ctx *, const int64_t *in, int64_t *out, int64_t n,
                          int64_t *total_dev);
int launch_scatter_flagged(sqd_ctx *, const uint64_t *in, const int64_t *flags,
                           const int64_t *pos, int64_t n, uint64_t *out);
int launch_fill_u64(sqd_ctx *, uint64_t *p, int64_t n, uint64_t v);
int launch_bitonic_sort_u64(sqd_ctx *, uint64_t *keys, int64_t n_pow2);
int launch_unique_flags(sqd_ctx *, const uint64_t *sorted, int64_t n, int64_t *flags);
int launch_check_sorted_unique(sqd_ctx *, const uint64_t *s, int64_t n, int norb, int ne,
                               int *bad_dev);
int launch_check_integrals(sqd_ctx *, const double *h, const double *V, int norb,
                           double *res_dev);

// tables
int launch_count_excitations(sqd_ctx *, const uint64_t *s, int64_t n, int norb, int kind,
                             int64_t *counts);
int launch_fill_excitations(sqd_ctx *, const uint64_t *s, int64_t n, int norb, int kind,
                            const int64_t *off, int64_t *cursor, uint64_t *keys);
int launch_finalize_singles(sqd_ctx *, const uint64_t *s, int norb, const uint64_t *keys,
                            int64_t nnz, const double *h, const double *V, int32_t *tgt,
                            uint16_t *pq, int8_t *sgn, double *val);
int launch_finalize_doubles(sqd_ctx *, const uint64_t *s, int norb, const uint64_t *keys,
                            int64_t nnz, const double *V, int32_t *tgt, uint32_t *orb,
                            int8_t *sgn, double *val);
int launch_string_terms(sqd_ctx *, const uint64_t *s, int64_t n, int norb, const double *h,
                        const double *V, double *energy, double *W, double *u);
int launch_diagonal(sqd_ctx *, const spin_tables *a, const spin_tables *b, int norb,
                    double ecore, const uint64_t *sa, double *diag);

// sigma
int launch_same_spin(sqd_ctx *, const spin_tables *rows, const spin_tables *cols,
                     int64_t nrows, int64_t ncols, const double *C, double *S,
                     const double *diag);
int launch_alpha_beta(sqd_ctx *, const sqd_tables *t, const double *C, double *S);
int measure_fp64_peaks(sqd_ctx *, double *dfma_tflops, double *dmma_tflops);
int set_ab_groups(sqd_ctx *, sqd_tables *t, double scale);
int tune_ab_groups(sqd_ctx *, sqd_tables *t, int mode,
                   int (*launch)(sqd_ctx *, sqd_tables *, const void *, double *), const void *C);
int launch_transpose(sqd_ctx *, const double *in, double *out, int64_t rows, int64_t cols,
                     bool add);

// davidson helpers
int launch_multidot(sqd_ctx *, const double *A, int64_t lda, int m, const double *x,
                    int64_t n, double *partial, int nblk, double *out);
int multidot_blocks(int64_t n);
int launch_gemv_sub(sqd_ctx *, const double *A, int64_t lda, int m, const double *c,
                    double *x, int64_t n);
int launch_combine(sqd_ctx *, const double *A, int64_t lda, int m, const double *Y,
                   int ldy, int k, double *out, int64_t ldo, int64_t n);
int launch_combine_sub(sqd_ctx *, const double *A, int64_t lda, int m, const double *Y,
                       int ldy, int k, double *out, int64_t ldo, int64_t n,
                       const int *gate = nullptr);
int launch_dgks_flag(sqd_ctx *, const double *P, int ldp, int m, int b, const double *tn2,
                     double loss, int *flag);
int block_dot_blocks(const sqd_ctx *, int64_t n);
int launch_block_dot(sqd_ctx *, const double *A, int64_t lda, int m, const double *X,
                     int64_t ldx, int b, int64_t n, double *partial, int nblk, double *out,
                     int ldo, const int *gate = nullptr);
int launch_ritz_block(sqd_ctx *, const double *V, const double *W, int64_t ld, int m,
                      const double *Y, const double *theta, const int *sel, int ks, double *X,
                      double *R, int64_t n, double *partial, int nblk, double *rnorm2);
int launch_project_g(sqd_ctx *, double *G, int ldg, int m, const double *Z, int ldz, int r,
                     double *GZ);
int launch_precondition_norm(sqd_ctx *, const double *R, const double *diag, double theta,
                             double floor_, int64_t n, double *T, double *partial,
                             double *norm2);
int launch_precondition_olsen(sqd_ctx *, const double *R, const double *X, const double *diag,
                              double theta, double floor_, int64_t n, double *T, double *partial,
                              double *norm2);
int launch_scale(sqd_ctx *, double *x, int64_t n, const double *s_dev, int invert_sqrt);
int launch_jacobi_eigh(sqd_ctx *, const double *G, int ldg, int m, double *evals, double *evecs,
                       int m_old = 0, const double *E_old = nullptr,
                       const double *th_old = nullptr);
// sym_n > 0: only positions (I, J) with I <= J of an sym_n x sym_n matrix;
// sym_n < 0: only I < J of a (-sym_n) x (-sym_n) matrix
int launch_argmin_k(sqd_ctx *, const double *d, int64_t n, int k, int64_t *idx_dev,
                    int64_t sym_n = 0);
int launch_set_unit(sqd_ctx *, double *V, int64_t ld, int k, const int64_t *idx_dev);
int launch_set_unit_sym(sqd_ctx *, double *V, int64_t ld, int k, const int64_t *idx_dev,
                        int64_t n, int sgn);
// spin-flip sector pieces (n x n vectors of a shared string set, C^T = sgn C;
// k_spin_flip.cu)
int launch_upper_half(sqd_ctx *, int sgn, const double *C, double *Ch, int64_t n);
int launch_sym_combine(sqd_ctx *, int sgn, const double *T, const double *Y, const double *D,
                       const double *C, double *S, int64_t n);
int launch_symmetrize(sqd_ctx *, int sgn, double *X, int64_t n);
int launch_alpha_beta_upper(sqd_ctx *, const sqd_tables *t, const double *Ch, double *Y);
int alpha_beta_upper_work(sqd_ctx *, sqd_tables *t, double *fmas);
int launch_fix_phase(sqd_ctx *, double *X, int64_t ld, int k, int64_t n, double *work_dev);
int launch_gdk_basis(sqd_ctx *, const double *Y, int m, int m2, const double *P, int mp, int k,
                     int ldp, double *Z, int ldz, int *r_dev);
int launch_identity_cols(sqd_ctx *, double *Y, int r, int k, int ld);
// one-root Davidson: fused passes (MD = fused_md(M): 16 or 32, 0 = unavailable)
int fused_md(int M);
int launch_ritz_prec_dot(sqd_ctx *, int MD, const double *V, const double *W, int64_t ld, int m,
                         const double *y, const double *theta, const double *diag, double floor_,
                         int64_t n, double *T, double *partial, int nblk, double *sums);
int launch_gs_update_dot(sqd_ctx *, int MD, const double *V, int64_t ld, int m, const double *P,
                         double *T, int64_t n, double *partial, int nblk, double *sums);
int launch_gs_update_scale(sqd_ctx *, int MD, const double *V, int64_t ld, int m,
                           const double *P, double scale, double *T, int64_t n, int nblk);
int launch_combine_inplace(sqd_ctx *, double *A, int64_t lda, int m, const double *Z, int ldz,
                           int r, int64_t n);
int launch_gram_tri(sqd_ctx *, const double *T, int64_t ld, int b, int64_t n, double *partial,
                    int nblk, double *out);
int launch_combine_tri(sqd_ctx *, double *T, int64_t ld, int b, const double *Z, int ldz,
                       int64_t n);
int launch_dots_one(sqd_ctx *, int MD, const double *V, int64_t ld, int m, const double *x,
                    int64_t n, double *partial, int nblk, double *out);
int launch_project_coeffs(sqd_ctx *, const double *Z, int ldz, int m, int r, const double *Pold,
                          double *Pnew);

// double-float sigma
int df_prepare(sqd_ctx *ctx, sqd_tables *t);
int sigma_df_one(sqd_ctx *ctx, sqd_tables *t, const double *Cv, double *Sv, double f_a,
                 double f_b, double f_ab);

// outer loop
int launch_string_weights(sqd_ctx *, const double *C, int64_t na, int64_t nb, double *wa,
                          double *wb);
int launch_select_strings(sqd_ctx *, const uint64_t *s, const double *w, int64_t n, double thr,
                          uint64_t *out, int64_t *n_out);
int launch_map_vector(sqd_ctx *, const uint64_t *oa, int64_t noa, const uint64_t *ob, int64_t nob,
                      const double *Cold, const uint64_t *nas, int64_t nna, const uint64_t *nbs,
                      int64_t nnb, double *Cnew, double *norm_out);

// stored H
int stored_build(sqd_ctx *ctx, sqd_tables *t, int64_t max_bytes, int64_t *nnz_out);
int stored_sigma(sqd_ctx *ctx, const sqd_tables *t, const double *C, double *S, int nvec);

// batched
// algorithmic FP64 flops of one sigma of one vector: alpha side (+ diagonal),
// beta side, alpha-beta paired singles
void sigma_work(const sqd_tables *t, double *f_a, double *f_b, double *f_ab);
int davidson_batched_impl(sqd_ctx *ctx, int nprob, sqd_tables *const *tables,
                          const sqd_options *o, double *h_energies, double *const *d_C,
                          int *h_iters, int *h_status);

// rdm
int launch_rdm(sqd_ctx *, const sqd_tables *t, const double *C, double *rdm1, double *rdm2);
int launch_orbital_gradient(sqd_ctx *, const sqd_tables *t, const double *g1, const double *g2,
                            double *grad);
