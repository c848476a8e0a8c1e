/*
 * sqd.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * sample-based quantum diagonalisation (SQD), arXiv 2601.16169.
 *
 * The method (Sections I-II): sampled electron configurations are filtered
 * into sets of alpha strings I_a and beta strings I_b; the Hamiltonian is
 * diagonalised on span{|I_a I_b>} by the Davidson method, whose cost is the
 * matrix-free product sigma = H C (96.5% of an iteration, Section VI) built
 * from one- and two-electron integrals through the Slater-Condon rules.
 *
 * Conventions used by every call
 * ------------------------------
 *  - Strings are uint64_t, bit k set = spatial orbital k occupied;
 *    norb <= 64.  String sets are sorted ascending and free of duplicates.
 *  - h is norb*norb doubles, h[p*norb+q] = h_pq; V is norb^4 doubles in
 *    chemist notation, V[((p*norb+q)*norb+r)*norb+s] = (pq|rs).  Both must
 *    be real-symmetric: h_pq = h_qp and V 8-fold symmetric (checked to
 *    1e-10 relative, else SQD_EINVAL).
 *  - H = E_core + sum_{pq,s} h_pq a+_{ps} a_{qs}
 *        + 1/2 sum_{pqrs,st} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}.
 *  - A determinant |I_a I_b> is the alpha-block-first product
 *    prod_{k in I_a} a+_{k,alpha} prod_{l in I_b} a+_{l,beta} |0>, both
 *    products in ascending orbital order.  Its index is ia * n_beta + ib,
 *    so a vector C is an n_alpha x n_beta row-major matrix (Section IV:
 *    work is threaded over the combined alpha x beta index space).
 *  - Pointers named d_* are device memory owned by the caller (e.g. torch
 *    tensors), h_* are host memory owned by the caller.  Opaque objects
 *    (sqd_ctx, sqd_tables) are owned by the library.
 *  - Every call returns an sqd_status; nothing aborts and no exception
 *    crosses the ABI.  On error, sqd_last_error(ctx) describes it.
 *  - Calls are enqueued on the context's stream.  Calls that return host
 *    scalars (sqd_build_strings, sqd_excitation_tables, sqd_davidson,
 *    sqd_tables_export) synchronise that stream before returning.
 *  - Calls on one context must not run concurrently from several threads.
 */
#ifndef SQD_H
#define SQD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sqd_ctx sqd_ctx;
typedef struct sqd_tables sqd_tables;

typedef enum {
    SQD_OK = 0,
    SQD_EINVAL = -1,        /* invalid argument */
    SQD_ENOMEM = -2,        /* device allocation failed */
    SQD_ECUDA = -3,         /* CUDA runtime error */
    SQD_ENOTCONVERGED = -4, /* Davidson hit max_iter; best estimate returned */
    SQD_EBREAKDOWN = -5,    /* Davidson basis could not be extended */
    SQD_ETIMEOUT = -6       /* reserved */
} sqd_status;

/* ------------------------------------------------------------- context -- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t owned by the caller (NULL = the legacy default stream); all
 * work of the context is enqueued on it. */
int sqd_create(sqd_ctx **ctx, int device, void *cuda_stream);

/* Replace the context's stream (caller-owned). */
int sqd_set_stream(sqd_ctx *ctx, void *cuda_stream);

/* Free the context (not the tables created with it: free those first). */
void sqd_destroy(sqd_ctx *ctx);

/* Text of the last error on this context ("" if none).  Owned by ctx. */
const char *sqd_last_error(const sqd_ctx *ctx);

/* Library version string, e.g. "sqd-gb300 0.1". */
const char *sqd_version(void);

/* -------------------------------------------- a1: string-set filtering -- */

/*
 * Filter sampled configurations into a string set (Sections I and V-A: the
 * sampled configurations are filtered on the classical side; strings are
 * one 64-bit word each, as with bit_length = norb in Section IV-A).
 *
 * d_raw[0..n_raw): raw strings (device).  Keeps those with exactly `nelec`
 * bits set and no bit at or above `norb`, sorts them ascending and removes
 * duplicates into d_out (device, capacity >= n_raw; may equal d_raw).
 * *n_out (host) receives the number of strings written.
 * Errors: SQD_EINVAL for norb outside [1, 64], nelec outside [0, norb],
 * n_raw < 0 or NULL pointers with n_raw > 0.
 */
int sqd_build_strings(sqd_ctx *ctx, const uint64_t *d_raw, int64_t n_raw,
                      int norb, int nelec, uint64_t *d_out, int64_t *n_out);

/*
 * sqd_build_strings_noalloc: the same filter as sqd_build_strings, for
 * callers that cannot allocate device memory -- for example a process whose
 * device memory is all reserved by another allocator (a framework's caching
 * allocator sized to the whole card), or a latency-critical loop that must
 * not pay the device-wide synchronisation that cudaMalloc/cudaFree imply.
 * The paper has no counterpart; it is an interface convenience.
 *
 * It allocates nothing: its scratch is a fixed 6.3 MB array in the
 * library's device memory, which every GPU that loads the library holds
 * until the process exits.  The caller passes the inputs and outputs exactly
 * as for sqd_build_strings (d_out may equal d_raw), with the same result.
 *  - n_raw may be at most 262144 (2^18); larger inputs return SQD_EINVAL
 *    (use sqd_build_strings).
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress) and keeps it for later calls.
 *  - Every call shares the one array and leaves its contents behind: calls
 *    that overlap on the GPU (from several streams, threads or contexts) race
 *    and must be serialised by the caller.
 */
int sqd_build_strings_noalloc(sqd_ctx *ctx, const uint64_t *d_raw, int64_t n_raw,
                              int norb, int nelec, uint64_t *d_out, int64_t *n_out);

/* ---------------------------------- a2-a4: excitation tables, diagonal -- */

/*
 * Build the excitation lists of both string sets and everything sigma needs
 * (Sections II and V-A: per-string excitation lists flattened into
 * offset + entry arrays; the integrals copied to the device once,
 * Section V-C).  The library copies strings and integrals; the caller's
 * buffers may be freed afterwards.
 *
 *   single entry of string I: target J = I - q + p (J in the set),
 *     p = orbital created, q = orbital annihilated,
 *     sign = <J| a+_p a_q |I> = (-1)^(number of occupied orbitals of I
 *     strictly between p and q), val = <I|H_s|J>;
 *   double entry of string I: target J = I - i - j + a + b, i < j, a < b,
 *     sign = <J| a+_a a+_b a_j a_i |I>, val = <I|H_s|J>;
 * H_s being the one-spin Hamiltonian (h plus the same-spin part of V).
 * Entries of a row are sorted by target index.
 *
 * d_alpha / d_beta: sorted unique string sets (device); they may be the same
 * buffer, in which case one table serves both spins.  nalpha_e / nbeta_e are
 * the electron counts of the sets (checked).  d_h, d_V as in the
 * conventions (device).  *tables receives the new object; free it with
 * sqd_free_tables.  n_alpha * n_beta must be below 2^40 and each set below
 * 2^31 strings.
 * Errors: SQD_EINVAL (sizes, popcounts, unsorted sets, asymmetric integrals,
 * non-finite integrals), SQD_ENOMEM.
 */
int sqd_excitation_tables(sqd_ctx *ctx, int norb,
                          const uint64_t *d_alpha, int64_t n_alpha, int nalpha_e,
                          const uint64_t *d_beta, int64_t n_beta, int nbeta_e,
                          const double *d_h, const double *d_V, double ecore,
                          sqd_tables **tables);

void sqd_free_tables(sqd_tables *tables);

/* Sizes of a table object.  info (host, 12 int64):
 *  [0] norb, [1] n_alpha, [2] n_beta, [3] nnz singles alpha, [4] nnz doubles
 *  alpha, [5] nnz singles beta, [6] nnz doubles beta, [7] shared (1 if one
 *  table serves both spins), [8] device bytes held, [9] max singles per
 *  string, [10] max doubles per string, [11] alpha row groups of the
 *  paired-singles work split (chosen by timing candidates on the first
 *  sigma of each sigma mode). */
int sqd_tables_info(const sqd_tables *tables, int64_t *info);

/*
 * Copy one excitation table to host buffers (for verification).
 * spin: 0 alpha, 1 beta.  kind: 1 singles, 2 doubles.
 * h_off (n+1 int64), h_tgt (nnz int32), h_orb (nnz*2 bytes p,q for kind 1;
 * nnz*4 bytes i,j,a,b for kind 2), h_sign (nnz int8), h_val (nnz double).
 * Any pointer may be NULL to skip that field.
 */
int sqd_tables_export(sqd_ctx *ctx, const sqd_tables *tables, int spin, int kind,
                      int64_t *h_off, int32_t *h_tgt, uint8_t *h_orb,
                      int8_t *h_sign, double *h_val);

/*
 * Diagonal H_II of every determinant into d_diag (device, n_alpha*n_beta):
 * E_core + E_a(I_a) + E_b(I_b) + sum_{k in I_a, l in I_b} (kk|ll), the
 * "diagonal terms" the Davidson time includes (Section VI).
 */
int sqd_diagonal(sqd_ctx *ctx, const sqd_tables *tables, double *d_diag);

/* ------------------------------------------------- a5-a7: sigma = H C -- */

/*
 * sigma = (P H P) C for nvec vectors (Section II: matrix-vector product
 * recomputing H_IJ; Section IV: three kinds of bra/ket pairs -- one or two
 * alpha excitations, one or two beta excitations, one alpha and one beta
 * excitation).  d_C and d_sigma are [nvec][n_alpha][n_beta] doubles
 * (device, distinct buffers).  Asynchronous on the context's stream.
 * Scratch (two n_alpha*n_beta vectors) is held by the tables object.
 */
int sqd_sigma(sqd_ctx *ctx, sqd_tables *tables, const double *d_C,
              double *d_sigma, int nvec);

/* ---------------------------------------------- SQD outer loop -- */

/*
 * Carry-over between SQD rounds (Section I: the diagonalisation also picks
 * the configurations carried into the next round of the iterative loop).
 *
 * sqd_string_weights: d_wa[i] = sum_j C(i,j)^2 (n_alpha doubles) and
 *   d_wb[j] = sum_i C(i,j)^2 (n_beta doubles) for the state d_C on the
 *   table's sets (device buffers; either output may be NULL).
 * sqd_select_strings: the strings d_str[i] with d_w[i] >= threshold, in
 *   their order, into d_out (capacity n); *n_out (host) their count.  The
 *   result, joined with newly sampled strings, is the raw input of the next
 *   sqd_build_strings.
 * sqd_map_vector: a warm-start guess for new sets from a state on old sets:
 *   d_new_C(I', J') = d_old_C(I', J') if both strings are in the old sets,
 *   else 0, normalised; *h_norm (host) receives the norm before
 *   normalisation (0: no overlap, the vector is left zero).  All string sets
 *   sorted ascending; vectors [n_alpha][n_beta] row-major on the device.
 */
int sqd_string_weights(sqd_ctx *ctx, const sqd_tables *tables, const double *d_C,
                       double *d_wa, double *d_wb);
int sqd_select_strings(sqd_ctx *ctx, const uint64_t *d_str, const double *d_w, int64_t n,
                       double threshold, uint64_t *d_out, int64_t *n_out);
int sqd_map_vector(sqd_ctx *ctx, const uint64_t *d_old_a, int64_t n_old_a,
                   const uint64_t *d_old_b, int64_t n_old_b, const double *d_old_C,
                   const uint64_t *d_new_a, int64_t n_new_a, const uint64_t *d_new_b,
                   int64_t n_new_b, double *d_new_C, double *h_norm);

/*
 * Arithmetic of the sigma products of one table object:
 *   mode 0 (default): native FP64 multiply-adds;
 *   mode 1: double-float -- every FP64 operand split into a pair of floats
 *     (48 of 53 bits), products formed exactly (Dekker) and summed
 *     error-free (Knuth TwoSum) on the FP32 pipe, results in FP64.  Relative
 *     error of a few 2^-48 per term; sigma agrees with mode 0 to ~1e-14.
 *     Not in the paper: GB300's FP32 pipe is ~58x its FP64 pipe, and the
 *     sigma terms are FP64-bound.
 * Applies to sqd_sigma and sqd_davidson on these tables (not to the batched
 * solver, the stored-H product or the RDMs, which stay FP64).
 * Mode 1 makes float-pair copies of the coefficient tables and the
 * diagonal on first use (the same bytes again) plus one scratch vector.
 */
int sqd_tables_set_sigma_mode(sqd_tables *tables, int mode);

/*
 * Spin-flip sectors (sector = +1 or -1; 0, the default, turns it off).
 * Only for tables built with one string set for both spins (the same device
 * array and electron count); otherwise SQD_EINVAL.
 *
 * With a shared string set, exchanging the alpha and beta strings of every
 * determinant, (Ia, Ib) -> (Ib, Ia), commutes with H (Section II's
 * Hamiltonian is spin-free and (pq|rs) = (rs|pq)), so the vectors, as
 * n x n matrices, split into a symmetric sector (C^T = C) and an
 * antisymmetric one (C^T = -C).  With this determinant ordering (all alpha
 * operators before the beta ones) an eigenstate of total spin S lies in
 * sector (-1)^S, whatever the electron count: singlets in +1, triplets in
 * -1.  On a vector of sector s the beta-beta part of sigma is
 * s times the transpose of the alpha-alpha part, and the alpha-beta part
 * commutes with the transposition, so with sector s set:
 *  - sqd_sigma forms sigma = (T + s T^T) + H_II C + (Y + s Y^T) with
 *    T = sigma_aa(C) and Y = sigma_ab(Ch), Ch the upper triangle of C (half
 *    its diagonal for s = +1): one same-spin pass instead of two and about
 *    half of the paired singles.  The caller states that every input vector
 *    lies in sector s; for any other vector the result is not H C.  Uses
 *    one more scratch vector of the table's size.
 *  - sqd_davidson searches sector s: its guess vectors are the sector's unit
 *    vectors e_II or (e_IJ + s e_JI)/sqrt(2) on the lowest H_II with
 *    Ia <= Ib (Ia < Ib for s = -1), or the caller's guess projected on the
 *    sector, and every correction vector is projected, (X + s X^T)/2,
 *    before it is orthogonalised, so the basis stays exactly in the sector.
 *    Its roots are the lowest of that sector, not necessarily of H.
 * Applies to the FP64 products (sigma mode 0); not to the batched solver,
 * the stored-H product or the RDMs.  Not in the paper, which forms the
 * three parts of sigma on every vector.
 */
int sqd_tables_set_spin_flip(sqd_tables *tables, int sector);

/* ------------------------------------------------ stored-H variant -- */

/*
 * The paper's second method (Section II): compute the Hamiltonian once,
 * store it, and re-use the stored elements in every iteration.
 * sqd_stored_h_build assembles P H P as a CSR matrix held by the table
 * object (12 bytes per nonzero: int32 column, FP64 value; rows in
 * determinant order; per row the diagonal, alpha, beta and alpha-beta
 * elements).  *nnz receives the nonzero count.  If the matrix would exceed
 * max_bytes (0: no limit) or 90% of the free device memory it returns
 * SQD_ENOMEM and builds nothing; N must be below 2^31.
 * sqd_sigma_stored applies it: same contract as sqd_sigma.  Setting
 * use_stored_h in sqd_options makes sqd_davidson use it.
 */
int sqd_stored_h_build(sqd_ctx *ctx, sqd_tables *tables, int64_t max_bytes, int64_t *nnz);
int sqd_sigma_stored(sqd_ctx *ctx, sqd_tables *tables, const double *d_C, double *d_sigma,
                     int nvec);

/* ---------------------------------------------------- a8: Davidson -- */

typedef struct {
    int nroots;          /* number of lowest eigenpairs, 1..28                 */
    int max_iter;        /* iteration limit (e.g. 200)                         */
    int max_subspace;    /* basis size limit; 0 = max(6*nroots, 16); values    */
                         /*    above 112 (the eigensolver's limit) are capped  */
    double tol_energy;   /* |theta - theta_previous| per root                  */
    double tol_residual; /* ||H x - theta x||_2 per root                       */
    double precond_floor;/* clamp of |theta - H_II| (e.g. 1e-8)                */
    int use_guess;       /* 1: d_C holds nroots initial vectors                */
    int use_stored_h;    /* 1: apply the stored matrix (sqd_stored_h_build)    */
    int correction;      /* 0: Davidson t = r/(theta - H_II); 1: Olsen's       */
                         /*    t = (r - eps x)/(theta - H_II) with x^T t = 0   */
} sqd_options;

/*
 * Davidson for the nroots lowest eigenpairs (Section I, Davidson 1975;
 * one sigma per new vector and iteration, diagonal preconditioner,
 * Gram-Schmidt, Section VI) with every step on the device.
 *
 * Guess: unit vectors on the nroots smallest H_II (ties: lower index), or
 * the nroots vectors in d_C if use_guess.  Correction t = r / (theta -
 * H_II) with |denominator| clamped to precond_floor (correction = 1: Olsen's
 * modification, t = (r - eps x) / (theta - H_II) with eps chosen so that
 * x^T t = 0, J. Olsen, P. Jorgensen, J. Simons, Chem. Phys. Lett. 169, 463
 * (1990); not in the paper, off by default).  The corrections of the
 * unconverged roots form one block, orthogonalised by classical
 * Gram-Schmidt against the basis (a second pass when a vector lost more
 * than half its squared norm, decided on the device) and then twice within
 * the block (from the block's Gram matrix, Cholesky QR twice, where every
 * vector keeps 1e-8 of its squared norm; vector by vector otherwise); a
 * vector is dropped if its norm after that is below 1e-12.  With
 * one root (and the Davidson correction, max_subspace <= 16) the passes are
 * fused and both run: the correction and its first projections come from
 * the pass that forms the Ritz pair, and the norm after the second pass
 * follows from Pythagoras, |t''|^2 = |t'|^2 - |V^T t'|^2, unless that
 * difference is not safely resolved (then it is taken explicitly).  At the
 * subspace limit the
 * basis restarts from the 2*nroots lowest Ritz vectors plus the nroots Ritz
 * vectors of the previous iteration orthonormalised against them (GD+k
 * restart; max_subspace must be >= 4*nroots).  Converged when every root
 * has ||r|| <= tol_residual and |delta theta| <= tol_energy (delta over the
 * last growth of the basis) in one iteration; a root that passed is not
 * re-formed until every root has passed.  Rayleigh-Ritz uses a one-block
 * Jacobi eigensolver in FP64, started from the previous eigenvectors while
 * the basis only grows.
 *
 * Outputs: h_energies[nroots] (host), d_C [nroots][n_alpha][n_beta] the
 * Ritz vectors (device, normalised, largest-magnitude component positive),
 * *h_iters (host, may be NULL), h_residuals[nroots] (host, may be NULL).
 * Returns SQD_ENOTCONVERGED (with the last estimates written) when max_iter
 * is reached, SQD_EBREAKDOWN if no new direction survives orthogonalisation
 * (or the basis spans the whole space) before convergence, SQD_EINVAL for
 * nroots outside [1, min(28, dimension)] or max_subspace < 4*nroots.
 */
int sqd_davidson(sqd_ctx *ctx, sqd_tables *tables, const sqd_options *opt,
                 double *h_energies, double *d_C, int *h_iters,
                 double *h_residuals);

/* -------------------------------------------- batched subspaces ----- */

/*
 * Ground states of nbatch independent subspaces at once (SQD produces many
 * subsampled configuration sets per round, Section I; each is one table
 * object from sqd_excitation_tables, all on this context's device).
 * Same Davidson readings as sqd_davidson with nroots == 1 (required),
 * max_subspace 0 meaning 16 (larger values are capped at 16), and the same
 * fused one-vector passes.  Every step runs as one launch over all
 * subspaces; one iteration is captured in a CUDA graph and replayed until
 * every subspace has converged or stopped.  The paired-singles tile is
 * autotuned at the start per size bucket (up to 4 buckets of equal count by
 * determinant count): for each bucket, the kernel variant (16 entries per
 * thread over 4096-entry chunks in a persistent work-queue kernel, or 8
 * entries per thread over 2048-entry chunks in a grid) and the alpha-row
 * group count (0.5, 1, 2 or 4 times the table's default split) are timed on
 * the first sigma of up to 4 of the bucket's largest subspaces.
 *
 * h_energies[nbatch] (host), d_C[b] (device, n_alpha*n_beta doubles each,
 * may be NULL to skip the vector; normalised, largest component positive),
 * h_iters[nbatch] and h_status[nbatch] (host, may be NULL; SQD_OK,
 * SQD_ENOTCONVERGED or SQD_EBREAKDOWN per subspace).  Returns the first
 * non-OK subspace status, or an error of the call itself.
 */
int sqd_davidson_batched(sqd_ctx *ctx, int nbatch, sqd_tables *const *tables,
                         const sqd_options *opt, double *h_energies, double *const *d_C,
                         int *h_iters, int *h_status);

/* What the last sqd_davidson_batched call chose (not in the paper; host
 * outputs, each may be NULL): the alpha-group scale of the paired-singles
 * split, and whether the iteration loop ran inside one graph (1: a
 * conditional WHILE node decided on the device) or as host-driven replays of
 * the captured iteration (0). */
int sqd_batched_tuning(const sqd_ctx *ctx, double *group_scale, int *device_loop);

/* Fix the paired-singles tile of later sqd_davidson_batched calls on this
 * context instead of autotuning it (not in the paper; for tests and
 * measurements): entries_per_thread 16 (persistent kernel, wide chunks) or 8
 * (grid kernel, standard chunks) with group_scale 0.5, 1, 2 or 4;
 * entries_per_thread 0 restores autotuning.  Errors: SQD_EINVAL. */
int sqd_batched_set_tile(sqd_ctx *ctx, int entries_per_thread, double group_scale);

/* The per-bucket tiles of the last sqd_davidson_batched call (not in the
 * paper): *nbuckets (host) receives the bucket count; for the first
 * min(*nbuckets, max_buckets) buckets, in increasing size, h_max_det[q] the
 * largest subspace of the bucket (determinants), h_scale[q] its alpha-group
 * scale and h_entries[q] its entries per thread (16: persistent, 8: grid).
 * Each array may be NULL. */
int sqd_batched_tuning_buckets(const sqd_ctx *ctx, int max_buckets, int *nbuckets,
                               int64_t *h_max_det, double *h_scale, int *h_entries);

/* ------------------------------------------------ adjoint: RDMs ----- */

/*
 * Spin-summed reduced density matrices of the normalised state d_C
 * ([n_alpha][n_beta], device): d_rdm1[p*norb+q] = sum_s <a+_{ps} a_{qs}>
 * and, unless d_rdm2 is NULL, d_rdm2[((p*norb+q)*norb+r)*norb+s] =
 * sum_{s,t} <a+_{ps} a+_{rt} a_{st} a_{qs}> (device outputs).  With C an
 * eigenvector of P H P these are dE/dh_pq and 2 dE/d(pq|rs) element-wise
 * (Hellmann-Feynman); E = E_core + sum h.rdm1 + 1/2 sum V.rdm2.
 * Not in the paper: the adjoint of the subspace energy.
 */
int sqd_rdm(sqd_ctx *ctx, sqd_tables *tables, const double *d_C,
            double *d_rdm1, double *d_rdm2);

/*
 * Orbital-rotation gradient of E for orbitals rotated by U = exp(kappa),
 * kappa antisymmetric, h' = U^T h U, V rotated on all four indices:
 * d_grad[p*norb+q] = dE/dkappa_pq at kappa = 0 = 2 (F_pq - F_qp) with the
 * generalized Fock matrix F_pq = sum_r h_pr rdm1_qr + sum_rst (pr|st)
 * rdm2_qrst (device buffers; rdm1, rdm2 as written by sqd_rdm, for the
 * integrals of `tables`).  Not in the paper.
 */
int sqd_orbital_gradient(sqd_ctx *ctx, sqd_tables *tables, const double *d_rdm1,
                         const double *d_rdm2, double *d_grad);

/* ------------------------------------------------------ measurement --- */

/*
 * Measurement counters (not in the paper; used to report throughput
 * against the roofline).  sqd_profile_enable(ctx, 1) resets the counters
 * and brackets every later kernel region of the library with CUDA events
 * on the context stream; 0 resets and stops timing.
 * Regions are booked in classes:
 *   0 same_spin_alpha, 1 same_spin_beta, 2 alpha_beta, 3 transpose,
 *   4 tables, 5 strings, 6 davidson (Ritz vectors, residuals,
 *   preconditioner, restart), 7 rdm, 8 stored, 9 ortho (Davidson
 *   Gram-Schmidt of the new block against the basis), 10 eigh (Rayleigh-Ritz
 *   eigensolver), 11 batched (a whole sqd_davidson_batched call),
 *   12 batched_sigma, 13 batched_vector, 14 batched_eigh (the stages of the
 *   batched iteration loop: timed on the device with the global timer at the
 *   stage boundaries inside the captured loop, one region per iteration;
 *   flops and bytes summed over the subspaces each stage served),
 *   15 gcols (Davidson: new columns of the projected matrix), 16 ortho_block
 *   (Davidson: orthonormalisation within the new block), 17 batched_sigma_ab
 *   (the paired-singles part of batched_sigma, timed the same way).
 * sqd_profile_read returns, for one class, the class name (static string),
 * the number of regions, their summed event time in ms, and the
 * algorithmic FP64 flops and compulsory bytes booked for them (host
 * outputs, each may be NULL).  It synchronises the stream.
 * sqd_launch_count returns the number of kernels launched on the context
 * since the last sqd_profile_enable call (counted with or without timing).
 */
int sqd_profile_enable(sqd_ctx *ctx, int enable);
int sqd_profile_read(sqd_ctx *ctx, int cls, const char **name, int64_t *regions,
                     double *ms, double *flops, double *bytes);
int sqd_launch_count(const sqd_ctx *ctx, int64_t *launches);

/*
 * FP64 throughput probes (not in the paper): the sigma and Davidson kernels
 * are bound by FP64 arithmetic, so their roofline needs the FP64 rate of
 * this GPU.  Runs a grid of independent FMA chains on the FP64 ALU pipe and
 * a grid of FP64 tensor-core MMAs (m8n8k4), each as the best of three timed
 * launches on the context stream after a warm-up, and returns TFLOP/s
 * (2 flop per multiply-add) in the host doubles given (either may be NULL).
 * Takes about a second; synchronises the stream.  Errors: SQD_EINVAL (NULL
 * ctx), SQD_ECUDA.
 */
int sqd_measure_fp64_peaks(sqd_ctx *ctx, double *dfma_tflops, double *dmma_tflops);

#ifdef __cplusplus
}
#endif

#endif /* SQD_H */
