// Batched SQD: many independent subspaces (each its own alpha/beta string
// sets over one Hamiltonian) solved together for their ground states.
//
// The paper solves one subspace per run; SQD itself produces many
// subsampled subspaces per round (Section I), which is what this serves.
//
// Design
//  - Every Davidson step runs as one launch over all subspaces: the sigma
//    stages are persistent kernels whose blocks pull (subspace, tile) work
//    items from an atomic counter; the vector kernels take (subspace,
//    slice) items; the small dense steps (Jacobi, GD+k restart basis) run
//    one block per subspace.
//  - Control lives on the device: each subspace has a state record
//    (basis size, active flag, theta, residual, ...) that every kernel
//    reads, so the kernel sequence of an iteration is the same for every
//    iteration and every subspace.  It is captured once in a CUDA graph and
//    replayed; the host reads one counter (active subspaces) per replay.
//  - The paired-singles tile is autotuned at setup per size bucket (up to
//    4 buckets of equal count by determinant count): the kernel variant (a
//    persistent work-queue kernel with 16 entries per thread over 4096-entry
//    chunks, or a plain grid with the single-problem tile, 8 entries per
//    thread over 2048-entry chunks at 3 blocks per SM) and the alpha-row
//    group count, timed on the first sigma of the bucket's largest subspaces.
//  - One root per subspace (the ground state), at most 16 basis vectors,
//    GD+k restart to 3 vectors.  The vector stages are the fused one-vector
//    passes of the single-problem solver (4 m + 6 vector passes per
//    iteration instead of 6 m + 14).
//  - With profiling on, a one-warp kernel stamps the global timer at the
//    stage boundaries inside the captured loop, so the sigma, vector and
//    eigensolver stages are timed per iteration on the device.
#include <algorithm>
#include <cmath>
#include <vector>

#include "davidson_body.cuh"
#include "sigma_body.cuh"

#define BV_SLICE 32768  // vector elements per slice item (128 per thread)
#define BV_THREADS 256

struct bdesc {
    int64_t na, nb, N, nsl;
    double sflops;   // algorithmic FP64 flops of one sigma (profiling)
    double abflops;  // the same for its paired-singles term
    ss_args ssa;  // alpha side (C, S filled from the state)
    ss_args ssb;  // beta side on T -> U
    ab_args ab;   // paired singles over the wide chunks (persistent kernel)
    ab_args abn;  // the same over the standard chunks (grid kernel)
    int64_t nch, nchn, ngr;
    double *V, *W, *X, *T, *U;  // V, W: M vectors each; T, U: sigma scratch
    double *G, *evals, *evecs, *Yprev, *Z, *partial, *coef;
    const double *diag;
};

struct bstate {
    int m, mprev, active, status, it, restart, newvec, r, expl;
    double theta, theta_old, rn, nrm2, scale;
    int64_t guess;
};

struct bparams {
    int nprob, M;
    double tol_r, tol_e, floor_;
    int max_iter;
};

__device__ __forceinline__ int find_prob(const int64_t *__restrict__ pre, int nprob,
                                         int64_t item) {
    int lo = 0, hi = nprob;  // pre[lo] <= item < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= item) lo = mid; else hi = mid;
    }
    return lo;
}

// pull the next work item of a persistent kernel (block-uniform)
__device__ __forceinline__ int64_t next_item(unsigned long long *counter) {
    __shared__ int64_t s_item;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_item = (int64_t)atomicAdd(counter, 1ull);
    __syncthreads();
    int64_t it = s_item;
    __syncthreads();
    return it;
}

// ------------------------------------------------------------ sigma stages --

template <bool ALPHA>
__global__ void __launch_bounds__(256) kb_same_spin(const bdesc *__restrict__ D,
                                                    const bstate *__restrict__ S,
                                                    const int64_t *__restrict__ pre, int nprob,
                                                    unsigned long long *counter) {
    const int64_t total = pre[nprob];
    for (;;) {
        const int64_t item = next_item(counter);
        if (item >= total) break;
        const int b = find_prob(pre, nprob, item);
        if (!S[b].newvec) continue;
        const bdesc &d = D[b];
        ss_args a = ALPHA ? d.ssa : d.ssb;
        if (ALPHA) {
            const int64_t slot = (int64_t)(S[b].m - 1) * d.N;
            a.C = d.V + slot;
            a.S = d.W + slot;
        } else {
            a.C = d.T;
            a.S = d.U;
        }
        const int64_t local = item - pre[b];
        same_spin_tile<ALPHA>(a, local % a.nrows, local / a.nrows);
    }
}

// dir 0: new vector (na x nb) -> T (nb x na); dir 1: W slot += U^T
template <int DIR>
__global__ void __launch_bounds__(256) kb_transpose(const bdesc *__restrict__ D,
                                                    const bstate *__restrict__ S,
                                                    const int64_t *__restrict__ pre, int nprob,
                                                    unsigned long long *counter) {
    const int64_t total = pre[nprob];
    for (;;) {
        const int64_t item = next_item(counter);
        if (item >= total) break;
        const int b = find_prob(pre, nprob, item);
        if (!S[b].newvec) continue;
        const bdesc &d = D[b];
        const int64_t slot = (int64_t)(S[b].m - 1) * d.N;
        const int64_t rows = DIR == 0 ? d.na : d.nb, cols = DIR == 0 ? d.nb : d.na;
        const int64_t tx = (cols + 31) / 32;
        const int64_t local = item - pre[b];
        const int64_t c0 = (local % tx) * 32, r0 = (local / tx) * 32;
        if (DIR == 0) transpose_tile<false>(d.V + slot, d.T, rows, cols, c0, r0);
        else transpose_tile<true>(d.U, d.W + slot, rows, cols, c0, r0);
    }
}

// persistent, KB_AB_MINB blocks per SM, AB_EPT_WIDE entries per thread over
// the tables' wide chunks: with 2 blocks per SM the work-queue state and 16
// entries fit the registers (8 entries at 3 blocks per SM spilled here and
// ran slower)
#ifndef KB_AB_MINB
#define KB_AB_MINB 2
#endif
__global__ void __launch_bounds__(AB_THREADS, KB_AB_MINB) kb_alpha_beta(const bdesc *__restrict__ D,
                                                               const bstate *__restrict__ S,
                                                               const int64_t *__restrict__ pre,
                                                               int nprob,
                                                               unsigned long long *counter) {
    const int64_t total = pre[nprob];
    for (;;) {
        const int64_t item = next_item(counter);
        if (item >= total) break;
        const int b = find_prob(pre, nprob, item);
        if (!S[b].newvec) continue;
        const bdesc &d = D[b];
        ab_args a = d.ab;
        const int64_t slot = (int64_t)(S[b].m - 1) * d.N;
        a.C = d.V + slot;
        a.S = d.W + slot;
        const int64_t local = item - pre[b];
        alpha_beta_block_t<AB_EPT_WIDE>(a, local % d.nch, local / d.nch);
    }
}

// the same stage as a plain grid over the items of the subspaces tuned to
// it: the single-problem kernel's tile (standard chunks of AB_ECAP entries,
// AB_EPT entries per thread) with the subspace looked
// up from the block index; blocks of subspaces without a new vector exit
// 3 blocks per SM: the subspace lookup adds registers to the single-problem
// tile, which spills at 4
#ifndef KB_GRID_MINB
#define KB_GRID_MINB 3
#endif
__global__ void __launch_bounds__(AB_THREADS, KB_GRID_MINB)
    kb_alpha_beta_grid(const bdesc *__restrict__ D, const bstate *__restrict__ S,
                       const int64_t *__restrict__ pre, int nprob) {
    const int64_t item = blockIdx.x;
    const int b = find_prob(pre, nprob, item);
    if (!S[b].newvec) return;
    const bdesc &d = D[b];
    ab_args a = d.abn;
    const int64_t slot = (int64_t)(S[b].m - 1) * d.N;
    a.C = d.V + slot;
    a.S = d.W + slot;
    const int64_t local = item - pre[b];
    alpha_beta_block_t<AB_EPT>(a, local % d.nchn, local / d.nchn);
}

// ---------------------------------------------------------- vector stages --

// decode a slice item: problem, element range
struct slice_t {
    int b;
    int64_t lo, hi, s;
};
__device__ __forceinline__ slice_t slice_of(const bdesc *D, const int64_t *pre, int nprob,
                                            int64_t item) {
    slice_t r;
    r.b = find_prob(pre, nprob, item);
    r.s = item - pre[r.b];
    r.lo = r.s * BV_SLICE;
    r.hi = min(D[r.b].N, r.lo + BV_SLICE);
    return r;
}

// The vector stages take the fused one-vector passes of the single-problem
// solver (m <= BM basis vectors per subspace, BM = 16):
//   kb_ritz_fused    : r = W y0 - theta V y0, t = r / (theta - H_II) into V[m]
//                      (or T when the subspace restarts first), partials of
//                      V_i . t, |r|^2, |t|^2 per slice;
//   kb_state_check   : sums them; convergence, restart decision;
//   kb_gs_update_dot : t' = t - V c with V_i . t' and |t'|^2;
//   kb_gs_accept     : |t''|^2 = |t'|^2 - |V^T t'|^2 (Pythagoras) when that is
//                      safely resolved, else the explicit norm is taken;
//   kb_gs_update2    : t'' = (t' - V c') * s.
// The Ritz vector itself is formed once, after the loop (kb_form_x).
#define BM 16

// The bodies are instantiated for the exact basis size MB of the block's
// subspace (a block-uniform switch): a predicated-off FP64 instruction would
// still take its FP64 issue slot, and the FP64 pipe bounds these passes.
template <int N>
struct bm_int {
    static constexpr int value = N;
};
#define BM_CASE(N, f) \
    case N:           \
        f(bm_int<N>{}); \
        break;
#define BM_DISPATCH(m, f)                                                                    \
    switch (m) {                                                                             \
        BM_CASE(1, f) BM_CASE(2, f) BM_CASE(3, f) BM_CASE(4, f) BM_CASE(5, f) BM_CASE(6, f)  \
        BM_CASE(7, f) BM_CASE(8, f) BM_CASE(9, f) BM_CASE(10, f) BM_CASE(11, f)             \
        BM_CASE(12, f) BM_CASE(13, f) BM_CASE(14, f) BM_CASE(15, f)                         \
        default: f(bm_int<16>{}); break;                                                     \
    }

// store the block sums of (projections [MB], extra [NX]) to rows 0..MB-1 and
// MB..MB+NX-1 of the subspace's partials
template <int MB, int NX>
__device__ __forceinline__ void store_sums(const bdesc &d, int64_t slice, const double (&acc)[MB],
                                           const double (&ex)[NX], double *red) {
    double vals[MB + NX];
#pragma unroll
    for (int i = 0; i < MB; i++) vals[i] = acc[i];
#pragma unroll
    for (int i = 0; i < NX; i++) vals[MB + i] = ex[i];
    int i;
    double v;
    if (block_sums<MB + NX>(vals, red, &i, &v)) d.partial[(int64_t)i * d.nsl + slice] = v;
}

template <int MB>
__device__ __forceinline__ void ritz_fused_body(const bdesc &d, const slice_t &sl, int M,
                                                double floor_, double *red) {
    const double th = d.evals[0];
    double *__restrict__ T = (MB + 1 > M) ? d.T : d.V + (int64_t)MB * d.N;
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    double s_r = 0.0, s_t = 0.0;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double vv[MB], ww[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) {
            vv[i] = d.V[(int64_t)i * d.N + n];
            ww[i] = d.W[(int64_t)i * d.N + n];
        }
        double x0 = 0.0, x1 = 0.0, w0 = 0.0, w1 = 0.0;  // two chains each
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            x0 = fma(vv[i], d.evecs[i], x0);
            w0 = fma(ww[i], d.evecs[i], w0);
            if (i + 1 < MB) {
                x1 = fma(vv[i + 1], d.evecs[i + 1], x1);
                w1 = fma(ww[i + 1], d.evecs[i + 1], w1);
            }
        }
        const double r = fma(-th, x0 + x1, w0 + w1);
        const double t = r * precond_recip(th - d.diag[n], floor_);
        T[n] = t;
        s_r = fma(r, r, s_r);
        s_t = fma(t, t, s_t);
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], t, acc[i]);
    }
    const double ex[2] = {s_r, s_t};
    store_sums<MB, 2>(d, sl.s, acc, ex, red);
}

// partial layout per subspace: partial[i * nsl + slice]: rows 0..m-1 the
// projections V_i . t, row m |r|^2, row m+1 |t|^2
__global__ void __launch_bounds__(BV_THREADS) kb_ritz_fused(const bdesc *__restrict__ D,
                                                            const bstate *__restrict__ S,
                                                            const int64_t *__restrict__ pre,
                                                            int nprob, int M, double floor_) {
    __shared__ double red[(BV_THREADS / 32) * (BM + 2)];
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.active) return;
    const bdesc &d = D[sl.b];
    auto go = [&](auto mb) { ritz_fused_body<decltype(mb)::value>(d, sl, M, floor_, red); };
    BM_DISPATCH(st.m, go);
}

// sum the slice partials of rows [0, cnt) into out (one block per subspace,
// one thread per row, fixed order)
__device__ __forceinline__ void sum_rows(const bdesc &d, int cnt, double *out) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        double s = 0.0;
        for (int64_t k = 0; k < d.nsl; k++) s += d.partial[(int64_t)i * d.nsl + k];
        out[i] = s;
    }
}

// convergence test and restart decision (one block per subspace): the
// projections V^T t go to coef, |r|^2 and |t|^2 to the state
__global__ void __launch_bounds__(64) kb_state_check(const bdesc *__restrict__ D,
                                                     bstate *__restrict__ S, bparams P) {
    const int b = blockIdx.x;
    bstate &st = S[b];
    if (threadIdx.x == 0) {
        st.newvec = 0;
        st.restart = 0;
    }
    if (!st.active) return;
    const bdesc &d = D[b];
    const int m = st.m;
    __shared__ double sums[BM + 2];
    sum_rows(d, m + 2, sums);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) d.coef[i] = sums[i];
    if (threadIdx.x != 0) return;
    st.rn = sqrt(sums[m]);
    st.theta = d.evals[0];
    if (st.rn <= P.tol_r && fabs(st.theta - st.theta_old) <= P.tol_e) {
        st.active = 0;
        st.status = 1;
        return;
    }
    if (st.it >= P.max_iter) {
        st.active = 0;
        st.status = SQD_ENOTCONVERGED;
        return;
    }
    st.it++;
    st.theta_old = st.theta;
    st.restart = (st.m + 1 > P.M) ? 1 : 0;
}

// GD+k restart basis Z and the projected G' = Z^T G Z (one block, 128
// threads, per restarting subspace); otherwise keep the Ritz coefficients
__global__ void __launch_bounds__(128) kb_restart_basis(const bdesc *__restrict__ D,
                                                        bstate *__restrict__ S, bparams P) {
    const int b = blockIdx.x;
    bstate &st = S[b];
    if (!st.active) return;
    const bdesc &d = D[b];
    const int m = st.m, M = P.M;
    if (!st.restart) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) d.Yprev[i] = d.evecs[i];
        if (threadIdx.x == 0) st.mprev = m;
        return;
    }
    const int r = gdk_block(d.evecs, m, min(2, m), st.mprev ? d.Yprev : nullptr, st.mprev, 1, M,
                            d.Z, M);
    // G' = Z^T G Z with G symmetric (upper triangle stored)
    __shared__ double GZ[JAC_MAX * 3];
    for (int t = threadIdx.x; t < m * r; t += blockDim.x) {
        const int i = t % m, j = t / m;
        double s = 0.0;
        for (int k = 0; k < m; k++) {
            const double g = (i <= k) ? d.G[i + (int64_t)k * M] : d.G[k + (int64_t)i * M];
            s = fma(g, d.Z[k + (int64_t)j * M], s);
        }
        GZ[i + j * m] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
        const int i = t % r, j = t / r;
        if (i > j) continue;
        double s = 0.0;
        for (int k = 0; k < m; k++) s = fma(d.Z[k + (int64_t)i * M], GZ[k + j * m], s);
        d.G[i + (int64_t)j * M] = s;
    }
    // projections of the correction on the new basis V Z: Z^T coef
    __shared__ double cz[3];
    if (threadIdx.x < r) {
        double s = 0.0;
        for (int k = 0; k < m; k++) s = fma(d.Z[k + (int64_t)threadIdx.x * M], d.coef[k], s);
        cz[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st.r = r;
        d.Yprev[0] = 1.0;
        for (int i = 1; i < r; i++) d.Yprev[i] = 0.0;
        st.mprev = r;
        // the Ritz vector is the first new basis vector (for a later exit)
        d.evecs[0] = 1.0;
        for (int i = 1; i < r; i++) d.evecs[i] = 0.0;
        for (int i = 0; i < r; i++) d.coef[i] = cz[i];
    }
}

// in place: V[0..r) = V Z, W[0..r) = W Z for restarting subspaces
__global__ void __launch_bounds__(BV_THREADS) kb_restart_combine(const bdesc *__restrict__ D,
                                                                 const bstate *__restrict__ S,
                                                                 const int64_t *__restrict__ pre,
                                                                 int nprob, int M) {
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.active || !st.restart) return;
    const bdesc &d = D[sl.b];
    const int m = st.m, r = st.r;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double av[3] = {0.0, 0.0, 0.0}, aw[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < m; i++) {
            const double v = d.V[(int64_t)i * d.N + n], w = d.W[(int64_t)i * d.N + n];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                if (j < r) {
                    const double z = d.Z[i + (int64_t)j * M];
                    av[j] = fma(v, z, av[j]);
                    aw[j] = fma(w, z, aw[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (j < r) {
                d.V[(int64_t)j * d.N + n] = av[j];
                d.W[(int64_t)j * d.N + n] = aw[j];
            }
        }
        d.V[(int64_t)r * d.N + n] = d.T[n];  // the correction, formed before the restart
    }
}

__global__ void kb_restart_finish(bstate *__restrict__ S, int nprob) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    bstate &st = S[b];
    if (st.active && st.restart) st.m = st.r;
}

template <int MB>
__device__ __forceinline__ void gs_update_dot_body(const bdesc &d, const slice_t &sl,
                                                   double *red) {
    double *__restrict__ T = d.V + (int64_t)MB * d.N;
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    double s_t = 0.0;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = d.V[(int64_t)i * d.N + n];
        const double t0 = T[n];
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            s0 = fma(vv[i], d.coef[i], s0);
            if (i + 1 < MB) s1 = fma(vv[i + 1], d.coef[i + 1], s1);
        }
        const double t = t0 - (s0 + s1);
        T[n] = t;
        s_t = fma(t, t, s_t);
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], t, acc[i]);
    }
    const double ex[1] = {s_t};
    store_sums<MB, 1>(d, sl.s, acc, ex, red);
}

// t' = t - V coef (t = V[m]) with partials of V_i . t' (rows 0..m-1) and
// |t'|^2 (row m)
__global__ void __launch_bounds__(BV_THREADS) kb_gs_update_dot(const bdesc *__restrict__ D,
                                                               const bstate *__restrict__ S,
                                                               const int64_t *__restrict__ pre,
                                                               int nprob) {
    __shared__ double red[(BV_THREADS / 32) * (BM + 1)];
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.active) return;
    const bdesc &d = D[sl.b];
    auto go = [&](auto mb) { gs_update_dot_body<decltype(mb)::value>(d, sl, red); };
    BM_DISPATCH(st.m, go);
}

// second-pass coefficients; the norm after the second pass by Pythagoras
// where safely resolved (else expl = 1: the norm is taken explicitly)
__global__ void __launch_bounds__(64) kb_gs_accept(const bdesc *__restrict__ D,
                                                   bstate *__restrict__ S) {
    const int b = blockIdx.x;
    bstate &st = S[b];
    if (!st.active) return;
    const bdesc &d = D[b];
    const int m = st.m;
    __shared__ double sums[BM + 1];
    sum_rows(d, m + 1, sums);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) d.coef[i] = sums[i];
    if (threadIdx.x != 0) return;
    double p2 = 0.0;
    for (int i = 0; i < m; i++) p2 += sums[i] * sums[i];
    const double n2a = sums[m], n2b = n2a - p2;
    if (p2 <= 0.5 * n2a && n2b >= 1e-20) {
        st.expl = 0;
        st.scale = 1.0 / sqrt(n2b);
    } else {
        st.expl = 1;
        st.scale = 1.0;
    }
}

template <int MB>
__device__ __forceinline__ void gs_update2_body(const bdesc &d, const slice_t &sl, double sc) {
    double *__restrict__ T = d.V + (int64_t)MB * d.N;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = d.V[(int64_t)i * d.N + n];
        const double t0 = T[n];
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            s0 = fma(vv[i], d.coef[i], s0);
            if (i + 1 < MB) s1 = fma(vv[i + 1], d.coef[i + 1], s1);
        }
        T[n] = (t0 - (s0 + s1)) * sc;
    }
}

// t'' = (t' - V coef) * scale
__global__ void __launch_bounds__(BV_THREADS) kb_gs_update2(const bdesc *__restrict__ D,
                                                            const bstate *__restrict__ S,
                                                            const int64_t *__restrict__ pre,
                                                            int nprob) {
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.active) return;
    const bdesc &d = D[sl.b];
    const double sc = st.scale;
    auto go = [&](auto mb) { gs_update2_body<decltype(mb)::value>(d, sl, sc); };
    BM_DISPATCH(st.m, go);
}

template <int MB>
__device__ __forceinline__ void gcol_body(const bdesc &d, const slice_t &sl, double *red) {
    const double *__restrict__ x = d.W + (int64_t)(MB - 1) * d.N;
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = d.V[(int64_t)i * d.N + n];
        const double xn = x[n];
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], xn, acc[i]);
    }
    const double ex[1] = {0.0};
    store_sums<MB, 1>(d, sl.s, acc, ex, red);  // rows 0..m-1 (row m unused)
}

// new column of G: partials of V[i] . W[m-1], i < m (after m was incremented),
// every basis value of an element loaded once
__global__ void __launch_bounds__(BV_THREADS) kb_gcol(const bdesc *__restrict__ D,
                                                      const bstate *__restrict__ S,
                                                      const int64_t *__restrict__ pre, int nprob) {
    __shared__ double red[(BV_THREADS / 32) * (BM + 1)];
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.newvec) return;
    const bdesc &d = D[sl.b];
    auto go = [&](auto mb) { gcol_body<decltype(mb)::value>(d, sl, red); };
    BM_DISPATCH(st.m, go);
}

// partial dot products on a slice.  mode 1: V[m] . V[m] (the explicit norm,
// subspaces with expl set); mode 2: V[i] . W[m-1], i < m (new column of G,
// after m was incremented)
__global__ void __launch_bounds__(BV_THREADS) kb_gram(const bdesc *__restrict__ D,
                                                      const bstate *__restrict__ S,
                                                      const int64_t *__restrict__ pre, int nprob,
                                                      int mode) {
    __shared__ double red[32];
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (mode == 2 ? !st.newvec : !(st.active && st.expl)) return;
    const bdesc &d = D[sl.b];
    const int m = st.m;
    const double *x = (mode == 2) ? d.W + (int64_t)(m - 1) * d.N : d.V + (int64_t)m * d.N;
    const int cnt = (mode == 1) ? 1 : m;
    int i = 0;
    for (; i + 4 <= cnt; i += 4) {  // four basis vectors per pass over the slice
        const double *a0 = d.V + (int64_t)i * d.N;
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
            const double xn = x[n];
#pragma unroll
            for (int u = 0; u < 4; u++) s[u] = fma(a0[(int64_t)u * d.N + n], xn, s[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const double t = block_sum(s[u], red);
            if (threadIdx.x == 0) d.partial[(int64_t)(i + u) * d.nsl + sl.s] = t;
        }
    }
    for (; i < cnt; i++) {
        const double *a = d.V + (int64_t)(mode == 1 ? m : i) * d.N;
        double s = 0.0;
        for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) s = fma(a[n], x[n], s);
        const double t = block_sum(s, red);
        if (threadIdx.x == 0) d.partial[(int64_t)i * d.nsl + sl.s] = t;
    }
}

// sum the partials: one block per subspace, one thread per coefficient
__global__ void kb_gram_final(const bdesc *__restrict__ D, bstate *__restrict__ S, int mode,
                              int M) {
    const int b = blockIdx.x;
    bstate &st = S[b];
    if (mode == 2 ? !st.newvec : !(st.active && st.expl)) return;
    const bdesc &d = D[b];
    const int cnt = (mode == 1) ? 1 : st.m;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        double s = 0.0;
        for (int64_t k = 0; k < d.nsl; k++) s += d.partial[(int64_t)i * d.nsl + k];
        if (mode == 1) st.nrm2 = s;
        else d.G[i + (int64_t)(st.m - 1) * M] = s;
    }
}

// keep or drop the orthogonalised correction
__global__ void kb_state_accept(bstate *__restrict__ S, bparams P) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= P.nprob) return;
    bstate &st = S[b];
    st.newvec = 0;
    if (!st.active) return;
    if (!st.expl) {  // normalised in kb_gs_update2
        st.m++;
        st.newvec = 1;
        return;
    }
    const double nrm = sqrt(st.nrm2);
    if (nrm >= 1e-12) {
        st.scale = 1.0 / nrm;
        st.m++;
        st.newvec = 1;
    } else {
        st.active = 0;
        st.status = (st.rn <= P.tol_r) ? 1 : SQD_EBREAKDOWN;
    }
}

// normalise a correction whose norm was taken explicitly
__global__ void __launch_bounds__(BV_THREADS) kb_scale_new(const bdesc *__restrict__ D,
                                                           const bstate *__restrict__ S,
                                                           const int64_t *__restrict__ pre,
                                                           int nprob) {
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    if (!st.newvec || !st.expl) return;
    const bdesc &d = D[sl.b];
    double *v = d.V + (int64_t)(st.m - 1) * d.N;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) v[n] *= st.scale;
}

// the Ritz vector of the final eigensolve, X = V y0 (after the loop)
__global__ void __launch_bounds__(BV_THREADS) kb_form_x(const bdesc *__restrict__ D,
                                                        const bstate *__restrict__ S,
                                                        const int64_t *__restrict__ pre,
                                                        int nprob) {
    const slice_t sl = slice_of(D, pre, nprob, blockIdx.x);
    const bstate &st = S[sl.b];
    const bdesc &d = D[sl.b];
    const int m = st.m;
    for (int64_t n = sl.lo + threadIdx.x; n < sl.hi; n += BV_THREADS) {
        double x = 0.0;
        for (int i = 0; i < m; i++) x = fma(d.V[(int64_t)i * d.N + n], d.evecs[i], x);
        d.X[n] = x;
    }
}

__global__ void __launch_bounds__(256) kb_jacobi(const bdesc *__restrict__ D,
                                                 const bstate *__restrict__ S, int M) {
    const int b = blockIdx.x;
    if (!S[b].active) return;
    const bdesc &d = D[b];
    jacobi_block(d.G, M, S[b].m, d.evals, d.evecs);
}

// end of a loop iteration on the device: run the body again while some
// subspace is active and the iteration limit is not reached
__global__ void kb_loop_control(const int *__restrict__ active, int *__restrict__ iters,
                                int limit, cudaGraphConditionalHandle h) {
    const int it = ++(*iters);
    cudaGraphSetConditional(h, (*active > 0 && it < limit) ? 1u : 0u);
}

// Stage timer of the batched loop (profiling only; one warp).  Stamped at
// the stage boundaries inside the captured loop: the global-timer interval
// since the previous stamp is booked to `stage` (0 sigma apart from its
// paired singles, 1 vector work, 2 eigensolve, 3 the paired singles; -1 only
// sets the start), with the algorithmic work of the subspaces the stage
// served: sigma flops of those given a new vector (booked by the stamp that
// ends the sigma stage, part 0; part 1 books time only), paired-singles flops;
// vector bytes and flops of the one-vector Davidson step (Ritz pair, residual,
// correction, two Gram-Schmidt passes, normalisation in three fused passes:
// 4 m + 6 vector passes and 12 m + 12 flops per element; part 1) or of the
// new G column (m + 1 passes, 2 m flops; part 2).
// acc: [0..4) ns, [4..8) flops, [8..12) bytes, [12..16) regions, [16] last stamp
__global__ void kb_stamp(const bdesc *__restrict__ D, const bstate *__restrict__ S, int nprob,
                         int stage, int part, double *__restrict__ acc) {
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    double f = 0.0, by = 0.0;
    if (stage >= 0) {
        for (int b = threadIdx.x; b < nprob; b += 32) {
            if (!S[b].newvec) continue;
            const double N = (double)D[b].N;
            const int m = S[b].m;  // after the new vector was appended
            if (stage == 0 && part == 0) {
                f += D[b].sflops;
            } else if (stage == 3) {
                f += D[b].abflops;
            } else if (stage == 1 && part == 1) {
                by += 8.0 * N * (4.0 * (m - 1) + 6.0);
                f += N * (12.0 * (m - 1) + 12.0);
            } else if (stage == 1) {
                by += 8.0 * N * (m + 1.0);
                f += 2.0 * N * m;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f += __shfl_down_sync(0xffffffffu, f, o);
            by += __shfl_down_sync(0xffffffffu, by, o);
        }
    }
    if (threadIdx.x == 0) {
        unsigned long long *last = reinterpret_cast<unsigned long long *>(acc + 16);
        if (stage >= 0) {
            acc[stage] += (double)(now - *last);
            acc[4 + stage] += f;
            acc[8 + stage] += by;
            if ((stage == 0 && part == 0) || (stage == 1 && part == 1) || stage == 2 ||
                stage == 3)
                acc[12 + stage] += 1.0;
        }
        *last = now;
    }
}

__global__ void kb_count_active(const bstate *__restrict__ S, int nprob, int *out) {
    __shared__ int c;
    if (threadIdx.x == 0) c = 0;
    __syncthreads();
    for (int b = threadIdx.x; b < nprob; b += blockDim.x)
        if (S[b].active) atomicAdd(&c, 1);
    __syncthreads();
    if (threadIdx.x == 0) *out = c;
}

// ---------------------------------------------------------------- setup --

// initial guess: the determinant of lowest H_II (lowest index on ties)
__global__ void __launch_bounds__(256) kb_guess(const bdesc *__restrict__ D,
                                                bstate *__restrict__ S) {
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    const int b = blockIdx.x;
    const bdesc &d = D[b];
    double bv = INFINITY;
    int64_t bi = -1;
    for (int64_t n = threadIdx.x; n < d.N; n += blockDim.x) {
        const double v = d.diag[n];
        if (bi < 0 || v < bv) {
            bv = v;
            bi = n;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double v2 = sv[threadIdx.x + o];
            const int64_t i2 = si[threadIdx.x + o];
            if (i2 >= 0 && (si[threadIdx.x] < 0 || v2 < sv[threadIdx.x] ||
                            (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x]))) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bstate &st = S[b];
        st = bstate();
        st.guess = si[0];
        st.m = 1;
        st.active = 1;
        st.newvec = 1;
        st.theta_old = INFINITY;
        d.V[si[0]] = 1.0;
    }
}

struct batched_plan {
    int nprob = 0, M = 0;
    double *stamps = nullptr;  // stage timer accumulators (profiling), 17 doubles
    std::vector<bdesc> hdesc;
    bdesc *D = nullptr;
    bstate *S = nullptr;
    int64_t *pre_ssa = nullptr, *pre_ssb = nullptr, *pre_ab = nullptr, *pre_t0 = nullptr,
            *pre_t1 = nullptr, *pre_vec = nullptr;
    int64_t tot_vec = 0;
    int64_t *pre_abg = nullptr;    // item prefix of the grid paired-singles kernel
    int64_t ab_items[2] = {0, 0};  // items of the persistent (0) and grid (1) kernels
    unsigned long long *counters = nullptr;  // 5 persistent-kernel queues
    int *d_active = nullptr;
    std::vector<void *> owned;  // device allocations
    std::vector<int64_t *> groups;  // per-problem alpha group arrays (owned)
};

static int plan_alloc(sqd_ctx *ctx, batched_plan &p, void **ptr, size_t bytes) {
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sqd_fail(ctx, e == cudaErrorMemoryAllocation ? SQD_ENOMEM : SQD_ECUDA,
                        "batched allocation of %zu bytes failed: %s", bytes,
                        cudaGetErrorString(e));
    }
    p.owned.push_back(*ptr);
    return SQD_OK;
}

static void plan_free(batched_plan &p) {
    for (void *q : p.owned) cudaFree(q);
    p.owned.clear();
}

static int upload_prefix(sqd_ctx *ctx, batched_plan &p, const std::vector<int64_t> &v,
                         int64_t **out) {
    SQD_TRY(plan_alloc(ctx, p, (void **)out, sizeof(int64_t) * v.size()));
    SQD_CUDA(ctx, cudaMemcpy(*out, v.data(), sizeof(int64_t) * v.size(), cudaMemcpyHostToDevice));
    return SQD_OK;
}

// alpha row groups of one subspace: `ng` groups of roughly equal single counts
static std::vector<int64_t> alpha_groups(const spin_tables *A, int64_t ng) {
    const std::vector<int64_t> &ao = A->h_off1;
    const int64_t total = ao[A->n];
    if (ng > A->n) ng = A->n;
    if (ng < 1) ng = 1;
    std::vector<int64_t> g{0};
    int64_t r = 0;
    for (int64_t k = 1; k < ng; k++) {
        const int64_t want = total * k / ng;
        while (r < A->n && ao[r] < want) r++;
        if (r > g.back()) g.push_back(r);
    }
    g.push_back(A->n);
    return g;
}

__global__ void kb_zero_counters(unsigned long long *c, int n) {
    if ((int)threadIdx.x < n) c[threadIdx.x] = 0ull;
}

// the paired-singles stage: the persistent kernel for the subspaces tuned
// to the wide tile, the grid kernel for the others
static int launch_ab_stage(sqd_ctx *ctx, batched_plan &p) {
    const size_t shm = sizeof(double) * 2 * AB_NA * AB_YW;
    if (p.ab_items[0] > 0) {
        kb_alpha_beta<<<KB_AB_MINB * ctx->sm_count, AB_THREADS, shm, ctx->stream>>>(
            p.D, p.S, p.pre_ab, p.nprob, p.counters + 2);
        SQD_LAUNCHED(ctx);
    }
    if (p.ab_items[1] > 0) {
        kb_alpha_beta_grid<<<(unsigned)p.ab_items[1], AB_THREADS, shm, ctx->stream>>>(
            p.D, p.S, p.pre_abg, p.nprob);
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

// launch the three sigma stages for every subspace flagged newvec (kernels
// only, so the sequence can be the body of a conditional graph node)
static int stamp(sqd_ctx *ctx, batched_plan &p, int stage, int part = 0);

// in_loop: inside the captured iteration, where the stage timer runs
static int launch_sigma_stages(sqd_ctx *ctx, batched_plan &p, bool in_loop = false) {
    const int n = p.nprob;
    const int sm = ctx->sm_count;
    kb_zero_counters<<<1, 32, 0, ctx->stream>>>(p.counters, 5);
    SQD_LAUNCHED(ctx);
    kb_same_spin<true><<<8 * sm, 256, 0, ctx->stream>>>(p.D, p.S, p.pre_ssa, n, p.counters + 0);
    SQD_LAUNCHED(ctx);
    kb_transpose<0><<<8 * sm, dim3(32, 8), 0, ctx->stream>>>(p.D, p.S, p.pre_t0, n,
                                                             p.counters + 1);
    SQD_LAUNCHED(ctx);
    if (in_loop) SQD_TRY(stamp(ctx, p, 0, 1));
    SQD_TRY(launch_ab_stage(ctx, p));
    if (in_loop) SQD_TRY(stamp(ctx, p, 3));
    kb_same_spin<false><<<8 * sm, 256, 0, ctx->stream>>>(p.D, p.S, p.pre_ssb, n,
                                                         p.counters + 3);
    SQD_LAUNCHED(ctx);
    kb_transpose<1><<<8 * sm, dim3(32, 8), 0, ctx->stream>>>(p.D, p.S, p.pre_t1, n,
                                                             p.counters + 4);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

static int launch_gram(sqd_ctx *ctx, batched_plan &p, int mode) {
    if (mode == 2)
        kb_gcol<<<(unsigned)p.tot_vec, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec,
                                                                     p.nprob);
    else
        kb_gram<<<(unsigned)p.tot_vec, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, p.nprob,
                                                                     mode);
    SQD_LAUNCHED(ctx);
    kb_gram_final<<<p.nprob, 128, 0, ctx->stream>>>(p.D, p.S, mode, p.M);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

static int stamp(sqd_ctx *ctx, batched_plan &p, int stage, int part) {
    if (!p.stamps) return SQD_OK;
    kb_stamp<<<1, 32, 0, ctx->stream>>>(p.D, p.S, p.nprob, stage, part, p.stamps);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// one Davidson iteration for every active subspace (the captured sequence)
static int launch_iteration(sqd_ctx *ctx, batched_plan &p, const bparams &P) {
    const int n = p.nprob;
    const unsigned vb = (unsigned)p.tot_vec;
    const unsigned tb = (unsigned)((n + 127) / 128);
    const size_t jshm = sizeof(double) * 2 * (size_t)((p.M + 1) & ~1) * (((p.M + 1) & ~1) + 1);
    SQD_TRY(stamp(ctx, p, -1));
    kb_jacobi<<<n, 256, jshm, ctx->stream>>>(p.D, p.S, p.M);
    SQD_LAUNCHED(ctx);
    SQD_TRY(stamp(ctx, p, 2));
    kb_ritz_fused<<<vb, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, n, p.M, P.floor_);
    SQD_LAUNCHED(ctx);
    kb_state_check<<<n, 64, 0, ctx->stream>>>(p.D, p.S, P);
    SQD_LAUNCHED(ctx);
    kb_restart_basis<<<n, 128, 0, ctx->stream>>>(p.D, p.S, P);
    SQD_LAUNCHED(ctx);
    kb_restart_combine<<<vb, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, n, p.M);
    SQD_LAUNCHED(ctx);
    kb_restart_finish<<<tb, 128, 0, ctx->stream>>>(p.S, n);
    SQD_LAUNCHED(ctx);
    kb_gs_update_dot<<<vb, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, n);
    SQD_LAUNCHED(ctx);
    kb_gs_accept<<<n, 64, 0, ctx->stream>>>(p.D, p.S);
    SQD_LAUNCHED(ctx);
    kb_gs_update2<<<vb, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, n);
    SQD_LAUNCHED(ctx);
    SQD_TRY(launch_gram(ctx, p, 1));  // explicit norms only where Pythagoras was not safe
    kb_state_accept<<<tb, 128, 0, ctx->stream>>>(p.S, P);
    SQD_LAUNCHED(ctx);
    kb_scale_new<<<vb, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, n);
    SQD_LAUNCHED(ctx);
    SQD_TRY(stamp(ctx, p, 1, 1));
    SQD_TRY(launch_sigma_stages(ctx, p, true));
    SQD_TRY(stamp(ctx, p, 0));
    SQD_TRY(launch_gram(ctx, p, 2));
    kb_count_active<<<1, 256, 0, ctx->stream>>>(p.S, n, p.d_active);
    SQD_LAUNCHED(ctx);
    SQD_TRY(stamp(ctx, p, 1, 2));
    return SQD_OK;
}

// Tile choices of the paired-singles stage, per subspace: the kernel
// variant (0: persistent, wide chunks of AB_ECAP_WIDE entries, 16 per
// thread, 2 blocks per SM; 1: grid, standard chunks, AB_EPT per thread,
// AB_MINB blocks per SM) and the alpha-row group count (the table's default
// split times a scale).  Group arrays are built once per candidate scale.
static const double kAbScales[] = {0.5, 1.0, 2.0, 4.0};
#define AB_NSCALE 4

struct ab_choice {
    std::vector<int64_t *> groups;  // per scale: device group rows
    std::vector<int64_t> ngr;       // per scale: group count
};

static int build_choices(sqd_ctx *ctx, batched_plan &p, const std::vector<sqd_tables *> &tabs,
                         std::vector<ab_choice> &ch) {
    ch.resize(p.nprob);
    for (int b = 0; b < p.nprob; b++) {
        const sqd_tables *t = tabs[b];
        // relative to the default split (the table's own split may be tuned)
        const double base = t->ab.ngroups / (t->ab.scale > 0.0 ? t->ab.scale : 1.0);
        for (int k = 0; k < AB_NSCALE; k++) {
            int64_t ng = (int64_t)std::llround(std::max(1.0, base * kAbScales[k]));
            if (ng > t->a.n) ng = std::max<int64_t>(1, t->a.n);
            std::vector<int64_t> g = alpha_groups(&t->a, ng);
            int64_t *dg = nullptr;
            SQD_TRY(plan_alloc(ctx, p, (void **)&dg, sizeof(int64_t) * g.size()));
            SQD_CUDA(ctx, cudaMemcpyAsync(dg, g.data(), sizeof(int64_t) * g.size(),
                                          cudaMemcpyHostToDevice, ctx->stream));
            SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            ch[b].groups.push_back(dg);
            ch[b].ngr.push_back((int64_t)g.size() - 1);
        }
    }
    SQD_TRY(plan_alloc(ctx, p, (void **)&p.pre_ab, sizeof(int64_t) * (p.nprob + 1)));
    SQD_TRY(plan_alloc(ctx, p, (void **)&p.pre_abg, sizeof(int64_t) * (p.nprob + 1)));
    return SQD_OK;
}

// apply (variant, scale index) per subspace; `on` (optional) limits the
// paired-singles items to the flagged subspaces (tuning)
static int apply_choices(sqd_ctx *ctx, batched_plan &p, const std::vector<sqd_tables *> &tabs,
                         const std::vector<ab_choice> &ch, const std::vector<int> &var,
                         const std::vector<int> &sck, const std::vector<char> *on) {
    std::vector<int64_t> pre0{0}, pre1{0};
    for (int b = 0; b < p.nprob; b++) {
        const sqd_tables *t = tabs[b];
        bdesc &d = p.hdesc[b];
        d.ab.group_rows = d.abn.group_rows = ch[b].groups[sck[b]];
        d.ngr = ch[b].ngr[sck[b]];
        const bool has = t->a.nnz1 > 0 && t->b->nnz1 > 0 && (!on || (*on)[b]);
        pre0.push_back(pre0.back() + ((has && var[b] == 0) ? d.nch * d.ngr : 0));
        pre1.push_back(pre1.back() + ((has && var[b] == 1) ? d.nchn * d.ngr : 0));
    }
    p.ab_items[0] = pre0.back();
    p.ab_items[1] = pre1.back();
    if (p.ab_items[1] > 2147483647LL) return sqd_fail(ctx, SQD_EINVAL, "batch too large");
    cudaStream_t st = ctx->stream;
    SQD_CUDA(ctx, cudaMemcpyAsync(p.D, p.hdesc.data(), sizeof(bdesc) * p.nprob,
                                  cudaMemcpyHostToDevice, st));
    SQD_CUDA(ctx, cudaMemcpyAsync(p.pre_ab, pre0.data(), sizeof(int64_t) * pre0.size(),
                                  cudaMemcpyHostToDevice, st));
    SQD_CUDA(ctx, cudaMemcpyAsync(p.pre_abg, pre1.data(), sizeof(int64_t) * pre1.size(),
                                  cudaMemcpyHostToDevice, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    return SQD_OK;
}

int davidson_batched_impl(sqd_ctx *ctx, int nprob, sqd_tables *const *tables,
                          const sqd_options *o, double *h_energies, double *const *d_C,
                          int *h_iters, int *h_status) {
    batched_plan p;
    p.nprob = nprob;
    // at most BM = 16 basis vectors per subspace (the fused vector passes
    // keep the projections in registers; a larger one-root basis did not
    // reduce the iterations: 176 / 175 / 174 at 16 / 24 / 32 on 4e8 dets)
    p.M = o->max_subspace > 0 ? std::min(o->max_subspace, BM) : BM;
    if (p.M < 4) return sqd_fail(ctx, SQD_EINVAL, "max_subspace must be >= 4");
    std::vector<sqd_tables *> tabs(tables, tables + nprob);
    p.hdesc.resize(nprob);
    std::vector<int64_t> pssa{0}, pssb{0}, pt0{0}, pt1{0}, pvec{0};
    const int M = p.M;
    int rc = SQD_OK;
    auto fail = [&](int r) {
        cudaStreamSynchronize(ctx->stream);
        plan_free(p);
        return r;
    };
    for (int b = 0; b < nprob; b++) {
        sqd_tables *t = tabs[b];
        bdesc &d = p.hdesc[b];
        d.na = t->a.n;
        d.nb = t->b->n;
        d.N = d.na * d.nb;
        const int Mb = (int)std::min<int64_t>(M, d.N);
        (void)Mb;
        d.nsl = (d.N + BV_SLICE - 1) / BV_SLICE;
        void *q;
#define BA(field, count)                                                             \
    if ((rc = plan_alloc(ctx, p, &q, sizeof(double) * (size_t)(count))) != SQD_OK)  \
        return fail(rc);                                                             \
    d.field = (double *)q;
        BA(V, (int64_t)M * d.N);
        BA(W, (int64_t)M * d.N);
        BA(X, d.N);
        BA(T, d.N);
        BA(U, d.N);
        BA(G, (int64_t)M * M);
        BA(evals, M);
        BA(evecs, (int64_t)M * M);
        BA(Yprev, M);
        BA(Z, (int64_t)M * 3);
        BA(partial, (int64_t)(M + 2) * d.nsl);
        BA(coef, M);
#undef BA
        if ((rc = (cudaMemsetAsync(d.V, 0, sizeof(double) * d.N, ctx->stream) == cudaSuccess
                       ? SQD_OK
                       : SQD_ECUDA)) != SQD_OK)
            return fail(sqd_fail(ctx, rc, "memset failed"));
        if (!t->diag) return fail(sqd_fail(ctx, SQD_EINVAL, "table without diagonal"));
        d.diag = t->diag;
        d.ssa = make_ss_args(&t->a, t->b, d.na, d.nb, nullptr, nullptr, t->diag);
        d.ssb = make_ss_args(t->b, &t->a, d.nb, d.na, nullptr, nullptr, nullptr);
        d.ab = make_ab_args(t, nullptr, nullptr);
        {
            double fa, fb, fab;
            sigma_work(t, &fa, &fb, &fab);
            d.sflops = fa + fb + fab;
            d.abflops = fab;
        }
        // persistent kernel: wide chunks; grid kernel: the standard ones
        d.abn = d.ab;
        d.ab.chunk_e = t->ab.chunk_e_wide;
        d.ab.chunk_y = t->ab.chunk_y_wide;
        d.nch = t->ab.nchunks_wide;
        d.nchn = t->ab.nchunks;
        d.ngr = t->ab.ngroups;
        pssa.push_back(pssa.back() + d.na * ((d.nb + 255) / 256));
        pssb.push_back(pssb.back() + d.nb * ((d.na + 255) / 256));
        pt0.push_back(pt0.back() + ((d.nb + 31) / 32) * ((d.na + 31) / 32));
        pt1.push_back(pt1.back() + ((d.na + 31) / 32) * ((d.nb + 31) / 32));
        pvec.push_back(pvec.back() + d.nsl);
    }
    p.tot_vec = pvec.back();
    if (p.tot_vec > 2147483647LL) return fail(sqd_fail(ctx, SQD_EINVAL, "batch too large"));
    if ((rc = plan_alloc(ctx, p, (void **)&p.D, sizeof(bdesc) * nprob)) != SQD_OK) return fail(rc);
    if ((rc = plan_alloc(ctx, p, (void **)&p.S, sizeof(bstate) * nprob)) != SQD_OK) return fail(rc);
    if ((rc = plan_alloc(ctx, p, (void **)&p.counters, sizeof(unsigned long long) * 8)) != SQD_OK)
        return fail(rc);
    if ((rc = plan_alloc(ctx, p, (void **)&p.d_active, sizeof(int))) != SQD_OK) return fail(rc);
    if (ctx->prof) {
        if ((rc = plan_alloc(ctx, p, (void **)&p.stamps, sizeof(double) * 17)) != SQD_OK)
            return fail(rc);
        if (cudaMemsetAsync(p.stamps, 0, sizeof(double) * 17, ctx->stream) != cudaSuccess)
            return fail(sqd_fail(ctx, SQD_ECUDA, "memset failed"));
    }
    if ((rc = upload_prefix(ctx, p, pssa, &p.pre_ssa)) != SQD_OK) return fail(rc);
    if ((rc = upload_prefix(ctx, p, pssb, &p.pre_ssb)) != SQD_OK) return fail(rc);
    if ((rc = upload_prefix(ctx, p, pt0, &p.pre_t0)) != SQD_OK) return fail(rc);
    if ((rc = upload_prefix(ctx, p, pt1, &p.pre_t1)) != SQD_OK) return fail(rc);
    if ((rc = upload_prefix(ctx, p, pvec, &p.pre_vec)) != SQD_OK) return fail(rc);

    // kernel attributes (dynamic shared memory)
    const size_t abshm = sizeof(double) * 2 * AB_NA * AB_YW;
    const int MM = (M + 1) & ~1;
    const size_t jshm = sizeof(double) * 2 * (size_t)MM * (MM + 1);
    if (cudaFuncSetAttribute(kb_alpha_beta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)abshm) != cudaSuccess ||
        cudaFuncSetAttribute(kb_alpha_beta_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)abshm) != cudaSuccess ||
        cudaFuncSetAttribute(kb_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)jshm) != cudaSuccess)
        return fail(sqd_fail(ctx, SQD_ECUDA, "cannot set shared memory limits"));

    // --- autotune the paired-singles tile per size bucket ------------------
    // The subspaces are split into up to 4 buckets of equal count by
    // determinant count.  For each bucket, every (kernel variant, group
    // scale) pair is timed on the paired-singles stage of the first sigma of
    // up to 4 of its largest subspaces; the fastest is kept for the bucket.
    std::vector<ab_choice> ch;
    if ((rc = build_choices(ctx, p, tabs, ch)) != SQD_OK) return fail(rc);
    std::vector<int> order(nprob);
    for (int b = 0; b < nprob; b++) order[b] = b;
    std::sort(order.begin(), order.end(),
              [&](int x, int y) { return p.hdesc[x].N < p.hdesc[y].N; });
    const int nbk = std::min(4, nprob);
    std::vector<int> var(nprob, 0), sck(nprob, 1);
    ctx->batched_buckets.clear();
    // the descriptors reach the device here for the first time: kb_guess and
    // every later kernel read them
    if ((rc = apply_choices(ctx, p, tabs, ch, var, sck, nullptr)) != SQD_OK) return fail(rc);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    kb_guess<<<nprob, 256, 0, ctx->stream>>>(p.D, p.S);
    SQD_LAUNCHED(ctx);
    int fk = -1;  // a fixed tile instead of tuning (sqd_batched_set_tile)
    for (int k = 0; k < AB_NSCALE; k++)
        if (ctx->batched_force_ept && kAbScales[k] == ctx->batched_force_scale) fk = k;
    for (int q = 0; q < nbk; q++) {
        const int lo = q * nprob / nbk, hi = (q + 1) * nprob / nbk;
        if (fk >= 0) {
            const int fv = ctx->batched_force_ept == AB_EPT_WIDE ? 0 : 1;
            for (int r = lo; r < hi; r++) {
                var[order[r]] = fv;
                sck[order[r]] = fk;
            }
            sqd_ctx::bucket_choice bc;
            bc.max_det = p.hdesc[order[hi - 1]].N;
            bc.scale = kAbScales[fk];
            bc.entries_per_thread = ctx->batched_force_ept;
            ctx->batched_buckets.push_back(bc);
            continue;
        }
        std::vector<char> on(nprob, 0);
        for (int r = std::max(lo, hi - 4); r < hi; r++) on[order[r]] = 1;
        double best_ms = INFINITY;
        int bv = 0, bs = 1;
        for (int v = 0; v < 2; v++) {
            for (int k = 0; k < AB_NSCALE; k++) {
                for (int r = lo; r < hi; r++) {
                    var[order[r]] = v;
                    sck[order[r]] = k;
                }
                if ((rc = apply_choices(ctx, p, tabs, ch, var, sck, &on)) != SQD_OK)
                    return fail(rc);
                float best_rep = INFINITY;
                for (int rep = 0; rep < 2; rep++) {
                    kb_zero_counters<<<1, 32, 0, ctx->stream>>>(p.counters, 5);
                    SQD_LAUNCHED(ctx);
                    cudaEventRecord(e0, ctx->stream);
                    if ((rc = launch_ab_stage(ctx, p)) != SQD_OK) return fail(rc);
                    cudaEventRecord(e1, ctx->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess)
                        return fail(sqd_fail(ctx, SQD_ECUDA, "sigma stage failed: %s",
                                             cudaGetErrorString(cudaGetLastError())));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    best_rep = std::min(best_rep, ms);
                }
                if (best_rep < best_ms) {
                    best_ms = best_rep;
                    bv = v;
                    bs = k;
                }
            }
        }
        for (int r = lo; r < hi; r++) {
            var[order[r]] = bv;
            sck[order[r]] = bs;
        }
        sqd_ctx::bucket_choice bc;
        bc.max_det = p.hdesc[order[hi - 1]].N;
        bc.scale = kAbScales[bs];
        bc.entries_per_thread = bv == 0 ? AB_EPT_WIDE : AB_EPT;
        ctx->batched_buckets.push_back(bc);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->batched_group_scale = kAbScales[sck[order[nprob - 1]]];
    if ((rc = apply_choices(ctx, p, tabs, ch, var, sck, nullptr)) != SQD_OK) return fail(rc);
    // the tuning sigma wrote W[0]: the guess and its sigma start afresh below

    // --- initial guess, its sigma and G[0][0] ------------------------------
    prof_begin(ctx, PROF_BATCHED);
    kb_guess<<<nprob, 256, 0, ctx->stream>>>(p.D, p.S);
    SQD_LAUNCHED(ctx);
    if ((rc = launch_sigma_stages(ctx, p)) != SQD_OK) return fail(rc);
    if ((rc = launch_gram(ctx, p, 2)) != SQD_OK) return fail(rc);

    bparams P;
    P.nprob = nprob;
    P.M = M;
    P.tol_r = o->tol_residual;
    P.tol_e = o->tol_energy;
    P.floor_ = o->precond_floor;
    P.max_iter = o->max_iter;

    // --- the iteration loop as one graph -------------------------------------
    // The iteration is captured once as the body of a conditional WHILE node
    // whose last kernel decides on the device whether to run it again, so
    // the whole solve is one graph launch with no host round trip.  Where
    // conditional nodes are unavailable, the captured iteration is replayed
    // from the host instead, reading the active count after each replay.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(sqd_fail(ctx, SQD_ECUDA, "cannot create capture stream"));
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        return fail(sqd_fail(ctx, SQD_ECUDA, "setup failed: %s",
                             cudaGetErrorString(cudaGetLastError())));
    const int limit = o->max_iter + 2;
    int *d_iters = nullptr;
    if ((rc = plan_alloc(ctx, p, (void **)&d_iters, sizeof(int))) != SQD_OK) return fail(rc);
    cudaStream_t user = ctx->stream;
    int64_t before = ctx->launches;
    bool device_loop = false;
    int irc = SQD_OK;
    {
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams cp = {};
        cudaGraphNode_t cnode;
        bool ok = cudaMemsetAsync(d_iters, 0, sizeof(int), user) == cudaSuccess &&
                  cudaStreamSynchronize(user) == cudaSuccess &&
                  cudaGraphCreate(&graph, 0) == cudaSuccess &&
                  cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) ==
                      cudaSuccess;
        if (ok) {
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            ok = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
        }
        if (ok) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            ctx->stream = cap;
            ok = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                irc = launch_iteration(ctx, p, P);
                kb_loop_control<<<1, 1, 0, cap>>>(p.d_active, d_iters, limit, h);
                ok = (cudaStreamEndCapture(cap, &body) == cudaSuccess) && irc == SQD_OK;
            }
            ctx->stream = user;
        }
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (ok) {
            device_loop = true;
        } else {
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            exec = nullptr;
            cudaGetLastError();
        }
    }
    const int64_t per_iter = ctx->launches - before;
    ctx->launches = before;
    if (!device_loop) {
        // fallback: one captured iteration replayed from the host
        ctx->stream = cap;
        bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        irc = ok ? launch_iteration(ctx, p, P) : SQD_ECUDA;
        ok = (cudaStreamEndCapture(cap, &graph) == cudaSuccess) && ok && irc == SQD_OK;
        ctx->launches = before;
        ctx->stream = user;
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (!ok) {
            if (graph) cudaGraphDestroy(graph);
            cudaStreamDestroy(cap);
            cudaGetLastError();
            return fail(sqd_fail(ctx, SQD_ECUDA, "graph capture of the batched iteration failed"));
        }
    }
    int iters = 0;
    if (device_loop) {
        if (cudaGraphLaunch(exec, ctx->stream) == cudaSuccess &&
            cudaMemcpyAsync(&iters, d_iters, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) ==
                cudaSuccess)
            cudaStreamSynchronize(ctx->stream);
        ctx->launches += per_iter * iters;
    } else {
        int active = nprob;
        while (active > 0 && iters < limit) {
            if (cudaGraphLaunch(exec, ctx->stream) != cudaSuccess) break;
            ctx->launches += per_iter;
            cudaMemcpyAsync(&active, p.d_active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
            if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) break;
            iters++;
        }
    }
    ctx->batched_device_loop = device_loop ? 1 : 0;
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    prof_end(ctx, 0.0, 0.0);
    if (p.stamps) {
        double acc[17];
        if (cudaMemcpyAsync(acc, p.stamps, sizeof(acc), cudaMemcpyDeviceToHost, ctx->stream) ==
                cudaSuccess &&
            cudaStreamSynchronize(ctx->stream) == cudaSuccess) {
            // the sigma class holds the whole stage, its paired singles included
            acc[0] += acc[3];
            const int cls[4] = {PROF_B_SIGMA, PROF_B_VECTOR, PROF_B_EIGH, PROF_B_SIGMA_AB};
            for (int q = 0; q < 4; q++) {
                ctx->cls_ms[cls[q]] += acc[q] * 1e-6;
                ctx->cls_flops[cls[q]] += acc[4 + q];
                ctx->cls_bytes[cls[q]] += acc[8 + q];
                ctx->cls_launches[cls[q]] += (int64_t)acc[12 + q];
            }
        }
    }
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess)
        return fail(sqd_fail(ctx, SQD_ECUDA, "batched Davidson failed: %s",
                             cudaGetErrorString(ce)));

    // --- outputs -----------------------------------------------------------
    kb_form_x<<<(unsigned)p.tot_vec, BV_THREADS, 0, ctx->stream>>>(p.D, p.S, p.pre_vec, nprob);
    SQD_LAUNCHED(ctx);
    std::vector<bstate> hs(nprob);
    if (cudaMemcpy(hs.data(), p.S, sizeof(bstate) * nprob, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(sqd_fail(ctx, SQD_ECUDA, "state copy failed"));
    double *work = nullptr;
    if ((rc = plan_alloc(ctx, p, (void **)&work, sizeof(double) * (3 * 4 * ctx->sm_count + 8))) !=
        SQD_OK)
        return fail(rc);
    int status = SQD_OK;
    for (int b = 0; b < nprob; b++) {
        const bdesc &d = p.hdesc[b];
        if (d_C && d_C[b]) {
            if (cudaMemcpyAsync(d_C[b], d.X, sizeof(double) * d.N, cudaMemcpyDeviceToDevice,
                                ctx->stream) != cudaSuccess)
                return fail(sqd_fail(ctx, SQD_ECUDA, "output copy failed"));
            if ((rc = launch_fix_phase(ctx, d_C[b], d.N, 1, d.N, work)) != SQD_OK) return fail(rc);
        }
        h_energies[b] = hs[b].theta;
        if (h_iters) h_iters[b] = hs[b].it;
        const int st = hs[b].status == 1 ? SQD_OK
                                         : (hs[b].status == 0 ? SQD_ENOTCONVERGED : hs[b].status);
        if (h_status) h_status[b] = st;
        if (st != SQD_OK && status == SQD_OK) status = st;
    }
    cudaStreamSynchronize(ctx->stream);
    plan_free(p);
    if (status != SQD_OK)
        return sqd_fail(ctx, status, "some subspaces did not converge (see h_status)");
    return SQD_OK;
}
