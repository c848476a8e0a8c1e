// Device bodies shared by the single-problem Davidson (k_davidson.cu) and
// the batched engine (k_batched.cu).
#pragma once

#include <cmath>

#include "sqd_internal.cuh"

#define RED_THREADS 256

__device__ __forceinline__ double block_sum(double v, double *sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) r += sh[i];
    }
    __syncthreads();
    return r;  // valid in thread 0
}

#define JAC_MAX SQD_MAX_SUBSPACE

// Block sums of CNT per-thread values at once: shuffles within each warp,
// one shared-memory exchange (sh holds (blockDim.x / 32) * CNT doubles), a
// single barrier.  Thread i < CNT returns the block sum of value i through
// *out_i and true; the others return false.  Summation order is fixed.
template <int CNT>
__device__ __forceinline__ bool block_sums(const double (&v)[CNT], double *sh, int *out_i,
                                           double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < CNT; i++) {
        double x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w * CNT + i] = x;
    }
    __syncthreads();
    if ((int)threadIdx.x >= CNT) return false;
    double s = 0.0;
    for (int q = 0; q < nw; q++) s += sh[q * CNT + threadIdx.x];
    *out_i = threadIdx.x;
    *out = s;
    return true;
}

// The preconditioner's 1 / (theta - H_II), |theta - H_II| clamped to floor_
// (sign kept, + for 0).  GB300's FP64 pipe runs 4 flop per clock per SM, so
// an IEEE division (a few tens of FP64 operations with its special cases)
// costs more than the whole projection of a correction on a small basis.
// Here: the hardware's approximate FP64 reciprocal (rcp.approx.ftz.f64, the
// special-function unit) refined by two Newton-Raphson steps for 1/d,
// x <- x + x (1 - d x), each of which squares the relative error; 4 DFMAs.
// The correction vector needs no correctly rounded quotient: it is
// orthonormalised against the basis afterwards, and the Davidson result
// does not depend on its last bits.
__device__ __forceinline__ double precond_recip(double d, double floor_) {
    if (fabs(d) < floor_) d = (d < 0.0) ? -floor_ : floor_;
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    double e = fma(-d, x, 1.0);
    x = fma(x, e, x);
    e = fma(-d, x, 1.0);
    return fma(x, e, x);
}

// Warm start (m_old > 0): the first m_old basis vectors are unchanged since
// the previous solve, whose eigenvectors E_old (m_old x m_old, column-major)
// and eigenvalues th_old are given.  The solver then works on
// Q^T G Q with Q = diag(E_old, I): its leading block is diag(th_old) (the
// previous solve converged), only the rows and columns of the appended
// vectors couple, and far fewer sweeps are needed; the eigenvectors are
// mapped back through Q at the end.
__device__ __forceinline__ void jacobi_block(const double *__restrict__ G, int ldg, int m,
                                             double *__restrict__ evals,
                                             double *__restrict__ evecs, int m_old = 0,
                                             const double *__restrict__ E_old = nullptr,
                                             const double *__restrict__ th_old = nullptr) {
    // A and Q live in dynamic shared memory, (M) x (M+1) doubles each
    extern __shared__ double jac_sh[];
    __shared__ double cs[JAC_MAX / 2], sn[JAC_MAX / 2];
    __shared__ int pp[JAC_MAX / 2], qq[JAC_MAX / 2];
    __shared__ int act[JAC_MAX / 2], wcnt[2];
    __shared__ double red[32];
    __shared__ int done;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int M = (m + 1) & ~1;  // even size; a padding row/col stays zero
    const int LD = M + 1;
    double *Ab = jac_sh, *Qb = jac_sh + (size_t)M * LD;
#define A(i, j) Ab[(i) * LD + (j)]
#define Q(i, j) Qb[(i) * LD + (j)]
    // only the upper triangle G[i + j*ldg], i <= j, is read
    for (int t = tid; t < M * M; t += nt) {
        int i = t / M, j = t % M;
        double v = 0.0;
        if (i < m && j < m) {
            if (i < m_old && j < m_old) {
                v = (i == j) ? th_old[i] : 0.0;
            } else if (i < m_old || j < m_old) {
                // coupling of old Ritz vector q to appended vector c
                const int q = min(i, j), c = max(i, j);
                double sacc = 0.0;
                for (int r = 0; r < m_old; r++)
                    sacc = fma(E_old[r + (int64_t)q * m_old], G[r + (int64_t)c * ldg], sacc);
                v = sacc;
            } else {
                v = (i <= j) ? G[i + (int64_t)j * ldg] : G[j + (int64_t)i * ldg];
            }
        }
        A(i, j) = v;
        Q(i, j) = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int npair = M / 2;
    for (int sweep = 0; sweep < 60; sweep++) {
        // convergence: off-diagonal Frobenius norm vs diagonal
        double off = 0.0, dia = 0.0;
        for (int t = tid; t < M * M; t += nt) {
            int i = t / M, j = t % M;
            double v = A(i, j);
            if (i != j) off += v * v; else dia += v * v;
        }
        double offs = block_sum(off, red);
        double dias = block_sum(dia, red);
        if (tid == 0) done = (offs <= 1e-30 * dias || offs == 0.0) ? 1 : 0;
        __syncthreads();
        if (done) break;
        for (int step = 0; step < M - 1; step++) {
            if (tid < npair) {
                // round-robin: player M-1 fixed, the others rotate
                int a, b;
                if (tid == 0) {
                    a = step;
                    b = M - 1;
                } else {
                    a = (step + tid) % (M - 1);
                    b = (step + M - 1 - tid) % (M - 1);
                }
                int p = min(a, b), q = max(a, b);
                double apq = A(p, q);
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    if (fabs(apq) <= 0x1p-60 * fmin(fabs(A(p, p)), fabs(A(q, q)))) {
                        // negligible against both diagonal entries: set to zero
                        // (no other pair of this step touches entry (p, q))
                        A(p, q) = 0.0;
                        A(q, p) = 0.0;
                    } else {
                        double tau = (A(q, q) - A(p, p)) / (2.0 * apq);
                        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                                : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                pp[tid] = p;
                qq[tid] = q;
                cs[tid] = c;
                sn[tid] = s;
            }
            // compact the pairs that rotate (s != 0): the updates below cost
            // FP64 issue per warp instruction, so identity rotations are dropped
            bool on = false;
            unsigned bal = 0u;
            if (tid < 64) {
                on = (tid < npair) && (sn[tid] != 0.0);
                bal = __ballot_sync(0xffffffffu, on);
                if ((tid & 31) == 0) wcnt[tid >> 5] = __popc(bal);
            }
            __syncthreads();
            if (on) act[__popc(bal & ((1u << (tid & 31)) - 1u)) + ((tid >> 5) ? wcnt[0] : 0)] = tid;
            const int nact = wcnt[0] + wcnt[1];
            __syncthreads();
            if (nact == 0) continue;  // uniform across the block
            // columns: A <- A J, Q <- Q J
            for (int t = tid; t < M * nact; t += nt) {
                int r = t / nact, k = act[t % nact];
                int p = pp[k], q = qq[k];
                double c = cs[k], s = sn[k];
                double ap = A(r, p), aq = A(r, q);
                A(r, p) = c * ap - s * aq;
                A(r, q) = s * ap + c * aq;
                double qp = Q(r, p), qv = Q(r, q);
                Q(r, p) = c * qp - s * qv;
                Q(r, q) = s * qp + c * qv;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int t = tid; t < M * nact; t += nt) {
                int col = t / nact, k = act[t % nact];
                int p = pp[k], q = qq[k];
                double c = cs[k], s = sn[k];
                double ap = A(p, col), aq = A(q, col);
                A(p, col) = c * ap - s * aq;
                A(q, col) = s * ap + c * aq;
            }
            __syncthreads();
        }
    }
    // sort ascending (selection of the order by one thread), write out
    __shared__ int order[JAC_MAX];
    if (tid == 0) {
        for (int i = 0; i < m; i++) order[i] = i;
        for (int i = 0; i < m; i++) {
            int best = i;
            for (int j = i + 1; j < m; j++) {
                double dj = A(order[j], order[j]), db = A(order[best], order[best]);
                if (dj < db || (dj == db && order[j] < order[best])) best = j;
            }
            int tmp = order[i];
            order[i] = order[best];
            order[best] = tmp;
        }
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
        int i = t % m, j = t / m;  // evecs[i + j*m] = (diag(E_old, I) Q)(i, order[j])
        double v;
        if (i < m_old) {
            v = 0.0;
            for (int q = 0; q < m_old; q++) v = fma(E_old[i + (int64_t)q * m_old], Q(q, order[j]), v);
        } else {
            v = Q(i, order[j]);
        }
        evecs[i + (int64_t)j * m] = v;
    }
    for (int j = tid; j < m; j += nt) evals[j] = A(order[j], order[j]);
}

__device__ __forceinline__ int gdk_block(const double *__restrict__ Y, int m, int m2,
                                         const double *__restrict__ P, int mp, int k, int ldp,
                                         double *__restrict__ Z, int ldz) {
    __shared__ double p[JAC_MAX];
    __shared__ double red[32];
    __shared__ double coef;
    const int i = threadIdx.x;
    for (int j = 0; j < m2; j++)
        if (i < m) Z[i + (int64_t)j * ldz] = Y[i + (int64_t)j * m];
    __syncthreads();
    int r = m2;
    for (int j = 0; j < k; j++) {
        if (i < m) p[i] = (i < mp && P) ? P[i + (int64_t)j * ldp] : 0.0;
        __syncthreads();
        for (int pass = 0; pass < 2; pass++) {
            for (int c = 0; c < r; c++) {
                double v = (i < m) ? Z[i + (int64_t)c * ldz] * p[i] : 0.0;
                double d = block_sum(v, red);
                if (i == 0) coef = d;
                __syncthreads();
                if (i < m) p[i] -= coef * Z[i + (int64_t)c * ldz];
                __syncthreads();
            }
        }
        double nv = (i < m) ? p[i] * p[i] : 0.0;
        double n2 = block_sum(nv, red);
        if (i == 0) coef = n2;
        __syncthreads();
        double nrm = sqrt(coef);
        if (nrm > 1e-8) {  // uniform across the block
            if (i < m) Z[i + (int64_t)r * ldz] = p[i] / nrm;
            r++;
        }
        __syncthreads();
    }
    return r;
}

