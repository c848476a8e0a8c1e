// Device kernels of the Davidson driver: block dot products of the new block
// with the basis (shared-memory tiles, every vector element read from HBM
// once), basis combinations and block Gram-Schmidt updates (one kernel per
// output-group width), Ritz vectors with residuals and their norms in one
// pass, the diagonal (Davidson) and Olsen corrections, the projected matrix
// Z^T G Z at restart, guess selection, sign fixing and a one-block parallel
// (round-robin) Jacobi eigensolver for the small Rayleigh-Ritz matrix,
// optionally warm-started from the previous eigenvectors.  All arithmetic
// is FP64; reductions run in a fixed order so results do not depend on
// scheduling.
#include <cmath>

#include "davidson_body.cuh"


int multidot_blocks(int64_t n) {
    int64_t b = (n + 4095) / 4096;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

// partial[i * nblk + blk] = sum over this block's slice of A_i[n] * x[n]
__global__ void __launch_bounds__(RED_THREADS)
    k_multidot_partial(const double *__restrict__ A, int64_t lda, int m,
                       const double *__restrict__ x, int64_t n, double *__restrict__ partial) {
    __shared__ double sh[32];
    int64_t per = (n + gridDim.x - 1) / gridDim.x;
    int64_t lo = per * blockIdx.x, hi = min(n, lo + per);
    for (int i = 0; i < m; i++) {
        const double *a = A + (int64_t)i * lda;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int64_t j = lo + threadIdx.x;
        for (; j + 3 * RED_THREADS < hi; j += 4 * RED_THREADS) {
            const double a0 = a[j], a1 = a[j + RED_THREADS], a2 = a[j + 2 * RED_THREADS],
                         a3 = a[j + 3 * RED_THREADS];
            const double x0 = x[j], x1 = x[j + RED_THREADS], x2 = x[j + 2 * RED_THREADS],
                         x3 = x[j + 3 * RED_THREADS];
            s0 = fma(a0, x0, s0);
            s1 = fma(a1, x1, s1);
            s2 = fma(a2, x2, s2);
            s3 = fma(a3, x3, s3);
        }
        for (; j < hi; j += RED_THREADS) s0 = fma(a[j], x[j], s0);
        double t = block_sum((s0 + s1) + (s2 + s3), sh);
        if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void k_multidot_final(const double *__restrict__ partial, int nblk, int m,
                                 double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partial[(int64_t)i * nblk + b];
    out[i] = s;
}

int launch_multidot(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *x,
                    int64_t n, double *partial, int nblk, double *out) {
    if (m == 0) return SQD_OK;
    k_multidot_partial<<<nblk, RED_THREADS, 0, ctx->stream>>>(A, lda, m, x, n, partial);
    SQD_LAUNCHED(ctx);
    k_multidot_final<<<(m + 63) / 64, 64, 0, ctx->stream>>>(partial, nblk, m, out);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// out_j[n] = sum_i A_i[n] Y[i + j*ldy], j < k  (sub: out_j[n] -= that sum).
// Each thread keeps 8 loads of A in flight (the basis does not fit in L2, so
// the loop is bound by HBM latency otherwise) and up to 8 outputs in
// registers; A is read once per group of 8 outputs.  The group width is a
// template parameter: predicated-off FP64 instructions would still take
// FP64 issue slots.
#define CB_U 8
template <int JN>
__device__ __forceinline__ void combine_group(const double *__restrict__ A, int64_t lda, int m,
                                              const double *__restrict__ Yj, int ldy,
                                              double *__restrict__ out, int64_t ldo, int64_t p,
                                              int sub) {
    double acc[JN];
#pragma unroll
    for (int q = 0; q < JN; q++) acc[q] = 0.0;
    int i = 0;
    for (; i + CB_U <= m; i += CB_U) {
        double a[CB_U];
#pragma unroll
        for (int u = 0; u < CB_U; u++) a[u] = A[(int64_t)(i + u) * lda + p];
#pragma unroll
        for (int u = 0; u < CB_U; u++) {
#pragma unroll
            for (int q = 0; q < JN; q++)
                acc[q] = fma(a[u], __ldg(Yj + i + u + (int64_t)q * ldy), acc[q]);
        }
    }
    for (; i < m; i++) {
        const double a = A[(int64_t)i * lda + p];
#pragma unroll
        for (int q = 0; q < JN; q++) acc[q] = fma(a, __ldg(Yj + i + (int64_t)q * ldy), acc[q]);
    }
#pragma unroll
    for (int q = 0; q < JN; q++) {
        double *o = out + (int64_t)q * ldo + p;
        *o = sub ? *o - acc[q] : acc[q];
    }
}

// one kernel per group width, so that a narrow group (one root, one new
// vector) is not held to the register count of the widest and runs at the
// occupancy its HBM streaming needs
template <int JN>
__global__ void __launch_bounds__(256) k_combine(const double *__restrict__ A, int64_t lda, int m,
                                                 const double *__restrict__ Yj, int ldy,
                                                 double *__restrict__ oj, int64_t ldo, int64_t n,
                                                 int sub, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;  // a pass the device decided to skip
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        combine_group<JN>(A, lda, m, Yj, ldy, oj, ldo, p, sub);
}

// out_j (-)= sum_i A_i Y_ij for j < k, one launch per group of 8 outputs;
// with gate, only if *gate != 0 (read on the device)
static int combine_launch(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *Y,
                          int ldy, int k, double *out, int64_t ldo, int64_t n, int sub,
                          const int *gate = nullptr) {
    if (k == 0 || n == 0) return SQD_OK;
    unsigned g = grid_1d(n, 256);
    if (g > 8u * (unsigned)ctx->sm_count * 8u) g = 8u * (unsigned)ctx->sm_count * 8u;
    for (int j0 = 0; j0 < k; j0 += 8) {
        const double *Yj = Y + (int64_t)j0 * ldy;
        double *oj = out + (int64_t)j0 * ldo;
        cudaStream_t st = ctx->stream;
        switch (min(8, k - j0)) {
            case 1: k_combine<1><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 2: k_combine<2><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 3: k_combine<3><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 4: k_combine<4><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 5: k_combine<5><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 6: k_combine<6><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            case 7: k_combine<7><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
            default: k_combine<8><<<g, 256, 0, st>>>(A, lda, m, Yj, ldy, oj, ldo, n, sub, gate); break;
        }
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

int launch_combine(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *Y, int ldy,
                   int k, double *out, int64_t ldo, int64_t n) {
    return combine_launch(ctx, A, lda, m, Y, ldy, k, out, ldo, n, 0);
}

// x[n] -= sum_i A_i[n] c[i]: one Gram-Schmidt update
int launch_gemv_sub(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *c,
                    double *x, int64_t n) {
    if (m == 0) return SQD_OK;
    return combine_launch(ctx, A, lda, m, c, m, 1, x, n, n, 1);
}

// out_j[n] -= sum_i A_i[n] Y[i + j*ldy], j < k: the update of block Gram-Schmidt
int launch_combine_sub(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *Y,
                       int ldy, int k, double *out, int64_t ldo, int64_t n, const int *gate) {
    if (m == 0) return SQD_OK;
    return combine_launch(ctx, A, lda, m, Y, ldy, k, out, ldo, n, 1, gate);
}

// ------------------------------------------------- block dot products ---
// out[i + j*ldo] = sum_n A_i[n] X_j[n] for i < m, j < b: a tall-skinny
// product split over n.  Each block walks its n-range in tiles of kc columns
// staged in shared memory (every element of A and X is read from HBM once),
// kc chosen so that the m + b rows of a tile fill about BD_TILE doubles.  The
// work of a tile is m*b outputs of kc multiply-adds; it is cut into m*b*g
// units (an output and every g-th column of the tile), g chosen on the host
// so that the units spread evenly over the 256 threads: with m*b = 320, for
// instance, one output per thread would leave 64 threads with a second one
// and the rest idle for half the tile, where g = 4 gives every thread 5
// units of kc/4 columns.  The g partial sums of an output are added in a
// fixed order at the end, and the per-block partials are summed in a fixed
// order too, so results do not depend on timing.
#define BD_TILE 4608
#define BD_MAXB 32
#define BD_OUT 16

int block_dot_blocks(const sqd_ctx *ctx, int64_t n) {
    int64_t b = (n + 4095) / 4096;
    const int64_t cap = 4LL * ctx->sm_count;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

static int block_dot_kc(int m, int b) {
    int kc = (BD_TILE / (m + b) - 1) / 32 * 32;
    return kc < 32 ? 32 : (kc > 512 ? 512 : kc);
}

// column split g (a power of two dividing kc, at most BD_OUT units per
// thread) with the shortest per-thread path ceil(mb g / 256) * kc / g; ties
// go to the smaller g
static int block_dot_split(int mb, int kc) {
    int best_g = 1;
    long best = -1;
    for (int g = 1; g <= RED_THREADS && g <= kc; g *= 2) {
        if ((long)mb * g > (long)RED_THREADS * BD_OUT) break;
        if (kc % g) continue;
        const long upt = ((long)mb * g + RED_THREADS - 1) / RED_THREADS;
        const long cost = upt * (kc / g);
        if (best < 0 || cost < best) {
            best = cost;
            best_g = g;
        }
    }
    return best_g;
}

__global__ void __launch_bounds__(RED_THREADS)
    k_block_dot_partial(const double *__restrict__ A, int64_t lda, int m,
                        const double *__restrict__ X, int64_t ldx, int b, int64_t n, int kc,
                        int g, double *__restrict__ partial, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;  // a pass the device decided to skip
    extern __shared__ double bd_sh[];
    const int ld = kc + 1;
    double *As = bd_sh, *Xs = bd_sh + (size_t)m * ld;
    const int mb = m * b;
    const int U = mb * g;  // units: (output, column group)
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x, hi = min(n, lo + per);
    double acc[BD_OUT];
#pragma unroll
    for (int q = 0; q < BD_OUT; q++) acc[q] = 0.0;
    for (int64_t c0 = lo; c0 < hi; c0 += kc) {
        const int len = (int)min((int64_t)kc, hi - c0);
        const int rows = m + b;
#pragma unroll 8
        for (int t = threadIdx.x; t < rows * kc; t += RED_THREADS) {
            const int r = t / kc, kk = t - r * kc;
            const double *src = (r < m) ? A + (int64_t)r * lda : X + (int64_t)(r - m) * ldx;
            bd_sh[(size_t)r * ld + kk] = (kk < len) ? src[c0 + kk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < BD_OUT; q++) {
            const int u = threadIdx.x + q * RED_THREADS;
            if (u < U) {
                const int o = u / g, tg = u - o * g;
                const double *ar = As + (size_t)(o % m) * ld, *xr = Xs + (size_t)(o / m) * ld;
                double s = acc[q];
#pragma unroll 4
                for (int kk = tg; kk < kc; kk += g) s = fma(ar[kk], xr[kk], s);
                acc[q] = s;
            }
        }
        __syncthreads();
    }
    // unit sums to shared memory (U <= 4096 doubles: the launch sizes the
    // dynamic shared memory for it), then each output adds its g units in order
#pragma unroll
    for (int q = 0; q < BD_OUT; q++) {
        const int u = threadIdx.x + q * RED_THREADS;
        if (u < U) bd_sh[u] = acc[q];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < mb; o += RED_THREADS) {
        double s = 0.0;
        for (int q = 0; q < g; q++) s += bd_sh[o * g + q];
        partial[(int64_t)blockIdx.x * mb + o] = s;
    }
}

__global__ void k_block_dot_final(const double *__restrict__ partial, int nblk, int m, int b,
                                  double *__restrict__ out, int ldo, const int *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int mb = m * b;
    if (o >= mb) return;
    double s = 0.0;
    for (int blk = 0; blk < nblk; blk++) s += partial[(int64_t)blk * mb + o];
    out[(o % m) + (int64_t)(o / m) * ldo] = s;
}

int launch_block_dot(sqd_ctx *ctx, const double *A, int64_t lda, int m, const double *X,
                     int64_t ldx, int b, int64_t n, double *partial, int nblk, double *out,
                     int ldo, const int *gate) {
    if (m == 0 || b == 0) return SQD_OK;
    if (m > JAC_MAX || b > BD_MAXB || m * b > RED_THREADS * BD_OUT)
        return sqd_fail(ctx, SQD_EINVAL, "block dot of %d x %d vectors out of range", m, b);
    const int kc = block_dot_kc(m, b);
    const int g = block_dot_split(m * b, kc);
    size_t shm = sizeof(double) * (size_t)(m + b) * (kc + 1);
    const size_t shu = sizeof(double) * (size_t)m * b * g;  // the unit sums
    if (shm < shu) shm = shu;
    // tiles fill about BD_TILE + (m + b) doubles, unit sums at most
    // RED_THREADS * BD_OUT doubles: 37 KB and 32 KB, within the default 48 KB
    k_block_dot_partial<<<nblk, RED_THREADS, shm, ctx->stream>>>(A, lda, m, X, ldx, b, n, kc, g,
                                                                  partial, gate);
    SQD_LAUNCHED(ctx);
    k_block_dot_final<<<(m * b + 127) / 128, 128, 0, ctx->stream>>>(partial, nblk, m, b, out, ldo,
                                                                    gate);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// Daniel-Gragg-Kaufman-Stewart test on the device: *flag = 1 if some vector
// of the block lost more than `loss` of its squared norm in the first
// Gram-Schmidt pass (|P_j|^2 > loss |t_j|^2, V orthonormal), else 0; the
// second pass is gated on it.  One block.
__global__ void k_dgks_flag(const double *__restrict__ P, int ldp, int m, int b,
                            const double *__restrict__ tn2, double loss, int *__restrict__ flag) {
    __shared__ int again;
    if (threadIdx.x == 0) again = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < b; j += blockDim.x) {
        double p2 = 0.0;
        for (int i = 0; i < m; i++) p2 = fma(P[i + (int64_t)j * ldp], P[i + (int64_t)j * ldp], p2);
        if (!(p2 <= loss * tn2[j])) atomicOr(&again, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *flag = again;
}

int launch_dgks_flag(sqd_ctx *ctx, const double *P, int ldp, int m, int b, const double *tn2,
                     double loss, int *flag) {
    k_dgks_flag<<<1, 32, 0, ctx->stream>>>(P, ldp, m, b, tn2, loss, flag);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------------- Ritz vectors, residuals --
// For the selected Ritz pairs j = sel[q], q < ks (theta_j, y_j = column j of
// Y, ld m): X_j = V y_j, R_j = W y_j - theta_j X_j, and per-block partial
// sums of |R_j|^2 (partial[blk*ks + q]).  V and W are read once per group of
// 8 selected roots (group width a template parameter, as in k_combine).
template <int JN>
__device__ __forceinline__ void ritz_group(const double *__restrict__ V,
                                           const double *__restrict__ W, int64_t ld, int m,
                                           const double *__restrict__ Y,
                                           const double *__restrict__ theta,
                                           const int *__restrict__ selq, double *__restrict__ X,
                                           double *__restrict__ R, int64_t n, double *ss) {
    int jj[JN];
    double th[JN];
#pragma unroll
    for (int q = 0; q < JN; q++) {
        jj[q] = __ldg(selq + q);
        th[q] = __ldg(theta + jj[q]);
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double xa[JN], wa[JN];
#pragma unroll
        for (int q = 0; q < JN; q++) xa[q] = wa[q] = 0.0;
        int i = 0;
        for (; i + 4 <= m; i += 4) {
            double v[4], w[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                v[u] = V[(int64_t)(i + u) * ld + p];
                w[u] = W[(int64_t)(i + u) * ld + p];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
#pragma unroll
                for (int q = 0; q < JN; q++) {
                    const double y = __ldg(Y + i + u + (int64_t)jj[q] * m);
                    xa[q] = fma(v[u], y, xa[q]);
                    wa[q] = fma(w[u], y, wa[q]);
                }
            }
        }
        for (; i < m; i++) {
            const double v = V[(int64_t)i * ld + p], w = W[(int64_t)i * ld + p];
#pragma unroll
            for (int q = 0; q < JN; q++) {
                const double y = __ldg(Y + i + (int64_t)jj[q] * m);
                xa[q] = fma(v, y, xa[q]);
                wa[q] = fma(w, y, wa[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < JN; q++) {
            const double r = fma(-th[q], xa[q], wa[q]);
            X[(int64_t)jj[q] * ld + p] = xa[q];
            R[(int64_t)jj[q] * ld + p] = r;
            ss[q] = fma(r, r, ss[q]);
        }
    }
}

template <int JN>
__global__ void __launch_bounds__(RED_THREADS)
    k_ritz_block(const double *__restrict__ V, const double *__restrict__ W, int64_t ld, int m,
                 const double *__restrict__ Y, const double *__restrict__ theta,
                 const int *__restrict__ selq, int ks, int j0, double *__restrict__ X,
                 double *__restrict__ R, int64_t n, double *__restrict__ partial) {
    __shared__ double red[32];
    double ss[JN];
#pragma unroll
    for (int q = 0; q < JN; q++) ss[q] = 0.0;
    ritz_group<JN>(V, W, ld, m, Y, theta, selq, X, R, n, ss);
#pragma unroll
    for (int q = 0; q < JN; q++) {
        const double t = block_sum(ss[q], red);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * ks + j0 + q] = t;
    }
}

__global__ void k_ritz_final(const double *__restrict__ partial, int nblk, int k,
                             double *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partial[(int64_t)b * k + j];
    out[j] = s;
}

// sel: device array of ks root indices; rnorm2[q] = |R_sel[q]|^2
int launch_ritz_block(sqd_ctx *ctx, const double *V, const double *W, int64_t ld, int m,
                      const double *Y, const double *theta, const int *sel, int ks, double *X,
                      double *R, int64_t n, double *partial, int nblk, double *rnorm2) {
    if (ks == 0 || n == 0) return SQD_OK;
    for (int j0 = 0; j0 < ks; j0 += 8) {  // one kernel per group of 8 roots
        const int *sq = sel + j0;
        cudaStream_t st = ctx->stream;
        switch (min(8, ks - j0)) {
#define RITZ_CASE(J)                                                                          \
    case J:                                                                                   \
        k_ritz_block<J><<<nblk, RED_THREADS, 0, st>>>(V, W, ld, m, Y, theta, sq, ks, j0, X, R, \
                                                       n, partial);                           \
        break;
            RITZ_CASE(1) RITZ_CASE(2) RITZ_CASE(3) RITZ_CASE(4) RITZ_CASE(5) RITZ_CASE(6)
            RITZ_CASE(7)
            default:
                k_ritz_block<8><<<nblk, RED_THREADS, 0, st>>>(V, W, ld, m, Y, theta, sq, ks, j0,
                                                              X, R, n, partial);
                break;
#undef RITZ_CASE
        }
        SQD_LAUNCHED(ctx);
    }
    k_ritz_final<<<(ks + 63) / 64, 64, 0, ctx->stream>>>(partial, nblk, ks, rnorm2);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------- projected matrix at restart --
// After V' = V Z, W' = W Z the projected matrix is G' = Z^T G Z (G symmetric,
// upper triangle stored with leading dimension ldg).  GZ (m x r, ld m) is a
// scratch buffer; the upper triangle of G'[0..r) overwrites G.
__global__ void k_gz(const double *__restrict__ G, int ldg, int m, const double *__restrict__ Z,
                     int ldz, int r, double *__restrict__ GZ) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * r) return;
    const int i = t % m, j = t / m;
    double s = 0.0;
    for (int q = 0; q < m; q++) {
        const double g = (i <= q) ? G[i + (int64_t)q * ldg] : G[q + (int64_t)i * ldg];
        s = fma(g, Z[q + (int64_t)j * ldz], s);
    }
    GZ[i + (int64_t)j * m] = s;
}

__global__ void k_ztgz(double *__restrict__ G, int ldg, int m, const double *__restrict__ Z,
                       int ldz, int r, const double *__restrict__ GZ) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= r * r) return;
    const int i = t % r, j = t / r;
    if (i > j) return;
    double s = 0.0;
    for (int q = 0; q < m; q++) s = fma(Z[q + (int64_t)i * ldz], GZ[q + (int64_t)j * m], s);
    G[i + (int64_t)j * ldg] = s;
}

int launch_project_g(sqd_ctx *ctx, double *G, int ldg, int m, const double *Z, int ldz, int r,
                     double *GZ) {
    if (m == 0 || r == 0) return SQD_OK;
    k_gz<<<(m * r + 127) / 128, 128, 0, ctx->stream>>>(G, ldg, m, Z, ldz, r, GZ);
    SQD_LAUNCHED(ctx);
    k_ztgz<<<(r * r + 127) / 128, 128, 0, ctx->stream>>>(G, ldg, m, Z, ldz, r, GZ);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// T = R / (theta - diag), |denominator| clamped to floor_ (sign kept, + for 0;
// the reciprocal by precond_recip);
// with partial != NULL also per-block partial sums of T^2
__global__ void __launch_bounds__(RED_THREADS)
    k_precondition(const double *__restrict__ R, const double *__restrict__ diag, double theta,
                   double floor_, int64_t n, double *__restrict__ T, double *__restrict__ partial) {
    __shared__ double red[32];
    double ss = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double t = R[p] * precond_recip(theta - diag[p], floor_);
        T[p] = t;
        ss = fma(t, t, ss);
    }
    if (partial) {
        const double tot = block_sum(ss, red);
        if (threadIdx.x == 0) partial[blockIdx.x] = tot;
    }
}

static unsigned precondition_grid(const sqd_ctx *ctx, int64_t n) {
    unsigned g = grid_1d(n, RED_THREADS);
    if (g > 4u * (unsigned)ctx->sm_count) g = 4u * (unsigned)ctx->sm_count;
    return g;
}

// T = R / (theta - diag) and *norm2 (device) = |T|^2; partial holds 4 * SMs doubles
int launch_precondition_norm(sqd_ctx *ctx, const double *R, const double *diag, double theta,
                             double floor_, int64_t n, double *T, double *partial,
                             double *norm2) {
    if (n == 0) return SQD_OK;
    const unsigned g = precondition_grid(ctx, n);
    k_precondition<<<g, RED_THREADS, 0, ctx->stream>>>(R, diag, theta, floor_, n, T, partial);
    SQD_LAUNCHED(ctx);
    k_multidot_final<<<1, 64, 0, ctx->stream>>>(partial, (int)g, 1, norm2);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// Olsen's correction: with d = theta - diag (clamped as above),
// a = sum x r / d and b = sum x x / d (per-block partials, 2 per block), then
// T = (R - (a/b) X) / d, so that X^T T = 0, and partials of |T|^2.
__global__ void __launch_bounds__(RED_THREADS)
    k_olsen_dots(const double *__restrict__ R, const double *__restrict__ X,
                 const double *__restrict__ diag, double theta, double floor_, int64_t n,
                 double *__restrict__ partial) {
    __shared__ double red[32];
    double sa = 0.0, sb = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double d = theta - diag[p];
        if (fabs(d) < floor_) d = (d < 0.0) ? -floor_ : floor_;
        const double x = X[p];
        sa += x * R[p] / d;
        sb += x * x / d;
    }
    const double ta = block_sum(sa, red);
    const double tb = block_sum(sb, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = ta;
        partial[gridDim.x + blockIdx.x] = tb;
    }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_olsen_apply(const double *__restrict__ R, const double *__restrict__ X,
                  const double *__restrict__ diag, double theta, double floor_, int64_t n,
                  const double *__restrict__ ab, double *__restrict__ T,
                  double *__restrict__ partial) {
    __shared__ double red[32];
    const double eps = (ab[1] != 0.0) ? ab[0] / ab[1] : 0.0;
    double ss = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double d = theta - diag[p];
        if (fabs(d) < floor_) d = (d < 0.0) ? -floor_ : floor_;
        const double t = (R[p] - eps * X[p]) / d;
        T[p] = t;
        ss = fma(t, t, ss);
    }
    const double tot = block_sum(ss, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// partial: 4 * SMs + 2 doubles; norm2 (device) = |T|^2
int launch_precondition_olsen(sqd_ctx *ctx, const double *R, const double *X, const double *diag,
                              double theta, double floor_, int64_t n, double *T, double *partial,
                              double *norm2) {
    if (n == 0) return SQD_OK;
    const unsigned g = precondition_grid(ctx, n);
    double *ab = partial + 2 * g;  // 2 doubles after the partials
    k_olsen_dots<<<g, RED_THREADS, 0, ctx->stream>>>(R, X, diag, theta, floor_, n, partial);
    SQD_LAUNCHED(ctx);
    k_multidot_final<<<1, 64, 0, ctx->stream>>>(partial, (int)g, 2, ab);
    SQD_LAUNCHED(ctx);
    k_olsen_apply<<<g, RED_THREADS, 0, ctx->stream>>>(R, X, diag, theta, floor_, n, ab, T, partial);
    SQD_LAUNCHED(ctx);
    k_multidot_final<<<1, 64, 0, ctx->stream>>>(partial, (int)g, 1, norm2);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// x *= s  (invert_sqrt: x *= 1/sqrt(s))
__global__ void k_scale(double *__restrict__ x, int64_t n, const double *__restrict__ s,
                        int invert_sqrt) {
    double f = invert_sqrt ? 1.0 / sqrt(*s) : *s;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        x[p] *= f;
}

int launch_scale(sqd_ctx *ctx, double *x, int64_t n, const double *s_dev, int invert_sqrt) {
    if (n == 0) return SQD_OK;
    unsigned g = grid_1d(n, 256);
    if (g > 8u * (unsigned)ctx->sm_count * 8u) g = 8u * (unsigned)ctx->sm_count * 8u;
    k_scale<<<g, 256, 0, ctx->stream>>>(x, n, s_dev, invert_sqrt);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------------------ Jacobi (1 block) --
// Symmetric eigenproblem of the m x m Rayleigh-Ritz matrix, m <= 128.
// Parallel cyclic Jacobi with the round-robin pair schedule: each step
// rotates m/2 disjoint (p,q) pairs chosen to zero A_pq (Golub & Van Loan,
// symmetric Schur decomposition 2x2), then applies all column rotations and
// all row rotations.  Sweeps until the off-diagonal norm is negligible.
// Output: evals ascending, evecs column-major (evecs[i + j*m] = Y_ij).

__global__ void __launch_bounds__(1024) k_jacobi(const double *__restrict__ G, int ldg, int m,
                                                 double *__restrict__ evals,
                                                 double *__restrict__ evecs, int m_old,
                                                 const double *__restrict__ E_old,
                                                 const double *__restrict__ th_old) {
    jacobi_block(G, ldg, m, evals, evecs, m_old, E_old, th_old);
}

int launch_jacobi_eigh(sqd_ctx *ctx, const double *G, int ldg, int m, double *evals,
                       double *evecs, int m_old, const double *E_old, const double *th_old) {
    if (m < 1 || m > JAC_MAX) return sqd_fail(ctx, SQD_EINVAL, "subspace size %d out of range", m);
    if (m_old < 0 || m_old > m || (m_old > 0 && (!E_old || !th_old)))
        return sqd_fail(ctx, SQD_EINVAL, "bad warm start for the projected eigenproblem");
    int M = (m + 1) & ~1;
    size_t shm = sizeof(double) * 2 * (size_t)M * (M + 1);
    SQD_CUDA(ctx, cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(double) * 2 * JAC_MAX * (JAC_MAX + 1))));
    k_jacobi<<<1, 1024, shm, ctx->stream>>>(G, ldg, m, evals, evecs, m_old, E_old, th_old);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------------------- guess selection --
// idx[t] = index of the t-th smallest diag entry in (value, index) order.
struct vi {
    double v;
    int64_t i;
};

__device__ __forceinline__ bool vi_less(double v1, int64_t i1, double v2, int64_t i2) {
    return v1 < v2 || (v1 == v2 && i1 < i2);
}

__global__ void __launch_bounds__(RED_THREADS)
    k_argmin_partial(const double *__restrict__ d, int64_t n, double lv, int64_t li,
                     int64_t sym_n, double *__restrict__ pv, int64_t *__restrict__ pi) {
    __shared__ double sv[RED_THREADS];
    __shared__ int64_t si[RED_THREADS];
    double bv = INFINITY;
    int64_t bi = -1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        // sym_n > 0: only I <= J of an sym_n x sym_n matrix; < 0: only I < J
        if (sym_n > 0 && p / sym_n > p % sym_n) continue;
        if (sym_n < 0 && p / (-sym_n) >= p % (-sym_n)) continue;
        double v = d[p];
        bool after = (li < 0) || vi_less(lv, li, v, p);
        if (after && (bi < 0 || vi_less(v, p, bv, bi))) {
            bv = v;
            bi = p;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double v2 = sv[threadIdx.x + o];
            int64_t i2 = si[threadIdx.x + o];
            if (i2 >= 0 && (si[threadIdx.x] < 0 || vi_less(v2, i2, sv[threadIdx.x], si[threadIdx.x]))) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = sv[0];
        pi[blockIdx.x] = si[0];
    }
}

__global__ void k_argmin_final(const double *pv, const int64_t *pi, int nblk, int t,
                               int64_t *idx, double *lastv) {
    double bv = INFINITY;
    int64_t bi = -1;
    for (int b = 0; b < nblk; b++)
        if (pi[b] >= 0 && (bi < 0 || vi_less(pv[b], pi[b], bv, bi))) {
            bv = pv[b];
            bi = pi[b];
        }
    idx[t] = bi;
    lastv[0] = bv;
}

int launch_argmin_k(sqd_ctx *ctx, const double *d, int64_t n, int k, int64_t *idx_dev,
                    int64_t sym_n) {
    int nblk = 4 * ctx->sm_count;
    double *pv = nullptr, *lastv = nullptr;
    int64_t *pi = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&pv, sizeof(double) * (nblk + 1), ctx->stream));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&pi, sizeof(int64_t) * nblk, ctx->stream));
    lastv = pv + nblk;
    double hv = 0.0;
    int64_t hi = -1;
    for (int t = 0; t < k; t++) {
        k_argmin_partial<<<nblk, RED_THREADS, 0, ctx->stream>>>(d, n, hv, hi, sym_n, pv, pi);
        SQD_LAUNCHED(ctx);
        k_argmin_final<<<1, 1, 0, ctx->stream>>>(pv, pi, nblk, t, idx_dev, lastv);
        SQD_LAUNCHED(ctx);
        SQD_CUDA(ctx, cudaMemcpyAsync(&hv, lastv, sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SQD_CUDA(ctx, cudaMemcpyAsync(&hi, idx_dev + t, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                      ctx->stream));
        SQD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (hi < 0) return sqd_fail(ctx, SQD_EINVAL, "fewer determinants than roots");
    }
    SQD_CUDA(ctx, cudaFreeAsync(pv, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(pi, ctx->stream));
    return SQD_OK;
}

__global__ void k_set_unit(double *V, int64_t ld, int k, const int64_t *idx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) V[(int64_t)j * ld + idx[j]] = 1.0;
}

int launch_set_unit(sqd_ctx *ctx, double *V, int64_t ld, int k, const int64_t *idx_dev) {
    k_set_unit<<<1, 128, 0, ctx->stream>>>(V, ld, k, idx_dev);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// the normalised unit vectors of one spin-flip sector at positions (I, J),
// I <= J, of an n x n matrix: e_II (sgn = +1 only), or
// (e_IJ + sgn e_JI) / sqrt(2)
__global__ void k_set_unit_sym(double *V, int64_t ld, int k, const int64_t *idx, int64_t n,
                               int sgn) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const int64_t p = idx[j], I = p / n, J = p % n;
    if (I == J) {
        V[(int64_t)j * ld + p] = 1.0;
    } else {
        V[(int64_t)j * ld + p] = M_SQRT1_2;
        V[(int64_t)j * ld + J * n + I] = sgn > 0 ? M_SQRT1_2 : -M_SQRT1_2;
    }
}

int launch_set_unit_sym(sqd_ctx *ctx, double *V, int64_t ld, int k, const int64_t *idx_dev,
                        int64_t n, int sgn) {
    k_set_unit_sym<<<1, 128, 0, ctx->stream>>>(V, ld, k, idx_dev, n, sgn);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ------------------------------------------------------- GD+k restart ---
// Z[:, 0..m2) = Y[:, 0..m2) (the lowest Ritz coefficients), then each of the
// k previous Ritz coefficient columns P[:, j] (rows >= mp are zero) is
// orthogonalised twice against the columns of Z so far and appended if its
// norm stays above 1e-8.  One block; m <= 112.  *r_out = columns of Z.
__global__ void __launch_bounds__(128) k_gdk_basis(const double *__restrict__ Y, int m, int m2,
                                                   const double *__restrict__ P, int mp, int k,
                                                   int ldp, double *__restrict__ Z, int ldz,
                                                   int *__restrict__ r_out) {
    int r = gdk_block(Y, m, m2, P, mp, k, ldp, Z, ldz);
    if (threadIdx.x == 0) *r_out = r;
}

int launch_gdk_basis(sqd_ctx *ctx, const double *Y, int m, int m2, const double *P, int mp,
                     int k, int ldp, double *Z, int ldz, int *r_dev) {
    if (m > JAC_MAX) return sqd_fail(ctx, SQD_EINVAL, "subspace too large");
    k_gdk_basis<<<1, 128, 0, ctx->stream>>>(Y, m, m2, P, mp, k, ldp, Z, ldz, r_dev);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// Yprev = first k columns of the identity (r rows, leading dimension ld)
__global__ void k_identity_cols(double *Y, int r, int k, int ld) {
    for (int t = threadIdx.x; t < r * k; t += blockDim.x) {
        int i = t % r, j = t / r;
        Y[i + (int64_t)j * ld] = (i == j) ? 1.0 : 0.0;
    }
}

int launch_identity_cols(sqd_ctx *ctx, double *Y, int r, int k, int ld) {
    k_identity_cols<<<1, 256, 0, ctx->stream>>>(Y, r, k, ld);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// ---------------------------------------------------------------- phase --
// Flip each vector so that its largest-magnitude component (lowest index on
// ties) is positive.
__global__ void __launch_bounds__(RED_THREADS)
    k_absmax_partial(const double *__restrict__ x, int64_t n, double *__restrict__ pv,
                     int64_t *__restrict__ pi) {
    __shared__ double sv[RED_THREADS];
    __shared__ int64_t si[RED_THREADS];
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double v = fabs(x[p]);
        if (v > bv) {  // first (lowest) index wins ties within a thread
            bv = v;
            bi = p;
        }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = RED_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double v2 = sv[threadIdx.x + o];
            int64_t i2 = si[threadIdx.x + o];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 >= 0 && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pv[blockIdx.x] = sv[0];
        pi[blockIdx.x] = si[0];
    }
}

__global__ void k_phase_final(const double *x, const double *pv, const int64_t *pi, int nblk,
                              double *sign_out) {
    double bv = -1.0;
    int64_t bi = -1;
    for (int b = 0; b < nblk; b++)
        if (pv[b] > bv || (pv[b] == bv && pi[b] >= 0 && pi[b] < bi)) {
            bv = pv[b];
            bi = pi[b];
        }
    *sign_out = (bi >= 0 && x[bi] < 0.0) ? -1.0 : 1.0;
}

int launch_fix_phase(sqd_ctx *ctx, double *X, int64_t ld, int k, int64_t n, double *work_dev) {
    int nblk = 4 * ctx->sm_count;
    double *pv = work_dev;                          // nblk
    int64_t *pi = (int64_t *)(work_dev + nblk);     // nblk
    double *sg = work_dev + 2 * nblk;               // 1
    for (int j = 0; j < k; j++) {
        double *x = X + (int64_t)j * ld;
        k_absmax_partial<<<nblk, RED_THREADS, 0, ctx->stream>>>(x, n, pv, pi);
        SQD_LAUNCHED(ctx);
        k_phase_final<<<1, 1, 0, ctx->stream>>>(x, pv, pi, nblk, sg);
        SQD_LAUNCHED(ctx);
        SQD_TRY(launch_scale(ctx, x, n, sg, 0));
    }
    return SQD_OK;
}

// ----------------------------------------------- one-vector fused passes --
// The one-root Davidson (a block of one new vector, m <= 16 basis vectors)
// is bound by HBM at large N: every pass over a basis vector costs 8 N bytes.
// These kernels cut the passes of an iteration from about 7 m + 16 vectors
// to 5 m + 8 by fusing what reads the same vectors:
//   k_ritz_prec_dot : x = V y, r = W y - theta x, t = r / (theta - H_II) and
//                     the projections V_i . t of the first Gram-Schmidt pass,
//                     with |r|^2 and |t|^2 (the Ritz vector is not stored);
//   k_gs_update_dot : t' = t - V p (first update) with V_i . t' (second pass
//                     projections) and |t'|^2;
//   k_gs_update_scale: t'' = (t' - V p') * s (second update and the
//                     normalisation; s = 1 / |t''| from |t''|^2 =
//                     |t'|^2 - |p'|^2, Pythagoras, V orthonormal).
// y, theta and p are read from device memory, so no host round trip sits
// between the eigensolve and the correction.  Per-block partials are summed
// in a fixed order by k_sum_partials.

// Each kernel is instantiated for the exact basis size MB (1..16): every
// load of an element's MB basis values is issued before its arithmetic, with
// no predicated-off slots, and the two Ritz sums run as two chains each.
template <int MB>
__global__ void __launch_bounds__(RED_THREADS)
    k_ritz_prec_dot(const double *__restrict__ V, const double *__restrict__ W, int64_t ld,
                    const double *__restrict__ y, const double *__restrict__ theta_p,
                    const double *__restrict__ diag, double floor_, int64_t n,
                    double *__restrict__ T, double *__restrict__ partial) {
    __shared__ double red[(RED_THREADS / 32) * (MB + 2)];
    __shared__ double ys[MB];
    if (threadIdx.x < MB) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    const double th = *theta_p;
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    double s_r = 0.0, s_t = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double vv[MB], ww[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) {
            vv[i] = V[(int64_t)i * ld + p];
            ww[i] = W[(int64_t)i * ld + p];
        }
        const double dg = diag[p];
        double x0 = 0.0, x1 = 0.0, w0 = 0.0, w1 = 0.0;
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            x0 = fma(vv[i], ys[i], x0);
            w0 = fma(ww[i], ys[i], w0);
            if (i + 1 < MB) {
                x1 = fma(vv[i + 1], ys[i + 1], x1);
                w1 = fma(ww[i + 1], ys[i + 1], w1);
            }
        }
        const double r = fma(-th, x0 + x1, w0 + w1);
        const double t = r * precond_recip(th - dg, floor_);
        T[p] = t;
        s_r = fma(r, r, s_r);
        s_t = fma(t, t, s_t);
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], t, acc[i]);
    }
    double vals[MB + 2];
#pragma unroll
    for (int i = 0; i < MB; i++) vals[i] = acc[i];
    vals[MB] = s_r;
    vals[MB + 1] = s_t;
    int i;
    double v;
    if (block_sums<MB + 2>(vals, red, &i, &v)) partial[(int64_t)blockIdx.x * (MB + 2) + i] = v;
}

template <int MB>
__global__ void __launch_bounds__(RED_THREADS)
    k_gs_update_dot(const double *__restrict__ V, int64_t ld, const double *__restrict__ P,
                    double *__restrict__ T, int64_t n, double *__restrict__ partial) {
    __shared__ double red[(RED_THREADS / 32) * (MB + 1)];
    __shared__ double ps[MB];
    if (threadIdx.x < MB) ps[threadIdx.x] = P[threadIdx.x];
    __syncthreads();
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    double s_t = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = V[(int64_t)i * ld + p];
        const double t0 = T[p];
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            s0 = fma(vv[i], ps[i], s0);
            if (i + 1 < MB) s1 = fma(vv[i + 1], ps[i + 1], s1);
        }
        const double t = t0 - (s0 + s1);
        T[p] = t;
        s_t = fma(t, t, s_t);
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], t, acc[i]);
    }
    double vals[MB + 1];
#pragma unroll
    for (int i = 0; i < MB; i++) vals[i] = acc[i];
    vals[MB] = s_t;
    int i;
    double v;
    if (block_sums<MB + 1>(vals, red, &i, &v)) partial[(int64_t)blockIdx.x * (MB + 1) + i] = v;
}

template <int MB>
__global__ void __launch_bounds__(RED_THREADS)
    k_gs_update_scale(const double *__restrict__ V, int64_t ld, const double *__restrict__ P,
                      double scale, double *__restrict__ T, int64_t n) {
    __shared__ double ps[MB];
    if (threadIdx.x < MB) ps[threadIdx.x] = P[threadIdx.x];
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = V[(int64_t)i * ld + p];
        const double t0 = T[p];
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < MB; i += 2) {
            s0 = fma(vv[i], ps[i], s0);
            if (i + 1 < MB) s1 = fma(vv[i + 1], ps[i + 1], s1);
        }
        T[p] = (t0 - (s0 + s1)) * scale;
    }
}

// compile-time basis size for the dispatch below
template <int N>
struct mb_int {
    static constexpr int value = N;
};
// call f(mb_int<m>{}) for m in [1, 16]
#define MB_CASE(N, f) \
    case N:           \
        f(mb_int<N>{}); \
        break;
#define MB_DISPATCH(m, f)                                                                     \
    switch (m) {                                                                              \
        MB_CASE(1, f) MB_CASE(2, f) MB_CASE(3, f) MB_CASE(4, f) MB_CASE(5, f) MB_CASE(6, f)   \
        MB_CASE(7, f) MB_CASE(8, f) MB_CASE(9, f) MB_CASE(10, f) MB_CASE(11, f)              \
        MB_CASE(12, f) MB_CASE(13, f) MB_CASE(14, f) MB_CASE(15, f)                          \
        default: f(mb_int<16>{}); break;                                                      \
    }
// the same for m in [1, 8]
#define MB8_DISPATCH(m, f)                                                                    \
    switch (m) {                                                                              \
        MB_CASE(1, f) MB_CASE(2, f) MB_CASE(3, f) MB_CASE(4, f) MB_CASE(5, f) MB_CASE(6, f)   \
        MB_CASE(7, f)                                                                         \
        default: f(mb_int<8>{}); break;                                                       \
    }

// V_i . x for i < MB (the new column of the projected matrix of a one-root
// solve, x = W_new): every load of an element's MB basis values in flight at
// once, per-block sums in one barrier.  A block-dot tile of m x 1 outputs
// leaves most threads idle; this pass keeps the FP64 pipe fed instead.
template <int MB>
__global__ void __launch_bounds__(RED_THREADS)
    k_dots_one(const double *__restrict__ V, int64_t ld, const double *__restrict__ x,
               int64_t n, double *__restrict__ partial) {
    __shared__ double red[(RED_THREADS / 32) * MB];
    double acc[MB];
#pragma unroll
    for (int i = 0; i < MB; i++) acc[i] = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double vv[MB];
#pragma unroll
        for (int i = 0; i < MB; i++) vv[i] = V[(int64_t)i * ld + p];
        const double xp = x[p];
#pragma unroll
        for (int i = 0; i < MB; i++) acc[i] = fma(vv[i], xp, acc[i]);
    }
    int i;
    double v;
    if (block_sums<MB>(acc, red, &i, &v)) partial[(int64_t)blockIdx.x * MB + i] = v;
}

// out[i] = sum over blocks b of partial[b * stride + i], i < cnt (fixed order)
__global__ void k_sum_partials(const double *__restrict__ partial, int nblk, int stride,
                               int cnt, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cnt) return;
    double s = 0.0;
    for (int b = 0; b < nblk; b++) s += partial[(int64_t)b * stride + i];
    out[i] = s;
}

// in place: A_j[n] = sum_i A_i[n] Z[i + j*ldz] for j < r <= 8 (every element
// is read by one thread before it writes, so the in-place update is safe)
template <int R>
__global__ void __launch_bounds__(256) k_combine_inplace(double *A, int64_t lda, int m,
                                                         const double *__restrict__ Z, int ldz,
                                                         int64_t n) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double acc[R];
#pragma unroll
        for (int j = 0; j < R; j++) acc[j] = 0.0;
        for (int i = 0; i < m; i++) {
            const double a = A[(int64_t)i * lda + p];
#pragma unroll
            for (int j = 0; j < R; j++) acc[j] = fma(a, __ldg(Z + i + (int64_t)j * ldz), acc[j]);
        }
#pragma unroll
        for (int j = 0; j < R; j++) A[(int64_t)j * lda + p] = acc[j];
    }
}

// Gram matrix of B vectors, upper triangle packed by columns:
// partial[blk * CNT + j(j+1)/2 + i] = block blk's share of T_i . T_j, i <= j.
// B(B+1)/2 multiply-adds per element, where a full B x B block dot does B^2.
template <int B>
__global__ void __launch_bounds__(RED_THREADS)
    k_gram_tri(const double *__restrict__ T, int64_t ld, int64_t n, double *__restrict__ partial) {
    constexpr int CNT = B * (B + 1) / 2;
    __shared__ double red[(RED_THREADS / 32) * CNT];
    double acc[CNT];
#pragma unroll
    for (int c = 0; c < CNT; c++) acc[c] = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double t[B];
#pragma unroll
        for (int i = 0; i < B; i++) t[i] = T[(int64_t)i * ld + p];
#pragma unroll
        for (int j = 0; j < B; j++)
#pragma unroll
            for (int i = 0; i <= j; i++) acc[j * (j + 1) / 2 + i] = fma(t[i], t[j], acc[j * (j + 1) / 2 + i]);
    }
    int i;
    double v;
    if (block_sums<CNT>(acc, red, &i, &v)) partial[(int64_t)blockIdx.x * CNT + i] = v;
}

// in place T_j = sum_{i <= j} T_i Z[i + j*ldz], j < B, for an upper
// triangular Z (the coefficients of Gram-Schmidt on the Gram matrix)
template <int B>
__global__ void __launch_bounds__(256) k_combine_tri(double *T, int64_t ld,
                                                     const double *__restrict__ Z, int ldz,
                                                     int64_t n) {
    constexpr int CNT = B * (B + 1) / 2;
    double z[CNT];
#pragma unroll
    for (int j = 0; j < B; j++)
#pragma unroll
        for (int i = 0; i <= j; i++) z[j * (j + 1) / 2 + i] = __ldg(Z + i + (int64_t)j * ldz);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double t[B];
#pragma unroll
        for (int i = 0; i < B; i++) t[i] = T[(int64_t)i * ld + p];
#pragma unroll
        for (int j = 0; j < B; j++) {
            double a = 0.0;
#pragma unroll
            for (int i = 0; i <= j; i++) a = fma(t[i], z[j * (j + 1) / 2 + i], a);
            T[(int64_t)j * ld + p] = a;
        }
    }
}

// P_new[j] = sum_i Z[i + j*ldz] P_old[i], j < r (the projections of a vector
// on the restarted basis V Z); one block
__global__ void k_project_coeffs(const double *__restrict__ Z, int ldz, int m, int r,
                                 const double *__restrict__ Pold, double *__restrict__ Pnew) {
    const int j = threadIdx.x;
    if (j >= r) return;
    double s = 0.0;
    for (int i = 0; i < m; i++) s = fma(Z[i + (int64_t)j * ldz], Pold[i], s);
    Pnew[j] = s;
}

int fused_md(int M) { return M <= 16 ? 16 : 0; }

// sums[0..m) = V^T t, sums[m] = |r|^2, sums[m+1] = |t|^2; partial: nblk*(m+2)
int launch_ritz_prec_dot(sqd_ctx *ctx, int MD, const double *V, const double *W, int64_t ld,
                         int m, const double *y, const double *theta, const double *diag,
                         double floor_, int64_t n, double *T, double *partial, int nblk,
                         double *sums) {
    if (m < 1 || m > MD || MD != 16)
        return sqd_fail(ctx, SQD_EINVAL, "fused Ritz pass: m = %d out of range", m);
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int MB = decltype(mb)::value;
        k_ritz_prec_dot<MB><<<nblk, RED_THREADS, 0, st>>>(V, W, ld, y, theta, diag, floor_, n, T,
                                                          partial);
    };
    MB_DISPATCH(m, go);
    SQD_LAUNCHED(ctx);
    k_sum_partials<<<1, 64, 0, st>>>(partial, nblk, m + 2, m + 2, sums);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// T -= V P; sums[0..m) = V^T T (after), sums[m] = |T|^2 (after)
int launch_gs_update_dot(sqd_ctx *ctx, int MD, const double *V, int64_t ld, int m,
                         const double *P, double *T, int64_t n, double *partial, int nblk,
                         double *sums) {
    if (m < 1 || m > MD || MD != 16)
        return sqd_fail(ctx, SQD_EINVAL, "fused Gram-Schmidt pass: m = %d out of range", m);
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int MB = decltype(mb)::value;
        k_gs_update_dot<MB><<<nblk, RED_THREADS, 0, st>>>(V, ld, P, T, n, partial);
    };
    MB_DISPATCH(m, go);
    SQD_LAUNCHED(ctx);
    k_sum_partials<<<1, 64, 0, st>>>(partial, nblk, m + 1, m + 1, sums);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// T = (T - V P) * scale
int launch_gs_update_scale(sqd_ctx *ctx, int MD, const double *V, int64_t ld, int m,
                           const double *P, double scale, double *T, int64_t n, int nblk) {
    if (m < 1 || m > MD || MD != 16)
        return sqd_fail(ctx, SQD_EINVAL, "fused Gram-Schmidt pass: m = %d out of range", m);
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int MB = decltype(mb)::value;
        k_gs_update_scale<MB><<<nblk, RED_THREADS, 0, st>>>(V, ld, P, scale, T, n);
    };
    MB_DISPATCH(m, go);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// out[i] = V_i . x for i < m <= MD (contiguous outputs); partial: nblk * m
int launch_dots_one(sqd_ctx *ctx, int MD, const double *V, int64_t ld, int m, const double *x,
                    int64_t n, double *partial, int nblk, double *out) {
    if (m < 1 || m > MD || MD != 16)
        return sqd_fail(ctx, SQD_EINVAL, "one-vector dots: m = %d out of range", m);
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int MB = decltype(mb)::value;
        k_dots_one<MB><<<nblk, RED_THREADS, 0, st>>>(V, ld, x, n, partial);
    };
    MB_DISPATCH(m, go);
    SQD_LAUNCHED(ctx);
    k_sum_partials<<<1, 64, 0, st>>>(partial, nblk, m, m, out);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

int launch_combine_inplace(sqd_ctx *ctx, double *A, int64_t lda, int m, const double *Z, int ldz,
                           int r, int64_t n) {
    if (r < 1 || r > 8 || r > m)
        return sqd_fail(ctx, SQD_EINVAL, "in-place combination of %d vectors", r);
    unsigned g = grid_1d(n, 256);
    if (g > 8u * (unsigned)ctx->sm_count * 8u) g = 8u * (unsigned)ctx->sm_count * 8u;
    cudaStream_t st = ctx->stream;
    switch (r) {
        case 1: k_combine_inplace<1><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 2: k_combine_inplace<2><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 3: k_combine_inplace<3><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 4: k_combine_inplace<4><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 5: k_combine_inplace<5><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 6: k_combine_inplace<6><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        case 7: k_combine_inplace<7><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
        default: k_combine_inplace<8><<<g, 256, 0, st>>>(A, lda, m, Z, ldz, n); break;
    }
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// out[j(j+1)/2 + i] = T_i . T_j for i <= j < b <= 8; partial: nblk * b(b+1)/2
int launch_gram_tri(sqd_ctx *ctx, const double *T, int64_t ld, int b, int64_t n, double *partial,
                    int nblk, double *out) {
    if (b < 1 || b > 8) return sqd_fail(ctx, SQD_EINVAL, "packed Gram matrix of %d vectors", b);
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int B = decltype(mb)::value;
        k_gram_tri<B><<<nblk, RED_THREADS, 0, st>>>(T, ld, n, partial);
    };
    MB8_DISPATCH(b, go);
    SQD_LAUNCHED(ctx);
    const int cnt = b * (b + 1) / 2;
    k_sum_partials<<<1, 64, 0, st>>>(partial, nblk, cnt, cnt, out);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// in place T_j = sum_{i <= j} T_i Z[i + j*ldz], j < b <= 8 (Z upper triangular)
int launch_combine_tri(sqd_ctx *ctx, double *T, int64_t ld, int b, const double *Z, int ldz,
                       int64_t n) {
    if (b < 1 || b > 8)
        return sqd_fail(ctx, SQD_EINVAL, "triangular combination of %d vectors", b);
    unsigned g = grid_1d(n, 256);
    if (g > 8u * (unsigned)ctx->sm_count * 8u) g = 8u * (unsigned)ctx->sm_count * 8u;
    cudaStream_t st = ctx->stream;
    auto go = [&](auto mb) {
        constexpr int B = decltype(mb)::value;
        k_combine_tri<B><<<g, 256, 0, st>>>(T, ld, Z, ldz, n);
    };
    MB8_DISPATCH(b, go);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

int launch_project_coeffs(sqd_ctx *ctx, const double *Z, int ldz, int m, int r,
                          const double *Pold, double *Pnew) {
    if (r < 1 || r > 128) return sqd_fail(ctx, SQD_EINVAL, "bad restart size %d", r);
    k_project_coeffs<<<1, 128, 0, ctx->stream>>>(Z, ldz, m, r, Pold, Pnew);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}
