// String-set filtering (popcount filter, bitonic sort, de-duplication), the
// exclusive scan used for every CSR offset array, and input checks.
#include <cstdarg>
#include <cstdio>

#include "sqd_internal.cuh"

int sqd_fail(sqd_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

// ------------------------------------------------------------- filter ---

__global__ void k_filter_flags(const uint64_t *__restrict__ raw, int64_t n, int norb,
                               int nelec, int64_t *__restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t x = raw[i];
    bool ok = (__popcll(x) == nelec) && (norb == 64 || (x >> norb) == 0);
    flags[i] = ok ? 1 : 0;
}

int launch_filter_flags(sqd_ctx *ctx, const uint64_t *raw, int64_t n, int norb, int nelec,
                        int64_t *flags) {
    if (n == 0) return SQD_OK;
    k_filter_flags<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(raw, n, norb, nelec, flags);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

__global__ void k_scatter_flagged(const uint64_t *__restrict__ in,
                                  const int64_t *__restrict__ flags,
                                  const int64_t *__restrict__ pos, int64_t n,
                                  uint64_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flags[i]) out[pos[i]] = in[i];
}

int launch_scatter_flagged(sqd_ctx *ctx, const uint64_t *in, const int64_t *flags,
                           const int64_t *pos, int64_t n, uint64_t *out) {
    if (n == 0) return SQD_OK;
    k_scatter_flagged<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(in, flags, pos, n, out);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

__global__ void k_fill_u64(uint64_t *p, int64_t n, uint64_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

int launch_fill_u64(sqd_ctx *ctx, uint64_t *p, int64_t n, uint64_t v) {
    if (n == 0) return SQD_OK;
    k_fill_u64<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(p, n, v);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

__global__ void k_unique_flags(const uint64_t *__restrict__ s, int64_t n,
                               int64_t *__restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flags[i] = (i == 0 || s[i] != s[i - 1]) ? 1 : 0;
}

int launch_unique_flags(sqd_ctx *ctx, const uint64_t *sorted, int64_t n, int64_t *flags) {
    if (n == 0) return SQD_OK;
    k_unique_flags<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(sorted, n, flags);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

// -------------------------------------------------------- bitonic sort ---
// Keys are sorted ascending in place; n is a power of two.  Stages whose
// partner distance is below BITONIC_LOCAL run inside one block in shared
// memory; longer distances run as one grid-wide compare-exchange pass each.

#define BITONIC_LOCAL 2048  // elements held by one block (1024 threads x 2)

__global__ void __launch_bounds__(1024) k_bitonic_local(uint64_t *keys, int64_t n,
                                                        int64_t k_from, int64_t k_to) {
    __shared__ uint64_t sh[BITONIC_LOCAL];
    int64_t base = (int64_t)blockIdx.x * BITONIC_LOCAL;
    for (int t = threadIdx.x; t < BITONIC_LOCAL; t += blockDim.x) sh[t] = keys[base + t];
    __syncthreads();
    // k_from == 2: full local sort (k = 2 .. BITONIC_LOCAL);
    // otherwise: finish the merge of size k_to for partner distances < BITONIC_LOCAL.
    for (int64_t k = k_from; k <= k_to; k <<= 1) {
        int64_t jstart = (k_from == 2) ? (k >> 1) : (BITONIC_LOCAL >> 1);
        for (int64_t j = jstart; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < BITONIC_LOCAL; t += blockDim.x) {
                int l = t ^ (int)j;
                if (l > t) {
                    int64_t gi = base + t;
                    bool asc = ((gi & k) == 0);
                    uint64_t a = sh[t], b = sh[l];
                    if ((a > b) == asc) {
                        sh[t] = b;
                        sh[l] = a;
                    }
                }
            }
            __syncthreads();
        }
        if (k_from != 2) break;
    }
    for (int t = threadIdx.x; t < BITONIC_LOCAL; t += blockDim.x) keys[base + t] = sh[t];
}

__global__ void k_bitonic_global(uint64_t *keys, int64_t n, int64_t k, int64_t j) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t l = i ^ j;
    if (l <= i) return;
    bool asc = ((i & k) == 0);
    uint64_t a = keys[i], b = keys[l];
    if ((a > b) == asc) {
        keys[i] = b;
        keys[l] = a;
    }
}

__global__ void k_bitonic_small(uint64_t *keys, int64_t n) {
    // one block, n <= BITONIC_LOCAL
    __shared__ uint64_t sh[BITONIC_LOCAL];
    for (int t = threadIdx.x; t < n; t += blockDim.x) sh[t] = keys[t];
    __syncthreads();
    for (int64_t k = 2; k <= n; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                int l = t ^ (int)j;
                if (l > t) {
                    bool asc = ((t & k) == 0);
                    uint64_t a = sh[t], b = sh[l];
                    if ((a > b) == asc) {
                        sh[t] = b;
                        sh[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < n; t += blockDim.x) keys[t] = sh[t];
}

int launch_bitonic_sort_u64(sqd_ctx *ctx, uint64_t *keys, int64_t n) {
    if (n <= 1) return SQD_OK;
    if (n & (n - 1)) return sqd_fail(ctx, SQD_EINVAL, "bitonic sort needs a power of two");
    if (n <= BITONIC_LOCAL) {
        k_bitonic_small<<<1, 1024, 0, ctx->stream>>>(keys, n);
        SQD_LAUNCHED(ctx);
        return SQD_OK;
    }
    unsigned nblk = (unsigned)(n / BITONIC_LOCAL);
    k_bitonic_local<<<nblk, 1024, 0, ctx->stream>>>(keys, n, 2, BITONIC_LOCAL);
    SQD_LAUNCHED(ctx);
    for (int64_t k = 2 * BITONIC_LOCAL; k <= n; k <<= 1) {
        for (int64_t j = k >> 1; j >= BITONIC_LOCAL; j >>= 1) {
            k_bitonic_global<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(keys, n, k, j);
            SQD_LAUNCHED(ctx);
        }
        k_bitonic_local<<<nblk, 1024, 0, ctx->stream>>>(keys, n, k, k);
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

// ---------------------------------------------------------------- scan ---
// Exclusive prefix sum of int64, hierarchical: per-block scans of 1024
// elements, a recursive scan of the block sums, then a uniform add.

#define SCAN_BLOCK 1024

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_blocks(const int64_t *__restrict__ in,
                                                            int64_t *__restrict__ out,
                                                            int64_t n,
                                                            int64_t *__restrict__ sums) {
    __shared__ int64_t wsum[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    int64_t inc = warp_incl_scan(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int64_t s = wsum[lane];
        s = warp_incl_scan(s);
        wsum[lane] = s;
    }
    __syncthreads();
    int64_t pre = (w > 0) ? wsum[w - 1] : 0;
    if (i < n) out[i] = pre + inc - v;
    if (threadIdx.x == SCAN_BLOCK - 1) sums[blockIdx.x] = pre + inc;
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n,
                           const int64_t *__restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void k_scan_total(const int64_t *in, const int64_t *out, int64_t n,
                             int64_t *total) {
    *total = (n > 0) ? out[n - 1] + in[n - 1] : 0;
}

static int scan_rec(sqd_ctx *ctx, const int64_t *in, int64_t *out, int64_t n) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    int64_t *sums = nullptr, *offs = nullptr;
    SQD_CUDA(ctx, cudaMallocAsync((void **)&sums, sizeof(int64_t) * (nb + 1), ctx->stream));
    SQD_CUDA(ctx, cudaMallocAsync((void **)&offs, sizeof(int64_t) * (nb + 1), ctx->stream));
    k_scan_blocks<<<(unsigned)nb, SCAN_BLOCK, 0, ctx->stream>>>(in, out, n, sums);
    SQD_LAUNCHED(ctx);
    if (nb > 1) {
        int r = scan_rec(ctx, sums, offs, nb);
        if (r != SQD_OK) return r;
        k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, ctx->stream>>>(out, n, offs);
        SQD_LAUNCHED(ctx);
    }
    SQD_CUDA(ctx, cudaFreeAsync(sums, ctx->stream));
    SQD_CUDA(ctx, cudaFreeAsync(offs, ctx->stream));
    return SQD_OK;
}

int launch_exclusive_scan(sqd_ctx *ctx, const int64_t *in, int64_t *out, int64_t n,
                          int64_t *total_dev) {
    if (n > 0) SQD_TRY(scan_rec(ctx, in, out, n));
    if (total_dev) {
        k_scan_total<<<1, 1, 0, ctx->stream>>>(in, out, n, total_dev);
        SQD_LAUNCHED(ctx);
    }
    return SQD_OK;
}

// --------------------------------------------------------------- checks ---

__global__ void k_check_strings(const uint64_t *__restrict__ s, int64_t n, int norb, int ne,
                                int *bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t x = s[i];
    int b = 0;
    if (__popcll(x) != ne) b |= 1;
    if (norb < 64 && (x >> norb) != 0) b |= 2;
    if (i + 1 < n && !(x < s[i + 1])) b |= 4;
    if (b) atomicOr(bad, b);
}

int launch_check_sorted_unique(sqd_ctx *ctx, const uint64_t *s, int64_t n, int norb, int ne,
                               int *bad_dev) {
    if (n == 0) return SQD_OK;
    k_check_strings<<<grid_1d(n, 256), 256, 0, ctx->stream>>>(s, n, norb, ne, bad_dev);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// res[0] = max asymmetry, res[1] = max |value|, res[2] = count of non-finite
__global__ void k_check_integrals(const double *__restrict__ h, const double *__restrict__ V,
                                  int norb, double *res) {
    int64_t n2 = (int64_t)norb * norb, n4 = n2 * n2;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2) {
        int p = (int)(i / norb), q = (int)(i % norb);
        double a = h[i], b = h[(int64_t)q * norb + p];
        if (!isfinite(a)) atomicAdd(&res[2], 1.0);
        else {
            atomic_max_nonneg(&res[0], fabs(a - b));
            atomic_max_nonneg(&res[1], fabs(a));
        }
    }
    if (i < n4) {
        int64_t t = i;
        int s_ = (int)(t % norb); t /= norb;
        int r = (int)(t % norb); t /= norb;
        int q = (int)(t % norb); t /= norb;
        int p = (int)t;
        double v = V[i];
        if (!isfinite(v)) {
            atomicAdd(&res[2], 1.0);
            return;
        }
        auto at = [&](int a, int b, int c, int d) {
            return V[(((int64_t)a * norb + b) * norb + c) * norb + d];
        };
        double d = fabs(v - at(q, p, r, s_));
        d = fmax(d, fabs(v - at(p, q, s_, r)));
        d = fmax(d, fabs(v - at(r, s_, p, q)));
        atomic_max_nonneg(&res[0], d);
        atomic_max_nonneg(&res[1], fabs(v));
    }
}

int launch_check_integrals(sqd_ctx *ctx, const double *h, const double *V, int norb,
                           double *res_dev) {
    int64_t n4 = (int64_t)norb * norb * norb * norb;
    k_check_integrals<<<grid_1d(n4, 256), 256, 0, ctx->stream>>>(h, V, norb, res_dev);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}
