// sqd_build_strings_noalloc: the string filter of sqd_build_strings with all
// of its scratch in a fixed device array, for callers that cannot allocate
// device memory.  The paper has no counterpart; see include/sqd.h.
#include <mutex>

#include "sqd_internal.cuh"

// Largest raw-string count this entry point accepts.
#define NOALLOC_MAX_RAW (1 << 18)
#define NOALLOC_SCAN_BLOCK 1024
#define NOALLOC_MAX_BLOCKS (NOALLOC_MAX_RAW / NOALLOC_SCAN_BLOCK)

// Scratch layout (int64 words): flags[MAX] | pos[MAX] | keys[MAX] |
// block sums[MAX_BLOCKS + 8] | block offsets[MAX_BLOCKS + 8] | totals[8].
#define NOALLOC_WORDS (3 * NOALLOC_MAX_RAW + 2 * (NOALLOC_MAX_BLOCKS + 8) + 8)

// Every GPU that loads the library holds this array (6 MB) until exit.
static __device__ __align__(256) int64_t g_noalloc_scratch[NOALLOC_WORDS];

// Device addresses of the array, looked up once per device.
static std::mutex g_noalloc_mu;
static int64_t *g_noalloc_ptr[128];

static int noalloc_scratch(sqd_ctx *ctx, int64_t **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 128)
        return sqd_fail(ctx, SQD_EINVAL, "device index out of range");
    if (!g_noalloc_ptr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return sqd_fail(ctx, SQD_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                            cudaGetErrorString(e));
        g_noalloc_ptr[ctx->device] = (int64_t *)p;
    }
    *out = g_noalloc_ptr[ctx->device];
    return SQD_OK;
}

// ---- exclusive scan on caller-provided workspace (n <= NOALLOC_MAX_RAW) --

__device__ __forceinline__ int64_t na_warp_scan(int64_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan of one block of NOALLOC_SCAN_BLOCK elements; block sum out
__global__ void __launch_bounds__(NOALLOC_SCAN_BLOCK)
    k_na_scan_blocks(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                     int64_t *__restrict__ sums) {
    __shared__ int64_t wsum[32];
    int64_t i = (int64_t)blockIdx.x * NOALLOC_SCAN_BLOCK + threadIdx.x;
    int64_t v = (i < n) ? in[i] : 0;
    int64_t inc = na_warp_scan(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) wsum[lane] = na_warp_scan(wsum[lane]);
    __syncthreads();
    int64_t pre = (w > 0) ? wsum[w - 1] : 0;
    if (i < n) out[i] = pre + inc - v;
    if (threadIdx.x == NOALLOC_SCAN_BLOCK - 1) sums[blockIdx.x] = pre + inc;
}

__global__ void k_na_scan_add(int64_t *__restrict__ out, int64_t n,
                              const int64_t *__restrict__ offs) {
    int64_t i = (int64_t)blockIdx.x * NOALLOC_SCAN_BLOCK + threadIdx.x;
    if (i < n) out[i] += offs[blockIdx.x];
}

__global__ void k_na_total(const int64_t *in, const int64_t *out, int64_t n, int64_t *total) {
    *total = (n > 0) ? out[n - 1] + in[n - 1] : 0;
}

// Two levels suffice: n <= 1024 * 1024.
static int na_scan(sqd_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, int64_t *sums,
                   int64_t *offs, int64_t *total) {
    if (n > 0) {
        int64_t nb = (n + NOALLOC_SCAN_BLOCK - 1) / NOALLOC_SCAN_BLOCK;
        k_na_scan_blocks<<<(unsigned)nb, NOALLOC_SCAN_BLOCK, 0, ctx->stream>>>(in, out, n, sums);
        SQD_LAUNCHED(ctx);
        if (nb > 1) {
            k_na_scan_blocks<<<1, NOALLOC_SCAN_BLOCK, 0, ctx->stream>>>(sums, offs, nb,
                                                                       sums + nb);
            SQD_LAUNCHED(ctx);
            k_na_scan_add<<<(unsigned)nb, NOALLOC_SCAN_BLOCK, 0, ctx->stream>>>(out, n, offs);
            SQD_LAUNCHED(ctx);
        }
    }
    k_na_total<<<1, 1, 0, ctx->stream>>>(in, out, n, total);
    SQD_LAUNCHED(ctx);
    return SQD_OK;
}

extern "C" int sqd_build_strings_noalloc(sqd_ctx *ctx, const uint64_t *d_raw, int64_t n_raw,
                                         int norb, int nelec, uint64_t *d_out,
                                         int64_t *n_out) {
    if (!ctx) return SQD_EINVAL;
    if (!n_out) return sqd_fail(ctx, SQD_EINVAL, "sqd_build_strings_noalloc: n_out is NULL");
    *n_out = 0;
    if (norb < 1 || norb > 64) return sqd_fail(ctx, SQD_EINVAL, "norb must be in [1, 64]");
    if (nelec < 0 || nelec > norb) return sqd_fail(ctx, SQD_EINVAL, "nelec must be in [0, norb]");
    if (n_raw < 0) return sqd_fail(ctx, SQD_EINVAL, "n_raw < 0");
    if (n_raw > NOALLOC_MAX_RAW)
        return sqd_fail(ctx, SQD_EINVAL,
                        "sqd_build_strings_noalloc accepts at most %d raw strings (got %lld); "
                        "use sqd_build_strings",
                        NOALLOC_MAX_RAW, (long long)n_raw);
    if (n_raw == 0) return SQD_OK;
    if (!d_raw || !d_out) return sqd_fail(ctx, SQD_EINVAL, "NULL string buffer");
    SQD_CUDA(ctx, cudaSetDevice(ctx->device));
    int64_t *ws = nullptr;
    SQD_TRY(noalloc_scratch(ctx, &ws));
    int64_t *flags = ws;
    int64_t *pos = ws + NOALLOC_MAX_RAW;
    uint64_t *keys = (uint64_t *)(ws + 2 * NOALLOC_MAX_RAW);
    int64_t *sums = ws + 3 * NOALLOC_MAX_RAW;
    int64_t *offs = sums + NOALLOC_MAX_BLOCKS + 8;
    int64_t *tot = offs + NOALLOC_MAX_BLOCKS + 8;
    cudaStream_t st = ctx->stream;

    SQD_TRY(launch_filter_flags(ctx, d_raw, n_raw, norb, nelec, flags));
    SQD_TRY(na_scan(ctx, flags, pos, n_raw, sums, offs, tot));
    int64_t m = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t P = 1;
    while (P < m) P <<= 1;
    SQD_TRY(launch_fill_u64(ctx, keys, P, ~0ull));
    SQD_TRY(launch_scatter_flagged(ctx, d_raw, flags, pos, n_raw, keys));
    SQD_TRY(launch_bitonic_sort_u64(ctx, keys, P));
    SQD_TRY(launch_unique_flags(ctx, keys, m, flags));
    SQD_TRY(na_scan(ctx, flags, pos, m, sums, offs, tot + 1));
    SQD_TRY(launch_scatter_flagged(ctx, keys, flags, pos, m, d_out));
    int64_t u = 0;
    SQD_CUDA(ctx, cudaMemcpyAsync(&u, tot + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SQD_CUDA(ctx, cudaStreamSynchronize(st));
    *n_out = m > 0 ? u : 0;
    return SQD_OK;
}
