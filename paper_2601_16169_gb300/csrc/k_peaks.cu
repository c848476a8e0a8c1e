// FP64 throughput probes: the roofline denominators of the sigma and
// Davidson kernels, which are bound by FP64 arithmetic rather than by HBM.
//
//  k_probe_dfma  independent FMA chains on the FP64 ALU pipe (8 chains per
//                thread, a grid of 8 blocks of 256 threads per SM).
//  k_probe_dmma  the FP64 tensor-core MMA (mma.sync m8n8k4, f64 in and out),
//                4 independent accumulators per warp; each instruction is
//                8 x 8 x 4 = 256 multiply-adds per warp.
//
// The results are written to memory only when a runtime flag is set, which
// the host never sets, so the compiler cannot drop the arithmetic.
#include "sqd_internal.cuh"

#define PROBE_THREADS 256

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double seed, int sink_flag,
                                                              double *sink) {
    double a[8];
    const double m = 1.0 + 1e-12 * seed, c = 1e-9 * seed;
#pragma unroll
    for (int u = 0; u < 8; u++) a[u] = seed + u + threadIdx.x * 1e-3;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 8; u++) a[u] = fma(a[u], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; u++) s += a[u];
    if (sink_flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void dmma_884(double &d0, double &d1, double a, double b) {
    asm volatile(
        "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
        : "+d"(d0), "+d"(d1)
        : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dmma(int iters, double seed, int sink_flag,
                                                              double *sink) {
    const double a = 1e-3 * seed + threadIdx.x * 1e-6, b = 1e-3 - seed * 1e-9;
    double d[8];
#pragma unroll
    for (int u = 0; u < 8; u++) d[u] = 0.0;
    for (int it = 0; it < iters; it++) {
        dmma_884(d[0], d[1], a, b);
        dmma_884(d[2], d[3], a, b);
        dmma_884(d[4], d[5], a, b);
        dmma_884(d[6], d[7], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; u++) s += d[u];
    if (sink_flag) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Time one probe: a warm-up launch, then the best of three timed launches.
static int time_probe(sqd_ctx *ctx, void (*kern)(int, double, int, double *), int iters,
                      double *sink, float *best_ms) {
    const unsigned grid = 8u * (unsigned)ctx->sm_count;
    cudaEvent_t e0, e1;
    SQD_CUDA(ctx, cudaEventCreate(&e0));
    SQD_CUDA(ctx, cudaEventCreate(&e1));
    *best_ms = INFINITY;
    int rc = SQD_OK;
    for (int rep = 0; rep < 4 && rc == SQD_OK; rep++) {
        cudaEventRecord(e0, ctx->stream);
        kern<<<grid, PROBE_THREADS, 0, ctx->stream>>>(iters, 1.0 + rep, 0, sink);
        if (cudaPeekAtLastError() != cudaSuccess) {
            rc = sqd_fail(ctx, SQD_ECUDA, "probe launch failed: %s",
                          cudaGetErrorString(cudaGetLastError()));
            break;
        }
        ctx->launches++;
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = sqd_fail(ctx, SQD_ECUDA, "probe failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < *best_ms) *best_ms = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int measure_fp64_peaks(sqd_ctx *ctx, double *dfma_tflops, double *dmma_tflops) {
    const double threads = 8.0 * ctx->sm_count * PROBE_THREADS;
    const int it_fma = 1 << 14, it_mma = 1 << 13;
    float ms = 0.f;
    if (dfma_tflops) {
        SQD_TRY(time_probe(ctx, k_probe_dfma, it_fma, nullptr, &ms));
        *dfma_tflops = 2.0 * 8.0 * it_fma * threads / (ms * 1e-3) / 1e12;
    }
    if (dmma_tflops) {
        const double warps = threads / 32.0;
        SQD_TRY(time_probe(ctx, k_probe_dmma, it_mma, nullptr, &ms));
        *dmma_tflops = 2.0 * 256.0 * 4.0 * it_mma * warps / (ms * 1e-3) / 1e12;
    }
    return SQD_OK;
}
