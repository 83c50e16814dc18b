// The GPU's FP64 fused multiply-add rate, measured (not in the paper).
//
// FP64 arithmetic is the co-bound of every FP64 sparse kernel of this
// library on a part whose FP64 pipe executes a few operations per clock per
// SM: one FMA per 12 bytes of matrix.  The rooflines of those kernels need
// that rate as a denominator, and a nominal figure is not a measurement.
// k_dfma_rate keeps CHAINS independent FMA chains per thread in flight on
// every SM (eight 256-thread blocks per SM), so the FP64 pipe, not latency,
// limits it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "ssg_ctx.h"
#include "ssg_internal.h"

namespace ssg {
namespace {

constexpr int kRateBlock = 256;
constexpr int kRateChains = 8;
constexpr int kRateBlocksPerSM = 8;

// a <- a m + c per chain; with 0 < m < 1 every chain converges to c / (1 - m),
// so no value overflows however long the loop.  The final test keeps the
// chains live (the compiler cannot know it never holds).
__global__ void __launch_bounds__(kRateBlock) k_dfma_rate(double *out, int32_t iters, double m, double c) {
    double a[kRateChains];
#pragma unroll
    for (int j = 0; j < kRateChains; ++j) a[j] = 1e-3 * (threadIdx.x + j);
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kRateChains; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kRateChains; ++j) s += a[j];
    if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace ssg

using namespace ssg;

extern "C" int ssg_measure_fp64_rate(ssg_ctx *ctx, int32_t iters, int32_t reps, double *tflops, double *best_ms) {
    if (!ctx || iters < 1 || reps < 1 || !tflops) {
        set_error("ssg_measure_fp64_rate: null context or result, or iters / reps < 1");
        return SSG_E_INVALID;
    }
    SSG_CUDA_TRY(cudaSetDevice(ctx->device));
    const int blocks = ctx->num_sms * kRateBlocksPerSM;
    double *sink = nullptr;
    SSG_CUDA_TRY(cudaMalloc(&sink, sizeof(double) * blocks));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {  // r = -1: warm-up
        e = cudaEventRecord(e0, ctx->stream);
        if (e == cudaSuccess) {
            k_dfma_rate<<<blocks, kRateBlock, 0, ctx->stream>>>(sink, iters, 0.9999999, 1e-7);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r >= 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) {
        set_error(std::string("ssg_measure_fp64_rate: ") + cudaGetErrorString(e));
        return SSG_E_CUDA;
    }
    const double fmas = static_cast<double>(blocks) * kRateBlock * kRateChains * static_cast<double>(iters);
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    if (best_ms) *best_ms = best;
    return SSG_OK;
}
