// FP32 FMA throughput of the GPU, measured in process: the denominator of the
// roofline of the CUDA-core kernels (the fused SLR tile kernel does its
// contraction as FP32 FMA chains).  Every thread runs kChains independent
// multiply-add chains, so the FMA pipes, not latency, bound the rate.
#include <cuda_runtime.h>

#include "slrcount.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;   // 2048 threads per SM: every warp slot filled

__device__ float g_peak_sink;

__global__ void __launch_bounds__(kThreads) ffma_peak_kernel(int iters, float a, float b) {
    float acc[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) acc[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) acc[j] = __fmaf_rn(acc[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += acc[j];
    // a store the compiler cannot prove dead; it never happens for these inputs
    if (s == -1.0f) g_peak_sink = s;
}

}  // namespace

extern "C" int slr_measure_fp32_peak(int device, int iters, double *tflops, double *ms) {
    if (!tflops || iters < 1) return SLR_EINVAL;
    cudaError_t e = cudaSetDevice(device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return SLR_ECUDA;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SLR_ECUDA;
    int rc = SLR_OK;
    float best = 1e30f;
    const int grid = sms * kBlocksPerSm;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SLR_ECUDA;
    // the first launch warms the clocks; the fastest of the next three counts
    for (int rep = 0; rep < 4 && rc == SLR_OK; ++rep) {
        cudaEventRecord(e0, s);
        ffma_peak_kernel<<<grid, kThreads, 0, s>>>(iters, 0.99999f, 1e-6f);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = SLR_ECUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < best) best = t;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc != SLR_OK) return rc;
    const double flop = 2.0 * kChains * (double)iters * (double)grid * kThreads;
    *tflops = flop / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return SLR_OK;
}
