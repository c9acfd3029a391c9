// sf_peak.cu -- measurement aid: the FP32 fused multiply-add rate this GPU
// sustains, the roofline denominator of the ALU-bound stages (the per-pixel
// assembly of the Gauss-Newton system, Section 5.1). Each thread runs eight
// independent FMA chains, so every SM sub-partition always has an FMA ready
// to issue; the rate is flops / the launch's CUDA-event time.
#include <cuda_runtime.h>

#include <algorithm>

#include "sf.h"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;

__device__ float g_fma_sink;

__global__ void __launch_bounds__(PEAK_THREADS) k_fma_rate(int iters, float a, float b)
{
    float x[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
    // a store the compiler cannot drop, taken only for an impossible value
    if (s == -1.0f) g_fma_sink = s;
}

} // namespace

extern "C" SF_API int sf_probe_fma_rate(int reps, double* flops_per_s, void* stream)
{
    if (!flops_per_s || reps < 1 || reps > 100) return SF_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_rate, PEAK_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    const int blocks = sms * std::max(per_sm, 1);
    const int iters = 1 << 14;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return SF_ERR_CUDA;
    }
    k_fma_rate<<<blocks, PEAK_THREADS, 0, st>>>(iters / 8, 1.0000001f, 1e-7f); // warm-up
    double best = 0.0;
    int rc = SF_OK;
    for (int r = 0; r < reps && rc == SF_OK; ++r) {
        cudaEventRecord(e0, st);
        k_fma_rate<<<blocks, PEAK_THREADS, 0, st>>>(iters, 1.0000001f, 1e-7f);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            rc = SF_ERR_CUDA;
            break;
        }
        const double flops = 2.0 * 4.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS;
        best = std::max(best, flops / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops_per_s = best;
    return rc;
}
