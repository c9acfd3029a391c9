// sf_watch.cu -- the library's bounded device-wide waits, exercised without a
// fault: the grid barrier (sf_common.cuh) that the PCG, Schwarz and trial
// kernels meet at, and the mbarrier wait (sf_tc.cuh) of the tensor-core
// GEMM, each run with a short limit on a condition the caller controls. A
// wait that runs out latches a status bit and returns; nothing traps.
#include <cuda_runtime.h>

#include "sf_launch.h"
#include "sf_tc.cuh"

namespace sfk {

namespace {

// one grid barrier; block `skip` never arrives
__global__ void k_barrier_probe(unsigned long long* ctr, int* status, int skip, long long limit, int* returned)
{
    unsigned long long target = grid_barrier_base(ctr, gridDim.x) + gridDim.x;
    if ((int)blockIdx.x == skip) return;
    grid_barrier(ctr, status, target, limit);
    if (threadIdx.x == 0) atomicAdd(returned, 1);
}

// one wait on an mbarrier of arrival count 1; thread 0 arrives first if `arrive`
__global__ void k_mbar_probe(int arrive, long long limit, int* completed)
{
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t mb = tc::smem_u32(&mbar);
    if (threadIdx.x == 0) tc::mbar_init(mb, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(mb) : "memory");
    const bool ok = tc::mbar_wait(mb, 0u, limit);
    const int all = __syncthreads_and(ok ? 1 : 0);
    if (threadIdx.x == 0) *completed = all;
}

} // namespace

} // namespace sfk

using namespace sfk;

extern "C" SF_API int sf_probe_barrier_timeout(int skip_block, long long limit_cycles, int* status, int* returned)
{
    if (!status || !returned || limit_cycles < 1 || limit_cycles > 4000000000LL) return SF_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    if (skip_block >= sms) return SF_ERR_ARG;
    unsigned long long* ctr = nullptr;
    int* words = nullptr; // [0] status, [1] blocks returned
    if (cudaMalloc(&ctr, sizeof(*ctr)) != cudaSuccess || cudaMalloc(&words, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctr);
        return SF_ERR_OOM;
    }
    cudaMemset(ctr, 0, sizeof(*ctr));
    cudaMemset(words, 0, 2 * sizeof(int));
    int* st = words;
    int* ret = words + 1;
    void* args[] = {(void*)&ctr, (void*)&st, (void*)&skip_block, (void*)&limit_cycles, (void*)&ret};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(sms), dim3(128), args, 0, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, words, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(ctr);
    cudaFree(words);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    *status = (h[0] & DEV_TIMEOUT) ? SF_ERR_TIMEOUT : (h[0] ? SF_ERR_STATE : SF_OK);
    *returned = h[1];
    return SF_OK;
}

extern "C" SF_API int sf_probe_mbarrier_timeout(int arrive, long long limit_cycles, int* completed)
{
    if (!completed || limit_cycles < 1 || limit_cycles > 4000000000LL) return SF_ERR_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_OOM;
    }
    cudaMemset(d, 0xff, sizeof(int));
    k_mbar_probe<<<1, 64>>>(arrive ? 1 : 0, limit_cycles, d);
    cudaError_t e = cudaDeviceSynchronize();
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SF_ERR_CUDA;
    }
    *completed = h;
    return SF_OK;
}

extern "C" SF_API int sf_probe_tagged_timeout(int mode, int skip_block, long long limit_cycles, int* status,
                                              int* returned)
{
    if (!status || !returned || (mode != 0 && mode != 1) || limit_cycles < 1 || limit_cycles > 4000000000LL)
        return SF_ERR_ARG;
    return sfk::tag_timeout_probe(mode, skip_block, limit_cycles, status, returned);
}
