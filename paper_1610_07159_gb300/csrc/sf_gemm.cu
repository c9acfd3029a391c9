// sf_gemm.cu -- BF16 x BF16 -> FP32 matrix product on the fifth-generation
// tensor cores (tcgen05), the one contraction of the warm-start network
// (every convolution of its forward and backward pass is lowered to it).
//
//   C[M, N] = A[M, K] * B[N, K]^T      (both operands K-major, K % 64 == 0)
//
// One CTA of four warps computes a 128 x BN tile (BN <= 256, a multiple of
// 16) over a range of K: per 64-wide K chunk the warps copy the A and B tiles
// into shared memory (cp.async, 16 bytes per copy, rows past the matrix
// zero-filled) in the tensor core's K-major layout without swizzling (8-row x
// 16-byte core matrices, contiguous along K), and one thread issues four
// 128 x BN x 16 MMAs into a tensor-memory accumulator and commits them to the
// stage's mbarrier. Two stages alternate: chunk k + 1 is copied while the
// MMAs of chunk k run, and a stage is refilled once its mbarrier reports the
// MMAs that read it done. The epilogue reads the accumulator lane by lane
// (tcgen05.ld, warp w owns rows 32w .. 32w + 31) and applies one of the
// epilogues below. Split-K (grid.y) writes FP32 partial products that a
// fixed-order reduction sums, so results do not depend on scheduling.
//
// Every mbarrier wait gives up after about one second; the CTA then waits
// once more for its MMAs in flight, frees its tensor memory, raises the
// error word (bit 0) and returns. If that second wait gives up too, MMAs may
// still be writing the tensor memory and reading the shared memory that the
// CTA released: bit 1 is raised as well, and the CUDA context is to be
// treated as poisoned (the process should not launch further work on it).
#include <cuda_bf16.h>

#include <mutex>

#include "sf_launch.h"
#include "sf_tc.cuh"

namespace sfk {

namespace {

constexpr int GT = 128;  // threads per CTA
constexpr int BM = 128;  // rows per tile
constexpr int BK = 64;   // K per chunk (128 bytes of BF16)
constexpr uint32_t LBO = 128;            // next core matrix along K
constexpr uint32_t SBO = 8 * LBO;        // next 8-row group

// byte offset of (row r, 16-byte vector v) of a tile in the K-major layout
__device__ __forceinline__ uint32_t tile_off(int r, int v) { return (uint32_t)((r >> 3) * SBO + v * LBO + (r & 7) * 16); }

// Starts the copies of rows [r0, r0 + rows) x K chunk kc of a row-major BF16
// matrix into a tile; rows at or past nrows are zero-filled.
__device__ __forceinline__ void stage_async(uint32_t tile, const __nv_bfloat16* src, int ld, int r0, int rows, int nrows,
                                            int kc)
{
    for (int i = threadIdx.x; i < rows * 8; i += GT) {
        const int r = i >> 3, v = i & 7;
        const bool ok = r0 + r < nrows;
        const __nv_bfloat16* g = ok ? src + (size_t)(r0 + r) * ld + kc * BK + v * 8 : src;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tile + tile_off(r, v)), "l"(g),
                     "r"(ok ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int EPI>
__global__ void __launch_bounds__(GT, 1) k_gemm(GemmArgs a)
{
    extern __shared__ uint8_t dsm[];
    // two stages, each an A tile (16 KiB) and a B tile (up to 32 KiB), 128-byte aligned
    uint8_t* base = dsm + ((128u - (tc::smem_u32(dsm) & 127u)) & 127u);
    constexpr uint32_t A_BYTES = BM * BK * 2, STAGE_BYTES = A_BYTES + 256 * BK * 2;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.z * a.BN, split = blockIdx.y;
    const int bn = min(a.BN, a.N - n0); // a multiple of 16
    const uint32_t ncols = bn <= 32 ? 32u : bn <= 64 ? 64u : bn <= 128 ? 128u : 256u;
    const uint32_t mb[2] = {tc::smem_u32(&mbar[0]), tc::smem_u32(&mbar[1])};
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_sh), ncols);
    if (tid == 0) {
        tc::mbar_init(mb[0], 1);
        tc::mbar_init(mb[1], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_sh;
    const uint32_t idesc = tc::idesc_bf16_f32(BM, bn);
    const int nkc = a.K / BK;
    const int kc0 = split * a.kc_per_split, kc1 = min(nkc, kc0 + a.kc_per_split);
    const uint32_t st0 = tc::smem_u32(base);

    uint32_t parity[2] = {0u, 0u};
    bool pending[2] = {false, false};
    bool failed = false, issued = false;
    auto wait_stage = [&](int s) -> bool {
        const bool w = tc::mbar_wait(mb[s], parity[s]);
        const bool any_fail = __syncthreads_or(!w) != 0;
        if (!any_fail) {
            parity[s] ^= 1u;
            pending[s] = false;
        }
        return !any_fail;
    };
    if (kc0 < kc1) {
        stage_async(st0, a.A, a.lda, m0, BM, a.M, kc0);
        stage_async(st0 + A_BYTES, a.B, a.ldb, n0, bn, a.N, kc0);
    }
    for (int kc = kc0; kc < kc1; ++kc) {
        const int s = (kc - kc0) & 1;
        const uint32_t sa = st0 + (uint32_t)s * STAGE_BYTES, sb = sa + A_BYTES;
        if (kc + 1 < kc1) {
            // the other stage is free once the MMAs of chunk kc - 1 are done
            if (pending[s ^ 1] && !wait_stage(s ^ 1)) {
                failed = true;
                break;
            }
            tc::fence_after_sync();
            const uint32_t na = st0 + (uint32_t)(s ^ 1) * STAGE_BYTES;
            stage_async(na, a.A, a.lda, m0, BM, a.M, kc + 1);
            stage_async(na + A_BYTES, a.B, a.ldb, n0, bn, a.N, kc + 1);
            cp_async_wait<2>(); // this thread's copies of chunk kc are in
        } else {
            cp_async_wait<0>();
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)
                tc::mma_bf16(tbase, tc::smem_desc(sa + 256u * j, LBO, SBO), tc::smem_desc(sb + 256u * j, LBO, SBO),
                             idesc, (kc > kc0 || j > 0) ? 1u : 0u);
            tc::mma_commit(mb[s]);
        }
        pending[s] = true;
        issued = true;
    }
    cp_async_wait<0>(); // no copy outlives the loop
    for (int s = 0; s < 2; ++s)
        if (!failed && pending[s] && !wait_stage(s)) failed = true;
    bool drained = true; // every committed MMA group has completed
    if (failed)
        for (int s = 0; s < 2; ++s)
            if (pending[s] && !wait_stage(s)) drained = false; // the MMAs still in flight, once more
    if (!drained && tid == 0) atomicOr(a.err, 2); // MMAs may still run: the context is poisoned
    tc::fence_after_sync();

    if (!failed) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < bn; c += 8) {
            float v[8];
            if (issued) {
                tc::tmem_ld8(trow + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = 0.f;
            }
            if (m >= a.M) continue;
            const int n = n0 + c;
            if (EPI == GEMM_F32) {
                float* dst = a.C + (size_t)split * a.split_stride + (size_t)m * a.ldc + n;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (n + i < a.n_store) dst[i] = v[i];
            } else if (EPI == GEMM_BIAS_RELU_BF16) {
                __nv_bfloat16* dst = a.Cb + (size_t)m * a.ldc + n;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (n + i < a.n_store) dst[i] = __float2bfloat16_rn(fmaxf(v[i] + a.bias[n + i], 0.f));
            } else { // GEMM_BIAS_NCHW_F32: image-major output [m / hw][n][m % hw]
                const int img = m / a.out_hw, px = m - img * a.out_hw;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (n + i < a.n_store)
                        a.C[((size_t)img * a.n_store + n + i) * a.out_hw + px] = v[i] + a.bias[n + i];
            }
        }
    } else if (tid == 0) {
        atomicOr(a.err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

} // namespace

int gemm_check(const GemmArgs& a)
{
    if (!a.A || !a.B || !a.err || a.M < 1 || a.N < 16 || a.N % 16 || a.K < BK || a.K % BK || a.lda < a.K ||
        a.ldb < a.K || a.lda % 8 || a.ldb % 8 || a.BN < 16 || a.BN > 256 || a.BN % 16 || a.kc_per_split < 1 ||
        a.n_store < 1)
        return SF_ERR_ARG;
    if (((uintptr_t)a.A | (uintptr_t)a.B) & 15) return SF_ERR_ARG;
    return SF_OK;
}

constexpr int GEMM_SMEM = 2 * (BM * BK * 2 + 256 * BK * 2) + 128;

template <int EPI>
void launch_epi(const GemmArgs& a, dim3 grid, cudaStream_t st)
{
    // the dynamic shared-memory limit is a function attribute of each device: set once per device
    static std::mutex mu;
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr[dev] &&
            cudaFuncSetAttribute(k_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM) == cudaSuccess)
            attr[dev] = true;
    }
    k_gemm<EPI><<<grid, GT, GEMM_SMEM, st>>>(a);
}

cudaError_t launch_gemm(const GemmArgs& a, int epi, int splits, cudaStream_t st)
{
    dim3 grid((a.M + BM - 1) / BM, splits, (a.N + a.BN - 1) / a.BN);
    if (epi == GEMM_F32)
        launch_epi<GEMM_F32>(a, grid, st);
    else if (epi == GEMM_BIAS_RELU_BF16)
        launch_epi<GEMM_BIAS_RELU_BF16>(a, grid, st);
    else
        launch_epi<GEMM_BIAS_NCHW_F32>(a, grid, st);
    return cudaGetLastError();
}

} // namespace sfk
