// sf_gemm.cu -- BF16 x BF16 -> FP32 matrix product on the fifth-generation
// tensor cores (tcgen05), the one contraction of the warm-start network
// (every convolution of its forward and backward pass is lowered to it).
//
//   C[M, N] = A[M, K] * B[N, K]^T      (both operands K-major, K % 64 == 0)
//
// One CTA of four warps computes a 128 x BN tile (BN <= 256, a multiple of
// 16) over a range of K. Thread 0 runs the main loop alone: per 64-wide K
// chunk it starts two TMA tile copies (A: 128 rows, B: BN rows, 128 bytes of
// K each, in the 128-byte swizzle layout; rows past the matrix arrive as
// zeros) that complete on the stage's "full" mbarrier, waits for them, issues
// four 128 x bn x 16 MMAs into a tensor-memory accumulator and commits them to
// the stage's "empty" mbarrier. Two stages alternate: the copies of chunk
// k + 1 run while the MMAs of chunk k do, and a stage is refilled once its
// empty barrier reports the MMAs that read it done. The epilogue reads the
// accumulator lane by lane (tcgen05.ld, warp w owns rows 32w .. 32w + 31) and
// applies one of the epilogues below. Split-K (grid.y) writes FP32 partial
// products that a fixed-order reduction sums, so results do not depend on
// scheduling.
//
// Every mbarrier wait gives up after about one second; the CTA then waits
// once more for its copies and MMAs in flight, frees its tensor memory,
// raises the error word (bit 0) and returns. If that second wait gives up
// too, copies or MMAs may still be writing the shared and tensor memory that
// the CTA released: bit 1 is raised as well, and the CUDA context is to be
// treated as poisoned (the process should not launch further work on it).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "sf_launch.h"
#include "sf_tc.cuh"

namespace sfk {

namespace {

constexpr int GT = 128;  // threads per CTA
constexpr int BM = 128;  // rows per tile
constexpr int BK = 64;   // K per chunk (128 bytes of BF16: one swizzle row)
constexpr uint32_t A_BYTES = BM * BK * 2;             // 16 KiB
constexpr uint32_t B_BYTES_MAX = 256 * BK * 2;        // 32 KiB
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES_MAX; // a multiple of 1024

template <int EPI>
__global__ void __launch_bounds__(GT, 1) k_gemm(GemmArgs a, const __grid_constant__ CUtensorMap tmA,
                                                const __grid_constant__ CUtensorMap tmB)
{
    extern __shared__ uint8_t dsm[];
    // two stages, each an A tile and a B tile; the swizzle layout wants every
    // tile on a 1024-byte boundary
    uint8_t* base = dsm + ((1024u - (tc::smem_u32(dsm) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ uint32_t tmem_sh;
    __shared__ int state_sh; // bit 0: a wait gave up; bit 1: work may still be in flight; bit 2: MMAs issued
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.z * a.BN, split = blockIdx.y;
    const int bn = min(a.BN, a.N - n0); // a multiple of 16
    const uint32_t ncols = bn <= 32 ? 32u : bn <= 64 ? 64u : bn <= 128 ? 128u : 256u;
    const uint32_t fb[2] = {tc::smem_u32(&full[0]), tc::smem_u32(&full[1])};
    const uint32_t eb[2] = {tc::smem_u32(&empty[0]), tc::smem_u32(&empty[1])};
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_sh), ncols);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(fb[s], 1);
            tc::mbar_init(eb[s], 1);
        }
        state_sh = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_sh;
    const int nkc = a.K / BK;
    const int kc0 = split * a.kc_per_split, kc1 = min(nkc, kc0 + a.kc_per_split);
    const uint32_t st0 = tc::smem_u32(base);

    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(BM, bn);
        const uint32_t tx_bytes = A_BYTES + (uint32_t)a.BN * BK * 2; // whole boxes, zero-filled past the matrix
        uint32_t fpar[2] = {0u, 0u}, epar[2] = {0u, 0u};
        bool fpend[2] = {false, false}, epend[2] = {false, false}; // copies / MMAs not yet waited for
        int state = 0;
        auto load = [&](int kc, int s) {
            const uint32_t sa = st0 + (uint32_t)s * STAGE_BYTES;
            tc::mbar_arrive_expect_tx(fb[s], tx_bytes);
            tc::tma_load_2d(sa, &tmA, kc * BK, m0, fb[s]);
            tc::tma_load_2d(sa + A_BYTES, &tmB, kc * BK, n0, fb[s]);
            fpend[s] = true;
        };
        auto wait_full = [&](int s) -> bool {
            if (!tc::mbar_wait(fb[s], fpar[s])) return false;
            fpar[s] ^= 1u;
            fpend[s] = false;
            return true;
        };
        auto wait_empty = [&](int s) -> bool {
            if (!tc::mbar_wait(eb[s], epar[s])) return false;
            epar[s] ^= 1u;
            epend[s] = false;
            return true;
        };
        if (kc0 < kc1) load(kc0, 0);
        for (int kc = kc0; kc < kc1; ++kc) {
            const int s = (kc - kc0) & 1;
            if (kc + 1 < kc1) {
                // the other stage is free once the MMAs of chunk kc - 1 are done
                if (epend[s ^ 1] && !wait_empty(s ^ 1)) {
                    state = 1;
                    break;
                }
                load(kc + 1, s ^ 1);
            }
            if (!wait_full(s)) {
                state = 1;
                break;
            }
            tc::fence_after_sync();
            const uint32_t sa = st0 + (uint32_t)s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j)
                tc::mma_bf16(tbase, tc::smem_desc_sw128(sa + 32u * j), tc::smem_desc_sw128(sb + 32u * j), idesc,
                             (kc > kc0 || j > 0) ? 1u : 0u);
            tc::mma_commit(eb[s]);
            epend[s] = true;
            state |= 4;
        }
        for (int s = 0; s < 2; ++s)
            if (!(state & 1) && epend[s] && !wait_empty(s)) state |= 1;
        if (state & 1) // the copies and MMAs still in flight, once more
            for (int s = 0; s < 2; ++s) {
                if (fpend[s] && !wait_full(s)) state |= 2;
                if (epend[s] && !wait_empty(s)) state |= 2;
            }
        state_sh = state;
    }
    __syncthreads();
    tc::fence_after_sync();
    const int state = state_sh;
    const bool failed = (state & 1) != 0, issued = (state & 4) != 0;
    if ((state & 2) && tid == 0) atomicOr(a.err, 2); // work may still run: the context is poisoned

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

constexpr int GEMM_SMEM = 2 * (int)STAGE_BYTES + 1024;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); looked up once per process.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The tile map of a row-major BF16 operand [rows][ld] (K-major, K columns
// used): boxes of 64 elements along K by box_rows rows, 128-byte swizzle,
// zeros past the matrix.
bool operand_map(CUtensorMap* m, const __nv_bfloat16* X, int rows, int ld, int K, int box_rows)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI>
void launch_epi(const GemmArgs& a, const CUtensorMap& ma, const CUtensorMap& mb, dim3 grid, cudaStream_t st)
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
    k_gemm<EPI><<<grid, GT, GEMM_SMEM, st>>>(a, ma, mb);
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

cudaError_t launch_gemm(const GemmArgs& a, int epi, int splits, cudaStream_t st)
{
    alignas(64) CUtensorMap ma, mb;
    if (!operand_map(&ma, a.A, a.M, a.lda, a.K, BM) || !operand_map(&mb, a.B, a.N, a.ldb, a.K, a.BN))
        return cudaErrorInvalidValue;
    dim3 grid((a.M + BM - 1) / BM, splits, (a.N + a.BN - 1) / a.BN);
    if (epi == GEMM_F32)
        launch_epi<GEMM_F32>(a, ma, mb, grid, st);
    else if (epi == GEMM_BIAS_RELU_BF16)
        launch_epi<GEMM_BIAS_RELU_BF16>(a, ma, mb, grid, st);
    else
        launch_epi<GEMM_BIAS_NCHW_F32>(a, ma, mb, grid, st);
    return cudaGetLastError();
}

} // namespace sfk
