// sf_tc.cuh -- Blackwell (sm_103a) tensor-core primitives written as inline
// PTX: shared-memory matrix descriptors, the tcgen05 instruction descriptor
// for BF16 x BF16 -> FP32, tensor-memory allocation, MMA issue and commit,
// tensor-memory loads, TMA tile copies, and mbarrier waits with a time limit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfk {

namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major operand without swizzling: the
// tile is made of 8-row x 16-byte core matrices stored contiguously (128 B
// each); `lbo` is the byte distance between core matrices adjacent along K,
// `sbo` between core matrices adjacent along M (or N). Bits: start address
// >> 4 in [0, 14), lbo >> 4 in [16, 30), sbo >> 4 in [32, 46), descriptor
// version 1 in [46, 48), base offset 0, swizzle mode 0 (none) in [61, 64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout that a TMA tile copy with CU_TENSOR_MAP_SWIZZLE_128B writes: rows of
// 128 bytes (64 BF16 along K), the 16-byte chunks of row r stored at chunk
// index (chunk ^ (r & 7)), 8-row groups 1024 bytes apart (sbo). The tile must
// start on a 1024-byte boundary; a K step inside the 128-byte row advances the
// start address (the swizzle is applied to the address bits). The leading
// byte offset is not used by this layout (field set to 1). Swizzle mode 2
// (128-byte) in [61, 64), descriptor version 1 in [46, 48), base offset 0.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16 with BF16 A and B (both
// K-major) and an FP32 accumulator: D format F32 (bits [4, 6) = 1), A and B
// format BF16 ([7, 10) = 1, [10, 13) = 1), N >> 3 in [17, 23), M >> 4 in
// [24, 29).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory allocation of `ncols` columns (a power of two >= 32) by one
// whole warp; the base address is written to shared memory at dst.
__device__ __forceinline__ void tmem_alloc(uint32_t dst_saddr, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_saddr), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core's (async proxy) reads.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D (tensor memory) = A * B^T (+ D if accumulate), one M x N x 16 step.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// Arrives once on the mbarrier when every MMA this thread issued so far has
// completed.
__device__ __forceinline__ void mma_commit(uint32_t mbar_saddr)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_saddr)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t saddr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival on the mbarrier that also expects `bytes` of asynchronous
// copies (TMA) to complete on it before the phase can end.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t saddr, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr), "r"(bytes) : "memory");
}

// TMA: copies the box of a 2-D tensor map at coordinates (x, y) (x along the
// contiguous dimension, in elements; x times the element size must be a
// multiple of 16 bytes) into shared memory at dst, completing `box bytes` of
// transactions on the mbarrier. Out-of-bound elements are filled with zeros.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t saddr, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(saddr), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// limit_cycles of SM clock (about one second by default); returns false on
// timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t saddr, uint32_t parity, long long limit_cycles = 2000000000LL)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(saddr, parity))
        if (clock64() - t0 > limit_cycles) return false;
    return true;
}

// Eight consecutive FP32 columns of this thread's tensor-memory lane (the
// warp covers 32 lanes starting at the lane field of taddr).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

} // namespace tc

} // namespace sfk
