// nep_tc.cuh -- Blackwell (sm_100 family) tensor-core building blocks in
// inline PTX: TMEM allocation, tcgen05.mma (kind::f16 with BF16 or FP16
// operands and FP32 accumulation), commit to an mbarrier, bounded mbarrier waits, TMEM
// loads and the proxy/ordering fences they need.
//
// Operands live in shared memory in the canonical K-major layout without
// swizzling: 8-row x 16-byte core matrices stored as 128 contiguous bytes,
// core matrices adjacent along K `lbo` bytes apart and along M/N `sbo` bytes
// apart.  All operand tiles here have K = 32 (four core matrices along K):
// lbo = 128, sbo = 512; the second K step of 16 starts 256 bytes in.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nep {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of a [rows x 32] K-major BF16 tile.
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int row, int k)
{
    return (uint32_t)(((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, the fixed version field (bits 46-48 = 0b001), no
// swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D in FP32, A and B in BF16, both
// K-major, dense, M x N tile.
__host__ __device__ __forceinline__ uint32_t idesc_bf16_f32(int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;                         // D format: FP32
    d |= 1u << 7;                         // A format: BF16
    d |= 1u << 10;                        // B format: BF16
    d |= (uint32_t)((N >> 3) & 0x3F) << 17;
    d |= (uint32_t)((M >> 4) & 0x1F) << 24;
    return d;
}

// The same with A and B in FP16 (both operands of one MMA have one type).
__host__ __device__ __forceinline__ uint32_t idesc_f16_f32(int M, int N)
{
    uint32_t d = 0;
    d |= 1u << 4;  // D format: FP32; A and B format fields 0: FP16
    d |= (uint32_t)((N >> 3) & 0x3F) << 17;
    d |= (uint32_t)((M >> 4) & 0x1F) << 24;
    return d;
}

// ---- TMEM allocation (one full warp executes these) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_result, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_result)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- MMA (one thread issues; the operand types come from idesc) ----
__device__ __forceinline__ void mma_kind_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate ? 1 : 0)
        : "memory");
}

// Arrive once on the mbarrier when every earlier tcgen05 operation of this
// thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Waits until the phase with the given parity has completed.  Gives up after
// max_polls polls and returns false, so a lost arrival can never hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_polls)
{
    const uint32_t a = smem_u32(mbar);
    for (uint32_t it = 0; it < max_polls; ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---- fences ----
// generic-proxy writes to shared memory -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- TMEM -> registers: 32 lanes x 8 consecutive 32-bit columns ----
// The destination words may only be read after tmem_ld_wait().
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace nep
