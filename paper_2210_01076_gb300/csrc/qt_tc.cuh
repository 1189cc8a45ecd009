// qt_tc.cuh -- 5th-generation tensor core (tcgen05) and tensor memory helpers
// for the fused-block op of the complex64 register kernel (sm_100a family).
//
// The block op multiplies the tile, viewed as a 128 x 64 fp32 matrix A (row:
// the seven tile bits outside the block; column: the block's 32 amplitudes,
// re and im), by the block's 64 x 64 real embedding B^T, D = A B^T, with
// tcgen05.mma kind::tf32 (M = 128, N = 64, K = 8 per instruction), the
// accumulator D in tensor memory.  fp32 accuracy comes from the 3xTF32 split
// (A = Ah + Al, B = Bh + Bl, D = Ah Bh + Ah Bl + Al Bh): each operand is
// rounded to tf32 and the residual rounded again.
//
// Shared-memory operands are K-major with the 128-byte swizzle: each row of a
// 32-element (128-byte) K atom is stored at row * 128 bytes inside 1024-byte
// groups of 8 rows, its 16-byte chunk c at chunk c ^ (row % 8).  A matrix
// descriptor addresses one K step (8 tf32 = 32 bytes) of such an atom: start
// address, stride between 8-row groups (1024 bytes), the sm_100 version bits
// and the swizzle mode.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace qt {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Tensor-memory columns held by one CTA: the 128 x 64 fp32 accumulator.
constexpr uint32_t kTmemCols = 64;

// One warp allocates; the address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy writes to shared memory become visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Instruction descriptor, kind::tf32: D fp32, A and B tf32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// Shared-memory descriptor of a K-major, 128-byte-swizzled operand at
// shared address `addr` (1024-byte aligned atom base plus the K step's byte
// offset inside the 128-byte row).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);         // start address
    d |= uint64_t(1) << 16;                       // leading byte offset (unused by this layout)
    d |= uint64_t((1024u >> 4) & 0x3FFFu) << 32;  // stride byte offset: 8 rows x 128 B
    d |= uint64_t(1) << 46;                       // descriptor version (sm_100)
    d |= uint64_t(2) << 61;                       // 128-byte swizzle
    return d;
}

// D (+)= A B^T for one K step; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 32 columns of 32-bit values of the warp's 32 tensor-memory lanes: thread i
// of the warp reads lane (taddr's lane + i), columns taddr's column .. +31.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// fp32 -> tf32, round to nearest (ties away from zero), in a 32-bit container.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace qt
