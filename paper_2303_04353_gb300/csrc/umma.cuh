// Fifth-generation tensor core (tcgen05) primitives for sm_103a in inline
// PTX: tensor-memory allocation, the shared-memory matrix descriptor and the
// instruction descriptor of a bf16 x bf16 -> FP32 MMA, the MMA itself, its
// completion signal on an mbarrier, and tensor-memory loads.
#pragma once
#include <cstdint>

namespace ddg {
namespace umma {

// Allocate `ncols` tensor-memory columns (a power of two, >= 32) for this
// CTA; executed by one whole warp.  The base address is written to shared
// memory at `dst`.
__device__ __forceinline__ void alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst),
                 "r"(ncols)
                 : "memory");
}

// Let other CTAs on this SM allocate (this CTA allocates once).
__device__ __forceinline__ void relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Order tensor-core operations around a thread synchronisation (a barrier
// or an mbarrier hand-off): `before` on the signalling side, `after` on the
// waiting side.
__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory descriptor of a K-major operand tile with 32-byte
// swizzling: rows of 32 bytes (16 bf16 along k) stored one after another,
// their two 16-byte halves exchanged in rows 4-7 of every 8 (the layout a
// TMA copy with CU_TENSOR_MAP_SWIZZLE_32B writes).  Groups of 8 rows are
// 256 bytes apart.  The tile must start on a 256-byte boundary.
//   bits  0-13  start address / 16
//   bits 16-29  leading-dimension byte offset / 16 (not used by K-major
//               swizzled layouts whose k extent is one swizzle row)
//   bits 32-45  stride-dimension byte offset / 16: 256 bytes
//   bits 46-48  descriptor version 1
//   bits 61-63  swizzle mode 6: 32 bytes
__device__ __forceinline__ uint64_t desc_k_sw32(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)6 << 61);
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major) and
// an FP32 accumulator, for an M x N x 16 product.
//   bits  4-5  accumulator format 1: FP32
//   bits  7-9  A format 1: bf16        bits 10-12  B format 1: bf16
//   bit  15/16 A/B major: 0 = K-major
//   bits 17-22 N / 8                   bits 24-28  M / 16
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

// D[tmem] = A B^T (accumulate = 0) or D += A B^T, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One arrival on the mbarrier once every tcgen05 operation this thread has
// issued so far has completed.
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// One to four loads of 4 consecutive 32-bit columns each (at t[0..N-1])
// for the 32 tensor-memory lanes of this warp's quadrant (lane i of the
// warp receives lane quadrant base + i), then one wait, all in one asm
// statement so that the registers are not read before the data has
// arrived: a group of diagonals pays the tensor-memory latency once.
__device__ __forceinline__ void ld_x4_n(const uint32_t (&t)[1], uint32_t (&r)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(t[0])
        : "memory");
}
__device__ __forceinline__ void ld_x4_n(const uint32_t (&t)[2], uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%8];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%9];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(t[0]), "r"(t[1])
        : "memory");
}
__device__ __forceinline__ void ld_x4_n(const uint32_t (&t)[3], uint32_t (&r)[12]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%12];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%13];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%14];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
        : "r"(t[0]), "r"(t[1]), "r"(t[2])
        : "memory");
}
__device__ __forceinline__ void ld_x4_n(const uint32_t (&t)[4], uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4, %5, %6, %7}, [%17];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%18];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12, %13, %14, %15}, [%19];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3])
        : "memory");
}

}  // namespace umma
}  // namespace ddg
