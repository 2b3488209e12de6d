// Inline-PTX helpers for the 5th-generation tensor cores of sm_103a
// (tcgen05: MMA issued by one thread, operands in shared memory, accumulator
// in tensor memory), mbarriers with bounded waits, and the descriptors they
// take.  Only what the half-step kernels use: cta_group::1, dense
// kind::tf32 and kind::f16 (BF16 inputs) with an FP32 accumulator, K-major
// operands in the no-swizzle canonical layout.
//
// Canonical K-major layout without swizzle (A: M x K, B: N x K).  The matrix
// is tiled into "core matrices" of 8 rows x 16 bytes (8 rows x 4 TF32 or
// 8 BF16 values), each stored as 128 contiguous bytes, row r of the core
// matrix at byte 16 r.  A shared-memory descriptor gives the start address,
// the byte distance between core matrices adjacent along K (leading byte
// offset, LBO) and between core matrices adjacent along M or N (stride byte
// offset, SBO).  One MMA instruction consumes 32 bytes of K per row (8 TF32
// or 16 BF16 values: two core matrices along K).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hermite {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (64 bits): start address >> 4 in bits
// 0-13, LBO >> 4 in bits 16-29, SBO >> 4 in bits 32-45, descriptor version 1
// in bits 46-47, base offset 0, layout type 0 (no swizzle) in bits 61-63.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor (32 bits) of a dense MMA with an FP32 accumulator
// and K-major A and B: D format F32 (1) in bits 4-5, A and B formats in bits
// 7-9 and 10-12 (kind::f16: 0 F16, 1 BF16; kind::tf32: 2 TF32), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
enum : uint32_t { kFmtBF16 = 1, kFmtTF32 = 2 };
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int m, int n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// ---- tensor memory --------------------------------------------------------
// Allocation by one whole warp; the TMEM address is written to `slot` (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- MMA (issued by a single thread) ---------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T; accumulate = 0 overwrites D.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on the mbarrier when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

// ---- ordering ---------------------------------------------------------------
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy); followed by a CTA barrier before the MMA.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}
// Waits for the phase with parity `phase` to complete, giving up after
// `max_tries` polls (each poll may suspend the thread briefly).  Returns
// false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase, uint32_t max_tries) {
  const uint32_t a = smem_addr(mbar);
  for (uint32_t i = 0; i < max_tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---- tensor memory -> registers --------------------------------------------
// Each thread of a warp reads 16 consecutive 32-bit columns of its own lane
// (lane = 32 * (warp % 4) + lane id, the warp's quarter of the 128 lanes);
// taddr carries the quarter's first lane in bits 16-31 and the column in 0-15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- operand splitting --------------------------------------------------------
// TF32 pieces: hi = x rounded to nearest (ties away) to 10 mantissa bits,
// lo = the remainder rounded the same way (x - hi is exact in FP32).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

}  // namespace tc
}  // namespace hermite
