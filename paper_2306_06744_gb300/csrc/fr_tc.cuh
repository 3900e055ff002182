// fr_tc.cuh -- inline-PTX wrappers for the fifth-generation tensor cores (tcgen05) of sm_103a:
// tensor-memory (TMEM) allocation, shared-memory matrix descriptors, BF16 MMA with FP32
// accumulation in TMEM, completion through an mbarrier with a bounded wait, and TMEM loads.
//
// Operand layout used throughout (no swizzle, K-major): a matrix of R rows and 64 BF16 columns is
// stored as core matrices of 8 rows x 8 columns (8 x 16 bytes, 128 contiguous bytes), element
// (r, k) at byte (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.  Adjacent core
// matrices along K are 128 bytes apart (leading byte offset), along the rows 1024 bytes apart
// (stride byte offset).  One MMA instruction consumes K = 16, i.e. two core matrices along K.
#pragma once
#include <cstdint>

namespace frg {
namespace tc {

constexpr uint32_t LBO = 128, SBO = 1024;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) in the 64-column operand layout above
__device__ __forceinline__ uint32_t canon_off(int r, int k) {
  return uint32_t((r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2);
}
// the same layout for a tile of `ncols` columns (a multiple of 8): 8-row groups ncols*16 bytes apart
__device__ __forceinline__ uint32_t canon_off_w(int r, int k, int ncols) {
  return uint32_t((r >> 3) * (ncols * 16) + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// descriptor version 1 at bit 46, base offset 0, relative leading offsets, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo = SBO) {
  return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((LBO >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}

// instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// D[M x N] (+)= A[M x 16] * B[N x 16]^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(uint32_t(accumulate))
      : "memory");
}

// the mbarrier receives one arrival when every MMA issued so far by this thread has completed
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// waits for the completion of the phase with the given parity; gives up after `limit` clock
// cycles and returns false.  Each round first tests without blocking, then checks the clock, then
// waits with try_wait (which may suspend the thread for a while inside the instruction), so a
// limit shorter than the completion's latency is honoured.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
}

// bulk copy (TMA, non-tensor) of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory; the issuing thread first announces the bytes on the mbarrier, whose
// phase then completes when they have landed
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// makes this thread's generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// warp-collective: allocate `ncols` TMEM columns (a power of two >= 32); the base address is
// written to the shared-memory word at `slot`
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// warp-collective: 16 consecutive 32-bit columns of 32 lanes; thread i of the warp receives the
// lane (lane field of taddr) + i
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc
}  // namespace frg
