// tcgen05 / mbarrier helpers shared by the tensor-core kernels (inline PTX, sm_103a).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace frbx {
namespace tc {

constexpr int kRows = 128;               // M of one MMA tile (TMEM lanes)
constexpr int kAtomBytes = kRows * 128;  // one 64-wide BF16 K atom of a 128-row tile (16 KB)

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(su32(b)) : "memory");
}
// Bounded wait for the completion of the phase with the given parity.  Returns false on
// timeout or when another role raised the abort flag (abort_flag may be null).  After a first
// probe, each try_wait may suspend the warp for up to kWaitSuspendNs (it wakes when the phase
// completes), so a waiting role takes no issue slots from the others; the limit and the abort
// flag are checked between probes.
constexpr uint32_t kWaitSuspendNs = 20000;
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag,
                                          long long limit) {
  const uint32_t addr = su32(b);
  uint32_t ok;
  asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
               : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
  if (ok) return true;
  const long long t0 = clock64();
  for (;;) {
    asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n selp.b32 %0, 1, 0, P;\n}\n"
                 : "=r"(ok) : "r"(addr), "r"(parity), "r"(kWaitSuspendNs) : "memory");
    if (ok) return true;
    if (abort_flag && *abort_flag) return false;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// byte offset of bf16 element (row, k) in a 128-row tile of 64-wide K atoms, 128B swizzle
__device__ __forceinline__ uint32_t a_offset(int row, int k) {
  return (uint32_t)((k >> 6) * kAtomBytes + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k & 63) >> 3) ^ (row & 7)) << 4) + (k & 7) * 2);
}

// byte offset of FP8 element (row, k): the same 128-byte rows and swizzle, 128 values per row
__device__ __forceinline__ uint32_t a_offset8(int row, int k) {
  return (uint32_t)((k >> 7) * kAtomBytes + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k & 127) >> 4) ^ (row & 7)) << 4) + (k & 15));
}

// true in exactly one lane of the (fully active) warp
__device__ __forceinline__ bool elect_one() {
  uint32_t p;
  asm volatile("{\n .reg .b32 rx;\n .reg .pred px;\n elect.sync rx|px, %1;\n selp.u32 %0, 1, 0, px;\n}\n"
               : "=r"(p) : "r"(0xffffffffu));
  return p != 0;
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Named barrier that also returns the OR of a predicate over its n threads (a uniform
// decision for the whole role).
__device__ __forceinline__ bool named_sync_or(int id, int n, bool pred) {
  uint32_t out;
  asm volatile("{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
               : "=r"(out) : "r"((uint32_t)pred), "r"(id), "r"(n) : "memory");
  return out != 0;
}

// 16-byte aligned global -> shared bulk copy whose completion is counted on an mbarrier
// (the barrier must expect the bytes first).
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

}  // namespace tc
}  // namespace frbx
