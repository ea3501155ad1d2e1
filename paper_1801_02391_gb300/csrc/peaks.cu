// Peak-rate probes of the GPU (libfrbx_peaks): the FP32 FMA pipe, scalar fma.rn.f32 and packed
// fma.rn.f32x2, and the tcgen05 tensor pipe, dense kind::f16 (BF16) and kind::f8f6f4 (E4M3)
// MMAs of M = 128, N = 256 with FP32 accumulation in tensor memory.  The bench divides its
// kernels' rates by these measured numbers; nothing of the search runs here.  Declarations and
// the contract: include/frbx_peaks.h.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/frbx_peaks.h"
#include "tc_common.cuh"

namespace {

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 16;      // independent accumulators per thread
constexpr int kMmaN = 256;          // MMA N (TMEM columns of the accumulator)
constexpr int kMmaSmem = 160 << 10; // dynamic shared memory: keeps one CTA per SM
constexpr long long kWaitCycles = 4000000000LL;

__global__ void __launch_bounds__(kFmaThreads) k_peak_fma(float *sink, int iters, float a, float b) {
  float x[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += x[k];
  if (s == -1.f) sink[0] = s;  // never true; keeps the chains alive
}

__global__ void __launch_bounds__(kFmaThreads) k_peak_fma2(float *sink, int iters, float a, float b) {
  uint64_t x[kFmaChains / 2], av, bv;
  asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
  for (int k = 0; k < kFmaChains / 2; ++k) {
    const float lo = (float)(threadIdx.x + 2 * k) * 1e-3f, hi = (float)(threadIdx.x + 2 * k + 1) * 1e-3f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x[k]) : "f"(lo), "f"(hi));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains / 2; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[k]) : "l"(av), "l"(bv));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kFmaChains / 2; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[k]));
    s += lo + hi;
  }
  if (s == -1.f) sink[0] = s;
}

// One CTA per SM; one thread issues `iters` x 4 MMAs (one 64-wide BF16 or 128-wide E4M3 K atom
// per 4) into one accumulator, then waits (bounded) for their completion.
template <bool kFp8>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, int *err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_done;
  __shared__ uint32_t tmem_base;
  unsigned char *sA = smem;                       // 128 rows x 128 B
  unsigned char *sB = smem + frbx::tc::kAtomBytes;  // 256 rows x 128 B
  // operands: small finite values from a hash of the byte index (E4M3 bytes below 0x38, BF16
  // exponents near 1), so the pipe does real work on non-zero data
  for (int i = threadIdx.x; i < (128 + kMmaN) * 128 / 4; i += blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u + blockIdx.x * 40503u;
    h ^= h >> 15;
    const uint32_t v = kFp8 ? (h & 0x37373737u) : ((h & 0x007F007Fu) | 0x3F003F00u);
    reinterpret_cast<uint32_t *>(sA)[i] = v;
  }
  if (threadIdx.x == 0) {
    frbx::tc::mbar_init(&bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(frbx::tc::su32(&tmem_base)),
                 "r"(kMmaN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    // D = F32; A, B = BF16 (format 1, kind::f16) or E4M3 (format 0, kind::f8f6f4); K-major
    const uint32_t ab = kFp8 ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
                           ((uint32_t)(frbx::tc::kRows >> 4) << 24);
    const uint64_t a0 = frbx::tc::desc_sw128(frbx::tc::su32(sA)), b0 = frbx::tc::desc_sw128(frbx::tc::su32(sB));
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t o = (uint64_t)((kk * 32) >> 4);
        const uint32_t acc = (i | kk) ? 1u : 0u;
        if (kFp8)
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(tmem), "l"(a0 + o), "l"(b0 + o), "r"(idesc), "r"(acc) : "memory");
        else
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(tmem), "l"(a0 + o), "l"(b0 + o), "r"(idesc), "r"(acc) : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(frbx::tc::su32(&bar_done)) : "memory");
    if (!frbx::tc::mbar_wait(&bar_done, 0, nullptr, kWaitCycles)) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kMmaN) : "memory");
}

}  // namespace

extern "C" int frbx_peak_probe(int32_t kind, int32_t iters, double *tflops, double *ms, void *stream) {
  if (!tflops || !ms || iters < 1 || kind < 0 || kind > 3) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -3;
  float *sink = nullptr;
  int *err = nullptr;
  if (cudaMalloc(&sink, 256) != cudaSuccess) return -2;
  err = reinterpret_cast<int *>(sink + 16);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(sink, 0, 256, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double flop = 0;
  auto launch = [&](int it) -> cudaError_t {
    if (kind <= 1) {
      const int blocks = n_sm * 8;  // 64 warps per SM
      if (kind == 0)
        k_peak_fma<<<blocks, kFmaThreads, 0, st>>>(sink, it, 0.9999f, 1e-4f);
      else
        k_peak_fma2<<<blocks, kFmaThreads, 0, st>>>(sink, it, 0.9999f, 1e-4f);
      flop = 2.0 * blocks * kFmaThreads * (double)it * kFmaChains;
    } else {
      const bool fp8 = kind == 3;
      auto kern = fp8 ? k_peak_mma<true> : k_peak_mma<false>;
      cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
      if (r != cudaSuccess) return r;
      kern<<<n_sm, 128, kMmaSmem, st>>>(it, err);
      flop = 2.0 * 128 * kMmaN * (fp8 ? 32 : 16) * 4.0 * (double)it * n_sm;
    }
    return cudaGetLastError();
  };
  if (e == cudaSuccess) e = launch(iters / 8 + 1);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = launch(iters);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  int bad = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(&bad, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -3;
  }
  if (bad) return -5;
  *ms = t;
  *tflops = flop / (t * 1e-3) / 1e12;
  return 0;
}
