// 32-point register FFT shared by the segment-fit kernels.  Each translation unit that
// includes this header owns its copy of the twiddle table and uploads it with upload_w32().
#pragma once

#include <cmath>

#include <cuda_runtime.h>

namespace frbx {

static __constant__ float2 c_w32[32];  // exp(-2 pi i e / 32), e = 0..31

// d * exp(-2 pi i e / 32) with the trivial factors resolved at compile time.
template <int E>
__device__ __forceinline__ float2 twiddle32(float2 d) {
  if constexpr (E == 0) {
    return d;
  } else if constexpr (E == 8) {
    return make_float2(d.y, -d.x);
  } else {
    const float2 w = c_w32[E];
    return make_float2(fmaf(d.x, w.x, -d.y * w.y), fmaf(d.x, w.y, d.y * w.x));
  }
}

// Radix-2 decimation-in-frequency butterflies of one stage (span S) on 32 values.
template <int S, int B, int K>
__device__ __forceinline__ void dif_bfly(float2 (&a)[32]) {
  const float2 u = a[B + K], v = a[B + K + S];
  a[B + K] = make_float2(u.x + v.x, u.y + v.y);
  a[B + K + S] = twiddle32<K * (16 / S)>(make_float2(u.x - v.x, u.y - v.y));
  if constexpr (K + 1 < S) dif_bfly<S, B, K + 1>(a);
}
template <int S, int B>
__device__ __forceinline__ void dif_stage(float2 (&a)[32]) {
  dif_bfly<S, B, 0>(a);
  if constexpr (B + 2 * S < 32) dif_stage<S, B + 2 * S>(a);
}
// In-place 32-point DFT (forward, exp(-i)); output k holds frequency bitrev5(k).
__device__ __forceinline__ void fft32_dif(float2 (&a)[32]) {
  dif_stage<16, 0>(a);
  dif_stage<8, 0>(a);
  dif_stage<4, 0>(a);
  dif_stage<2, 0>(a);
  dif_stage<1, 0>(a);
}

static inline cudaError_t upload_w32() {
  float2 w[32];
  const double two_pi = 6.283185307179586476925286766559;
  for (int e = 0; e < 32; ++e) {
    w[e].x = (float)std::cos(two_pi * e / 32.0);
    w[e].y = (float)-std::sin(two_pi * e / 32.0);
  }
  return cudaMemcpyToSymbol(c_w32, w, sizeof(w));
}

}  // namespace frbx
