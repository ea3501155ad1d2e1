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

// Radix-2 decimation-in-frequency butterflies of one stage (span S) on NP values; the
// twiddle of butterfly K at span S is exp(-2 pi i K / (2 S)) = w32^(K * 16 / S).
template <int NP, int S, int B, int K>
__device__ __forceinline__ void dif_bfly(float2 (&a)[NP]) {
  const float2 u = a[B + K], v = a[B + K + S];
  a[B + K] = make_float2(u.x + v.x, u.y + v.y);
  a[B + K + S] = twiddle32<K * (16 / S)>(make_float2(u.x - v.x, u.y - v.y));
  if constexpr (K + 1 < S) dif_bfly<NP, S, B, K + 1>(a);
}
template <int NP, int S, int B>
__device__ __forceinline__ void dif_stage(float2 (&a)[NP]) {
  dif_bfly<NP, S, B, 0>(a);
  if constexpr (B + 2 * S < NP) dif_stage<NP, S, B + 2 * S>(a);
}
// In-place 32-point DFT (forward, exp(-i)); output k holds frequency bitrev5(k).
__device__ __forceinline__ void fft32_dif(float2 (&a)[32]) {
  dif_stage<32, 16, 0>(a);
  dif_stage<32, 8, 0>(a);
  dif_stage<32, 4, 0>(a);
  dif_stage<32, 2, 0>(a);
  dif_stage<32, 1, 0>(a);
}
// In-place 16-point DFT (forward, exp(-i)); output k holds frequency bitrev4(k).
__device__ __forceinline__ void fft16_dif(float2 (&a)[16]) {
  dif_stage<16, 8, 0>(a);
  dif_stage<16, 4, 0>(a);
  dif_stage<16, 2, 0>(a);
  dif_stage<16, 1, 0>(a);
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
