// Device helpers shared by the segment-fit kernels (Eq. 3 gather, argmax, output).
#pragma once

#include <climits>

#include "frbx_internal.h"

namespace frbx {

__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Keep the larger power; on equal power the lower linear cell index (m * Lm + q).
__device__ __forceinline__ void better(float &bp, int &bi, float p, int i) {
  if (p > bp || (p == bp && i < bi)) {
    bp = p;
    bi = i;
  }
}

__host__ __device__ constexpr int bitrev5(int k) {
  return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

struct Seg {
  int bl, d, l, k0;
  long long out;
  bool valid;
};

// Window ranges of the time tile a CTA fits in the implicit layout (blockIdx = (DM trial, time
// tile of TT APs, baseline)): window w contributes the slots s in [s_lo, s_lo + cnt) whose start
// k0 = s * step(l) falls in the tile; slots at or beyond the DM's valid count are written as
// empty.  DM trials vary fastest across the grid, so the CTAs resident at one time read the
// same stretch of the cube (plus its dispersion halo) from L2.
struct TileWin {
  int s_lo[kMaxWin], cum[kMaxWin + 1], len[kMaxWin], off[kMaxWin], nval[kMaxWin];
};

__device__ __forceinline__ void tile_windows(const FitArgs &a, TileWin &tw) {
  if (threadIdx.x == 0) {
    const int t0 = blockIdx.y * a.TT;
    int c = 0;
    for (int w = 0; w < a.n_win; ++w) {
      const int l = a.win_len[w], step = max(1, l / 2);
      const int ns = a.T >= l ? (a.T - l) / step + 1 : 0;
      const int lo = (t0 + step - 1) / step, hi = min((t0 + a.TT + step - 1) / step, ns);
      tw.s_lo[w] = lo;
      tw.cum[w] = c;
      c += max(0, hi - lo);
      tw.len[w] = l;
      tw.off[w] = a.win_off[w];
      tw.nval[w] = a.n_valid[blockIdx.x * a.n_win + w];
    }
    tw.cum[a.n_win] = c;
  }
}

// Segment number i of this CTA.  List mode: rows [blockIdx.x * tile, ...) of the list.
__device__ __forceinline__ bool tile_segment(const FitArgs &a, bool list, int i, const TileWin &tw, Seg &s) {
  if (list) {
    const long long r = (long long)blockIdx.x * a.tile + i;
    if (i >= a.tile || r >= a.n_seg) return false;
    const int4 row = reinterpret_cast<const int4 *>(a.seg)[r];
    s.bl = row.x;
    s.d = row.y;
    s.l = row.z;
    s.k0 = row.w;
    s.out = r;
    s.valid = true;
    return true;
  }
  if (i >= tw.cum[a.n_win]) return false;
  int w = 0;
  while (i >= tw.cum[w + 1]) ++w;
  const int sidx = tw.s_lo[w] + (i - tw.cum[w]);
  s.bl = blockIdx.z;
  s.d = blockIdx.x;
  s.l = tw.len[w];
  s.k0 = sidx * max(1, s.l / 2);
  s.valid = sidx < tw.nval[w];
  s.out = ((long long)s.bl * a.n_dm + s.d) * a.S_tot + tw.off[w] + sidx;
  return true;
}

// Eq. 3 gather of one segment into X (row stride xs), weighted and rotated.
__device__ __forceinline__ void gather_segment(const FitArgs &a, const Seg &s, float2 *X, int xs) {
  const int *dk = a.dk + (size_t)s.d * a.C;
  const size_t base = (size_t)s.bl * a.T + s.k0;
  for (int c = threadIdx.x; c < a.C; c += blockDim.x) {
    const float2 *p = a.vis + (base + __ldg(dk + c)) * a.C + c;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int i = 0; i < s.l; ++i) {
      const float2 v = __ldg(p + (size_t)i * a.C);
      acc.x += v.x;
      acc.y += v.y;
    }
    const int n = c / a.J, j = c - n * a.J;
    X[n * xs + j] = cmul(acc, __ldg(a.wrot + c));
  }
}

// Block-wide argmax of (bp, bi); thread 0 gets the result.
__device__ __forceinline__ void block_best(float &bp, int &bi, float *rp, int *ri) {
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const float p2 = __shfl_xor_sync(0xffffffffu, bp, off);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, off);
    better(bp, bi, p2, i2);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    rp[warp] = bp;
    ri[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) better(bp, bi, rp[w], ri[w]);
  }
}

__device__ __forceinline__ void write_fit(const FitArgs &a, const Seg &s, float bp, int bi) {
  frbx_seg r;
  if (s.valid && bp >= 0.f) {
    r.amp = sqrtf(bp);
    r.sbd_idx = (uint16_t)(bi >> a.log2Lm);
    r.mbd_idx = (uint16_t)(bi & (a.Lm - 1));
  } else {
    r.amp = -1.f;
    r.sbd_idx = 0;
    r.mbd_idx = 0;
  }
  a.out[s.out] = r;
}

}  // namespace frbx
