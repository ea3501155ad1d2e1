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

// The work item a CTA fits: one (baseline, time tile of TT APs, DM trial) of one scan.  Plain
// launches take it from blockIdx = (DM trial, time tile, baseline) -- DM trials vary fastest, so
// the CTAs resident at one time read the same stretch of the cube and its dispersion halo from
// L2; batched launches claim items from a device counter across all scans of a setup.
struct ItemCtx {
  const float2 *vis;  // cube of the scan [n_bl][T][C]
  frbx_seg *out;      // its series [n_bl][n_dm][S_tot]
  const int *nval;    // its valid-segment counts [n_dm][n_win]
  const int *woff;    // first slot of each window in one of its series [n_win]
  int T, S_tot, bl, d, tt;
};

__device__ __forceinline__ ItemCtx plain_item(const FitArgs &a) {
  ItemCtx c;
  c.vis = a.vis;
  c.out = a.out;
  c.nval = a.n_valid;
  c.woff = a.win_off;
  c.T = a.T;
  c.S_tot = a.S_tot;
  c.bl = blockIdx.z;
  c.d = blockIdx.x;
  c.tt = blockIdx.y;
  return c;
}

// Global item -> scan and coordinates (items of scan k are [item0[k], item0[k + 1])).
__device__ __forceinline__ ItemCtx batch_item(const FitArgs &a, const BatchScan *scans, int n_scans, long long item) {
  int lo = 0, hi = n_scans;  // scans[lo].item0 <= item < scans[hi].item0
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (scans[mid].item0 <= item) lo = mid; else hi = mid;
  }
  const BatchScan &sc = scans[lo];
  const long long local = item - sc.item0;
  ItemCtx c;
  c.vis = sc.vis;
  c.out = sc.out;
  c.nval = sc.n_valid;
  c.woff = sc.win_off;
  c.T = sc.T;
  c.S_tot = sc.S_tot;
  c.d = (int)(local % a.n_dm);
  const long long r = local / a.n_dm;
  c.tt = (int)(r % sc.n_tt);
  c.bl = (int)(r / sc.n_tt);
  return c;
}

// Window w contributes the slots s in [s_lo, s_lo + cnt) whose start k0 = s * step(l) falls in
// the tile; slots at or beyond the DM's valid count are written as empty.
struct TileWin {
  int s_lo[kMaxWin], cum[kMaxWin + 1], len[kMaxWin], off[kMaxWin], nval[kMaxWin];
};

__device__ __forceinline__ void tile_windows(const FitArgs &a, const ItemCtx &c, TileWin &tw) {
  if (threadIdx.x == 0) {
    const int t0 = c.tt * a.TT;
    int n = 0;
    for (int w = 0; w < a.n_win; ++w) {
      const int l = a.win_len[w], step = max(1, l / 2);
      const int ns = c.T >= l ? (c.T - l) / step + 1 : 0;
      const int lo = (t0 + step - 1) / step, hi = min((t0 + a.TT + step - 1) / step, ns);
      tw.s_lo[w] = lo;
      tw.cum[w] = n;
      n += max(0, hi - lo);
      tw.len[w] = l;
      tw.off[w] = c.woff[w];
      tw.nval[w] = c.nval[c.d * a.n_win + w];
    }
    tw.cum[a.n_win] = n;
  }
}

// Segment number i of this item.  List mode: rows [blockIdx.x * tile, ...) of the list.
__device__ __forceinline__ bool tile_segment(const FitArgs &a, bool list, int i, const TileWin &tw,
                                             const ItemCtx &c, Seg &s) {
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
  s.bl = c.bl;
  s.d = c.d;
  s.l = tw.len[w];
  s.k0 = sidx * max(1, s.l / 2);
  s.valid = sidx < tw.nval[w];
  s.out = ((long long)s.bl * a.n_dm + s.d) * c.S_tot + tw.off[w] + sidx;
  return true;
}

// Eq. 3 gather of one segment into X (row stride xs), weighted and rotated.
__device__ __forceinline__ void gather_segment(const FitArgs &a, const ItemCtx &c, const Seg &s, float2 *X, int xs) {
  const int *dk = a.dk + (size_t)s.d * a.C;
  const size_t base = (size_t)s.bl * c.T + s.k0;
  for (int p = threadIdx.x; p < a.C; p += blockDim.x) {
    const float2 *src = c.vis + (base + __ldg(dk + p)) * a.C + p;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int i = 0; i < s.l; ++i) {
      const float2 v = __ldg(src + (size_t)i * a.C);
      acc.x += v.x;
      acc.y += v.y;
    }
    const int n = p / a.J, j = p - n * a.J;
    X[n * xs + j] = cmul(acc, __ldg(a.wrot + p));
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

__device__ __forceinline__ void write_fit(const FitArgs &a, frbx_seg *out, const Seg &s, float bp, int bi) {
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
  out[s.out] = r;
}

}  // namespace frbx
