// Fringe-fit kernels: dedispersed time segment (Eq. 3), 2-D delay transform on the
// SBD x MBD grid (Eq. 5 as the 2-D DFT of Sec. 5.1) and the grid maximum, one CTA
// per tile of segments.
//
// Two kernels compute the same thing:
//  * k_fit_direct: direct DFT sums from shared-memory twiddle tables; any grid size.
//  * k_fit_fft:    four-step decomposition with a 32-point register FFT for both axes;
//                  needs Ls and Lm multiples of 32.
//      SBD: with j = 32 j1 + j2 and m = m1 + (Ls/32) m2,
//           Y(n, m) = sum_j2 w32^(j2 m2) [ sum_j1 X(n, j) wLs^(j m1) ]
//      MBD: with g = 32 g1 + g2 and q = q1 + (Lm/32) q2,
//           G(m, q) = sum_g2 w32^(g2 q2) [ sum_{n: g_n = g2 mod 32} Y(n, m) wLm^(g_n q1) ]
//      The inner sums run over the occupied points / channels only (the MBD input of a
//      zero-padded channel grid is sparse), the outer 32-point DFTs run in registers.
#include <climits>

#include "frbx_internal.h"

namespace frbx {

__constant__ float2 c_w32[32];  // exp(-2 pi i e / 32), e = 0..31

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

struct Seg {
  int bl, d, l, k0;
  long long out;
  bool valid;
};

// Segment number i of this CTA's tile.  Implicit layout: blockIdx = (slot tile, d, bl).
__device__ __forceinline__ bool tile_segment(const FitArgs &a, bool list, int i, const int *win_off,
                                             const int *win_len, const int *nval, Seg &s) {
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
  const int slot = blockIdx.x * a.tile + i;
  if (i >= a.tile || slot >= a.S_tot) return false;
  int w = 0;
  while (w + 1 < a.n_win && slot >= win_off[w + 1]) ++w;
  const int sidx = slot - win_off[w];
  s.bl = blockIdx.z;
  s.d = blockIdx.y;
  s.l = win_len[w];
  s.k0 = sidx * max(1, s.l / 2);
  s.valid = sidx < nval[w];
  s.out = ((long long)s.bl * a.n_dm + s.d) * a.S_tot + slot;
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

// --------------------------------------------------------------------------------------
// Direct-DFT kernel (any grid)
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFitThreads) k_fit_direct(FitArgs a, int list) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *X = reinterpret_cast<float2 *>(smem);  // [C]
  float2 *Y = X + a.C;                           // [N][Ls]
  float2 *tws = Y + a.N * a.Ls;                  // [Ls]
  float2 *twm = tws + a.Ls;                      // [Lm]
  int *gsh = reinterpret_cast<int *>(twm + a.Lm);  // [N]
  int *win_off = gsh + a.N;                      // [kMaxWin]
  int *win_len = win_off + kMaxWin;              // [kMaxWin]
  int *nval = win_len + kMaxWin;                 // [kMaxWin]
  float *rp = reinterpret_cast<float *>(nval + kMaxWin);  // [32]
  int *ri = reinterpret_cast<int *>(rp + 32);    // [32]

  for (int i = threadIdx.x; i < a.Ls; i += blockDim.x) tws[i] = a.tw_s[i];
  for (int i = threadIdx.x; i < a.Lm; i += blockDim.x) twm[i] = a.tw_m[i];
  for (int i = threadIdx.x; i < a.N; i += blockDim.x) gsh[i] = a.g[i];
  if (!list) {
    for (int i = threadIdx.x; i < a.n_win; i += blockDim.x) {
      win_off[i] = a.win_off[i];
      win_len[i] = a.win_len[i];
      nval[i] = a.n_valid[blockIdx.y * a.n_win + i];
    }
  }
  __syncthreads();

  const int Ls = a.Ls, Lm = a.Lm, J = a.J, N = a.N;
  for (int it = 0;; ++it) {
    Seg s;
    if (!tile_segment(a, list, it, win_off, win_len, nval, s)) break;
    if (!s.valid) {
      if (threadIdx.x == 0) write_fit(a, s, -1.f, 0);
      continue;
    }
    gather_segment(a, s, X, J);
    __syncthreads();
    // Eq. 5, sum over j = 1 .. J-1 for every (n, m)
    for (int o = threadIdx.x; o < N * Ls; o += blockDim.x) {
      const int n = o / Ls, m = o - n * Ls;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = 1; j < J; ++j) acc = cfma(acc, X[n * J + j], tws[(j * m) & (Ls - 1)]);
      Y[o] = acc;
    }
    __syncthreads();
    // Eq. 5, sum over n for every (m, q), |G|^2 and the maximum
    float bp = -1.f;
    int bi = INT_MAX;
    for (int o = threadIdx.x; o < Ls * Lm; o += blockDim.x) {
      const int m = o >> a.log2Lm, q = o & (Lm - 1);
      if (((m - a.m_lo) & (Ls - 1)) >= a.m_len || ((q - a.q_lo) & (Lm - 1)) >= a.q_len) continue;
      float2 acc = make_float2(0.f, 0.f);
      for (int n = 0; n < N; ++n) acc = cfma(acc, Y[n * Ls + m], twm[(gsh[n] * q) & (Lm - 1)]);
      const float p = fmaf(acc.x, acc.x, acc.y * acc.y);
      if (p > bp) {  // o increases per thread, so '>' keeps the lowest index on ties
        bp = p;
        bi = o;
      }
    }
    block_best(bp, bi, rp, ri);
    if (threadIdx.x == 0) write_fit(a, s, bp, bi);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------------------
// FFT kernel (Ls, Lm multiples of 32)
// --------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFitThreads, 2) k_fit_fft(FitArgs a, int list) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, Ls = a.Ls, Lm = a.Lm;
  const int PS = Ls >> 5, PM = Lm >> 5;
  const int JP = a.J1 * 32;       // padded points per channel
  const int xs = JP + 1;          // X row stride (odd: conflict-free column reads)
  const int ys = Ls + 4;          // Y row stride
  float2 *X = reinterpret_cast<float2 *>(smem);  // [N][xs]
  float2 *Y = X + N * xs;                        // [N][ys]
  float2 *stw = Y + N * ys;                      // [PS][JP]
  float2 *mtw = stw + PS * JP;                   // [N][PM]
  int *slot = reinterpret_cast<int *>(mtw + N * PM);  // [32][occ]
  int *win_off = slot + 32 * a.occ;
  int *win_len = win_off + kMaxWin;
  int *nval = win_len + kMaxWin;
  float *rp = reinterpret_cast<float *>(nval + kMaxWin);
  int *ri = reinterpret_cast<int *>(rp + 32);

  for (int i = threadIdx.x; i < N * xs; i += blockDim.x) X[i] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < PS * JP; i += blockDim.x) stw[i] = a.sbd_tw[i];
  for (int i = threadIdx.x; i < N * PM; i += blockDim.x) mtw[i] = a.mbd_tw[i];
  for (int i = threadIdx.x; i < 32 * a.occ; i += blockDim.x) slot[i] = a.slot[i];
  if (!list) {
    for (int i = threadIdx.x; i < a.n_win; i += blockDim.x) {
      win_off[i] = a.win_off[i];
      win_len[i] = a.win_len[i];
      nval[i] = a.n_valid[blockIdx.y * a.n_win + i];
    }
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    Seg s;
    if (!tile_segment(a, list, it, win_off, win_len, nval, s)) break;
    if (!s.valid) {
      if (threadIdx.x == 0) write_fit(a, s, -1.f, 0);
      continue;
    }
    gather_segment(a, s, X, xs);
    __syncthreads();

    // SBD transform: task (n, m1)
    for (int t = threadIdx.x; t < N * PS; t += blockDim.x) {
      const int n = t / PS, m1 = t - n * PS;
      float2 A[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) A[k] = make_float2(0.f, 0.f);
      const float2 *xr = X + n * xs;
      const float2 *wr = stw + m1 * JP;
      for (int j1 = 0; j1 < a.J1; ++j1) {
#pragma unroll
        for (int j2 = 0; j2 < 32; ++j2) A[j2] = cfma(A[j2], xr[j1 * 32 + j2], wr[j1 * 32 + j2]);
      }
      fft32_dif(A);
      float2 *yr = Y + n * ys + m1;
#pragma unroll
      for (int k = 0; k < 32; ++k) yr[PS * bitrev5(k)] = A[k];
    }
    __syncthreads();

    // MBD transform + |G|^2 + maximum: task (m, q1)
    float bp = -1.f;
    int bi = INT_MAX;
    for (int t = threadIdx.x; t < Ls * PM; t += blockDim.x) {
      const int m = t / PM, q1 = t - m * PM;
      if (((m - a.m_lo) & (Ls - 1)) >= a.m_len) continue;
      float2 A[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) A[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int g2 = 0; g2 < 32; ++g2) {
        for (int o = 0; o < a.occ; ++o) {
          const int n = slot[g2 * a.occ + o];
          if (n >= 0) A[g2] = cfma(A[g2], Y[n * ys + m], mtw[n * PM + q1]);
        }
      }
      fft32_dif(A);
      float tp = -1.f;
      int tq = 0;
#pragma unroll
      for (int q2 = 0; q2 < 32; ++q2) {  // q increases with q2: '>' keeps the lowest q
        const float2 v = A[bitrev5(q2)];
        const float p = fmaf(v.x, v.x, v.y * v.y);
        const int q = q1 + PM * q2;
        if (p > tp && ((q - a.q_lo) & (Lm - 1)) < a.q_len) {
          tp = p;
          tq = q;
        }
      }
      if (tp >= 0.f) better(bp, bi, tp, m * Lm + tq);
    }
    block_best(bp, bi, rp, ri);
    if (threadIdx.x == 0) write_fit(a, s, bp, bi);
    __syncthreads();
  }
}

// --------------------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------------------
static size_t direct_smem(const FitArgs &a) {
  return sizeof(float2) * ((size_t)a.C + (size_t)a.N * a.Ls + a.Ls + a.Lm) +
         sizeof(int) * ((size_t)a.N + 3 * kMaxWin) + 64 * sizeof(int);
}

static size_t fft_smem(const FitArgs &a) {
  const size_t JP = (size_t)a.J1 * 32, xs = JP + 1, ys = (size_t)a.Ls + 4;
  return sizeof(float2) * ((size_t)a.N * xs + (size_t)a.N * ys + (size_t)(a.Ls / 32) * JP +
                           (size_t)a.N * (a.Lm / 32)) +
         sizeof(int) * (32 * (size_t)a.occ + 3 * kMaxWin) + 64 * sizeof(int);
}

static size_t max_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

bool fft_supported(int Ls, int Lm, int J) { return Ls % 32 == 0 && Lm % 32 == 0 && J <= Ls; }

void set_fft_constants() {
  float2 w[32];
  const double two_pi = 6.283185307179586476925286766559;
  for (int e = 0; e < 32; ++e) {
    w[e].x = (float)std::cos(two_pi * e / 32.0);
    w[e].y = (float)-std::sin(two_pi * e / 32.0);
  }
  cudaMemcpyToSymbol(c_w32, w, sizeof(w));
}

cudaError_t launch_fit(const FitArgs &a, int n_bl, bool list_mode, int kernel, cudaStream_t st,
                       int64_t *launches) {
  const bool use_fft = kernel == 2 || (kernel == 0 && fft_supported(a.Ls, a.Lm, a.J));
  const size_t smem = use_fft ? fft_smem(a) : direct_smem(a);
  if (smem > max_smem()) return cudaErrorInvalidConfiguration;
  dim3 grid;
  if (list_mode) {
    const long long nb = (a.n_seg + a.tile - 1) / a.tile;
    if (nb == 0) return cudaSuccess;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    grid = dim3((unsigned)nb, 1, 1);
  } else {
    const int nb = (a.S_tot + a.tile - 1) / a.tile;
    if (nb == 0 || a.n_dm == 0 || n_bl == 0) return cudaSuccess;
    if (a.n_dm > 65535 || n_bl > 65535) return cudaErrorInvalidConfiguration;
    grid = dim3((unsigned)nb, (unsigned)a.n_dm, (unsigned)n_bl);
  }
  cudaError_t e;
  if (use_fft) {
    e = cudaFuncSetAttribute(k_fit_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fit_fft<<<grid, kFitThreads, smem, st>>>(a, list_mode ? 1 : 0);
  } else {
    e = cudaFuncSetAttribute(k_fit_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fit_direct<<<grid, kFitThreads, smem, st>>>(a, list_mode ? 1 : 0);
  }
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
