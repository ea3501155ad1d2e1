// Fringe-fit kernels: dedispersed time segment (Eq. 3), 2-D delay transform on the
// SBD x MBD grid (Eq. 5 as the 2-D DFT of Sec. 5.1) and the grid maximum, one CTA
// per tile of segments.
//
// Two kernels compute the same thing:
//  * k_fit_direct: direct DFT sums from shared-memory twiddle tables; any grid size.
//  * k_fit_fft (kernels_fft.cu): four-step decomposition with 32-point register FFTs;
//                  needs Ls and Lm multiples of 32.
#include <algorithm>

#include "fit_common.cuh"

namespace frbx {

// --------------------------------------------------------------------------------------
// Direct-DFT kernel (any grid)
// --------------------------------------------------------------------------------------
template <bool kBatch>
__global__ void __launch_bounds__(kFitThreads)
    k_fit_direct(const __grid_constant__ FitArgs a, int list, const BatchScan *scans, int n_scans, long long total,
                 unsigned int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *X = reinterpret_cast<float2 *>(smem);  // [C]
  float2 *Y = X + a.C;                           // [N][Ls]
  float2 *tws = Y + a.N * a.Ls;                  // [Ls]
  float2 *twm = tws + a.Ls;                      // [Lm]
  int *gsh = reinterpret_cast<int *>(twm + a.Lm);  // [N]
  float *rp = reinterpret_cast<float *>(gsh + a.N);  // [32]
  int *ri = reinterpret_cast<int *>(rp + 32);    // [32]

  for (int i = threadIdx.x; i < a.Ls; i += blockDim.x) tws[i] = a.tw_s[i];
  for (int i = threadIdx.x; i < a.Lm; i += blockDim.x) twm[i] = a.tw_m[i];
  for (int i = threadIdx.x; i < a.N; i += blockDim.x) gsh[i] = a.g[i];
  __shared__ TileWin tw;
  __shared__ long long s_item;

  const int Ls = a.Ls, Lm = a.Lm, J = a.J, N = a.N;
  for (int pass = 0;; ++pass) {
    ItemCtx c;
    if (kBatch) {
      if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1u);
      __syncthreads();
      const long long item = s_item;
      if (item >= total) break;
      c = batch_item(a, scans, n_scans, item);
    } else {
      if (pass > 0) break;
      c = plain_item(a);
    }
    if (!list) tile_windows(a, c, tw);
    __syncthreads();
  for (int it = 0;; ++it) {
    Seg s;
    if (!tile_segment(a, list, it, tw, c, s)) break;
    if (!s.valid) {
      if (threadIdx.x == 0) write_fit(a, c.out, s, -1.f, 0);
      continue;
    }
    gather_segment(a, c, s, X, J);
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
    if (threadIdx.x == 0) write_fit(a, c.out, s, bp, bi);
    __syncthreads();
  }
    __syncthreads();  // the tile table and the item slot are reused by the next item
  }
}

// --------------------------------------------------------------------------------------
// Launcher
// --------------------------------------------------------------------------------------
static size_t direct_smem(const FitArgs &a) {
  return sizeof(float2) * ((size_t)a.C + (size_t)a.N * a.Ls + a.Ls + a.Lm) +
         sizeof(int) * ((size_t)a.N + 3 * kMaxWin) + 64 * sizeof(int);
}

size_t max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

bool fit_grid(const FitArgs &a, int n_bl, bool list_mode, dim3 *grid) {
  if (list_mode) {
    const long long nb = (a.n_seg + a.tile - 1) / a.tile;
    if (nb > 0x7fffffffLL) return false;
    *grid = dim3((unsigned)nb, 1, 1);
  } else {
    if (n_bl > 65535) return false;
    if (a.S_tot == 0) {
      *grid = dim3(0, 1, 1);
      return true;
    }
    const long long n_tt = ((long long)a.T + a.TT - 1) / a.TT;
    if (n_tt > 65535) return false;
    *grid = dim3((unsigned)a.n_dm, (unsigned)n_tt, (unsigned)n_bl);
  }
  return true;
}

cudaError_t launch_fit(const FitArgs &a, int n_bl, bool list_mode, int kernel, cudaStream_t st,
                       int64_t *launches) {
  const bool use_fft = kernel == 2 || (kernel == 0 && fft_supported(a.Ls, a.Lm, a.J) && a.occ <= 4);
  if (use_fft) return launch_fit_fft(a, n_bl, list_mode, st, launches);
  const size_t smem = direct_smem(a);
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  dim3 grid;
  if (!fit_grid(a, n_bl, list_mode, &grid)) return cudaErrorInvalidConfiguration;
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_fit_direct<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_fit_direct<false><<<grid, kFitThreads, smem, st>>>(a, list_mode ? 1 : 0, nullptr, 0, 0, nullptr);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_fit_batch(const FitArgs &a, const BatchScan *scans, int n_scans, long long total,
                             unsigned int *counter, int kernel, int ctas_per_sm, cudaStream_t st, int64_t *launches) {
  const bool use_fft = kernel == 2 || (kernel == 0 && fft_supported(a.Ls, a.Lm, a.J) && a.occ <= 4);
  if (use_fft) return launch_fit_fft_batch(a, scans, n_scans, total, counter, ctas_per_sm, st, launches);
  const size_t smem = direct_smem(a);
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaFuncSetAttribute(k_fit_direct<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fit_direct<true>, kFitThreads, smem);
  if (e != cudaSuccess) return e;
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, std::max(occ, 1)) : std::max(occ, 1);
  k_fit_direct<true><<<(unsigned)(sms * per_sm), kFitThreads, smem, st>>>(a, 0, scans, n_scans, total, counter);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
