// Segment fit with four-step register FFTs (Eq. 3 gather, Eq. 5 on the Sec. 5.1 grid, maximum).
//
//  SBD: with j = 32 j1 + j2 and m = m1 + (Ls/32) m2,
//       Y(n, m) = sum_j2 w32^(j2 m2) [ sum_j1 X(n, j) wLs^(j m1) ]
//  MBD: with g = 32 g1 + g2 and q = q1 + (Lm/32) q2,
//       G(m, q) = sum_g2 w32^(g2 q2) [ sum_{n: g_n = g2 mod 32} Y(n, m) wLm^(g_n q1) ]
//
// One CTA of 128 threads fits a tile of segments one after the other: gather into shared
// memory, one SBD task (n, m1) per thread, then Ls * Lm / 32 MBD tasks (m, q1) that each end
// in a 32-point register FFT and the maximum of its 32 cells.  The channel of each residue
// class g2 comes from the kernel parameters (uniform across the CTA), so the MBD inner sum is
// unrolled over the occupied channels only.  The per-task maximum packs the cell's q2 into the
// 6 low mantissa bits of |G|^2 (a 2^-17 relative truncation) and takes an integer max.
#include "fit_common.cuh"
#include "fft32.cuh"

namespace frbx {

constexpr int kFftThreads = 128;

struct FftSmem {
  int xs, ys, ts;
  size_t bytes;
};

__host__ __device__ inline FftSmem fft_smem_layout(int N, int Ls, int Lm, int J1) {
  FftSmem l;
  const int JP = J1 * 32;
  l.xs = JP + 1;   // odd stride: column reads of 8 channel rows hit distinct banks
  l.ys = Ls + 4;
  l.ts = JP + 1;
  l.bytes = sizeof(float2) * ((size_t)N * l.xs + (size_t)N * l.ys + (size_t)(Ls / 32) * l.ts +
                              (size_t)N * (Lm / 32)) +
            16 * sizeof(int);  // block reduction (4 warps)
  return l;
}

template <int OCC, bool kFull, bool kBatch>
__global__ void __launch_bounds__(kFftThreads, 4)
    k_fit_fft(const __grid_constant__ FitArgs a, int list, const BatchScan *scans, int n_scans, long long total,
              unsigned int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int N = a.N, Ls = a.Ls, Lm = a.Lm;
  const int PS = Ls >> 5, PM = Lm >> 5;
  const int lps = __ffs(PS) - 1, lpm = __ffs(PM) - 1;
  const int JP = a.J1 * 32;
  const FftSmem L = fft_smem_layout(N, Ls, Lm, a.J1);
  float2 *X = reinterpret_cast<float2 *>(smem);  // [N][xs]
  float2 *Y = X + N * L.xs;                      // [N][ys]
  float2 *stw = Y + N * L.ys;                    // [PS][ts]
  float2 *mtw = stw + PS * L.ts;                 // [N][PM]
  float *rp = reinterpret_cast<float *>(mtw + N * PM);
  int *ri = reinterpret_cast<int *>(rp + 8);

  for (int i = threadIdx.x; i < N * L.xs; i += blockDim.x) X[i] = make_float2(0.f, 0.f);
  for (int i = threadIdx.x; i < PS * JP; i += blockDim.x) {
    const int r = i / JP, c = i - r * JP;
    stw[r * L.ts + c] = a.sbd_tw[i];
  }
  for (int i = threadIdx.x; i < N * PM; i += blockDim.x) mtw[i] = a.mbd_tw[i];
  __shared__ TileWin tw;
  __shared__ long long s_item;

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
    gather_segment(a, c, s, X, L.xs);
    __syncthreads();

    // SBD transform, task (n, m1)
    for (int t = threadIdx.x; t < N * PS; t += blockDim.x) {
      const int n = t >> lps, m1 = t & (PS - 1);
      float2 A[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) A[k] = make_float2(0.f, 0.f);
      const float2 *xr = X + n * L.xs;
      const float2 *wr = stw + m1 * L.ts;
      for (int j1 = 0; j1 < a.J1; ++j1) {
#pragma unroll
        for (int j2 = 0; j2 < 32; ++j2) A[j2] = cfma(A[j2], xr[j1 * 32 + j2], wr[j1 * 32 + j2]);
      }
      fft32_dif(A);
      float2 *yr = Y + n * L.ys + m1;
#pragma unroll
      for (int k = 0; k < 32; ++k) yr[PS * bitrev5(k)] = A[k];
    }
    __syncthreads();

    // MBD transform, |G|^2 and the maximum, task (m, q1)
    float bp = -1.f;
    int bi = INT_MAX;
    for (int t = threadIdx.x; t < Ls * PM; t += blockDim.x) {
      const int m = t >> lpm, q1 = t & (PM - 1);
      if (!kFull && ((m - a.m_lo) & (Ls - 1)) >= a.m_len) continue;
      const float2 *ym = Y + m;
      const float2 *tq = mtw + q1;
      float2 A[32];
#pragma unroll
      for (int g2 = 0; g2 < 32; ++g2) {
        A[g2] = make_float2(0.f, 0.f);
#pragma unroll
        for (int o = 0; o < OCC; ++o) {
          const int n = a.slot_n[g2][o];
          if (n >= 0) A[g2] = cfma(A[g2], ym[n * L.ys], tq[n * PM]);
        }
      }
      fft32_dif(A);
      unsigned key = 0u;
#pragma unroll
      for (int q2 = 0; q2 < 32; ++q2) {
        const float2 v = A[bitrev5(q2)];
        const float p = fmaf(v.x, v.x, v.y * v.y);
        unsigned k = (__float_as_uint(p) & ~63u) | (unsigned)(32 - q2);
        if (!kFull && (((q1 + PM * q2) - a.q_lo) & (Lm - 1)) >= a.q_len) k = 0u;
        key = max(key, k);
      }
      if (key != 0u) better(bp, bi, __uint_as_float(key & ~63u), m * Lm + q1 + PM * (32 - (int)(key & 63u)));
    }
    block_best(bp, bi, rp, ri);
    if (threadIdx.x == 0) write_fit(a, c.out, s, bp, bi);
  }
    __syncthreads();  // the tile table and the item slot are reused by the next item
  }
}

void set_fft_constants() {
  upload_w32();
  set_mma_constants();
  set_tree_constants();
}

bool fft_supported(int Ls, int Lm, int J) { return Ls % 32 == 0 && Lm % 32 == 0 && J <= Ls; }

template <int OCC, bool kFull, bool kBatch>
static cudaError_t launch_one(const FitArgs &a, dim3 grid, size_t smem, int list, cudaStream_t st,
                              const BatchScan *scans = nullptr, int n_scans = 0, long long total = 0,
                              unsigned int *counter = nullptr) {
  cudaError_t e = cudaFuncSetAttribute(k_fit_fft<OCC, kFull, kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_fit_fft<OCC, kFull, kBatch><<<grid, kFftThreads, smem, st>>>(a, list, scans, n_scans, total, counter);
  return cudaGetLastError();
}

cudaError_t launch_fit_fft(const FitArgs &a, int n_bl, bool list_mode, cudaStream_t st, int64_t *launches) {
  if (!fft_supported(a.Ls, a.Lm, a.J) || a.occ > 4 || a.occ < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = fft_smem_layout(a.N, a.Ls, a.Lm, a.J1).bytes;
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  dim3 grid;
  if (!fit_grid(a, n_bl, list_mode, &grid)) return cudaErrorInvalidConfiguration;
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
  const bool full = a.m_lo == 0 && a.m_len == a.Ls && a.q_lo == 0 && a.q_len == a.Lm;
  const int list = list_mode ? 1 : 0;
  cudaError_t e;
  if (a.occ == 1) e = full ? launch_one<1, true, false>(a, grid, smem, list, st) : launch_one<1, false, false>(a, grid, smem, list, st);
  else if (a.occ == 2) e = full ? launch_one<2, true, false>(a, grid, smem, list, st) : launch_one<2, false, false>(a, grid, smem, list, st);
  else e = full ? launch_one<4, true, false>(a, grid, smem, list, st) : launch_one<4, false, false>(a, grid, smem, list, st);
  ++*launches;
  return e;
}

cudaError_t launch_fit_fft_batch(const FitArgs &a, const BatchScan *scans, int n_scans, long long total,
                                 unsigned int *counter, int ctas_per_sm, cudaStream_t st, int64_t *launches) {
  if (!fft_supported(a.Ls, a.Lm, a.J) || a.occ > 4 || a.occ < 1) return cudaErrorInvalidConfiguration;
  const size_t smem = fft_smem_layout(a.N, a.Ls, a.Lm, a.J1).bytes;
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  if (total <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = ctas_per_sm > 0 ? ctas_per_sm : 4;
  const dim3 grid((unsigned)(sms * per_sm));
  const bool full = a.m_lo == 0 && a.m_len == a.Ls && a.q_lo == 0 && a.q_len == a.Lm;
  cudaError_t e;
  if (a.occ == 1) e = full ? launch_one<1, true, true>(a, grid, smem, 0, st, scans, n_scans, total, counter) : launch_one<1, false, true>(a, grid, smem, 0, st, scans, n_scans, total, counter);
  else if (a.occ == 2) e = full ? launch_one<2, true, true>(a, grid, smem, 0, st, scans, n_scans, total, counter) : launch_one<2, false, true>(a, grid, smem, 0, st, scans, n_scans, total, counter);
  else e = full ? launch_one<4, true, true>(a, grid, smem, 0, st, scans, n_scans, total, counter) : launch_one<4, false, true>(a, grid, smem, 0, st, scans, n_scans, total, counter);
  ++*launches;
  return e;
}

}  // namespace frbx
