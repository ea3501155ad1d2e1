// Dispersion shift table (Eq. 1-2) and the normalisation / threshold stage (Eq. 6,
// Sec. 2.4.1 step a) for baselines and for baseline combinations (Sec. 2.4.2 step b).
#include <cfloat>

#include "frbx_internal.h"

namespace frbx {

// ---------------------------------------------------------------- Eq. 1-2
// dk = floor(0.5 + ((4.15e6 * DM) * (1/(f*f) - 1/(fref*fref))) / t_ap), every step a
// correctly rounded FP64 operation (explicit _rn intrinsics: no contraction), so the
// table is reproducible bit for bit on any IEEE host.
__global__ void k_shift_table(const double *__restrict__ f, int C, double inv_fref2,
                              const double *__restrict__ dm, int n_dm, double t_ap,
                              int *__restrict__ dk) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n_dm * C) return;
  const int d = (int)(i / C), c = (int)(i - (long long)d * C);
  const double fc = f[c];
  const double b = __dsub_rn(__ddiv_rn(1.0, __dmul_rn(fc, fc)), inv_fref2);
  const double dt = __dmul_rn(__dmul_rn(4.15e6, dm[d]), b);
  double x = __dadd_rn(0.5, __ddiv_rn(dt, t_ap));
  x = fmin(x, 1.0e9);  // keeps the int conversion defined for absurd DM; no segment is then valid
  dk[i] = (int)floor(x);
}

__global__ void k_row_max(const int *__restrict__ dk, int C, int *__restrict__ out) {
  __shared__ int red[32];
  const int d = blockIdx.x;
  int m = 0;
  for (int c = threadIdx.x; c < C; c += blockDim.x) m = max(m, dk[(size_t)d * C + c]);
#pragma unroll
  for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    out[d] = m;
  }
}

cudaError_t launch_shift_table(const double *f, int C, double fref, const double *dm, int n_dm,
                               double t_ap, int *dk, int *dk_max, cudaStream_t st,
                               int64_t *launches) {
  const long long n = (long long)n_dm * C;
  if (n == 0) return cudaSuccess;
  const double inv_fref2 = 1.0 / (fref * fref);
  const int threads = 256;
  k_shift_table<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(f, C, inv_fref2, dm,
                                                                            n_dm, t_ap, dk);
  ++*launches;
  k_row_max<<<n_dm, 256, 0, st>>>(dk, C, dk_max);
  ++*launches;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Eq. 6 + threshold
// Amplitude of slot i of series s at DM d: a baseline's |G|, or for a combination the
// sum of |G| over its baselines (Sec. 2.4.2: the "power" summed is the amplitude).
__device__ __forceinline__ double series_value(const StatsArgs &a, int s, int d, int slot) {
  if (!a.masks) return (double)a.series[((size_t)s * a.n_dm + d) * a.S_tot + slot].amp;
  const unsigned long long mask = a.masks[s];
  double v = 0.0;
  for (int b = 0; b < a.n_bl; ++b)
    if ((mask >> b) & 1ull) v += (double)a.series[((size_t)b * a.n_dm + d) * a.S_tot + slot].amp;
  return v;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int warp = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// One CTA per (window, DM, series): population mean and std over the valid segments,
// then the count of P = (A - mean) / std > threshold; optionally writes P.
__global__ void __launch_bounds__(256) k_stats_count(StatsArgs a) {
  __shared__ double red[32];
  const int w = blockIdx.x, d = blockIdx.y, s = blockIdx.z;
  const int nv = a.n_valid[d * a.n_win + w];
  const int off = a.win_off[w];
  const size_t sid = ((size_t)s * a.n_dm + d) * a.n_win + w;
  double sum = 0.0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) sum += series_value(a, s, d, off + i);
  const double mean = nv > 0 ? block_sum(sum, red) / nv : 0.0;
  double sq = 0.0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double dv = series_value(a, s, d, off + i) - mean;
    sq += dv * dv;
  }
  const double sd = nv > 0 ? sqrt(block_sum(sq, red) / nv) : 0.0;
  int cnt = 0;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double p = sd > 0.0 ? (series_value(a, s, d, off + i) - mean) / sd : 0.0;
    if (p > a.threshold) ++cnt;
    if (a.pnorm) a.pnorm[((size_t)s * a.n_dm + d) * a.S_tot + off + i] = (float)p;
  }
  const double total = block_sum((double)cnt, red);
  if (threadIdx.x == 0) {
    a.mean_std[2 * sid] = mean;
    a.mean_std[2 * sid + 1] = sd;
    a.counts[sid] = (int)total;
  }
}

// Exclusive scan of the per-(series, DM, window) counts into offsets (one CTA).
__global__ void __launch_bounds__(1024) k_scan(const int *__restrict__ counts, long long n,
                                               long long *__restrict__ offsets) {
  __shared__ long long part[1024];
  const long long chunk = (n + blockDim.x - 1) / blockDim.x;
  const long long lo = threadIdx.x * chunk, hi = min(n, lo + chunk);
  long long s = 0;
  for (long long i = lo; i < hi; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const long long v = part[t];
      part[t] = run;
      run += v;
    }
    offsets[n] = run;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (long long i = lo; i < hi; ++i) {
    offsets[i] = run;
    run += counts[i];
  }
}

// Ordered compaction of the crossings of one (window, DM, series) in ascending k0.
__global__ void __launch_bounds__(256) k_events(StatsArgs a) {
  __shared__ int wsum[8];
  __shared__ int base_s;
  const int w = blockIdx.x, d = blockIdx.y, s = blockIdx.z;
  const int nv = a.n_valid[d * a.n_win + w];
  const int off = a.win_off[w], step = a.win_step[w];
  const size_t sid = ((size_t)s * a.n_dm + d) * a.n_win + w;
  const double mean = a.mean_std[2 * sid], sd = a.mean_std[2 * sid + 1];
  long long out = a.offsets[sid];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < nv; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    double v = 0.0, p = 0.0;
    bool hit = false;
    if (i < nv) {
      v = series_value(a, s, d, off + i);
      p = sd > 0.0 ? (v - mean) / sd : 0.0;
      hit = p > a.threshold;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        const int t = wsum[k];
        wsum[k] = run;
        run += t;
      }
      base_s = run;
    }
    __syncthreads();
    if (hit) {
      const long long pos = out + wsum[warp] + __popc(bal & ((1u << lane) - 1u));
      frbx_event e;
      e.series = a.series_base + s;
      e.dm_idx = d;
      e.win_idx = w;
      e.k0 = i * step;
      e.amp = (float)v;
      e.pnorm = (float)p;
      if (!a.masks) {
        const frbx_seg sg = a.series[((size_t)s * a.n_dm + d) * a.S_tot + off + i];
        e.sbd_idx = sg.sbd_idx;
        e.mbd_idx = sg.mbd_idx;
      } else {
        e.sbd_idx = 0;
        e.mbd_idx = 0;
      }
      a.events[pos] = e;
    }
    out += base_s;
    __syncthreads();
  }
}

cudaError_t launch_stats_count(const StatsArgs &a, cudaStream_t st, int64_t *launches) {
  if (a.n_series == 0 || a.n_dm == 0 || a.n_win == 0) return cudaSuccess;
  k_stats_count<<<dim3(a.n_win, a.n_dm, a.n_series), 256, 0, st>>>(a);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_scan(const StatsArgs &a, cudaStream_t st, int64_t *launches) {
  const long long n = (long long)a.n_series * a.n_dm * a.n_win;
  k_scan<<<1, 1024, 0, st>>>(a.counts, n, a.offsets);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_events(const StatsArgs &a, cudaStream_t st, int64_t *launches) {
  if (a.n_series == 0 || a.n_dm == 0 || a.n_win == 0) return cudaSuccess;
  k_events<<<dim3(a.n_win, a.n_dm, a.n_series), 256, 0, st>>>(a);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
