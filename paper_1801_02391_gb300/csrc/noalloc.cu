// frbx_fit_segments_noalloc: the segment fit of frbx_fit_segments without any device
// allocation.  Its scratch (setup tables, shift table, segment rows, error flag) lives in
// one file-scope __device__ array of fixed size; see include/frbx.h for the contract.
#include <cmath>
#include <cstring>

#include "frbx_internal.h"

namespace frbx {

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB on every device that loads the library

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  Looked up on every call: the
// lookup allocates nothing once the library's module is loaded on the device (the first call
// there loads it), and a cached pointer would go stale after cudaDeviceReset or in another
// context.
cudaError_t scratch_address(void **out) { return cudaGetSymbolAddress(out, g_noalloc_scratch); }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct SetupParams {
  int N, J, C, Ls, Lm;
  double f_bw, f_ref;
  int g[kMaxChan];
};

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }

// Point frequencies (FP64, the order of frbx_create), weight x calibration rotation, and the
// SBD / MBD twiddle tables, computed on the device from the copied setup arrays.
__global__ void k_noalloc_tables(SetupParams sp, const double *f0, const double *dtau, const double *dphi,
                                 const uint8_t *flag, int have_dtau, int have_dphi, int have_flag, double *f,
                                 float2 *wrot, float2 *tws, float2 *twm, int *g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double two_pi = 6.283185307179586476925286766559;
  if (i < sp.C) {
    const int n = i / sp.J, j = i - n * sp.J;
    const double fj = __ddiv_rn(__dmul_rn((double)j, sp.f_bw), (double)sp.J);
    f[i] = __dadd_rn(f0[n], fj);
    const bool used = j > 0 && !(have_flag && flag[i]);
    const double dt = have_dtau ? dtau[n] : 0.0, dp = have_dphi ? dphi[n] : 0.0;
    // the calibration phase of Eq. 5 in frbx_create's order, each step rounded on its own
    // (no contraction): ((2 pi (f_j - f_bw / 2)) dtau) 1e-3 + dphi
    const double ph = dadd(dmul(dmul(dmul(two_pi, __dsub_rn(fj, __ddiv_rn(sp.f_bw, 2.0))), dt), 1e-3), dp);
    double sn, cs;
    sincos(ph, &sn, &cs);
    wrot[i] = used ? make_float2((float)cs, (float)-sn) : make_float2(0.f, 0.f);
  }
  if (i < sp.Ls) {
    double sn, cs;
    sincos(__ddiv_rn(dmul(two_pi, (double)i), (double)sp.Ls), &sn, &cs);
    tws[i] = make_float2((float)cs, (float)-sn);
  }
  if (i < sp.Lm) {
    double sn, cs;
    sincos(__ddiv_rn(dmul(two_pi, (double)i), (double)sp.Lm), &sn, &cs);
    twm[i] = make_float2((float)cs, (float)-sn);
  }
  if (i < sp.N) g[i] = sp.g[i];
}

// Every row must read inside the cube: 0 <= bl < n_bl, 0 <= d < n_dm, l >= 1, k0 >= 0,
// k0 + max_c dk(d, c) + l <= T.  A bad row raises the flag (checked before the fit runs).
__global__ void k_noalloc_check(const int4 *segs, long long n_seg, const int *dk_max, int n_bl, int n_dm, int T,
                                int *bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_seg) return;
  const int4 r = segs[i];
  const bool ok = r.x >= 0 && r.x < n_bl && r.y >= 0 && r.y < n_dm && r.z >= 1 && r.w >= 0 &&
                  (long long)r.w + dk_max[r.y] + r.z <= (long long)T;
  if (!ok) atomicExch(bad, 1);
}

}  // namespace

}  // namespace frbx

extern "C" int frbx_fit_segments_noalloc(const frbx_setup *s, const void *vis_dev, int32_t n_bl, int32_t T,
                                         const double *dm, int32_t n_dm, const int32_t *segs, int64_t n_seg,
                                         frbx_seg *out_dev, void *cuda_stream) {
  using namespace frbx;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!s || !s->f0_mhz || !vis_dev || !dm || n_dm < 1 || n_bl < 1 || n_bl > kMaxBl || T < 1 || n_seg < 0 ||
      (n_seg > 0 && (!segs || !out_dev)))
    return FRBX_EINVAL;
  if (((uintptr_t)vis_dev & 7u) != 0 || ((uintptr_t)out_dev & 7u) != 0) return FRBX_EINVAL;
  for (int d = 0; d < n_dm; ++d)
    if (!(dm[d] >= 0) || !std::isfinite(dm[d])) return FRBX_EINVAL;
  // setup scalars on the host (stack only), by the code frbx_create uses
  SetupGrid sg;
  const int rc = setup_grid(s, &sg);
  if (rc != FRBX_OK) return rc;
  const int N = sg.N, J = sg.J;
  SetupParams sp{};
  sp.N = N;
  sp.J = J;
  sp.C = sg.C;
  sp.Ls = sg.Ls;
  sp.Lm = sg.Lm;
  sp.f_bw = s->f_bw_mhz;
  sp.f_ref = sg.f_ref;
  for (int n = 0; n < N; ++n) sp.g[n] = sg.g[n];
  // scratch layout, checked against the fixed size
  const int C = sp.C;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_err = take(sizeof(int)), o_f0 = take(8 * (size_t)N), o_dtau = take(8 * (size_t)N),
               o_dphi = take(8 * (size_t)N), o_flag = take((size_t)C), o_f = take(8 * (size_t)C),
               o_wrot = take(8 * (size_t)C), o_tws = take(8 * (size_t)sp.Ls), o_twm = take(8 * (size_t)sp.Lm),
               o_g = take(4 * (size_t)N), o_dm = take(8 * (size_t)n_dm), o_dkmax = take(4 * (size_t)n_dm),
               o_dk = take(4 * (size_t)n_dm * C), o_seg = take(16 * (size_t)std::max<int64_t>(n_seg, 1));
  if (off > kScratchBytes) return FRBX_EINVAL;  // needs more than the fixed 16 MiB
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return FRBX_ECUDA;
  unsigned char *b = (unsigned char *)base;
  cudaError_t e = cudaMemsetAsync(b + o_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_f0, s->f0_mhz, 8 * (size_t)N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && s->chan_delay_ns)
    e = cudaMemcpyAsync(b + o_dtau, s->chan_delay_ns, 8 * (size_t)N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && s->chan_phase_rad)
    e = cudaMemcpyAsync(b + o_dphi, s->chan_phase_rad, 8 * (size_t)N, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && s->flag) e = cudaMemcpyAsync(b + o_flag, s->flag, (size_t)C, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_dm, dm, 8 * (size_t)n_dm, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_seg > 0)
    e = cudaMemcpyAsync(b + o_seg, segs, 16 * (size_t)n_seg, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return FRBX_ECUDA;
  const int nt = std::max(C, std::max(sp.Ls, sp.Lm));
  k_noalloc_tables<<<(nt + 255) / 256, 256, 0, st>>>(
      sp, (const double *)(b + o_f0), (const double *)(b + o_dtau), (const double *)(b + o_dphi),
      (const uint8_t *)(b + o_flag), s->chan_delay_ns != nullptr, s->chan_phase_rad != nullptr, s->flag != nullptr,
      (double *)(b + o_f), (float2 *)(b + o_wrot), (float2 *)(b + o_tws), (float2 *)(b + o_twm), (int *)(b + o_g));
  int64_t launches = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_shift_table((const double *)(b + o_f), C, sp.f_ref, (const double *)(b + o_dm), n_dm, s->t_ap_ms,
                           (int *)(b + o_dk), (int *)(b + o_dkmax), st, &launches);
  if (e != cudaSuccess) return FRBX_ECUDA;
  if (n_seg == 0) return cudaStreamSynchronize(st) == cudaSuccess ? FRBX_OK : FRBX_ECUDA;
  k_noalloc_check<<<(unsigned)((n_seg + 255) / 256), 256, 0, st>>>((const int4 *)(b + o_seg), n_seg,
                                                                  (const int *)(b + o_dkmax), n_bl, n_dm, T,
                                                                  (int *)(b + o_err));
  int bad = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, b + o_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return FRBX_ECUDA;
  if (bad) return FRBX_EINVAL;  // a row reads outside the cube; nothing was fitted
  FitArgs a{};
  a.vis = (const float2 *)vis_dev;
  a.T = T;
  a.C = C;
  a.N = N;
  a.J = J;
  a.n_dm = n_dm;
  a.dk = (const int *)(b + o_dk);
  a.wrot = (const float2 *)(b + o_wrot);
  a.tw_s = (const float2 *)(b + o_tws);
  a.tw_m = (const float2 *)(b + o_twm);
  a.g = (const int *)(b + o_g);
  a.Ls = sp.Ls;
  a.Lm = sp.Lm;
  int l2 = 0;
  while ((1 << l2) < sp.Lm) ++l2;
  a.log2Lm = l2;
  a.m_lo = 0;
  a.m_len = sp.Ls;
  a.q_lo = 0;
  a.q_len = sp.Lm;
  a.seg = (const int *)(b + o_seg);
  a.n_seg = n_seg;
  a.tile = 16;
  a.out = out_dev;
  e = launch_fit(a, n_bl, true, 1, st, &launches);
  if (e == cudaErrorInvalidConfiguration) return FRBX_EUNSUPPORTED;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? FRBX_OK : FRBX_ECUDA;
}
