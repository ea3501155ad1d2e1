// Appendix A on the device: the calibrator's long segment, and per channel the delay that
// maximises the channel power after the common SBD is removed, then the residual phase.
//
//   X(n, j)  = sum_{k0 <= k < k0 + l} S(n, j, k)                         (FP64 sum)
//   z_j      = w(n, j) X(n, j) exp(-i 2 pi f_j SBD)
//   D(tau)   = sum_j z_j exp(-i omega_j tau),  omega_j = 2 pi (f_j - f_bw/2) 1e-3 (rad / ns)
//   tau_n    = argmax |D|^2: grid of 8 J delays (step J / (8 J f_bw) us), three-point parabola,
//              then Newton steps on |D(tau)|^2 while its curvature is negative
//   phi_n    = arg sum_j w X exp(-i 2 pi [f_j SBD + (f0_n - min f0) MBD + (f_j - f_bw/2) tau_n] 1e-3)
// The grid fit for SBD / MBD runs through the ordinary fit kernel on the summed spectrum.
#include "frbx_internal.h"

namespace frbx {

namespace {
constexpr int kCalPad = 8;
constexpr int kCalNewton = 8;
}  // namespace

// One thread per (baseline, point): FP64 sum of the calibrator APs; a complex64 copy of the
// sum (one "AP" per baseline) feeds the grid fit, and the unit weights (no calibration
// rotation: the extraction starts from zero delays and phases) go alongside.
__global__ void k_cal_sum(const float2 *vis, int T, int C, int n_bl, int k0, int l, const float2 *wrot,
                          double2 *xsum, float2 *xcube, float2 *wunit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_bl * C) return;
  const int b = i / C, c = i - b * C;
  const float2 *p = vis + ((size_t)b * T + k0) * C + c;
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < l; ++k) {
    const float2 v = p[(size_t)k * C];
    sr += (double)v.x;
    si += (double)v.y;
  }
  xsum[i] = make_double2(sr, si);
  xcube[i] = make_float2((float)sr, (float)si);
  if (b == 0) {
    const float2 w = wrot[c];
    wunit[c] = (w.x != 0.f || w.y != 0.f) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void dsum_phase(const double2 *z, const double *omega, int J, double tau, double &dr,
                                           double &di, double &d1r, double &d1i, double &d2r, double &d2i) {
  dr = di = d1r = d1i = d2r = d2i = 0.0;
  for (int j = 0; j < J; ++j) {
    double s, c;
    sincos(-omega[j] * tau, &s, &c);
    const double er = z[j].x * c - z[j].y * s, ei = z[j].x * s + z[j].y * c;  // z e^{-i w tau}
    dr += er;
    di += ei;
    d1r += omega[j] * ei;  // (-i w) e: real part = w * imag
    d1i += -omega[j] * er;
    d2r += -omega[j] * omega[j] * er;
    d2i += -omega[j] * omega[j] * ei;
  }
}

// One thread per (baseline, channel).
__global__ void k_cal_channels(const double2 *xsum, const float2 *wrot, int n_bl, int N, int J, double f_bw,
                               const double *f0, double f0_min, const double *sbd_mbd, double *delay_ns,
                               double *phase_rad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_bl * N) return;
  const int b = i / N, n = i - b * N;
  const double two_pi = 6.283185307179586476925286766559;
  const double sbd = sbd_mbd[2 * b], mbd = sbd_mbd[2 * b + 1];
  double2 z[kMaxPoint];
  double omega[kMaxPoint];
  for (int j = 0; j < J; ++j) {
    const double fj = ((double)j * f_bw) / (double)J;
    const float2 w = wrot[n * J + j];
    const bool used = (w.x != 0.f || w.y != 0.f);
    const double2 x = xsum[(size_t)b * N * J + n * J + j];
    double s, c;
    sincos(-two_pi * fj * sbd * 1e-3, &s, &c);
    z[j] = used ? make_double2(x.x * c - x.y * s, x.x * s + x.y * c) : make_double2(0.0, 0.0);
    omega[j] = two_pi * (fj - f_bw / 2.0) * 1e-3;
  }
  // grid search over L = 8 J delays
  const int L = kCalPad * J;
  const double step = ((double)J * 1000.0) / ((double)L * f_bw);
  double best = -1.0, pw_m = 0.0, pw_p = 0.0;
  int kb = 0;
  auto power_at = [&](int p) {
    const int sp = p < L / 2 ? p : p - L;
    double dr, di, a, bb, cc, dd;
    dsum_phase(z, omega, J, sp * step, dr, di, a, bb, cc, dd);
    return dr * dr + di * di;
  };
  for (int p = 0; p < L; ++p) {
    const double pw = power_at(p);
    if (pw > best) {
      best = pw;
      kb = p;
    }
  }
  pw_m = power_at((kb - 1 + L) % L);
  pw_p = power_at((kb + 1) % L);
  const double den = pw_m - 2.0 * best + pw_p;
  const double off = den == 0.0 ? 0.0 : 0.5 * (pw_m - pw_p) / den;
  double tau = ((kb < L / 2 ? kb : kb - L) + off) * step;
  for (int it = 0; it < kCalNewton; ++it) {
    double dr, di, d1r, d1i, d2r, d2i;
    dsum_phase(z, omega, J, tau, dr, di, d1r, d1i, d2r, d2i);
    const double f1 = 2.0 * (dr * d1r + di * d1i);
    const double f2 = 2.0 * (d1r * d1r + d1i * d1i + dr * d2r + di * d2i);
    if (!(f2 < 0.0)) break;
    tau -= f1 / f2;
  }
  // residual phase with the common SBD / MBD and the channel delay removed
  double sr = 0.0, si = 0.0;
  for (int j = 0; j < J; ++j) {
    const double fj = ((double)j * f_bw) / (double)J;
    const float2 w = wrot[n * J + j];
    if (w.x == 0.f && w.y == 0.f) continue;
    const double2 x = xsum[(size_t)b * N * J + n * J + j];
    const double ph = two_pi * (fj * sbd + (f0[n] - f0_min) * mbd + (fj - f_bw / 2.0) * tau) * 1e-3;
    double s, c;
    sincos(-ph, &s, &c);
    sr += x.x * c - x.y * s;
    si += x.x * s + x.y * c;
  }
  delay_ns[i] = tau;
  phase_rad[i] = atan2(si, sr);
}

cudaError_t launch_cal_sum(const float2 *vis, int T, int C, int n_bl, int k0, int l, const float2 *wrot,
                           double2 *xsum, float2 *xcube, float2 *wunit, cudaStream_t st, int64_t *launches) {
  const int n = n_bl * C;
  k_cal_sum<<<(n + 127) / 128, 128, 0, st>>>(vis, T, C, n_bl, k0, l, wrot, xsum, xcube, wunit);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_cal_channels(const double2 *xsum, const float2 *wrot, int n_bl, int N, int J, double f_bw,
                                const double *f0, double f0_min, const double *sbd_mbd, double *delay_ns,
                                double *phase_rad, cudaStream_t st, int64_t *launches) {
  const int n = n_bl * N;
  k_cal_channels<<<(n + 31) / 32, 32, 0, st>>>(xsum, wrot, n_bl, N, J, f_bw, f0, f0_min, sbd_mbd, delay_ns,
                                               phase_rad);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
