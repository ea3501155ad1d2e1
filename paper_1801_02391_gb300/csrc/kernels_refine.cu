// Candidate refinement below the grid spacing: coherent power of Eq. 4 (delay-rate term kept)
// for a window whose start follows the dispersion sweep continuously, and its adjoint.
//
//   u(n,j)   = t0 + 4.15e6 DM (f^-2 - f_ref^-2) / t_ap                  (FP64)
//   X(i)     = sum_{m=-1..2} w_m(phi) S(n, j, k + m),  k + phi = u + i  (cubic Catmull-Rom)
//   Phi      = 2 pi [ (f_j tau_s + (f0_n - f0_min) tau_m) 1e-3 + f0_n rho t_ap (u + i) 1e-6 ]
//              (argument formed and reduced modulo one cycle in FP64, sine / cosine in FP32)
//   G_b      = sum_{n, j>=1} c(n, j) sum_{i<l} X(i) exp(-i Phi),   P = sum_b |G_b|^2
//
// One CTA per (candidate, baseline); the adjoint accumulates dG_b/dtheta with the same walk
// and contracts it with 2 conj(G_b) dL/dP.  Samples whose taps would leave the cube count as
// zero and raise the candidate's status flag.
#include "frbx_internal.h"

namespace frbx {

namespace {

constexpr int kRefThreads = 256;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

struct PointConst {
  double f, fj, f0n, fmbd, ddm;  // frequencies (MHz) and du/dDM (APs per pc cm^-3)
  float2 wrot;
};

__device__ __forceinline__ PointConst point_const(const RefineArgs &r, int c) {
  PointConst p;
  const int n = c / r.J, j = c - n * r.J;
  p.f = r.f[c];
  p.fj = __ddiv_rn(__dmul_rn((double)j, r.f_bw), (double)r.J);
  p.f0n = r.f0[n];
  p.fmbd = p.f0n - r.f0_min;
  p.ddm = __ddiv_rn(__dmul_rn(4.15e6, __dsub_rn(__ddiv_rn(1.0, __dmul_rn(p.f, p.f)), r.inv_fref2)), r.t_ap);
  p.wrot = r.wrot[c];
  return p;
}

__device__ __forceinline__ void cr_weights(float t, float w[4], float dw[4]) {
  const float t2 = t * t, t3 = t2 * t;
  w[0] = 0.5f * (-t3 + 2.f * t2 - t);
  w[1] = 0.5f * (3.f * t3 - 5.f * t2 + 2.f);
  w[2] = 0.5f * (-3.f * t3 + 4.f * t2 + t);
  w[3] = 0.5f * (t3 - t2);
  dw[0] = 0.5f * (-3.f * t2 + 4.f * t - 1.f);
  dw[1] = 0.5f * (9.f * t2 - 10.f * t);
  dw[2] = 0.5f * (-9.f * t2 + 8.f * t + 1.f);
  dw[3] = 0.5f * (3.f * t2 - 2.f * t);
}

// exp(-2 pi i cycles), the argument reduced modulo one in FP64 first
__device__ __forceinline__ float2 phasor(double cycles) {
  const double red = cycles - floor(cycles);
  float s, c;
  sincospif(2.f * (float)red, &s, &c);
  return make_float2(c, -s);
}

template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float *red) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k * 32 + warp] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float s = 0.f;
      for (int w = 0; w < nw; ++w) s += red[k * 32 + w];
      v[k] = s;
    }
}

}  // namespace

__global__ void __launch_bounds__(kRefThreads) k_refine_fwd(RefineArgs r) {
  __shared__ float red[2 * 32];
  const int cand = blockIdx.x, b = blockIdx.y;
  const double *th = r.params + (size_t)cand * r.n_par;
  const double dm = th[0], t0 = th[1], tau_s = th[2 + 3 * b], tau_m = th[3 + 3 * b], rho = th[4 + 3 * b];
  const int l = r.width[cand];
  const float2 *vb = r.vis + (size_t)b * r.T * r.C;
  float acc[2] = {0.f, 0.f};
  bool edge = false;
  for (int c = threadIdx.x; c < r.C; c += blockDim.x) {
    const PointConst p = point_const(r, c);
    if (p.wrot.x == 0.f && p.wrot.y == 0.f) continue;  // j = 0 or flagged
    const double u = t0 + dm * p.ddm;
    const double base = (p.fj * tau_s + p.fmbd * tau_m) * 1e-3;
    const double rate = p.f0n * rho * r.t_ap * 1e-6;
    for (int i = 0; i < l; ++i) {
      const double x = u + i;
      const double kf = floor(x);
      const long long k = (long long)kf;
      if (k - 1 < 0 || k + 2 > r.T - 1) {
        edge = true;
        continue;
      }
      float w[4], dw[4];
      cr_weights((float)(x - kf), w, dw);
      const float2 *s = vb + (size_t)(k - 1) * r.C + c;
      float2 smp = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 v = __ldg(s + (size_t)m * r.C);
        smp.x = fmaf(w[m], v.x, smp.x);
        smp.y = fmaf(w[m], v.y, smp.y);
      }
      const float2 t = cmulf(cmulf(p.wrot, smp), phasor(base + rate * x));
      acc[0] += t.x;
      acc[1] += t.y;
    }
  }
  if (edge) r.status[cand] = 1;
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) {
    r.g[2 * ((size_t)cand * r.n_bl + b)] = acc[0];
    r.g[2 * ((size_t)cand * r.n_bl + b) + 1] = acc[1];
  }
}

__global__ void k_refine_power(RefineArgs r) {
  const int cand = blockIdx.x * blockDim.x + threadIdx.x;
  if (cand >= r.n_cand) return;
  float p = 0.f;
  for (int b = 0; b < r.n_bl; ++b) {
    const float gr = r.g[2 * ((size_t)cand * r.n_bl + b)], gi = r.g[2 * ((size_t)cand * r.n_bl + b) + 1];
    p = fmaf(gr, gr, fmaf(gi, gi, p));
  }
  r.power[cand] = p;
}

__global__ void __launch_bounds__(kRefThreads) k_refine_adjoint(RefineArgs r) {
  __shared__ float red[10 * 32];
  const int cand = blockIdx.x, b = blockIdx.y;
  const double *th = r.params + (size_t)cand * r.n_par;
  const double dm = th[0], t0 = th[1], tau_s = th[2 + 3 * b], tau_m = th[3 + 3 * b], rho = th[4 + 3 * b];
  const int l = r.width[cand];
  const float2 *vb = r.vis + (size_t)b * r.T * r.C;
  // sums: term * f_j, term * fmbd, term * f0n t_ap x, dG/du, dG/du * ddm (complex each)
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.f;
  for (int c = threadIdx.x; c < r.C; c += blockDim.x) {
    const PointConst p = point_const(r, c);
    if (p.wrot.x == 0.f && p.wrot.y == 0.f) continue;
    const double u = t0 + dm * p.ddm;
    const double base = (p.fj * tau_s + p.fmbd * tau_m) * 1e-3;
    const double rate = p.f0n * rho * r.t_ap * 1e-6;
    const float arate = (float)(6.283185307179586 * p.f0n * rho * r.t_ap * 1e-6);  // dPhi/du
    float2 du_sum = make_float2(0.f, 0.f);
    for (int i = 0; i < l; ++i) {
      const double x = u + i;
      const double kf = floor(x);
      const long long k = (long long)kf;
      if (k - 1 < 0 || k + 2 > r.T - 1) continue;
      float w[4], dw[4];
      cr_weights((float)(x - kf), w, dw);
      const float2 *s = vb + (size_t)(k - 1) * r.C + c;
      float2 smp = make_float2(0.f, 0.f), dsmp = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const float2 v = __ldg(s + (size_t)m * r.C);
        smp.x = fmaf(w[m], v.x, smp.x);
        smp.y = fmaf(w[m], v.y, smp.y);
        dsmp.x = fmaf(dw[m], v.x, dsmp.x);
        dsmp.y = fmaf(dw[m], v.y, dsmp.y);
      }
      const float2 e = phasor(base + rate * x);
      const float2 t = cmulf(cmulf(p.wrot, smp), e);
      const float fj = (float)p.fj, fm = (float)p.fmbd, fx = (float)(p.f0n * r.t_ap * x);
      acc[0] = fmaf(t.x, fj, acc[0]);
      acc[1] = fmaf(t.y, fj, acc[1]);
      acc[2] = fmaf(t.x, fm, acc[2]);
      acc[3] = fmaf(t.y, fm, acc[3]);
      acc[4] = fmaf(t.x, fx, acc[4]);
      acc[5] = fmaf(t.y, fx, acc[5]);
      // d/du of the sample: c X'(x) e^{-i Phi} + t (-i dPhi/du), dPhi/du = 2 pi f0_n rho t_ap 1e-6
      const float2 td = cmulf(cmulf(p.wrot, dsmp), e);
      du_sum.x += td.x + arate * t.y;
      du_sum.y += td.y - arate * t.x;
    }
    acc[6] += du_sum.x;
    acc[7] += du_sum.y;
    acc[8] = fmaf(du_sum.x, (float)p.ddm, acc[8]);
    acc[9] = fmaf(du_sum.y, (float)p.ddm, acc[9]);
  }
  block_sum<10>(acc, red);
  if (threadIdx.x == 0) {
    const float gr = r.g[2 * ((size_t)cand * r.n_bl + b)], gi = r.g[2 * ((size_t)cand * r.n_bl + b) + 1];
    const float up = r.dpower[cand];
    // dP/dtheta = 2 Re(conj(G) dG/dtheta); dG/dtau_s = -2 pi i 1e-3 A0, etc.
    auto re_conj_g = [&](float ar, float ai) { return gr * ar + gi * ai; };        // Re(conj(G) A)
    auto im_conj_g = [&](float ar, float ai) { return gr * ai - gi * ar; };        // Im(conj(G) A)
    const float two_pi = 6.283185307179586f;
    // Re(conj(G) (-i c A)) = c Im(conj(G) A)
    float *dp = r.dparams + (size_t)cand * r.n_par;
    dp[2 + 3 * b] = 2.f * up * two_pi * 1e-3f * im_conj_g(acc[0], acc[1]);
    dp[3 + 3 * b] = 2.f * up * two_pi * 1e-3f * im_conj_g(acc[2], acc[3]);
    dp[4 + 3 * b] = 2.f * up * two_pi * 1e-6f * im_conj_g(acc[4], acc[5]);
    float *part = r.partial + 2 * ((size_t)cand * r.n_bl + b);
    part[0] = 2.f * up * re_conj_g(acc[8], acc[9]);  // DM
    part[1] = 2.f * up * re_conj_g(acc[6], acc[7]);  // t0
  }
}

__global__ void k_refine_shared_grads(RefineArgs r) {
  const int cand = blockIdx.x * blockDim.x + threadIdx.x;
  if (cand >= r.n_cand) return;
  float ddm = 0.f, dt0 = 0.f;
  for (int b = 0; b < r.n_bl; ++b) {
    ddm += r.partial[2 * ((size_t)cand * r.n_bl + b)];
    dt0 += r.partial[2 * ((size_t)cand * r.n_bl + b) + 1];
  }
  r.dparams[(size_t)cand * r.n_par] = ddm;
  r.dparams[(size_t)cand * r.n_par + 1] = dt0;
}

cudaError_t launch_refine(const RefineArgs &r, bool adjoint, cudaStream_t st, int64_t *launches) {
  if (r.n_cand == 0) return cudaSuccess;
  const dim3 grid((unsigned)r.n_cand, (unsigned)r.n_bl);
  if (!adjoint) {
    k_refine_fwd<<<grid, kRefThreads, 0, st>>>(r);
    k_refine_power<<<(r.n_cand + 255) / 256, 256, 0, st>>>(r);
  } else {
    k_refine_adjoint<<<grid, kRefThreads, 0, st>>>(r);
    k_refine_shared_grads<<<(r.n_cand + 255) / 256, 256, 0, st>>>(r);
  }
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace frbx
