// C ABI of libfrbx: argument checking, setup tables, scratch management and the
// orchestration of the hot path (shift table -> fit -> normalise/threshold -> host
// extraction).  Declarations and the contract of every entry point: include/frbx.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "frbx_internal.h"

using frbx::FitArgs;
using frbx::StatsArgs;

namespace {

int fail(frbx_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(frbx_handle *h, cudaError_t e, const char *what) {
  const int code = (e == cudaErrorMemoryAllocation) ? FRBX_ENOMEM : FRBX_ECUDA;
  cudaGetLastError();  // clear a sticky-free error so the next call starts clean
  return fail(h, code, std::string(what) + ": " + cudaGetErrorString(e));
}

#define FRBX_CK(h, call)                                        \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
  } while (0)

// Grow a scratch buffer to at least `bytes` (contents are not kept).
cudaError_t ensure(frbx_handle::Buf &b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  const size_t want = std::max<size_t>(bytes, 256);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e == cudaSuccess) b.bytes = want;
  return e;
}

// The same for a handle's own scratch, counted against its scratch cap (frbx_limits): growing
// past the cap fails as an allocation failure (FRBX_ENOMEM) and keeps the old buffer.
cudaError_t ensure(frbx_handle *h, frbx_handle::Buf &b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  const size_t want = std::max<size_t>(bytes, 256);
  const size_t cap = (size_t)h->lim.scratch_cap_bytes;
  if (cap > 0 && h->scratch_total - b.bytes + want > cap) return cudaErrorMemoryAllocation;
  h->scratch_total -= b.bytes;
  const cudaError_t e = ensure(b, want);
  h->scratch_total += b.bytes;
  return e;
}

// Pipeline-wait limit of the tensor-core kernels, and the limit of the waits that drain work in
// flight before a CTA exits.
constexpr long long kDrainCycles = 2000000000LL;
long long wait_cycles(const frbx_handle *h) { return h->lim.wait_cycles > 0 ? h->lim.wait_cycles : kDrainCycles; }

template <class T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(1, src.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// Nearest E4M3 value (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, no infinities,
// largest finite 448), ties to even, saturating; built from the format's definition.
uint8_t to_e4m3(double v) {
  const uint8_t sgn = v < 0 ? 0x80 : 0x00;
  const double a = std::fabs(v);
  if (!(a < 448.0)) return sgn | 0x7E;  // 448 = 2^8 x 1.75
  int e = a > 0 ? (int)std::floor(std::log2(a)) : -6;
  if (e < -6) e = -6;                    // subnormals share the smallest exponent
  double r = std::nearbyint(std::ldexp(a, 3 - e));  // mantissa in units of 2^(e-3), ties to even
  if (r >= 16.0) {
    r = 8.0;
    ++e;
  }
  if (e > 8 || (e == 8 && r > 14.0)) return sgn | 0x7E;
  if (r < 8.0) return sgn | (uint8_t)r;  // subnormal (e = -6)
  return sgn | (uint8_t)(((e + 7) << 3) | ((int)r - 8));
}

int next_pow2(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

int window_step(int l) { return std::max(1, l / 2); }

int n_slots(int T, int l) { return T >= l ? (T - l) / window_step(l) + 1 : 0; }

int n_valid(int T, int l, int dk_max) {
  const long long r = (long long)T - dk_max - l;
  return r >= 0 ? (int)(r / window_step(l) + 1) : 0;
}

// A delay window as the wrapped index interval [lo, lo + len) of an axis of L cells
// whose value is v(s) for the signed index s = i (i < L/2) or i - L.
template <class F>
bool axis_window(int L, const double win[2], F value, int *lo, int *len) {
  if (!(win[0] <= win[1])) {
    *lo = 0;
    *len = L;
    return true;
  }
  int s_lo = INT32_MAX, s_hi = INT32_MIN;
  for (int s = -L / 2; s < L / 2; ++s) {
    const double v = value(s);
    if (v >= win[0] && v <= win[1]) {
      s_lo = std::min(s_lo, s);
      s_hi = std::max(s_hi, s);
    }
  }
  if (s_lo > s_hi) return false;
  *lo = ((s_lo % L) + L) % L;
  *len = s_hi - s_lo + 1;
  return true;
}

std::once_flag g_const_once;

struct Layout {
  std::vector<int> win_len, win_off, win_step, n_valid;  // n_valid [n_dm][n_win]
  int S_tot = 0;
};

}  // namespace

namespace frbx {

int setup_grid(const frbx_setup *s, SetupGrid *o) {
  if (!s || !s->f0_mhz || !o) return FRBX_EINVAL;
  const int N = s->n_chan, J = s->n_point;
  if (N < 1 || N > kMaxChan || J < 2 || J > kMaxPoint) return FRBX_EINVAL;
  if (!(s->f_bw_mhz > 0) || !(s->t_ap_ms > 0) || !std::isfinite(s->f_bw_mhz) || !std::isfinite(s->t_ap_ms))
    return FRBX_EINVAL;
  o->N = N;
  o->J = J;
  o->C = N * J;
  double fmax = 0, fmin0 = 0;
  for (int n = 0; n < N; ++n) {
    const double f0 = s->f0_mhz[n];
    if (!(f0 > 0) || !std::isfinite(f0)) return FRBX_EINVAL;
    fmin0 = n == 0 ? f0 : std::min(fmin0, f0);
    for (int j = 0; j < J; ++j) fmax = std::max(fmax, f0 + ((double)j * s->f_bw_mhz) / (double)J);
  }
  o->fmin0 = fmin0;
  o->f_ref = s->f_ref_dm_mhz != 0.0 ? s->f_ref_dm_mhz : fmax;
  if (!(o->f_ref >= fmax)) return FRBX_EINVAL;  // a reference below the band would make negative shifts
  // MBD grid: GCD of the channel offsets in whole kHz
  long long off_khz[kMaxChan], gcd = 0;
  for (int n = 0; n < N; ++n) {
    const double v = (s->f0_mhz[n] - fmin0) * 1000.0, r = std::nearbyint(v);
    if (std::fabs(v - r) > 1e-3) return FRBX_EINVAL;
    off_khz[n] = (long long)r;
    if (r != 0) gcd = std::gcd(gcd, (long long)r);
  }
  if (gcd == 0) gcd = (long long)std::nearbyint(s->f_bw_mhz * 1000.0);
  if (gcd <= 0) return FRBX_EINVAL;
  o->df_grid = (double)gcd / 1000.0;
  int gmax = 0;
  for (int n = 0; n < N; ++n) {
    const long long gv = off_khz[n] / gcd;
    if (gv > kMaxLm) return FRBX_EUNSUPPORTED;
    o->g[n] = (int)gv;
    gmax = std::max(gmax, (int)gv);
  }
  const int sp = s->sbd_pad ? s->sbd_pad : 2, mp = s->mbd_pad ? s->mbd_pad : 2;
  if (sp < 1 || mp < 1) return FRBX_EINVAL;
  o->Ls = sp * J;
  o->Lm = mp * next_pow2(gmax + 1);
  if (!is_pow2(o->Ls) || !is_pow2(o->Lm) || o->Ls > kMaxLs || o->Lm > kMaxLm || (long long)o->Ls * o->Lm > (1LL << 20))
    return FRBX_EUNSUPPORTED;
  return FRBX_OK;
}

}  // namespace frbx

extern "C" {

void frbx_default_params(frbx_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->threshold = 3.0f;
  p->nwin_min = 3;
  p->sbd_win_ns[0] = 1.0;
  p->sbd_win_ns[1] = -1.0;
  p->mbd_win_ns[0] = 1.0;
  p->mbd_win_ns[1] = -1.0;
  p->combos = nullptr;
  p->n_combo = 0;
  p->kernel = 0;
}

int frbx_create(const frbx_setup *s, frbx_handle **out) {
  if (!out) return FRBX_EINVAL;
  *out = nullptr;
  frbx::SetupGrid sg;
  const int rc = frbx::setup_grid(s, &sg);
  if (rc != FRBX_OK) return rc;
  const int N = sg.N, J = sg.J;
  auto *h = new frbx_handle();
  for (auto &row : h->slot_n)
    for (short &v : row) v = -1;
  h->N = N;
  h->J = J;
  h->C = sg.C;
  h->f_bw = s->f_bw_mhz;
  h->t_ap = s->t_ap_ms;
  h->f0.assign(s->f0_mhz, s->f0_mhz + N);
  h->f.resize((size_t)h->C);
  for (int n = 0; n < N; ++n)
    for (int j = 0; j < J; ++j) h->f[(size_t)n * J + j] = h->f0[(size_t)n] + ((double)j * s->f_bw_mhz) / (double)J;
  h->f_ref = sg.f_ref;
  h->df_grid = sg.df_grid;
  h->g.assign(sg.g, sg.g + N);
  h->Ls = sg.Ls;
  h->Lm = sg.Lm;
  h->J1 = (J + 31) / 32;
  // weight x calibration rotation exp(-i[2 pi (f_j - f_bw/2) dtau0_n + dphi0_n]) (Eq. 5)
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<float2> wrot((size_t)h->C);
  for (int n = 0; n < N; ++n)
    for (int j = 0; j < J; ++j) {
      const int c = n * J + j;
      const bool used = j > 0 && !(s->flag && s->flag[c]);
      const double fj = ((double)j * s->f_bw_mhz) / (double)J;
      const double dt = s->chan_delay_ns ? s->chan_delay_ns[n] : 0.0;
      const double dp = s->chan_phase_rad ? s->chan_phase_rad[n] : 0.0;
      const double ph = two_pi * (fj - s->f_bw_mhz / 2.0) * dt * 1e-3 + dp;
      wrot[(size_t)c] = used ? make_float2((float)std::cos(ph), (float)-std::sin(ph))
                             : make_float2(0.f, 0.f);
    }
  auto tw = [&](int L) {
    std::vector<float2> t((size_t)L);
    for (int k = 0; k < L; ++k)
      t[(size_t)k] = make_float2((float)std::cos(two_pi * k / L), (float)-std::sin(two_pi * k / L));
    return t;
  };
  std::vector<float2> tws = tw(h->Ls), twm = tw(h->Lm);
  // FFT-kernel tables
  std::vector<float2> sbd_tw, mbd_tw, tree_tw;
  std::vector<int> slot, tree_slot;
  if (h->Ls % 32 == 0) {  // SBD four-step table (FFT and tensor-core fits)
    const int PS = h->Ls / 32, JP = h->J1 * 32;
    sbd_tw.assign((size_t)PS * JP, make_float2(0.f, 0.f));
    for (int m1 = 0; m1 < PS; ++m1)
      for (int j = 0; j < J; ++j) sbd_tw[(size_t)m1 * JP + j] = tws[(size_t)(((long long)j * m1) % h->Ls)];
  }
  if (h->Ls % 32 == 0 && h->Lm % 32 == 0) {  // MBD four-step tables (FFT fit)
    const int PM = h->Lm / 32;
    mbd_tw.resize((size_t)N * PM);
    for (int n = 0; n < N; ++n)
      for (int q1 = 0; q1 < PM; ++q1)
        mbd_tw[(size_t)n * PM + q1] = twm[(size_t)(((long long)h->g[(size_t)n] * q1) % h->Lm)];
    std::vector<std::vector<int>> res(32);
    for (int n = 0; n < N; ++n) res[(size_t)(h->g[(size_t)n] % 32)].push_back(n);
    h->occ = 1;
    for (auto &r : res) h->occ = std::max(h->occ, (int)r.size());
    slot.assign((size_t)32 * h->occ, -1);
    for (int g2 = 0; g2 < 32; ++g2)
      for (size_t o = 0; o < res[(size_t)g2].size(); ++o) slot[(size_t)g2 * h->occ + o] = res[(size_t)g2][o];
    for (int g2 = 0; g2 < 32; ++g2)
      for (int o = 0; o < 4; ++o)
        h->slot_n[g2][o] = (short)(o < (int)res[(size_t)g2].size() ? res[(size_t)g2][(size_t)o] : -1);
  }
  if (h->Ls % 32 == 0 && (h->Lm % 32 == 0 || h->Lm == 16)) {
    // Lm = 16: the tree uses the h = 0 half alone (one thread per row, all 16 cells), whose
    // twiddles below are 1 (q1 = 0)
    const int PM = std::max(1, h->Lm / 32);
    // window-tree fit: channel n sits in slot (g_n mod 16) + 16 o of a Y row (o its rank in
    // the class); half h of the 32-point DIF over residues g2 = g_n mod 32 takes it with
    // exp(-2 pi i [(g_n q1 mod Lm) / Lm + h (g_n mod 32) / 32]) -- the MBD twiddle times the
    // first-stage factor (+1, or -w32^(g mod 16) for the odd half), from the exact index;
    // stored as [slot / 2][q1][h][slot mod 2] so a thread reads two slots' twiddles at once
    std::vector<int> cnt16(16, 0);
    tree_slot.resize((size_t)N);
    for (int n = 0; n < N; ++n) {
      const int r = (int)(h->g[(size_t)n] % 16);
      tree_slot[(size_t)n] = r + 16 * cnt16[(size_t)r]++;
    }
    h->tree_s16 = *std::max_element(cnt16.begin(), cnt16.end());
    const int NS = 16 * h->tree_s16;
    tree_tw.assign((size_t)NS * PM * 2, make_float2(0.f, 0.f));
    for (int n = 0; n < N; ++n)
      for (int q1 = 0; q1 < PM; ++q1)
        for (int hh = 0; hh < 2; ++hh) {
          const long long g = h->g[(size_t)n];
          const long long ex = ((g * q1) % h->Lm) * 32 + hh * (g % 32) * h->Lm;
          const double th = two_pi * (double)(ex % (32LL * h->Lm)) / (32.0 * h->Lm);
          const size_t sl = (size_t)tree_slot[(size_t)n];
          tree_tw[(((sl >> 1) * PM + q1) * 2 + hh) * 2 + (sl & 1)] = make_float2((float)std::cos(th), (float)-std::sin(th));
        }
  }
  // BF16 DFT matrix of the MBD transform for the tensor-core fit, in its shared-memory image
  // (rows: chunks of NC output columns, first half Re G, second half Im G; K-major, 64-wide
  // K atoms, 128-byte swizzle); phases from the exact index g_n q mod Lm, cos/sin in FP64
  std::vector<uint16_t> bimg;
  std::vector<uint8_t> bimg8;
  if (frbx::mma_supported(h->Ls, h->Lm, N, J)) {
    const int KA = (2 * N + 63) / 64, rows = 2 * h->Lm, NC = std::min(256, rows), half = NC / 2;
    bimg.assign((size_t)KA * rows * 64, 0);
    auto bf16 = [](double v) {
      const float f = (float)v;
      uint32_t u;
      std::memcpy(&u, &f, 4);
      u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
      return (uint16_t)(u >> 16);
    };
    auto put = [&](int R, int k, double v) {
      const size_t off = (size_t)(k / 64) * rows * 128 + (size_t)(R / 8) * 1024 + (size_t)(R % 8) * 128 +
                         (size_t)((((k % 64) / 8) ^ (R % 8)) * 16) + (size_t)(k % 8) * 2;
      bimg[off / 2] = bf16(v);
    };
    for (int R = 0; R < rows; ++R) {
      const int c = R / NC, r = R % NC, q = c * half + (r % half);
      const bool im = r >= half;
      for (int n = 0; n < N; ++n) {
        const long long ex = ((long long)h->g[(size_t)n] * q) % h->Lm;
        const double th = two_pi * (double)ex / (double)h->Lm;
        put(R, n, im ? -std::sin(th) : std::cos(th));
        put(R, N + n, im ? std::cos(th) : std::sin(th));
      }
    }
    h->KA = KA;
    h->NC = NC;
    h->b_atom_bytes = rows * 128;
    h->b_bytes = KA * rows * 128;
    // E4M3 image: the same rows and swizzle, 128 values per 128-byte row of an atom
    const int KA8 = (2 * N + 127) / 128;
    bimg8.assign((size_t)KA8 * rows * 128, 0);
    auto put8 = [&](int R, int k, double v) {
      const size_t off = (size_t)(k / 128) * rows * 128 + (size_t)(R / 8) * 1024 + (size_t)(R % 8) * 128 +
                         (size_t)((((k % 128) / 16) ^ (R % 8)) * 16) + (size_t)(k % 16);
      bimg8[off] = to_e4m3(v);
    };
    for (int R = 0; R < rows; ++R) {
      const int c = R / NC, r = R % NC, q = c * half + (r % half);
      const bool im = r >= half;
      for (int n = 0; n < N; ++n) {
        const long long ex = ((long long)h->g[(size_t)n] * q) % h->Lm;
        const double th = two_pi * (double)ex / (double)h->Lm;
        put8(R, n, im ? -std::sin(th) : std::cos(th));
        put8(R, N + n, im ? std::cos(th) : std::sin(th));
      }
    }
    h->b_bytes8 = KA8 * rows * 128;
  }
  // window-tree tensor-core fit: per block of 32 MBD columns q, the DFT rows (Re G of the 32
  // q, then Im G) split as W = W_hi + W_lo in BF16, in 128-byte swizzled images; per 64-wide
  // K atom the 64 hi rows are followed by the 64 lo rows, so [W_hi; W_lo] is one 128-row operand
  std::vector<uint16_t> wtree;
  std::vector<uint8_t> wtree8;
  if (frbx::tree_mma_supported(h->Ls, h->Lm, N, J)) {
    const int KA = (2 * N + 63) / 64, rows = 64, n_qb = h->Lm / 32, atom = rows * 128;
    const int wb = 2 * KA * atom;  // bytes per block: per K atom, hi rows then lo rows
    wtree.assign((size_t)n_qb * wb / 2, 0);
    auto bf16 = [](double v) {
      const float f = (float)v;
      uint32_t u;
      std::memcpy(&u, &f, 4);
      u += 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
      return (uint16_t)(u >> 16);
    };
    auto bf16f = [](uint16_t b) {
      const uint32_t u = (uint32_t)b << 16;
      float f;
      std::memcpy(&f, &u, 4);
      return (double)f;
    };
    auto put = [&](int qb, int lo, int R, int k, uint16_t v) {
      const size_t off = (size_t)qb * wb + (size_t)(k / 64) * 2 * atom + (size_t)lo * atom + (size_t)(R / 8) * 1024 +
                         (size_t)(R % 8) * 128 + (size_t)((((k % 64) / 8) ^ (R % 8)) * 16) + (size_t)(k % 8) * 2;
      wtree[off / 2] = v;
    };
    for (int qb = 0; qb < n_qb; ++qb)
      for (int R = 0; R < rows; ++R) {
        const int q = qb * 32 + (R % 32);
        const bool im = R >= 32;
        for (int n = 0; n < N; ++n) {
          const long long ex = ((long long)h->g[(size_t)n] * q) % h->Lm;
          const double th = two_pi * (double)ex / (double)h->Lm;
          const double vr = im ? -std::sin(th) : std::cos(th), vi = im ? std::cos(th) : std::sin(th);
          const uint16_t rh = bf16(vr), ih = bf16(vi);
          put(qb, 0, R, n, rh);
          put(qb, 0, R, N + n, ih);
          put(qb, 1, R, n, bf16(vr - bf16f(rh)));
          put(qb, 1, R, N + n, bf16(vi - bf16f(ih)));
        }
      }
    h->wtree_bytes = wb;
    // the E4M3 form: per block of 32 q, the same 64 rows (Re G of the 32 q, then Im G) rounded
    // once to E4M3, 128 K values per 128-byte row
    const int KA8 = (2 * N + 127) / 128, wb8 = KA8 * rows * 128;
    wtree8.assign((size_t)n_qb * wb8, 0);
    auto put8 = [&](int qb, int R, int k, double v) {
      const size_t off = (size_t)qb * wb8 + (size_t)(k / 128) * rows * 128 + (size_t)(R / 8) * 1024 +
                         (size_t)(R % 8) * 128 + (size_t)((((k % 128) / 16) ^ (R % 8)) * 16) + (size_t)(k % 16);
      wtree8[off] = to_e4m3(v);
    };
    for (int qb = 0; qb < n_qb; ++qb)
      for (int R = 0; R < rows; ++R) {
        const int q = qb * 32 + (R % 32);
        const bool im = R >= 32;
        for (int n = 0; n < N; ++n) {
          const long long ex = ((long long)h->g[(size_t)n] * q) % h->Lm;
          const double th = two_pi * (double)ex / (double)h->Lm;
          put8(qb, R, n, im ? -std::sin(th) : std::cos(th));
          put8(qb, R, N + n, im ? std::cos(th) : std::sin(th));
        }
      }
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = upload(&h->d_f, h->f);
  if (e == cudaSuccess) e = upload(&h->d_f0, h->f0);
  if (e == cudaSuccess) e = upload(&h->d_wrot, wrot);
  if (e == cudaSuccess) e = upload(&h->d_tw_s, tws);
  if (e == cudaSuccess) e = upload(&h->d_tw_m, twm);
  if (e == cudaSuccess) e = upload(&h->d_g, h->g);
  if (e == cudaSuccess) e = upload(&h->d_sbd_tw, sbd_tw);
  if (e == cudaSuccess) e = upload(&h->d_mbd_tw, mbd_tw);
  if (e == cudaSuccess) e = upload(&h->d_slot, slot);
  if (e == cudaSuccess) e = upload(&h->d_tree_tw, tree_tw);
  if (e == cudaSuccess) e = upload(&h->d_tree_slot, tree_slot);
  if (e == cudaSuccess && !bimg.empty()) e = upload((uint16_t **)&h->d_bimg, bimg);
  if (e == cudaSuccess && !bimg8.empty()) e = upload((uint8_t **)&h->d_bimg8, bimg8);
  if (e == cudaSuccess && !wtree.empty()) e = upload((uint16_t **)&h->d_wtree, wtree);
  if (e == cudaSuccess && !wtree8.empty()) e = upload((uint8_t **)&h->d_wtree8, wtree8);
  if (e == cudaSuccess) {
    std::call_once(g_const_once, frbx::set_fft_constants);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? FRBX_ENOMEM : FRBX_ECUDA;
    cudaGetLastError();
    frbx_destroy(h);
    return code;
  }
  *out = h;
  return FRBX_OK;
}

void frbx_destroy(frbx_handle *h) {
  if (!h) return;
  void *ptrs[] = {h->d_f,      h->d_f0,     h->d_wrot, h->d_tw_s, h->d_tw_m,     h->d_g,
                  h->d_sbd_tw, h->d_mbd_tw, h->d_slot, h->d_bimg, h->d_tree_tw, h->d_tree_slot, h->d_bimg8,
                  h->d_wtree,  h->d_wtree8};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->tree_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->tree_kev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t x : h->tree_st)
    if (x) cudaStreamDestroy(x);
  for (cudaEvent_t e : h->vis_ev)
    if (e) cudaEventDestroy(e);
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  frbx_handle::Buf *bufs[] = {&h->vis, &h->dk, &h->dk_max, &h->series, &h->pnorm, &h->stats,
                              &h->counts, &h->offsets, &h->events, &h->small, &h->seglist, &h->masks,
                              &h->errflag, &h->refine, &h->calib, &h->ytree};
  for (auto *b : bufs)
    if (b->p) cudaFree(b->p);
  delete h;
}

const char *frbx_last_error(const frbx_handle *h) { return h ? h->err.c_str() : "null handle"; }

int frbx_grid_info(const frbx_handle *h, int32_t *Ls, int32_t *Lm, double *df_grid_mhz,
                   int32_t *g_out) {
  if (!h) return FRBX_EINVAL;
  if (Ls) *Ls = h->Ls;
  if (Lm) *Lm = h->Lm;
  if (df_grid_mhz) *df_grid_mhz = h->df_grid;
  if (g_out)
    for (int n = 0; n < h->N; ++n) g_out[n] = h->g[(size_t)n];
  return FRBX_OK;
}

int64_t frbx_series_layout(int32_t T, const int32_t *windows, int32_t n_win, int64_t *offset) {
  if (T < 1 || n_win < 1 || n_win > frbx::kMaxWin || !windows) return FRBX_EINVAL;
  int64_t tot = 0;
  for (int w = 0; w < n_win; ++w) {
    if (windows[w] < 1) return FRBX_EINVAL;
    if (offset) offset[w] = tot;
    tot += n_slots(T, windows[w]);
  }
  return tot;
}

int64_t frbx_last_launch_count(const frbx_handle *h) { return h ? h->launches : -1; }

int frbx_set_limits(frbx_handle *h, const frbx_limits *lim) {
  if (!h) return FRBX_EINVAL;
  if (!lim) {
    h->lim = frbx_limits{};
    return FRBX_OK;
  }
  if (lim->tree_chunk_bytes < 0 || lim->wait_cycles < 0 || lim->scratch_cap_bytes < 0 || lim->hold_producers < 0)
    return fail(h, FRBX_EINVAL, "limits must be >= 0");
  h->lim = *lim;
  h->lim.reserved = 0;
  return FRBX_OK;
}

int frbx_get_limits(const frbx_handle *h, frbx_limits *lim) {
  if (!h || !lim) return FRBX_EINVAL;
  *lim = h->lim;
  return FRBX_OK;
}

int64_t frbx_scratch_bytes(const frbx_handle *h) { return h ? (int64_t)h->scratch_total : -1; }

}  // extern "C"

namespace {

// Shift table for dm[] into h->dk / h->dk_max; dk_max copied to host.
int run_shift_table(frbx_handle *h, const double *dm, int n_dm, std::vector<int> *dk_max,
                    cudaStream_t st) {
  for (int d = 0; d < n_dm; ++d)
    if (!(dm[d] >= 0) || !std::isfinite(dm[d])) return fail(h, FRBX_EINVAL, "DM trials must be finite and >= 0");
  FRBX_CK(h, ensure(h, h->small, sizeof(double) * (size_t)n_dm + 4096));
  FRBX_CK(h, ensure(h, h->dk, sizeof(int) * (size_t)n_dm * h->C));
  FRBX_CK(h, ensure(h, h->dk_max, sizeof(int) * (size_t)n_dm));
  double *d_dm = (double *)h->small.p;
  FRBX_CK(h, cudaMemcpyAsync(d_dm, dm, sizeof(double) * n_dm, cudaMemcpyHostToDevice, st));
  FRBX_CK(h, frbx::launch_shift_table(h->d_f, h->C, h->f_ref, d_dm, n_dm, h->t_ap, (int *)h->dk.p,
                                      (int *)h->dk_max.p, st, &h->launches));
  dk_max->resize((size_t)n_dm);
  FRBX_CK(h, cudaMemcpyAsync(dk_max->data(), h->dk_max.p, sizeof(int) * n_dm, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

int check_params(frbx_handle *h, const frbx_params *p, int n_bl, FitArgs *a) {
  if (!(p->threshold == p->threshold)) return fail(h, FRBX_EINVAL, "threshold is NaN");
  if (p->nwin_min < 1) return fail(h, FRBX_EINVAL, "nwin_min must be >= 1");
  if (p->n_combo < 0 || (p->n_combo > 0 && !p->combos)) return fail(h, FRBX_EINVAL, "bad combos");
  for (int c = 0; c < p->n_combo; ++c) {
    const uint64_t m = p->combos[c];
    if (m == 0 || (n_bl < 64 && (m >> n_bl) != 0)) return fail(h, FRBX_EINVAL, "combo mask names a missing baseline");
  }
  const int J = h->J, Ls = h->Ls, Lm = h->Lm;
  const double fbw = h->f_bw, dfg = h->df_grid;
  if (!axis_window(Ls, p->sbd_win_ns, [&](int s) { return (((double)s * J) * 1000.0) / ((double)Ls * fbw); },
                   &a->m_lo, &a->m_len))
    return fail(h, FRBX_EINVAL, "SBD window holds no grid cell");
  if (!axis_window(Lm, p->mbd_win_ns, [&](int s) { return ((double)s * 1000.0) / ((double)Lm * dfg); },
                   &a->q_lo, &a->q_len))
    return fail(h, FRBX_EINVAL, "MBD window holds no grid cell");
  if (p->kernel < 0 || p->kernel > 8) return fail(h, FRBX_EINVAL, "kernel must be 0 to 8");
  if (p->kernel == 3 || p->kernel == 5) {
    if (!h->d_bimg) return fail(h, FRBX_EUNSUPPORTED, "tensor-core fit needs Ls of 64 or 128, 2 Lm >= 32, N <= 64");
    if (a->m_len != Ls || a->q_len != Lm)
      return fail(h, FRBX_EUNSUPPORTED, "tensor-core fit searches the whole grid (no delay windows)");
  }
  if (p->kernel == 2 && !frbx::fft_supported(h->Ls, h->Lm, h->J))
    return fail(h, FRBX_EUNSUPPORTED, "FFT kernel needs Ls and Lm multiples of 32");
  return FRBX_OK;
}

void fill_fit_tables(frbx_handle *h, FitArgs *a, const float2 *vis, int T, int n_dm) {
  a->vis = vis;
  a->T = T;
  a->C = h->C;
  a->N = h->N;
  a->J = h->J;
  a->n_dm = n_dm;
  a->dk = (const int *)h->dk.p;
  a->wrot = h->d_wrot;
  a->tw_s = h->d_tw_s;
  a->tw_m = h->d_tw_m;
  a->g = h->d_g;
  a->Ls = h->Ls;
  a->Lm = h->Lm;
  a->log2Lm = ilog2(h->Lm);
  a->slot = h->d_slot;
  a->occ = h->occ;
  a->sbd_tw = h->d_sbd_tw;
  a->mbd_tw = h->d_mbd_tw;
  a->J1 = h->J1;
  std::memcpy(a->slot_n, h->slot_n, sizeof(a->slot_n));
}

// With `copied` (host input of a search), the copy runs on the handle's copy stream one
// baseline at a time and *copied receives the events that mark each baseline done (null for
// device input); without it, the copy is one transfer on st.
int check_vis(frbx_handle *h, const void *vis, int vis_on_device, int n_bl, int T, cudaStream_t st,
              const float2 **dvis, const cudaEvent_t **copied = nullptr) {
  if (copied) *copied = nullptr;
  if (!vis) return fail(h, FRBX_EINVAL, "vis is NULL");
  if (n_bl < 1 || n_bl > frbx::kMaxBl) return fail(h, FRBX_EINVAL, "n_bl must be 1..64");
  if (T < 1) return fail(h, FRBX_EINVAL, "T must be >= 1");
  if (((uintptr_t)vis & 7u) != 0) return fail(h, FRBX_EINVAL, "vis must be 8-byte aligned");
  const size_t bytes = sizeof(float2) * (size_t)n_bl * T * h->C;
  if (vis_on_device) {
    *dvis = (const float2 *)vis;
    return FRBX_OK;
  }
  FRBX_CK(h, ensure(h, h->vis, bytes));
  *dvis = (const float2 *)h->vis.p;
  if (!copied) {
    FRBX_CK(h, cudaMemcpyAsync(h->vis.p, vis, bytes, cudaMemcpyHostToDevice, st));
    return FRBX_OK;
  }
  if (!h->copy_st) FRBX_CK(h, cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking));
  while ((int)h->vis_ev.size() < n_bl + 1) {
    cudaEvent_t ev = nullptr;
    FRBX_CK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    h->vis_ev.push_back(ev);
  }
  FRBX_CK(h, cudaEventRecord(h->vis_ev[(size_t)n_bl], st));
  FRBX_CK(h, cudaStreamWaitEvent(h->copy_st, h->vis_ev[(size_t)n_bl], 0));
  const size_t per_bl = bytes / (size_t)n_bl;
  for (int b = 0; b < n_bl; ++b) {
    FRBX_CK(h, cudaMemcpyAsync((char *)h->vis.p + (size_t)b * per_bl, (const char *)vis + (size_t)b * per_bl, per_bl,
                               cudaMemcpyHostToDevice, h->copy_st));
    FRBX_CK(h, cudaEventRecord(h->vis_ev[(size_t)b], h->copy_st));
  }
  *copied = h->vis_ev.data();
  return FRBX_OK;
}

void to_cand(const frbx_handle *h, const frbx::Pulse &p, const double *dm, const Layout &,
             bool combined, frbx_cand *c) {
  std::memset(c, 0, sizeof(*c));
  c->series = p.series;
  c->dm_idx = p.d;
  c->win_idx = p.w;
  c->width = p.l;
  c->k0 = p.k0;
  c->sbd_idx = combined ? 0 : p.m;
  c->mbd_idx = combined ? 0 : p.q;
  c->n_win = p.n_win;
  c->group = p.group;
  c->amp = p.amp;
  c->pnorm = p.p;
  c->t_s = (double)p.k0 * h->t_ap * 1e-3;
  const int sm = p.m < h->Ls / 2 ? p.m : p.m - h->Ls;
  const int sq = p.q < h->Lm / 2 ? p.q : p.q - h->Lm;
  c->sbd_ns = combined ? 0.0 : (((double)sm * h->J) * 1000.0) / ((double)h->Ls * h->f_bw);
  c->mbd_ns = combined ? 0.0 : ((double)sq * 1000.0) / ((double)h->Lm * h->df_grid);
  c->dm = dm[p.d];
}

// Tensor-core fit of n_valid segments (implicit layout of the search, or the list in a).
int run_fit_mma(frbx_handle *h, const FitArgs &a, int n_bl, bool list_mode, long long n_valid, bool fp8,
                cudaStream_t st) {
  frbx::MmaArgs mm{};
  mm.fp8 = fp8 ? 1 : 0;
  mm.bimg = fp8 ? h->d_bimg8 : h->d_bimg;
  mm.b_bytes = fp8 ? h->b_bytes8 : h->b_bytes;
  mm.b_atom_bytes = h->b_atom_bytes;
  mm.KA = h->KA;
  mm.NC = h->NC;
  mm.n_chunk = 2 * h->Lm / h->NC;
  mm.kk_steps = fp8 ? (2 * h->N + 31) / 32 : (2 * h->N + 15) / 16;  // K per MMA: 32 (E4M3), 16 (BF16)
  int cols = 32;
  while (cols < 2 * h->NC) cols *= 2;
  mm.tmem_cols = cols;
  mm.spt = 128 / h->Ls;
  mm.n_valid = n_valid;
  mm.n_items = list_mode ? 0 : (long long)n_bl * ((a.T + a.TT - 1) / a.TT) * a.n_dm;
  mm.timeout = wait_cycles(h);
  mm.drain_timeout = kDrainCycles;
  mm.hold = h->lim.hold_producers ? 1 : 0;
  FRBX_CK(h, ensure(h, h->errflag, sizeof(int)));
  FRBX_CK(h, cudaMemsetAsync(h->errflag.p, 0, sizeof(int), st));
  mm.err = (int *)h->errflag.p;
  cudaError_t e = frbx::launch_fit_mma(a, mm, n_bl, list_mode, st, &h->launches);
  if (e == cudaErrorInvalidConfiguration) return fail(h, FRBX_EUNSUPPORTED, "tensor-core fit does not fit this shape");
  FRBX_CK(h, e);
  int flag = 0;
  FRBX_CK(h, cudaMemcpyAsync(&flag, h->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  if (flag) return fail(h, FRBX_ETIMEOUT, "tensor-core fit: a bounded wait gave up");
  return FRBX_OK;
}

// Normalise + threshold + ordered events of n_series series (baselines or combos).
int run_stats(frbx_handle *h, StatsArgs sa, cudaStream_t st, std::vector<frbx_event> *ev) {
  const size_t ns = (size_t)sa.n_series * sa.n_dm * sa.n_win;
  FRBX_CK(h, ensure(h, h->stats, sizeof(double) * 2 * ns));
  FRBX_CK(h, ensure(h, h->counts, sizeof(int) * (ns + 1)));
  FRBX_CK(h, ensure(h, h->offsets, sizeof(long long) * (ns + 1)));
  sa.mean_std = (double *)h->stats.p;
  sa.counts = (int *)h->counts.p;
  sa.offsets = (long long *)h->offsets.p;
  FRBX_CK(h, frbx::launch_stats_count(sa, st, &h->launches));
  FRBX_CK(h, frbx::launch_scan(sa, st, &h->launches));
  long long total = 0;
  FRBX_CK(h, cudaMemcpyAsync(&total, sa.offsets + ns, sizeof(long long), cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  ev->resize((size_t)total);
  if (total == 0) return FRBX_OK;
  FRBX_CK(h, ensure(h, h->events, sizeof(frbx_event) * (size_t)total));
  sa.events = (frbx_event *)h->events.p;
  FRBX_CK(h, frbx::launch_events(sa, st, &h->launches));
  FRBX_CK(h, cudaMemcpyAsync(ev->data(), sa.events, sizeof(frbx_event) * (size_t)total,
                             cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

}  // namespace

// Multi-window fit through the matrix additivity of Sec. 5.1 (kernels_tree.cu): per chunk of
// (baseline, DM) series, the SBD pass writes the transformed one-AP spectra, the MBD pass
// builds every window from them and merges the maxima into the series buffer (as 64-bit
// keys, zeroed first); a last pass turns the keys into frbx_seg records.  d_tab holds the
// window tables and valid-segment counts in the layout frbx_search uploads.
// Time tile of the window-tree fit (APs per MBD CTA, a multiple of 64; frbx_search doubles it
// for long scans on the tensor cores); frbx_search_batch measures the candidates per setup.
constexpr int kTreeTT = 1024;
constexpr int kTreeTuneTT[] = {512, 1024, 2048};

struct TreeRun {
  frbx::TreeArgs t{};
  bool full = true;
  std::vector<int2> ser;  // (bl, d) of the series whose sweep fits the scan, baseline-major
  size_t chunk = 1, y_bytes = 0, a_bytes = 0;
  size_t sc_off = 0;  // E4M3 form: offset of the per-AP scales in a buffer set
  int n_bl = 0;
  size_t need() const { return 2 * (y_bytes + a_bytes); }  // two buffer sets: chunks alternate
};

// Host planning: kernel arguments, series list and chunk size for `budget` bytes per set.
// form: -1 = the FP32 tree (k_tree_mbd), else the tensor-core form of k_tree_mma (0 split BF16 x3,
// 1 BF16, 2 E4M3).
void plan_tree(const frbx_handle *h, const FitArgs &a, int nlev, const int32_t *windows, int n_win,
               const std::vector<int> &dkm, int n_bl, int T, int n_dm, const int *win_off, int S_tot, size_t budget,
               int form, TreeRun *r, int TT = kTreeTT) {
  const bool mma = form >= 0;
  frbx::TreeArgs &t = r->t;
  t = frbx::TreeArgs{};
  r->n_bl = n_bl;
  t.dk_max = (const int *)h->dk_max.p;
  t.T = T;
  t.keys = reinterpret_cast<unsigned long long *>(a.out);
  t.n_dm = n_dm;
  t.S_tot = S_tot;
  t.win_off = win_off;
  t.N = h->N;
  t.NS = 16 * h->tree_s16;
  t.slot_of = h->d_tree_slot;
  t.Ls = h->Ls;
  t.Lm = h->Lm;
  t.PM = std::max(1, h->Lm / 32);
  t.half = h->Lm == 16;
  t.RB = frbx::tree_rows_per_block(h->Ls, h->Lm);
  t.n_mb = h->Ls / t.RB;
  t.nlev = nlev;
  for (int &e : t.emit_w) e = -1;
  for (int w = 0; w < n_win; ++w) t.emit_w[__builtin_ctz((unsigned)windows[w])] = w;
  t.m_lo = a.m_lo;
  t.m_len = a.m_len;
  t.q_lo = a.q_lo;
  t.q_len = a.q_len;
  t.tw = h->d_tree_tw;
  t.TT = TT;
  t.n_tt = (T + t.TT - 1) / t.TT;
  t.k_per_cta = 16;
  t.n_ktile = (T + t.k_per_cta - 1) / t.k_per_cta;
  t.y_series = (size_t)T * h->Ls * h->N;
  r->full = a.m_lo == 0 && a.m_len == h->Ls && a.q_lo == 0 && a.q_len == h->Lm;
  if (mma) {  // tensor-core MBD pass: A tiles per AP in their shared-memory image instead of FP32 rows
    t.mma = 1;
    t.form = form;
    t.KA = form == 2 ? (2 * h->N + 127) / 128 : (2 * h->N + 63) / 64;
    t.k8_steps = (2 * h->N + 31) / 32;
    t.tile_bytes = frbx::tree_mma_tile_bytes(form, h->N);
    t.wimg = (const unsigned char *)(form == 2 ? h->d_wtree8 : h->d_wtree);
    t.w_bytes = frbx::tree_mma_w_bytes(form, h->N);
    // delay windows: rotate the SBD rows so the searched ones come first (in groups of 8)
    t.rot = r->full ? 0 : (a.m_lo & ~7);
    // rows searched after the rotation: [m_lo mod 8, m_lo mod 8 + m_len) in 32-row quarters
    const int nq = r->full ? 4 : ((a.m_lo & 7) + a.m_len + 31) / 32;
    t.pack = nq == 1 ? 4 : nq == 2 ? 2 : 1;
    t.prow = 128 / t.pack;
    t.piece_bytes = t.tile_bytes / t.pack;
    t.n_tg = (t.n_tt + t.pack - 1) / t.pack;
    t.n_qb = h->Lm / 32;
    t.log2Lm = a.log2Lm;
    t.err = (int *)h->errflag.p;
    t.timeout = wait_cycles(h);
    t.drain_timeout = kDrainCycles;
    t.hold = h->lim.hold_producers ? 1 : 0;
    t.yt_series = (size_t)T * t.piece_bytes;
    t.y_series = t.yt_series / sizeof(float2);
  }
  r->ser.clear();
  for (int b = 0; b < n_bl; ++b)
    for (int d = 0; d < n_dm; ++d)
      if (T - dkm[(size_t)d] >= 1) r->ser.push_back(make_int2(b, d));
  // per series: its transformed spectra, the E4M3 form's per-AP scales and the deep anchors of
  // its MBD CTAs
  const size_t anc_per = mma ? 0 : sizeof(float2) * frbx::tree_anchor_floats(nlev) * t.n_mb * t.n_tt;
  const size_t sc_per = form == 2 ? sizeof(float) * (size_t)T : 0;
  const size_t per = sizeof(float2) * t.y_series + sc_per + anc_per;
  r->chunk = std::max<size_t>(1, std::min(std::max<size_t>(r->ser.size(), 1), budget / per));
  r->sc_off = (sizeof(float2) * t.y_series * r->chunk + 255) & ~(size_t)255;
  r->y_bytes = r->sc_off + ((sc_per * r->chunk + 255) & ~(size_t)255);
  r->a_bytes = (anc_per * r->chunk + 255) & ~(size_t)255;
}

// Enqueue on st: zero the keys, the chunk passes (SBD passes on one library stream, MBD
// passes on the other, so the SBD pass of chunk i + 1 overlaps the MBD pass of chunk i;
// chunk parity picks the buffer set at `bufs`), then the key -> record pass.  d_ser holds
// r.ser on the device.  With `timing`, every pass is bracketed by events for the stage times.
// copied: per-baseline events of a cube copy still in flight (check_vis), or null; the SBD pass
// of a chunk waits only for the baselines its series read (r.ser is baseline-major).
int enqueue_tree(frbx_handle *h, const FitArgs &a, const TreeRun &r, const int2 *d_ser, char *bufs, bool timing,
                 int n_win, const int *win_len, const int *win_off, const int *n_valid, cudaStream_t st,
                 const cudaEvent_t *copied = nullptr) {
  const frbx::TreeArgs &t = r.t;
  const size_t n_el = (size_t)r.n_bl * t.n_dm * t.S_tot;
  if (n_el == 0) return FRBX_OK;
  FRBX_CK(h, cudaMemsetAsync(a.out, 0, sizeof(frbx_seg) * n_el, st));
  if (!r.ser.empty()) {
    cudaStream_t sA = h->tree_st[0], sB = h->tree_st[1];
    cudaEvent_t ev_start = h->tree_ev[0], *evA = h->tree_ev + 1, *evB = h->tree_ev + 3;
    FRBX_CK(h, cudaEventRecord(ev_start, st));
    FRBX_CK(h, cudaStreamWaitEvent(sA, ev_start, 0));
    FRBX_CK(h, cudaStreamWaitEvent(sB, ev_start, 0));
    const int n_chunks = (int)((r.ser.size() + r.chunk - 1) / r.chunk);
    if (timing) {
      while ((int)h->tree_kev.size() < 4 * n_chunks) {
        cudaEvent_t ev = nullptr;
        FRBX_CK(h, cudaEventCreate(&ev));
        h->tree_kev.push_back(ev);
      }
      h->tree_chunks = n_chunks;
      h->tree_tensor = t.mma ? 1 : 0;
    }
    int ci = 0;
    for (size_t c0 = 0; c0 < r.ser.size(); c0 += r.chunk, ++ci) {
      const int par = ci & 1;
      frbx::TreeArgs tc = t;
      char *base = bufs + (size_t)par * (r.y_bytes + r.a_bytes);
      tc.Y = (float2 *)base;
      tc.Yt = (const unsigned char *)base;
      tc.anc_g = (float2 *)(base + r.y_bytes);
      tc.ascale = t.form == 2 ? (float *)(base + r.sc_off) : nullptr;
      tc.series = d_ser + c0;
      tc.n_s = (int)std::min(r.chunk, r.ser.size() - c0);
      cudaEvent_t *kev = timing ? h->tree_kev.data() + 4 * ci : nullptr;
      cudaError_t e = cudaSuccess;
      if (ci >= 2) e = cudaStreamWaitEvent(sA, evB[par], 0);  // the MBD pass two chunks back is done with this set
      if (e == cudaSuccess && copied) e = cudaStreamWaitEvent(sA, copied[r.ser[c0 + (size_t)tc.n_s - 1].x], 0);
      if (e == cudaSuccess && kev) e = cudaEventRecord(kev[0], sA);
      if (e == cudaSuccess) e = frbx::launch_tree_sbd(a, tc, sA, &h->launches);
      if (e == cudaSuccess && kev) e = cudaEventRecord(kev[1], sA);
      if (e == cudaSuccess) e = cudaEventRecord(evA[par], sA);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sB, evA[par], 0);
      if (e == cudaSuccess && kev) e = cudaEventRecord(kev[2], sB);
      if (e == cudaSuccess)
        e = t.mma ? frbx::launch_tree_mma(tc, r.full, sB, &h->launches)
                  : frbx::launch_tree_mbd(tc, r.full, sB, &h->launches);
      if (e == cudaSuccess && kev) e = cudaEventRecord(kev[3], sB);
      if (e == cudaSuccess) e = cudaEventRecord(evB[par], sB);
      if (e == cudaErrorInvalidConfiguration) return fail(h, FRBX_EUNSUPPORTED, "window-tree fit does not fit this shape");
      FRBX_CK(h, e);
    }
    FRBX_CK(h, cudaEventRecord(evA[0], sA));
    FRBX_CK(h, cudaStreamWaitEvent(st, evA[0], 0));
    FRBX_CK(h, cudaEventRecord(evB[0], sB));
    FRBX_CK(h, cudaStreamWaitEvent(st, evB[0], 0));
  }
  FRBX_CK(h, frbx::launch_tree_finalize(a.out, (long long)n_el, t.S_tot, t.n_dm, n_win, win_len, win_off, n_valid,
                                         a.log2Lm, h->Lm, st, &h->launches));
  return FRBX_OK;
}

// Streams and events of the window-tree fit, made before any stream capture uses them.
int tree_prepare(frbx_handle *h) {
  for (int i = 0; i < 2; ++i)
    if (!h->tree_st[i]) FRBX_CK(h, cudaStreamCreateWithFlags(&h->tree_st[i], cudaStreamNonBlocking));
  for (cudaEvent_t &ev : h->tree_ev)
    if (!ev) FRBX_CK(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  return FRBX_OK;
}

// frbx_search's window-tree fit: plan with a budget of a quarter of the free memory (at most
// 16 GiB per buffer set), size the handle's scratch, upload the series list, enqueue.
int run_fit_tree(frbx_handle *h, const FitArgs &a, int nlev, int form, const int32_t *windows, int n_win,
                 const std::vector<int> &dkm, int n_bl, int T, int n_dm, const int *d_tab, int S_tot, cudaStream_t st,
                 const cudaEvent_t *copied) {
  size_t free_b = 0, total_b = 0;
  FRBX_CK(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = h->lim.tree_chunk_bytes > 0 ? (size_t)h->lim.tree_chunk_bytes
                                                    : std::min<size_t>((size_t)16 << 30, (free_b + h->ytree.bytes) / 4);
  const bool mma = form >= 0;
  if (mma) {
    FRBX_CK(h, ensure(h, h->errflag, sizeof(int)));
    FRBX_CK(h, cudaMemsetAsync(h->errflag.p, 0, sizeof(int), st));
  }
  // long scans on the tensor cores take time tiles of 2 x kTreeTT APs: half the trailing APs
  // each tile re-reads and half the per-CTA setup, while the grid still spans many waves
  const int TT = mma && T >= 8 * kTreeTT ? 2 * kTreeTT : kTreeTT;
  TreeRun r;
  plan_tree(h, a, nlev, windows, n_win, dkm, n_bl, T, n_dm, d_tab + frbx::kMaxWin, S_tot, budget, form, &r, TT);
  int rc = tree_prepare(h);
  if (rc) return rc;
  const size_t ser_bytes = (sizeof(int2) * std::max<size_t>(r.ser.size(), 1) + 255) & ~(size_t)255;
  FRBX_CK(h, ensure(h, h->ytree, ser_bytes + r.need()));
  int2 *d_ser = (int2 *)h->ytree.p;
  if (!r.ser.empty())
    FRBX_CK(h, cudaMemcpyAsync(d_ser, r.ser.data(), sizeof(int2) * r.ser.size(), cudaMemcpyHostToDevice, st));
  rc = enqueue_tree(h, a, r, d_ser, (char *)h->ytree.p + ser_bytes, true, n_win, d_tab, d_tab + frbx::kMaxWin,
                    d_tab + 3 * frbx::kMaxWin, st, copied);
  // the call's stream also follows the whole copy (series that read no baseline past some b, or
  // none at all, leave later copies unwaited otherwise)
  if (copied) FRBX_CK(h, cudaStreamWaitEvent(st, copied[n_bl - 1], 0));
  if (rc || !mma) return rc;
  int flag = 0;
  FRBX_CK(h, cudaMemcpyAsync(&flag, h->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  if (flag) return fail(h, FRBX_ETIMEOUT, "window-tree tensor-core fit: a bounded wait gave up");
  return FRBX_OK;
}

// Everything after the fit (Eq. 6 and threshold on the device, then the host extraction of
// Sec. 2.4.1 b-d, the DM merge of Sec. 5.3, cross-matching and the power sums of Sec. 2.4.2)
// for one scan whose segment series are at `series`; d_tab holds the window tables and the
// scan's valid-segment counts in the layout frbx_search uploads.
int finish_search(frbx_handle *h, const frbx_seg *series, int n_bl, int T, const double *dm, int n_dm, int n_win,
                  const Layout &L, const int *d_tab, const frbx_params &p, frbx_results *res, cudaStream_t st) {
  int rc = FRBX_OK;
  const size_t n_series_el = (size_t)n_bl * n_dm * L.S_tot;
  // normalised power and threshold crossings of every baseline series
  const bool want_p = res->pnorm && res->series_cap >= (int64_t)n_series_el;
  float *pn = nullptr;
  if (want_p) {
    if (res->series_on_device) {
      pn = res->pnorm;
    } else {
      FRBX_CK(h, ensure(h, h->pnorm, sizeof(float) * n_series_el));
      pn = (float *)h->pnorm.p;
    }
    FRBX_CK(h, cudaMemsetAsync(pn, 0, sizeof(float) * n_series_el, st));
  }
  StatsArgs sa{};
  sa.series = series;
  sa.n_bl = n_bl;
  sa.n_dm = n_dm;
  sa.S_tot = L.S_tot;
  sa.n_win = n_win;
  sa.win_off = d_tab + frbx::kMaxWin;
  sa.win_step = d_tab + 2 * frbx::kMaxWin;
  sa.n_valid = d_tab + 3 * frbx::kMaxWin;
  sa.threshold = (double)p.threshold;
  sa.n_series = n_bl;
  sa.masks = nullptr;
  sa.pnorm = pn;
  sa.series_base = 0;
  std::vector<frbx_event> ev_bl, ev_cb;
  rc = run_stats(h, sa, st, &ev_bl);
  if (rc) return rc;
  FRBX_CK(h, cudaEventRecord(h->ev[4], st));
  if (p.n_combo > 0) {
    FRBX_CK(h, ensure(h, h->masks, sizeof(uint64_t) * (size_t)p.n_combo));
    FRBX_CK(h, cudaMemcpyAsync(h->masks.p, p.combos, sizeof(uint64_t) * p.n_combo, cudaMemcpyHostToDevice, st));
    sa.masks = (const unsigned long long *)h->masks.p;
    sa.n_series = p.n_combo;
    sa.pnorm = nullptr;
    rc = run_stats(h, sa, st, &ev_cb);
    if (rc) return rc;
  }
  FRBX_CK(h, cudaEventRecord(h->ev[5], st));
  FRBX_CK(h, cudaEventSynchronize(h->ev[5]));
  {
    float ms = 0.f;
    const int pairs[4][2] = {{0, 1}, {2, 3}, {3, 4}, {4, 5}};
    for (int k = 0; k < 4; ++k) {
      FRBX_CK(h, cudaEventElapsedTime(&ms, h->ev[pairs[k][0]], h->ev[pairs[k][1]]));
      h->stage_ms[k] = ms;
    }
    // window-tree fit: device time of its SBD and MBD kernels, summed over the chunks
    h->stage_ms[5] = h->stage_ms[6] = h->stage_ms[7] = 0.0;
    for (int c = 0; c < h->tree_chunks; ++c) {
      const cudaEvent_t *kev = h->tree_kev.data() + 4 * c;
      FRBX_CK(h, cudaEventElapsedTime(&ms, kev[0], kev[1]));
      h->stage_ms[5] += ms;
      FRBX_CK(h, cudaEventElapsedTime(&ms, kev[2], kev[3]));
      h->stage_ms[6] += ms;
    }
    h->stage_ms[7] = h->tree_chunks;
    h->stage_ms[8] = h->tree_chunks > 0 ? h->tree_tensor : 0;
  }
  const auto host_t0 = std::chrono::steady_clock::now();

  // host extraction (Sec. 2.4.1 b-d, Sec. 5.3 merge, cross-matching, Sec. 2.4.2)
  frbx::ExtractConfig cfg{T, n_dm, n_win, p.nwin_min, h->Lm, L.win_len.data()};
  std::vector<frbx::Pulse> pre, merged, comb;
  std::vector<frbx::GroupOut> groups;
  frbx::extract_pulses(cfg, ev_bl.data(), (int64_t)ev_bl.size(), n_bl, true, &pre, &merged);
  frbx::cross_match(T, &merged, n_bl, &groups);
  if (p.n_combo > 0)
    frbx::extract_pulses(cfg, ev_cb.data(), (int64_t)ev_cb.size(), p.n_combo, false, nullptr, &comb);

  h->stage_ms[4] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host_t0).count();
  bool trunc = false;
  auto put_cands = [&](const std::vector<frbx::Pulse> &v, bool combined, frbx_cand *dst, int64_t cap,
                       int64_t *count) {
    *count = (int64_t)v.size();
    if (cap > 0 && (int64_t)v.size() > cap) trunc = true;
    if (!dst) return;
    const int64_t n = std::min<int64_t>(cap, (int64_t)v.size());
    for (int64_t i = 0; i < n; ++i) to_cand(h, v[(size_t)i], dm, L, combined, &dst[i]);
  };
  put_cands(merged, false, res->pulses, res->pulses_cap, &res->pulses_count);
  put_cands(comb, true, res->combined, res->combined_cap, &res->combined_count);
  put_cands(pre, false, res->pulses_dm, res->pulses_dm_cap, &res->pulses_dm_count);
  res->groups_count = (int64_t)groups.size();
  if (res->groups) {
    const int64_t n = std::min<int64_t>(res->groups_cap, (int64_t)groups.size());
    for (int64_t i = 0; i < n; ++i) {
      res->groups[i].bl_mask = groups[(size_t)i].mask;
      res->groups[i].n_baselines = groups[(size_t)i].n_baselines;
      res->groups[i].n_pulses = groups[(size_t)i].n_pulses;
    }
  }
  if (res->groups_cap > 0 && (int64_t)groups.size() > res->groups_cap) trunc = true;
  res->events_count = (int64_t)(ev_bl.size() + ev_cb.size());
  res->events_baseline_count = (int64_t)ev_bl.size();
  if (res->events) {
    int64_t k = 0;
    for (const auto &ev : {&ev_bl, &ev_cb})
      for (const frbx_event &x : *ev) {
        if (k >= res->events_cap) break;
        res->events[k++] = x;
      }
  }
  if (res->events_cap > 0 && res->events_count > res->events_cap) trunc = true;
  res->series_count = (int64_t)n_series_el;
  if (res->series && res->series_cap >= (int64_t)n_series_el) {
    FRBX_CK(h, cudaMemcpyAsync(res->series, series, sizeof(frbx_seg) * n_series_el,
                               res->series_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (want_p && !res->series_on_device)
    FRBX_CK(h, cudaMemcpyAsync(res->pnorm, pn, sizeof(float) * n_series_el, cudaMemcpyDeviceToHost, st));
  if ((res->series || res->pnorm) && res->series_cap < (int64_t)n_series_el) trunc = true;
  FRBX_CK(h, cudaStreamSynchronize(st));
  if (trunc) return fail(h, FRBX_ETRUNC, "an output array was too small");
  return FRBX_OK;
}

extern "C" int frbx_shift_table(frbx_handle *h, const double *dm, int32_t n_dm, int32_t *dk_out,
                                void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  if (!dm || !dk_out || n_dm < 1) return fail(h, FRBX_EINVAL, "bad DM list or output");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  h->launches = 0;
  std::vector<int> dkm;
  int rc = run_shift_table(h, dm, n_dm, &dkm, st);
  if (rc) return rc;
  FRBX_CK(h, cudaMemcpyAsync(dk_out, h->dk.p, sizeof(int) * (size_t)n_dm * h->C, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

static int fit_segments_impl(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl,
                             int32_t T, const double *dm, int32_t n_dm, const int32_t *segs,
                             int64_t n_seg, const frbx_params *params, frbx_seg *out,
                             void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  h->launches = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!dm || n_dm < 1 || n_seg < 0 || (n_seg > 0 && (!segs || !out)))
    return fail(h, FRBX_EINVAL, "bad DM list, segment list or output");
  frbx_params p;
  if (params) p = *params; else frbx_default_params(&p);
  FitArgs a{};
  int rc = check_params(h, &p, n_bl, &a);
  if (rc) return rc;
  const float2 *dvis = nullptr;
  rc = check_vis(h, vis, vis_on_device, n_bl, T, st, &dvis);
  if (rc) return rc;
  std::vector<int> dkm;
  rc = run_shift_table(h, dm, n_dm, &dkm, st);
  if (rc) return rc;
  for (int64_t i = 0; i < n_seg; ++i) {
    const int32_t *r = segs + 4 * i;
    if (r[0] < 0 || r[0] >= n_bl || r[1] < 0 || r[1] >= n_dm || r[2] < 1 || r[3] < 0 ||
        (long long)r[3] + dkm[(size_t)r[1]] + r[2] > T)
      return fail(h, FRBX_EINVAL, "segment row " + std::to_string(i) + " reads outside the cube");
  }
  if (n_seg == 0) return FRBX_OK;
  FRBX_CK(h, ensure(h, h->seglist, sizeof(int32_t) * 4 * (size_t)n_seg));
  FRBX_CK(h, ensure(h, h->series, sizeof(frbx_seg) * (size_t)n_seg));
  FRBX_CK(h, cudaMemcpyAsync(h->seglist.p, segs, sizeof(int32_t) * 4 * (size_t)n_seg, cudaMemcpyHostToDevice, st));
  if (p.kernel == 4 || p.kernel >= 6) p.kernel = 0;  // explicit segment lists have no window structure to exploit
  fill_fit_tables(h, &a, dvis, T, n_dm);
  a.seg = (const int *)h->seglist.p;
  a.n_seg = n_seg;
  a.tile = 16;
  a.out = (frbx_seg *)h->series.p;
  if (p.kernel == 3 || p.kernel == 5) {
    rc = run_fit_mma(h, a, n_bl, true, n_seg, p.kernel == 5, st);
    if (rc) return rc;
  } else {
    cudaError_t e = frbx::launch_fit(a, n_bl, true, p.kernel, st, &h->launches);
    if (e == cudaErrorInvalidConfiguration) return fail(h, FRBX_EUNSUPPORTED, "fit kernel does not fit this shape");
    FRBX_CK(h, e);
  }
  FRBX_CK(h, cudaMemcpyAsync(out, h->series.p, sizeof(frbx_seg) * (size_t)n_seg, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

static int search_impl(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl,
                       int32_t T, const double *dm, int32_t n_dm, const int32_t *windows,
                       int32_t n_win, const frbx_params *params, frbx_results *res,
                       void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  h->launches = 0;
  h->err.clear();
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!res) return fail(h, FRBX_EINVAL, "results is NULL");
  if (!dm || n_dm < 1) return fail(h, FRBX_EINVAL, "need at least one DM trial");
  if (!windows || n_win < 1 || n_win > frbx::kMaxWin) return fail(h, FRBX_EINVAL, "need 1..16 windows");
  for (int w = 0; w < n_win; ++w) {
    if (windows[w] < 1) return fail(h, FRBX_EINVAL, "window lengths must be >= 1");
    for (int v = 0; v < w; ++v)
      if (windows[v] == windows[w]) return fail(h, FRBX_EINVAL, "window lengths must be distinct");
  }
  frbx_params p;
  if (params) p = *params; else frbx_default_params(&p);
  FitArgs a{};
  int rc = check_params(h, &p, n_bl, &a);
  if (rc) return rc;
  for (double &v : h->stage_ms) v = 0.0;
  h->tree_chunks = 0;
  for (cudaEvent_t &ev : h->ev)
    if (!ev) FRBX_CK(h, cudaEventCreate(&ev));
  const float2 *dvis = nullptr;
  const cudaEvent_t *copied = nullptr;  // host input: the cube's copy runs beside the shift table
  rc = check_vis(h, vis, vis_on_device, n_bl, T, st, &dvis, &copied);
  if (rc) return rc;
  std::vector<int> dkm;
  FRBX_CK(h, cudaEventRecord(h->ev[0], st));
  rc = run_shift_table(h, dm, n_dm, &dkm, st);
  if (rc) return rc;
  FRBX_CK(h, cudaEventRecord(h->ev[1], st));

  // layout of a (baseline, DM) series and the valid-segment counts (host)
  Layout L;
  L.win_len.assign(windows, windows + n_win);
  long long stot = 0;
  for (int w = 0; w < n_win; ++w) {
    L.win_off.push_back((int)stot);
    L.win_step.push_back(window_step(windows[w]));
    stot += n_slots(T, windows[w]);
  }
  if (stot > (1LL << 30)) return fail(h, FRBX_EUNSUPPORTED, "too many segments per series");
  L.S_tot = (int)stot;
  L.n_valid.resize((size_t)n_dm * n_win);
  for (int d = 0; d < n_dm; ++d)
    for (int w = 0; w < n_win; ++w) L.n_valid[(size_t)d * n_win + w] = n_valid(T, windows[w], dkm[(size_t)d]);
  // small tables: win_len | win_off | win_step | n_valid | masks
  std::vector<int> tab;
  tab.insert(tab.end(), L.win_len.begin(), L.win_len.end());
  tab.resize(frbx::kMaxWin, 0);
  tab.insert(tab.end(), L.win_off.begin(), L.win_off.end());
  tab.resize(2 * frbx::kMaxWin, 0);
  tab.insert(tab.end(), L.win_step.begin(), L.win_step.end());
  tab.resize(3 * frbx::kMaxWin, 0);
  tab.insert(tab.end(), L.n_valid.begin(), L.n_valid.end());
  FRBX_CK(h, ensure(h, h->small, sizeof(int) * tab.size() + 4096));
  int *d_tab = (int *)h->small.p;
  FRBX_CK(h, cudaMemcpyAsync(d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, st));
  const size_t n_series_el = (size_t)n_bl * n_dm * L.S_tot;
  FRBX_CK(h, ensure(h, h->series, sizeof(frbx_seg) * n_series_el));

  // fit every segment
  fill_fit_tables(h, &a, dvis, T, n_dm);
  a.n_win = n_win;
  a.win_len = d_tab;
  a.win_off = d_tab + frbx::kMaxWin;
  a.n_valid = d_tab + 3 * frbx::kMaxWin;
  a.S_tot = L.S_tot;
  a.tile = 64;
  a.TT = 64;
  a.out = (frbx_seg *)h->series.p;
  FRBX_CK(h, cudaEventRecord(h->ev[2], st));
  int nlev = 0;
  const bool tree_ok = frbx::tree_supported(h->Ls, h->Lm, h->N, h->J, h->tree_s16, windows, n_win, &nlev);
  // tensor-core window tree: kernel 6 (split BF16, FP32-equivalent), 7 (BF16), 8 (E4M3)
  const bool tree_tc_shape = tree_ok && h->d_wtree && frbx::tree_mma_supported(h->Ls, h->Lm, h->N, h->J);
  const int tc_form = p.kernel == 7 ? 1 : p.kernel == 8 ? 2 : 0;
  const bool tree_tc = tree_tc_shape && frbx::tree_mma_fits(tc_form, h->N, nlev);
  if ((p.kernel == 4 && !tree_ok) || (p.kernel >= 6 && !tree_tc))
    return fail(h, FRBX_EUNSUPPORTED,
                "window-tree fit needs power-of-two windows <= 64, Ls a multiple of 32 and Lm 16 or a multiple of 32 "
                "(tensor cores: Ls 128, "
                "2N <= 128, Lm a multiple of 32)");
  if (p.kernel == 4 || p.kernel >= 6 || (p.kernel == 0 && tree_ok)) {
    const int form = p.kernel >= 6 || (p.kernel == 0 && tree_tc) ? tc_form : -1;
    rc = run_fit_tree(h, a, nlev, form, windows, n_win, dkm, n_bl, T, n_dm, d_tab, L.S_tot, st, copied);
    if (rc) return rc;
  } else if (p.kernel == 3 || p.kernel == 5) {
    if (copied) FRBX_CK(h, cudaStreamWaitEvent(st, copied[n_bl - 1], 0));
    long long nv = 0;
    for (int v : L.n_valid) nv += v;
    rc = run_fit_mma(h, a, n_bl, false, nv * n_bl, p.kernel == 5, st);
    if (rc) return rc;
  } else {
    if (copied) FRBX_CK(h, cudaStreamWaitEvent(st, copied[n_bl - 1], 0));
    cudaError_t e = frbx::launch_fit(a, n_bl, false, p.kernel, st, &h->launches);
    if (e == cudaErrorInvalidConfiguration) return fail(h, FRBX_EUNSUPPORTED, "fit kernel does not fit this shape");
    FRBX_CK(h, e);
  }
  FRBX_CK(h, cudaEventRecord(h->ev[3], st));

  return finish_search(h, (const frbx_seg *)h->series.p, n_bl, T, dm, n_dm, n_win, L, d_tab, p, res, st);
}

namespace {
// After a failed call: wait for the work it queued (caller stream and the library's own
// streams), so the caller may release its buffers, and clear a non-sticky CUDA error.
void settle(frbx_handle *h, cudaStream_t st) {
  cudaStreamSynchronize(st);
  for (cudaStream_t x : h->tree_st)
    if (x) cudaStreamSynchronize(x);
  if (h->copy_st) cudaStreamSynchronize(h->copy_st);
  cudaGetLastError();
}
}  // namespace

extern "C" int frbx_fit_segments(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl,
                                 int32_t T, const double *dm, int32_t n_dm, const int32_t *segs,
                                 int64_t n_seg, const frbx_params *params, frbx_seg *out,
                                 void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  const int rc = fit_segments_impl(h, vis, vis_on_device, n_bl, T, dm, n_dm, segs, n_seg, params, out, cuda_stream);
  if (rc != FRBX_OK) settle(h, (cudaStream_t)cuda_stream);
  return rc;
}

extern "C" int frbx_search(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl,
                           int32_t T, const double *dm, int32_t n_dm, const int32_t *windows,
                           int32_t n_win, const frbx_params *params, frbx_results *res,
                           void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  const int rc = search_impl(h, vis, vis_on_device, n_bl, T, dm, n_dm, windows, n_win, params, res, cuda_stream);
  if (rc != FRBX_OK && rc != FRBX_ETRUNC) settle(h, (cudaStream_t)cuda_stream);
  return rc;
}

extern "C" int frbx_extract_events(const frbx_event *events, int64_t n_events, int32_t n_series,
                                   int32_t T, int32_t n_dm, const int32_t *windows, int32_t n_win,
                                   int32_t Lm, int32_t nwin_min, int32_t cross_match,
                                   frbx_cand *pulses, int64_t pulses_cap, int64_t *pulses_count,
                                   frbx_group *groups, int64_t groups_cap, int64_t *groups_count,
                                   frbx_cand *pre_merge, int64_t pre_cap, int64_t *pre_count) {
  if (n_events < 0 || (n_events > 0 && !events) || n_series < 1 || n_series > 64 || T < 1 || n_dm < 1 ||
      !windows || n_win < 1 || n_win > frbx::kMaxWin || Lm < 0 || nwin_min < 1)
    return FRBX_EINVAL;
  for (int w = 0; w < n_win; ++w) {
    if (windows[w] < 1) return FRBX_EINVAL;
    for (int v = 0; v < w; ++v)
      if (windows[v] == windows[w]) return FRBX_EINVAL;
  }
  for (int64_t i = 0; i < n_events; ++i) {
    const frbx_event &e = events[i];
    if (e.series < 0 || e.series >= n_series || e.dm_idx < 0 || e.dm_idx >= n_dm || e.win_idx < 0 ||
        e.win_idx >= n_win || e.k0 < 0 || e.k0 >= T || (Lm > 0 && e.mbd_idx >= Lm))
      return FRBX_EINVAL;
    if (i > 0) {
      const frbx_event &f = events[i - 1];
      const long long a[4] = {f.series, f.dm_idx, f.win_idx, f.k0}, b[4] = {e.series, e.dm_idx, e.win_idx, e.k0};
      if (!std::lexicographical_compare(a, a + 4, b, b + 4)) return FRBX_EINVAL;
    }
  }
  frbx::ExtractConfig cfg{T, n_dm, n_win, nwin_min, Lm, windows};
  std::vector<frbx::Pulse> pre, merged;
  std::vector<frbx::GroupOut> gr;
  frbx::extract_pulses(cfg, events, n_events, n_series, Lm > 0, &pre, &merged);
  if (cross_match) frbx::cross_match(T, &merged, n_series, &gr);
  bool trunc = false;
  auto put = [&](const std::vector<frbx::Pulse> &v, frbx_cand *dst, int64_t cap, int64_t *count) {
    if (count) *count = (int64_t)v.size();
    if (cap > 0 && (int64_t)v.size() > cap) trunc = true;
    if (!dst) return;
    for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)v.size()); ++i) {
      const frbx::Pulse &p = v[(size_t)i];
      frbx_cand &c = dst[i];
      std::memset(&c, 0, sizeof(c));
      c.series = p.series;
      c.dm_idx = p.d;
      c.win_idx = p.w;
      c.width = p.l;
      c.k0 = p.k0;
      c.sbd_idx = p.m;
      c.mbd_idx = p.q;
      c.n_win = p.n_win;
      c.group = p.group;
      c.amp = p.amp;
      c.pnorm = p.p;
    }
  };
  put(merged, pulses, pulses_cap, pulses_count);
  put(pre, pre_merge, pre_cap, pre_count);
  if (groups_count) *groups_count = (int64_t)gr.size();
  if (groups)
    for (int64_t i = 0; i < std::min<int64_t>(groups_cap, (int64_t)gr.size()); ++i) {
      groups[i].bl_mask = gr[(size_t)i].mask;
      groups[i].n_baselines = gr[(size_t)i].n_baselines;
      groups[i].n_pulses = gr[(size_t)i].n_pulses;
    }
  if (groups_cap > 0 && (int64_t)gr.size() > groups_cap) trunc = true;
  return trunc ? FRBX_ETRUNC : FRBX_OK;
}

extern "C" int frbx_last_stage_times(const frbx_handle *h, double *ms_out, int32_t n) {
  if (!h || !ms_out || n < 0) return FRBX_EINVAL;
  const int k = std::min(n, 9);
  for (int i = 0; i < k; ++i) ms_out[i] = h->stage_ms[i];
  return k;
}

namespace {

int refine_common(frbx_handle *h, const void *vis_dev, int32_t n_bl, int32_t T, const double *params_dev,
                  const int32_t *width_dev, int32_t n_cand, frbx::RefineArgs *r) {
  if (!vis_dev || !params_dev || !width_dev || n_cand < 0 || n_cand > 65535 * 256)
    return fail(h, FRBX_EINVAL, "bad refinement arguments");
  if (n_bl < 1 || n_bl > frbx::kMaxBl || n_bl > 65535 || T < 4) return fail(h, FRBX_EINVAL, "bad n_bl or T");
  if (((uintptr_t)vis_dev & 7u) != 0) return fail(h, FRBX_EINVAL, "vis must be 8-byte aligned");
  r->vis = (const float2 *)vis_dev;
  r->T = T;
  r->C = h->C;
  r->J = h->J;
  r->n_bl = n_bl;
  r->n_cand = n_cand;
  r->n_par = 2 + 3 * n_bl;
  r->f = h->d_f;
  r->f0 = h->d_f0;
  r->wrot = h->d_wrot;
  r->f0_min = *std::min_element(h->f0.begin(), h->f0.end());
  r->inv_fref2 = 1.0 / (h->f_ref * h->f_ref);
  r->f_bw = h->f_bw;
  r->t_ap = h->t_ap;
  r->params = params_dev;
  r->width = width_dev;
  return FRBX_OK;
}

}  // namespace

extern "C" int frbx_refine_power(frbx_handle *h, const void *vis_dev, int32_t n_bl, int32_t T,
                                 const double *params_dev, const int32_t *width_dev, int32_t n_cand,
                                 float *power_dev, float *g_dev, int32_t *status_dev, void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  h->launches = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  frbx::RefineArgs r{};
  int rc = refine_common(h, vis_dev, n_bl, T, params_dev, width_dev, n_cand, &r);
  if (rc) return rc;
  if (n_cand > 0 && (!power_dev || !g_dev || !status_dev)) return fail(h, FRBX_EINVAL, "missing output");
  r.g = g_dev;
  r.power = power_dev;
  r.status = status_dev;
  if (n_cand > 0) FRBX_CK(h, cudaMemsetAsync(status_dev, 0, sizeof(int32_t) * (size_t)n_cand, st));
  FRBX_CK(h, frbx::launch_refine(r, false, st, &h->launches));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

extern "C" int frbx_refine_adjoint(frbx_handle *h, const void *vis_dev, int32_t n_bl, int32_t T,
                                   const double *params_dev, const int32_t *width_dev, int32_t n_cand,
                                   const float *g_dev, const float *dpower_dev, float *dparams_dev,
                                   void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  h->launches = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  frbx::RefineArgs r{};
  int rc = refine_common(h, vis_dev, n_bl, T, params_dev, width_dev, n_cand, &r);
  if (rc) return rc;
  if (n_cand > 0 && (!g_dev || !dpower_dev || !dparams_dev)) return fail(h, FRBX_EINVAL, "missing input or output");
  FRBX_CK(h, ensure(h, h->refine, sizeof(float) * 2 * (size_t)n_cand * n_bl + 16));
  r.g = const_cast<float *>(g_dev);
  r.dpower = dpower_dev;
  r.dparams = dparams_dev;
  r.partial = (float *)h->refine.p;
  FRBX_CK(h, frbx::launch_refine(r, true, st, &h->launches));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

extern "C" int frbx_calibrate(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl, int32_t T,
                              int32_t k0, int32_t l, double *sbd_ns, double *mbd_ns, double *delay_ns,
                              double *phase_rad, void *cuda_stream) {
  if (!h) return FRBX_EINVAL;
  h->launches = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!sbd_ns || !mbd_ns || !delay_ns || !phase_rad) return fail(h, FRBX_EINVAL, "missing output");
  if (k0 < 0 || l < 1 || (long long)k0 + l > T) return fail(h, FRBX_EINVAL, "calibrator segment outside the scan");
  const float2 *dvis = nullptr;
  int rc = check_vis(h, vis, vis_on_device, n_bl, T, st, &dvis);
  if (rc) return rc;
  const int C = h->C, N = h->N;
  // scratch: FP64 sums, complex64 copy, unit weights, zero shifts, rows, fits, delays
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_xs = take(16 * (size_t)n_bl * C), o_xc = take(8 * (size_t)n_bl * C), o_w = take(8 * (size_t)C),
               o_dk = take(4 * (size_t)C), o_rows = take(16 * (size_t)n_bl), o_fit = take(8 * (size_t)n_bl),
               o_sm = take(16 * (size_t)n_bl), o_d = take(8 * (size_t)n_bl * N), o_p = take(8 * (size_t)n_bl * N);
  FRBX_CK(h, ensure(h, h->calib, off));
  unsigned char *b = (unsigned char *)h->calib.p;
  FRBX_CK(h, frbx::launch_cal_sum(dvis, T, C, n_bl, k0, l, h->d_wrot, (double2 *)(b + o_xs), (float2 *)(b + o_xc),
                                  (float2 *)(b + o_w), st, &h->launches));
  FRBX_CK(h, cudaMemsetAsync(b + o_dk, 0, 4 * (size_t)C, st));
  std::vector<int32_t> rows((size_t)4 * n_bl);
  for (int i = 0; i < n_bl; ++i) {
    rows[4 * i] = i;
    rows[4 * i + 1] = 0;
    rows[4 * i + 2] = 1;
    rows[4 * i + 3] = 0;
  }
  FRBX_CK(h, cudaMemcpyAsync(b + o_rows, rows.data(), 16 * (size_t)n_bl, cudaMemcpyHostToDevice, st));
  // (c) common fringe fit on the grid, no calibration rotation
  FitArgs a{};
  fill_fit_tables(h, &a, (const float2 *)(b + o_xc), 1, 1);
  a.dk = (const int *)(b + o_dk);
  a.wrot = (const float2 *)(b + o_w);
  a.m_lo = 0;
  a.m_len = h->Ls;
  a.q_lo = 0;
  a.q_len = h->Lm;
  a.seg = (const int *)(b + o_rows);
  a.n_seg = n_bl;
  a.tile = 16;
  a.out = (frbx_seg *)(b + o_fit);
  cudaError_t e = frbx::launch_fit(a, n_bl, true, 0, st, &h->launches);
  if (e == cudaErrorInvalidConfiguration) return fail(h, FRBX_EUNSUPPORTED, "fit kernel does not fit this shape");
  FRBX_CK(h, e);
  std::vector<frbx_seg> fits((size_t)n_bl);
  FRBX_CK(h, cudaMemcpyAsync(fits.data(), b + o_fit, 8 * (size_t)n_bl, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  std::vector<double> sm((size_t)2 * n_bl);
  for (int i = 0; i < n_bl; ++i) {
    const int m = fits[(size_t)i].sbd_idx, q = fits[(size_t)i].mbd_idx;
    const int sm_ = m < h->Ls / 2 ? m : m - h->Ls, sq = q < h->Lm / 2 ? q : q - h->Lm;
    sm[(size_t)2 * i] = (((double)sm_ * h->J) * 1000.0) / ((double)h->Ls * h->f_bw);
    sm[(size_t)2 * i + 1] = ((double)sq * 1000.0) / ((double)h->Lm * h->df_grid);
    sbd_ns[i] = sm[(size_t)2 * i];
    mbd_ns[i] = sm[(size_t)2 * i + 1];
  }
  FRBX_CK(h, cudaMemcpyAsync(b + o_sm, sm.data(), 16 * (size_t)n_bl, cudaMemcpyHostToDevice, st));
  const double f0_min = *std::min_element(h->f0.begin(), h->f0.end());
  FRBX_CK(h, frbx::launch_cal_channels((const double2 *)(b + o_xs), h->d_wrot, n_bl, N, h->J, h->f_bw, h->d_f0,
                                       f0_min, (const double *)(b + o_sm), (double *)(b + o_d),
                                       (double *)(b + o_p), st, &h->launches));
  FRBX_CK(h, cudaMemcpyAsync(delay_ns, b + o_d, 8 * (size_t)n_bl * N, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaMemcpyAsync(phase_rad, b + o_p, 8 * (size_t)n_bl * N, cudaMemcpyDeviceToHost, st));
  FRBX_CK(h, cudaStreamSynchronize(st));
  return FRBX_OK;
}

// ======================================================================================
// Batched search over many scans (several setups, uneven lengths) with a persistent,
// graph-captured fit and an autotuned time tile.
// ======================================================================================
struct frbx_batch {
  std::string err;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string key;
  int captures = 0, replays = 0;
  std::map<std::string, int> tuned_tt;  // setup shape + DM grid + windows -> time tile
  frbx_handle::Buf desc, tables, series, counters, tree_ser;
  std::vector<int> last_tt;
  double last_fit_ms = 0.0;
  int64_t launches = 0, graph_kernels = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t cap = nullptr;  // capture only (the legacy default stream cannot be captured)
};

namespace {

int bfail(frbx_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  return code;
}

#define FRBX_BCK(b, call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      cudaGetLastError();                                                                  \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? FRBX_ENOMEM : FRBX_ECUDA,        \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    }                                                                                      \
  } while (0)

struct ScanPlan {
  int setup;          // index into the unique setups
  Layout L;
  size_t series_off;  // element offset in the batch series buffer
  size_t nval_off;    // int offset of its valid-count table in the tables buffer
};

constexpr int kTuneTT[] = {32, 64, 128};

}  // namespace

extern "C" int frbx_batch_create(frbx_batch **out) {
  if (!out) return FRBX_EINVAL;
  *out = new frbx_batch();
  return FRBX_OK;
}

extern "C" void frbx_batch_destroy(frbx_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (frbx_handle::Buf *x : {&b->desc, &b->tables, &b->series, &b->counters, &b->tree_ser})
    if (x->p) cudaFree(x->p);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

extern "C" const char *frbx_batch_last_error(const frbx_batch *b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int frbx_batch_info(const frbx_batch *b, frbx_batch_stats *st) {
  if (!b || !st) return FRBX_EINVAL;
  std::memset(st, 0, sizeof(*st));
  st->graph_captures = b->captures;
  st->graph_replays = b->replays;
  st->n_setups = (int32_t)b->last_tt.size();
  for (size_t i = 0; i < b->last_tt.size() && i < 16; ++i) st->time_tile[i] = b->last_tt[i];
  st->fit_ms = b->last_fit_ms;
  st->launches = b->launches;
  return FRBX_OK;
}

extern "C" int frbx_search_batch(frbx_batch *b, const frbx_scan *scans, int32_t n_scans, const double *dm,
                                 int32_t n_dm, const int32_t *windows, int32_t n_win, const frbx_params *params,
                                 frbx_results *results, void *cuda_stream) {
  if (!b) return FRBX_EINVAL;
  b->err.clear();
  b->launches = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!scans || n_scans < 1 || n_scans > 4096 || !results) return bfail(b, FRBX_EINVAL, "need 1..4096 scans and results");
  if (!dm || n_dm < 1) return bfail(b, FRBX_EINVAL, "need at least one DM trial");
  if (!windows || n_win < 1 || n_win > frbx::kMaxWin) return bfail(b, FRBX_EINVAL, "need 1..16 windows");
  for (int w = 0; w < n_win; ++w) {
    if (windows[w] < 1) return bfail(b, FRBX_EINVAL, "window lengths must be >= 1");
    for (int v = 0; v < w; ++v)
      if (windows[v] == windows[w]) return bfail(b, FRBX_EINVAL, "window lengths must be distinct");
  }
  frbx_params p;
  if (params) p = *params; else frbx_default_params(&p);
  if (p.kernel < 0 || p.kernel > 6 || p.kernel == 3 || p.kernel == 5)
    return bfail(b, FRBX_EINVAL, "batched search runs kernels 0, 1, 2, 4 or 6");
  // unique setups in order of first appearance
  std::vector<frbx_handle *> setups;
  std::vector<ScanPlan> plan((size_t)n_scans);
  for (int i = 0; i < n_scans; ++i) {
    const frbx_scan &sc = scans[i];
    if (!sc.setup || !sc.vis_dev || sc.n_bl < 1 || sc.n_bl > frbx::kMaxBl || sc.T < 1 ||
        ((uintptr_t)sc.vis_dev & 7u))
      return bfail(b, FRBX_EINVAL, "scan " + std::to_string(i) + ": bad setup, cube, n_bl or T");
    for (int c = 0; c < p.n_combo; ++c)
      if (p.combos && sc.n_bl < 64 && (p.combos[c] >> sc.n_bl) != 0)
        return bfail(b, FRBX_EINVAL, "scan " + std::to_string(i) + ": combo mask names a missing baseline");
    auto it = std::find(setups.begin(), setups.end(), sc.setup);
    plan[(size_t)i].setup = (int)(it - setups.begin());
    if (it == setups.end()) setups.push_back(sc.setup);
  }
  if (setups.size() > 16) return bfail(b, FRBX_EINVAL, "at most 16 setups per batch");
  // per setup: parameter checks and the shift table of the DM grid (h->dk, read by the fit)
  std::vector<FitArgs> fa(setups.size());
  std::vector<std::vector<int>> dkm(setups.size());
  for (size_t g = 0; g < setups.size(); ++g) {
    frbx_handle *h = setups[g];
    h->err.clear();
    int rc = check_params(h, &p, 64, &fa[g]);
    if (!rc) rc = run_shift_table(h, dm, n_dm, &dkm[g], st);
    if (rc) return bfail(b, rc, "setup " + std::to_string(g) + ": " + h->err);
  }
  // window-tree fit where it applies (kernel 0) or is asked for (kernel 4)
  std::vector<int> tree_lev(setups.size(), -1);
  std::vector<char> tree_tc(setups.size(), 0);
  for (size_t g = 0; g < setups.size(); ++g) {
    frbx_handle *h = setups[g];
    int nlev = 0;
    const bool ok = frbx::tree_supported(h->Ls, h->Lm, h->N, h->J, h->tree_s16, windows, n_win, &nlev);
    const FitArgs &ag = fa[g];
    const bool tc_ok = ok && h->d_wtree && frbx::tree_mma_supported(h->Ls, h->Lm, h->N, h->J) &&
                       frbx::tree_mma_fits(0, h->N, nlev);
    (void)ag;
    if ((p.kernel == 4 && !ok) || (p.kernel == 6 && !tc_ok))
      return bfail(b, FRBX_EUNSUPPORTED, "setup " + std::to_string(g) + ": window-tree fit does not apply");
    if (ok && (p.kernel == 0 || p.kernel == 4 || p.kernel == 6)) {
      tree_lev[g] = nlev;
      tree_tc[g] = (p.kernel == 6 || (p.kernel == 0 && tc_ok)) ? 1 : 0;
    }
  }
  // layouts, valid-segment counts, window offsets and series offsets of every scan; one device
  // table: win_len[16] | per scan: win_off[16], n_valid[n_dm][n_win]
  std::vector<int> tab(windows, windows + n_win);
  tab.resize(frbx::kMaxWin, 0);
  std::vector<size_t> woff_at((size_t)n_scans);
  size_t series_total = 0;
  for (int i = 0; i < n_scans; ++i) {
    ScanPlan &sp = plan[(size_t)i];
    const int T = scans[i].T;
    long long stot = 0;
    sp.L.win_len.assign(windows, windows + n_win);
    for (int w = 0; w < n_win; ++w) {
      sp.L.win_off.push_back((int)stot);
      sp.L.win_step.push_back(window_step(windows[w]));
      stot += n_slots(T, windows[w]);
    }
    if (stot > (1LL << 30)) return bfail(b, FRBX_EUNSUPPORTED, "too many segments per series");
    sp.L.S_tot = (int)stot;
    sp.L.n_valid.resize((size_t)n_dm * n_win);
    for (int d = 0; d < n_dm; ++d)
      for (int w = 0; w < n_win; ++w)
        sp.L.n_valid[(size_t)d * n_win + w] = n_valid(T, windows[w], dkm[(size_t)sp.setup][(size_t)d]);
    woff_at[(size_t)i] = tab.size();
    tab.insert(tab.end(), sp.L.win_off.begin(), sp.L.win_off.end());
    tab.resize(tab.size() + (size_t)(frbx::kMaxWin - n_win), 0);
    sp.nval_off = tab.size();
    tab.insert(tab.end(), sp.L.n_valid.begin(), sp.L.n_valid.end());
    sp.series_off = series_total;
    series_total += (size_t)scans[i].n_bl * n_dm * sp.L.S_tot;
  }
  FRBX_BCK(b, ensure(b->tables, sizeof(int) * tab.size()));
  FRBX_BCK(b, cudaMemcpyAsync(b->tables.p, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, st));
  FRBX_BCK(b, ensure(b->series, sizeof(frbx_seg) * std::max<size_t>(series_total, 1)));
  FRBX_BCK(b, ensure(b->counters, 256 * (setups.size() + 1)));
  FRBX_BCK(b, ensure(b->desc, sizeof(frbx::BatchScan) * (size_t)n_scans * 2));
  const int *d_tab = (const int *)b->tables.p;
  frbx_seg *d_series = (frbx_seg *)b->series.p;
  frbx::BatchScan *d_desc = (frbx::BatchScan *)b->desc.p;
  unsigned int *d_cnt = (unsigned int *)b->counters.p;
  if (!b->e0) FRBX_BCK(b, cudaEventCreate(&b->e0));
  if (!b->e1) FRBX_BCK(b, cudaEventCreate(&b->e1));

  // descriptors of the scans of setup g (in scan order), with time tile TT
  auto make_desc = [&](int g, int TT, std::vector<frbx::BatchScan> *desc) {
    long long item = 0;
    desc->clear();
    for (int i = 0; i < n_scans; ++i) {
      if (plan[(size_t)i].setup != g) continue;
      frbx::BatchScan d{};
      d.vis = (const float2 *)scans[i].vis_dev;
      d.out = d_series + plan[(size_t)i].series_off;
      d.n_valid = d_tab + plan[(size_t)i].nval_off;
      d.win_off = d_tab + woff_at[(size_t)i];
      d.T = scans[i].T;
      d.S_tot = plan[(size_t)i].L.S_tot;
      d.n_bl = scans[i].n_bl;
      d.n_tt = (scans[i].T + TT - 1) / TT;
      d.item0 = item;
      item += (long long)d.n_bl * d.n_tt * n_dm;
      desc->push_back(d);
    }
    return item;
  };
  auto fit_args = [&](int g, int TT) {
    FitArgs a;
    std::memcpy(&a, &fa[(size_t)g], sizeof(a));
    fill_fit_tables(setups[(size_t)g], &a, nullptr, 0, n_dm);
    a.n_win = n_win;
    a.win_len = d_tab;
    a.win_off = nullptr;
    a.n_valid = nullptr;
    a.TT = TT;
    a.tile = 64;
    return a;
  };

  // time tile per setup: measured once per (setup shape, DM count, windows, kernel) and kept.
  // Every candidate fits the same leading stretch of the setup's items (4096 AP-baselines of
  // every DM trial, or all of them), twice; the faster minimum wins.
  b->last_tt.assign(setups.size(), 64);
  std::vector<frbx::BatchScan> desc;
  for (size_t g = 0; g < setups.size(); ++g) {
    frbx_handle *h = setups[g];
    if (tree_lev[g] >= 0) {  // the window tree's time tile is measured with its own passes below
      b->last_tt[g] = kTreeTT;
      continue;
    }
    std::string tkey = std::to_string(h->N) + "x" + std::to_string(h->J) + "/" + std::to_string(h->Ls) + "/" +
                       std::to_string(h->Lm) + "/" + std::to_string(n_dm);
    for (int w = 0; w < n_win; ++w) tkey += "," + std::to_string(windows[w]);
    tkey += "/" + std::to_string(p.kernel) + "/" + std::to_string(fa[g].m_len) + "x" + std::to_string(fa[g].q_len);
    auto hit = b->tuned_tt.find(tkey);
    if (hit != b->tuned_tt.end()) {
      b->last_tt[g] = hit->second;
      continue;
    }
    float best_ms = 1e30f;
    int best_tt = 64;
    for (int TT : kTuneTT) {
      const long long total = make_desc((int)g, TT, &desc);
      FRBX_BCK(b, cudaMemcpyAsync(d_desc, desc.data(), sizeof(frbx::BatchScan) * desc.size(), cudaMemcpyHostToDevice,
                                  st));
      const FitArgs a = fit_args((int)g, TT);
      const long long sample = std::min<long long>(total, (long long)n_dm * (4096 / TT));
      float ms_min = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        FRBX_BCK(b, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned int), st));
        FRBX_BCK(b, cudaEventRecord(b->e0, st));
        cudaError_t e = frbx::launch_fit_batch(a, d_desc, (int)desc.size(), sample, d_cnt, p.kernel, 0, st,
                                               &b->launches);
        if (e == cudaErrorInvalidConfiguration)
          return bfail(b, FRBX_EUNSUPPORTED, "fit kernel does not fit setup " + std::to_string(g));
        FRBX_BCK(b, e);
        FRBX_BCK(b, cudaEventRecord(b->e1, st));
        FRBX_BCK(b, cudaEventSynchronize(b->e1));
        float ms = 0.f;
        FRBX_BCK(b, cudaEventElapsedTime(&ms, b->e0, b->e1));
        ms_min = std::min(ms_min, ms);
      }
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best_tt = TT;
      }
    }
    b->tuned_tt[tkey] = best_tt;
    b->last_tt[g] = best_tt;
  }

  // descriptors with the chosen tiles; the graph is re-captured only when they change
  const size_t half = (size_t)n_scans;  // second half of the descriptor buffer: graph copies
  std::vector<frbx::BatchScan> all;
  std::vector<long long> totals(setups.size());
  std::vector<size_t> first(setups.size());
  for (size_t g = 0; g < setups.size(); ++g) {
    totals[g] = make_desc((int)g, b->last_tt[g], &desc);
    if (totals[g] > 0x7fffffffLL) return bfail(b, FRBX_EUNSUPPORTED, "too many work items for one setup");
    first[g] = all.size();
    all.insert(all.end(), desc.begin(), desc.end());
  }
  FRBX_BCK(b, cudaMemcpyAsync(d_desc + half, all.data(), sizeof(frbx::BatchScan) * all.size(), cudaMemcpyHostToDevice,
                              st));
  // window-tree scans: plans, per-setup scratch sized for the largest, series lists uploaded
  std::vector<TreeRun> truns((size_t)n_scans);
  std::vector<FitArgs> targs((size_t)n_scans);
  std::vector<size_t> tser_off((size_t)n_scans, 0);
  std::vector<size_t> need_h(setups.size(), 0);
  std::vector<int2> tser_all;
  size_t n_tree_setups = 0;
  for (size_t g = 0; g < setups.size(); ++g) n_tree_setups += tree_lev[g] >= 0;
  int64_t tree_launches = 0;
  if (n_tree_setups) {
    for (size_t g = 0; g < setups.size(); ++g)
      if (tree_lev[g] >= 0) FRBX_BCK(b, ensure(setups[g], setups[g]->errflag, sizeof(int)));
    size_t free_b = 0, total_b = 0;
    FRBX_BCK(b, cudaMemGetInfo(&free_b, &total_b));
    auto tree_budget = [&](const frbx_handle *h) {
      return h->lim.tree_chunk_bytes > 0
                 ? (size_t)h->lim.tree_chunk_bytes
                 : std::min<size_t>((size_t)16 << 30, (free_b + h->ytree.bytes) / (4 * n_tree_setups));
    };
    auto tree_args = [&](int i) {
      const int g = plan[(size_t)i].setup;
      FitArgs a = fit_args(g, 1024);
      fill_fit_tables(setups[(size_t)g], &a, (const float2 *)scans[i].vis_dev, scans[i].T, n_dm);
      a.win_off = d_tab + woff_at[(size_t)i];
      a.n_valid = d_tab + plan[(size_t)i].nval_off;
      a.S_tot = plan[(size_t)i].L.S_tot;
      a.out = d_series + plan[(size_t)i].series_off;
      return a;
    };
    // the window tree's time tile per setup: measured once per (setup shape, DM count, windows,
    // form, delay window) on one chunk of the series of the setup's longest scan, twice per
    // candidate; the faster minimum wins (the real fit below rewrites that scan's series)
    for (size_t g = 0; g < setups.size(); ++g) {
      if (tree_lev[g] < 0) continue;
      frbx_handle *h = setups[g];
      std::string tkey = "tree/" + std::to_string(h->N) + "x" + std::to_string(h->J) + "/" + std::to_string(h->Ls) +
                         "/" + std::to_string(h->Lm) + "/" + std::to_string(n_dm) + "/" + std::to_string(tree_tc[g]);
      for (int w = 0; w < n_win; ++w) tkey += "," + std::to_string(windows[w]);
      tkey += "/" + std::to_string(fa[g].m_lo) + "+" + std::to_string(fa[g].m_len) + "x" + std::to_string(fa[g].q_lo) +
              "+" + std::to_string(fa[g].q_len);
      auto hit = b->tuned_tt.find(tkey);
      if (hit != b->tuned_tt.end()) {
        b->last_tt[g] = hit->second;
        continue;
      }
      int i_g = -1;
      for (int i = 0; i < n_scans; ++i)
        if (plan[(size_t)i].setup == (int)g && (i_g < 0 || scans[i].T > scans[i_g].T)) i_g = i;
      float best_ms = 1e30f;
      int best_tt = kTreeTT;
      for (int TT : kTreeTuneTT) {
        if (i_g < 0) break;
        const FitArgs a = tree_args(i_g);
        TreeRun r;
        plan_tree(h, a, tree_lev[g], windows, n_win, dkm[g], scans[i_g].n_bl, scans[i_g].T, n_dm, a.win_off, a.S_tot,
                  tree_budget(h), tree_tc[g] != 0 ? 0 : -1, &r, TT);
        if (r.ser.empty()) break;
        r.ser.resize(std::min(r.ser.size(), r.chunk));
        if (ensure(h, h->ytree, r.need()) != cudaSuccess || tree_prepare(h) != FRBX_OK) {
          cudaGetLastError();
          return bfail(b, FRBX_ENOMEM, "setup " + std::to_string(g) + ": window-tree scratch");
        }
        FRBX_BCK(b, ensure(b->tree_ser, sizeof(int2) * r.ser.size()));
        FRBX_BCK(b, cudaMemcpyAsync(b->tree_ser.p, r.ser.data(), sizeof(int2) * r.ser.size(), cudaMemcpyHostToDevice,
                                    st));
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          FRBX_BCK(b, cudaEventRecord(b->e0, st));
          const int rc = enqueue_tree(h, a, r, (const int2 *)b->tree_ser.p, (char *)h->ytree.p, false, n_win, d_tab,
                                      d_tab + woff_at[(size_t)i_g], d_tab + plan[(size_t)i_g].nval_off, st);
          if (rc) return bfail(b, rc, "setup " + std::to_string(g) + ": " + h->err);
          FRBX_BCK(b, cudaEventRecord(b->e1, st));
          FRBX_BCK(b, cudaEventSynchronize(b->e1));
          float ms = 0.f;
          FRBX_BCK(b, cudaEventElapsedTime(&ms, b->e0, b->e1));
          ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
          best_ms = ms_min;
          best_tt = TT;
        }
      }
      b->tuned_tt[tkey] = best_tt;
      b->last_tt[g] = best_tt;
    }
    for (int i = 0; i < n_scans; ++i) {
      const int g = plan[(size_t)i].setup;
      if (tree_lev[(size_t)g] < 0) continue;
      frbx_handle *h = setups[(size_t)g];
      const FitArgs a = tree_args(i);
      targs[(size_t)i] = a;
      plan_tree(h, a, tree_lev[(size_t)g], windows, n_win, dkm[(size_t)g], scans[i].n_bl, scans[i].T, n_dm,
                a.win_off, a.S_tot, tree_budget(h), tree_tc[(size_t)g] != 0 ? 0 : -1, &truns[(size_t)i],
                b->last_tt[(size_t)g]);
      need_h[(size_t)g] = std::max(need_h[(size_t)g], truns[(size_t)i].need());
      tser_off[(size_t)i] = tser_all.size();
      tser_all.insert(tser_all.end(), truns[(size_t)i].ser.begin(), truns[(size_t)i].ser.end());
      tree_launches += 2 * (int64_t)((truns[(size_t)i].ser.size() + truns[(size_t)i].chunk - 1) / truns[(size_t)i].chunk) + 1;
    }
    for (size_t g = 0; g < setups.size(); ++g) {
      if (tree_lev[g] < 0) continue;
      frbx_handle *h = setups[g];
      if (ensure(h, h->errflag, sizeof(int)) != cudaSuccess || ensure(h, h->ytree, need_h[g]) != cudaSuccess ||
          tree_prepare(h) != FRBX_OK) {
        cudaGetLastError();
        return bfail(b, FRBX_ENOMEM, "setup " + std::to_string(g) + ": window-tree scratch");
      }
    }
    FRBX_BCK(b, ensure(b->tree_ser, sizeof(int2) * std::max<size_t>(tser_all.size(), 1)));
    if (!tser_all.empty())
      FRBX_BCK(b, cudaMemcpyAsync(b->tree_ser.p, tser_all.data(), sizeof(int2) * tser_all.size(),
                                  cudaMemcpyHostToDevice, st));
  }
  std::string key = std::to_string(n_scans) + ":" + std::to_string(n_dm) + ":" + std::to_string(p.kernel) + ":" +
                    std::to_string((uintptr_t)b->desc.p) + ":" + std::to_string((uintptr_t)b->counters.p);
  for (size_t g = 0; g < setups.size(); ++g) {
    // the launch parameters baked into the graph, byte for byte
    const FitArgs a = fit_args((int)g, b->last_tt[g]);
    key += "|" + std::to_string(totals[g]) + "/" + std::to_string(first[g]) + "/";
    key.append(reinterpret_cast<const char *>(&a), sizeof(a));
  }
  for (int i = 0; i < n_scans; ++i) {
    if (tree_lev[(size_t)plan[(size_t)i].setup] < 0) continue;
    const frbx::TreeArgs &tt = truns[(size_t)i].t;
    key += "|t" + std::to_string(i) + ":" + std::to_string(truns[(size_t)i].chunk) + ":" +
           std::to_string((uintptr_t)setups[(size_t)plan[(size_t)i].setup]->ytree.p) + ":" +
           std::to_string((uintptr_t)b->tree_ser.p) + "/";
    key.append(reinterpret_cast<const char *>(&tt), sizeof(tt));
    key.append(reinterpret_cast<const char *>(&targs[(size_t)i]), sizeof(FitArgs));
  }
  if (b->key != key || !b->exec) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->key.clear();
    // the graph is recorded on a private stream and launched on the caller's
    if (!b->cap) FRBX_BCK(b, cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    cudaStream_t cs = b->cap;
    FRBX_BCK(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaError_t ce = cudaSuccess;
    int64_t graph_launches = 0;
    for (size_t g = 0; g < setups.size() && ce == cudaSuccess; ++g) {
      if (tree_lev[g] >= 0) continue;
      unsigned int *cnt = d_cnt + 64 * (g + 1);
      ce = cudaMemsetAsync(cnt, 0, sizeof(unsigned int), cs);
      if (ce == cudaSuccess) {
        const size_t nd = (g + 1 < setups.size() ? first[g + 1] : all.size()) - first[g];
        ce = frbx::launch_fit_batch(fit_args((int)g, b->last_tt[g]), d_desc + half + first[g], (int)nd, totals[g],
                                    cnt, p.kernel, 0, cs, &graph_launches);
      }
    }
    int trc = FRBX_OK;
    for (size_t g = 0; g < setups.size() && ce == cudaSuccess; ++g)
      if (tree_lev[g] >= 0) ce = cudaMemsetAsync(setups[g]->errflag.p, 0, sizeof(int), cs);
    for (int i = 0; i < n_scans && ce == cudaSuccess && trc == FRBX_OK; ++i) {
      const int g = plan[(size_t)i].setup;
      if (tree_lev[(size_t)g] < 0) continue;
      frbx_handle *h = setups[(size_t)g];
      trc = enqueue_tree(h, targs[(size_t)i], truns[(size_t)i], (const int2 *)b->tree_ser.p + tser_off[(size_t)i],
                         (char *)h->ytree.p, false, n_win, d_tab, d_tab + woff_at[(size_t)i],
                         d_tab + plan[(size_t)i].nval_off, cs);
      if (trc) b->err = "scan " + std::to_string(i) + ": " + h->err;
    }
    graph_launches += tree_launches;
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (trc != FRBX_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return bfail(b, trc, b->err);
    }
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return bfail(b, ce == cudaErrorInvalidConfiguration ? FRBX_EUNSUPPORTED : FRBX_ECUDA,
                   std::string("fit graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      b->exec = nullptr;
      cudaGetLastError();
      return bfail(b, FRBX_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
    }
    b->graph = graph;
    b->graph_kernels = graph_launches;
    b->key = key;
    ++b->captures;
  } else {
    ++b->replays;
  }
  FRBX_BCK(b, cudaEventRecord(b->e0, st));
  FRBX_BCK(b, cudaGraphLaunch(b->exec, st));
  FRBX_BCK(b, cudaEventRecord(b->e1, st));
  FRBX_BCK(b, cudaEventSynchronize(b->e1));
  {
    float ms = 0.f;
    FRBX_BCK(b, cudaEventElapsedTime(&ms, b->e0, b->e1));
    b->last_fit_ms = ms;
  }
  b->launches += b->graph_kernels;
  for (size_t g = 0; g < setups.size(); ++g) {
    if (!tree_tc[g]) continue;
    int flag = 0;
    FRBX_BCK(b, cudaMemcpy(&flag, setups[g]->errflag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return bfail(b, FRBX_ETIMEOUT, "setup " + std::to_string(g) + ": a bounded wait of the fit gave up");
  }

  // per scan: Eq. 6 and threshold on the device, then the host extraction, as in frbx_search;
  // the scan's window tables go to the head of its setup's small buffer in that layout
  bool trunc = false;
  for (int i = 0; i < n_scans; ++i) {
    frbx_handle *h = setups[(size_t)plan[(size_t)i].setup];
    const Layout &L = plan[(size_t)i].L;
    std::vector<int> t2(3 * frbx::kMaxWin, 0);
    for (int w = 0; w < n_win; ++w) {
      t2[(size_t)w] = windows[w];
      t2[(size_t)frbx::kMaxWin + w] = L.win_off[(size_t)w];
      t2[(size_t)2 * frbx::kMaxWin + w] = L.win_step[(size_t)w];
    }
    t2.insert(t2.end(), L.n_valid.begin(), L.n_valid.end());
    h->err.clear();
    h->launches = 0;
    h->tree_chunks = 0;
    int rc = FRBX_OK;
    if (ensure(h, h->small, sizeof(int) * t2.size() + 4096) != cudaSuccess ||
        cudaMemcpyAsync(h->small.p, t2.data(), sizeof(int) * t2.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, FRBX_ECUDA, "scan " + std::to_string(i) + ": table upload failed");
    }
    for (cudaEvent_t &ev : h->ev)
      if (!ev && cudaEventCreate(&ev) != cudaSuccess) return bfail(b, FRBX_ECUDA, "cudaEventCreate failed");
    for (int k = 0; k < 4; ++k) cudaEventRecord(h->ev[k], st);
    rc = finish_search(h, d_series + plan[(size_t)i].series_off, scans[i].n_bl, scans[i].T, dm, n_dm, n_win, L,
                       (const int *)h->small.p, p, &results[i], st);
    b->launches += h->launches;
    if (rc == FRBX_ETRUNC) trunc = true;
    else if (rc) return bfail(b, rc, "scan " + std::to_string(i) + ": " + h->err);
  }
  if (trunc) return bfail(b, FRBX_ETRUNC, "an output array was too small");
  return FRBX_OK;
}
