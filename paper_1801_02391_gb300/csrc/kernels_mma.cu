// Segment fit with the MBD transform as a BF16 or FP8 (E4M3) DFT-GEMM on the tcgen05 tensor cores
// (Eq. 3 gather and the SBD transform in FP32 on the CUDA cores, Eq. 5's sum over channels
// as a dense GEMM with FP32 accumulation in tensor memory, grid maximum on the CUDA cores).
//
// For one M = 128 row tile (Ls = 128: one segment; Ls = 64: two), with K = 2N real inputs
// per row (Re Y, Im Y of every channel) and the output columns split in chunks of NC:
//     D[m][c] = sum_k A[m][k] B[c][k],  A[m][n] = Re Y(n, m), A[m][N + n] = Im Y(n, m),
//     B rows of a chunk: first NC/2 give Re G(m, q), the next NC/2 give Im G(m, q) with
//     Re G = sum_n Re Y cos th + Im Y sin th,  Im G = sum_n Im Y cos th - Re Y sin th,
//     th = 2 pi (g_n q mod Lm) / Lm  (the phase index is exact; only cos/sin are rounded).
// FP8 form: A holds s Y in E4M3 with s the power of two for which s times the L1 norm of the
// segment's spectrum is at most 448 (so no element can leave E4M3's finite range), B holds
// cos / sin in E4M3, the MMA is kind::f8f6f4 with K = 32 per instruction, and the epilogue
// divides the segment's maximum |G|^2 by s^2.
//
// Roles (416 threads): two producer groups (warps 0-3 and 4-7) each gather a segment and run
// its SBD FFT into an A tile (BF16, 128B-swizzled, K-major) of a three-tile ring; warp 12
// allocates tensor memory and one lane issues tcgen05.mma per chunk into one of two
// accumulator slots; warps 8-11 read the slot back with tcgen05.ld (warp w reads lanes
// 32 (w % 4) ..), form |G|^2 and keep the maximum.  Hand-offs use mbarriers; every wait is
// bounded by a clock limit after which the kernel records FRBX_ETIMEOUT, drains, frees its
// tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fft32.cuh"
#include "fit_common.cuh"
#include "tc_common.cuh"

namespace frbx {

using tc::a_offset;
using tc::a_offset8;
using tc::desc_sw128;
using tc::mbar_arrive;
using tc::mbar_init;
using tc::mbar_wait;
using tc::named_sync;
using tc::named_sync_or;
using tc::su32;

namespace {

constexpr int kGroups = 2;                         // producer groups, each fits its own segment
constexpr int kGroupWarps = 4;
constexpr int kGroupThreads = kGroupWarps * 32;    // 128
constexpr int kEpiWarps = 4;                       // one per TMEM lane quarter
constexpr int kEpiWarp0 = kGroups * kGroupWarps;   // warps 8..11: lane quarter = warp % 4
constexpr int kMmaWarp = kEpiWarp0 + kEpiWarps;    // warp 12
constexpr int kMmaThreads = (kMmaWarp + 1) * 32;   // 416: 13 warps, at most 4 per SM sub-partition
constexpr int kABufs = 3;                          // ring of A tiles
constexpr int kRows = 128;                         // M of one MMA tile
constexpr int kAtomBytes = kRows * 128;            // one 64-wide K atom of an A tile (16 KB)
constexpr int kGatherBatch = 16;                   // independent loads in flight per thread
constexpr int kBarGroup0 = 1, kBarEpi = 3;         // named barrier ids (group g uses 1 + g)
constexpr int kListItem = 64;                      // list mode: rows per work item
constexpr int kScaleRing = 16;                     // FP8: per-tile segment scales in flight

struct MmaLayout {
  size_t b_off, a_off, x_off, stw_off, bytes;
  int xs, ts;
};

__host__ __device__ inline MmaLayout mma_layout(const MmaArgs &m, int N, int Ls, int J1) {
  MmaLayout l;
  l.b_off = 0;
  l.a_off = (size_t)m.b_bytes;
  l.x_off = l.a_off + kABufs * (size_t)m.KA * kAtomBytes;
  l.xs = J1 * 32 + 1;
  l.ts = J1 * 32 + 1;
  l.stw_off = l.x_off + kGroups * sizeof(float2) * (size_t)N * l.xs;
  l.bytes = l.stw_off + sizeof(float2) * (size_t)(Ls / 32) * l.ts + 1024;  // +1024: base alignment
  return l;
}

// The valid segments of one work item (baseline, time tile of TT APs, DM trial), window by
// window in the caller's order, then by start AP.  Items are numbered with the DM fastest,
// so the CTAs working at one time cover one stretch of the cube and its dispersion halo.
struct ItemTab {
  int lo[kMaxWin], cum[kMaxWin + 1], len[kMaxWin], off[kMaxWin];
  int bl, d, nseg, tiles;
};

__device__ __forceinline__ void item_decode(const FitArgs &a, long long item, int &bl, int &tt, int &d) {
  d = (int)(item % a.n_dm);
  const long long r = item / a.n_dm;
  const int n_tt = (a.T + a.TT - 1) / a.TT;
  tt = (int)(r % n_tt);
  bl = (int)(r / n_tt);
}

// Valid-segment count of window w in the item (and its first slot).
__device__ __forceinline__ int item_window(const FitArgs &a, int tt, int d, int w, int &lo) {
  const int t0 = tt * a.TT;
  const int l = a.win_len[w], step = max(1, l / 2);
  const int ns = a.T >= l ? (a.T - l) / step + 1 : 0;
  lo = (t0 + step - 1) / step;
  const int hi = min(min((t0 + a.TT + step - 1) / step, ns), a.n_valid[d * a.n_win + w]);
  return max(0, hi - lo);
}

__device__ __forceinline__ int item_tiles(const FitArgs &a, long long item, int spt) {
  int bl, tt, d, lo, n = 0;
  item_decode(a, item, bl, tt, d);
  for (int w = 0; w < a.n_win; ++w) n += item_window(a, tt, d, w, lo);
  return (n + spt - 1) / spt;
}

__device__ __forceinline__ void item_table(const FitArgs &a, long long item, int spt, ItemTab &t) {
  int tt;
  item_decode(a, item, t.bl, tt, t.d);
  int c = 0;
  for (int w = 0; w < a.n_win; ++w) {
    int lo;
    const int n = item_window(a, tt, t.d, w, lo);
    t.lo[w] = lo;
    t.cum[w] = c;
    t.len[w] = a.win_len[w];
    t.off[w] = a.win_off[w];
    c += n;
  }
  t.cum[a.n_win] = c;
  t.nseg = c;
  t.tiles = (c + spt - 1) / spt;
}

// Segment k of the current item (implicit layout) or row v of the list.
__device__ __forceinline__ void item_segment(const FitArgs &a, const ItemTab &t, int k, int n_win, int &l,
                                             int &k0, long long &out) {
  int w = 0;
  while (k >= t.cum[w + 1]) ++w;
  const int s = t.lo[w] + (k - t.cum[w]);
  l = t.len[w];
  k0 = s * max(1, l / 2);
  out = ((long long)t.bl * a.n_dm + t.d) * a.S_tot + t.off[w] + s;
  (void)n_win;
}

// Tile sequence of a CTA: items blockIdx.x, blockIdx.x + gridDim.x, ... (list mode: one
// "item" holding rows [0, n_seg)), each cut into tiles of spt segments.
struct Cursor {
  long long item;
  int tile_in_item, tiles;
};

}  // namespace

template <bool kFp8>
__global__ void __launch_bounds__(kMmaThreads, 1)
    k_fit_mma(const __grid_constant__ FitArgs a, const __grid_constant__ MmaArgs mm, int list) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_afull[kABufs], bar_aempty[kABufs], bar_accfull[2], bar_accempty[2], bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float red_p[kEpiWarps];
  __shared__ int red_i[kEpiWarps];
  __shared__ ItemTab tabs[kGroups + 1];  // producer groups, epilogue
  // FP8: 1/s^2 of each segment of a tile (A holds s Y, s a power of two), tagged by tile number
  __shared__ float sc_inv2[kScaleRing][2];
  __shared__ long long sc_tag[kScaleRing];
  __shared__ float l1_part[kGroups][kGroupWarps];

  const int N = a.N, Ls = a.Ls, Lm = a.Lm, C = a.C;
  const int PS = Ls >> 5, lps = __ffs(PS) - 1;
  const MmaLayout L = mma_layout(mm, N, Ls, a.J1);
  unsigned char *sB = smem + L.b_off;
  unsigned char *sA = smem + L.a_off;
  float2 *stw = reinterpret_cast<float2 *>(smem + L.stw_off);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int JP = a.J1 * 32;
  const int SPT = mm.spt;
  // list mode: items are runs of kListItem rows; implicit: n_bl * n_tt * n_dm items
  const long long n_items = list ? (mm.n_valid + kListItem - 1) / kListItem : mm.n_items;

  // ---- set-up: constant operand B, SBD twiddles, zeroed A tiles and X, barriers, TMEM
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(mm.bimg);
    uint4 *dst = reinterpret_cast<uint4 *>(sB);
    for (int i = tid; i < mm.b_bytes / 16; i += blockDim.x) dst[i] = src[i];
    uint4 *za = reinterpret_cast<uint4 *>(sA);
    for (int i = tid; i < (int)((L.stw_off - L.a_off) / 16); i += blockDim.x) za[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < PS * JP; i += blockDim.x) {
      const int r = i / JP, c = i - r * JP;
      stw[r * L.ts + c] = a.sbd_tw[i];
    }
  }
  if (tid == 0) {
    for (int i = 0; i < kABufs; ++i) {
      mbar_init(&bar_afull[i], kGroupThreads);
      mbar_init(&bar_aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bar_accfull[i], 1);
      mbar_init(&bar_accempty[i], kEpiWarps * 32);
    }
    mbar_init(&bar_drain, 1);
    abort_flag = 0;
    for (int i = 0; i < kScaleRing; ++i) sc_tag[i] = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(mm.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int *abortp = &abort_flag;

  if (warp < kEpiWarp0) {
    // ================= producers: gather (Eq. 3) + SBD FFT -> BF16 A tile =================
    const int g = warp / kGroupWarps, gtid = tid - g * kGroupThreads, bar = kBarGroup0 + g;
    ItemTab &tab = tabs[g];
    float2 *X = reinterpret_cast<float2 *>(smem + L.x_off) + (size_t)g * N * L.xs;
    long long i = 0;  // CTA-local tile counter
    const long long n_prod = mm.hold ? 0 : n_items;  // test aid: with hold, the producers issue nothing
    for (long long item = blockIdx.x; item < n_prod; item += gridDim.x) {
      if (gtid == 0) {
        if (list) {
          tab.nseg = (int)min((long long)kListItem, mm.n_valid - item * kListItem);
          tab.tiles = (tab.nseg + SPT - 1) / SPT;
        } else {
          item_table(a, item, SPT, tab);
        }
      }
      named_sync(bar, kGroupThreads);
      const int tiles = tab.tiles, nseg = tab.nseg;
      bool stop = false;
      for (int ti = 0; ti < tiles; ++ti, ++i) {
        if ((int)(i % kGroups) != g) continue;
        const int b = (int)(i % kABufs);
        const uint32_t use = (uint32_t)(i / kABufs);
        const bool got = mbar_wait(&bar_aempty[b], (use & 1) ^ 1, abortp, mm.timeout);
        if (named_sync_or(bar, kGroupThreads, !got)) {
          stop = true;
          break;
        }
        unsigned char *At = sA + (size_t)b * mm.KA * kAtomBytes;
        for (int sl = 0; sl < SPT; ++sl) {
          const int k = ti * SPT + sl;
          if (k >= nseg) break;
          int bl, d, l, k0;
          long long out;
          if (list) {
            const int4 row = reinterpret_cast<const int4 *>(a.seg)[item * kListItem + k];
            bl = row.x;
            d = row.y;
            l = row.z;
            k0 = row.w;
          } else {
            item_segment(a, tab, k, a.n_win, l, k0, out);
            bl = tab.bl;
            d = tab.d;
          }
          // gather: kGatherBatch independent point loads in flight per thread
          float l1 = 0.f;
          const int *dk = a.dk + (size_t)d * C;
          const float2 *vb = a.vis + (size_t)bl * a.T * C;
          for (int p0 = gtid; p0 < C; p0 += kGroupThreads * kGatherBatch) {
            int off[kGatherBatch];
            float2 acc[kGatherBatch];
#pragma unroll
            for (int q = 0; q < kGatherBatch; ++q) {
              const int c = p0 + q * kGroupThreads;
              off[q] = c < C ? (k0 + __ldg(dk + c)) * C + c : 0;
              acc[q] = make_float2(0.f, 0.f);
            }
            for (int r = 0; r < l; ++r) {
#pragma unroll
              for (int q = 0; q < kGatherBatch; ++q) {
                if (p0 + q * kGroupThreads < C) {
                  const float2 v = __ldg(vb + off[q]);
                  acc[q].x += v.x;
                  acc[q].y += v.y;
                  off[q] += C;
                }
              }
            }
#pragma unroll
            for (int q = 0; q < kGatherBatch; ++q) {
              const int c = p0 + q * kGroupThreads;
              if (c < C) {
                const int n = c / a.J, j = c - n * a.J;
                const float2 x = cmul(acc[q], __ldg(a.wrot + c));
                X[n * L.xs + j] = x;
                if (kFp8) l1 += fabsf(x.x) + fabsf(x.y);
              }
            }
          }
          if (kFp8) {
#pragma unroll
            for (int off = 16; off; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
            if (lane == 0) l1_part[g][gtid >> 5] = l1;
          }
          named_sync(bar, kGroupThreads);
          // FP8: every |Re Y|, |Im Y| is at most the L1 norm of the segment's spectrum, so the
          // power of two s with s L1 <= 448 keeps A within E4M3's finite range
          float sc = 1.f;
          if (kFp8) {
            float tot = 0.f;
#pragma unroll
            for (int w = 0; w < kGroupWarps; ++w) tot += l1_part[g][w];
            int ex = 1;
            if (tot > 1e-30f) frexpf(448.f / tot, &ex);
            sc = ldexpf(1.f, max(-100, min(100, ex - 1)));
            if (gtid == 0) sc_inv2[i % kScaleRing][sl] = 1.f / (sc * sc);
          }
          // SBD four-step FFT, task (n, m1); rows sl * Ls + m of the A tile
          for (int t = gtid; t < N * PS; t += kGroupThreads) {
            const int n = t >> lps, m1 = t & (PS - 1);
            float2 A[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) A[q] = make_float2(0.f, 0.f);
            const float2 *xr = X + n * L.xs;
            const float2 *wr = stw + m1 * L.ts;
            for (int j1 = 0; j1 < a.J1; ++j1) {
#pragma unroll
              for (int j2 = 0; j2 < 32; ++j2) A[j2] = cfma(A[j2], xr[j1 * 32 + j2], wr[j1 * 32 + j2]);
            }
            fft32_dif(A);
#pragma unroll
            for (int q = 0; q < 32; ++q) {
              const int row = sl * Ls + m1 + PS * bitrev5(q);
              if (kFp8) {
                At[a_offset8(row, n)] = (unsigned char)__nv_cvt_float_to_fp8(A[q].x * sc, __NV_SATFINITE, __NV_E4M3);
                At[a_offset8(row, N + n)] = (unsigned char)__nv_cvt_float_to_fp8(A[q].y * sc, __NV_SATFINITE, __NV_E4M3);
              } else {
                *reinterpret_cast<__nv_bfloat16 *>(At + a_offset(row, n)) = __float2bfloat16_rn(A[q].x);
                *reinterpret_cast<__nv_bfloat16 *>(At + a_offset(row, N + n)) = __float2bfloat16_rn(A[q].y);
              }
            }
          }
          named_sync(bar, kGroupThreads);  // X is reused by the next segment
        }
        if (kFp8 && gtid == 0) sc_tag[i % kScaleRing] = i;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&bar_afull[b]);
      }
      if (stop) {
        *abortp = 1;
        break;
      }
    }
  } else if (warp == kMmaWarp) {
    // ================= MMA issuer =================
    long long i = 0, chunk_ctr = 0;
    bool ok = true;
    // D = F32; A, B = BF16 (kind::f16) or E4M3 (kind::f8f6f4, format code 0); K-major; N, M
    const uint32_t ab = kFp8 ? 0u : 1u;
    const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(mm.NC >> 3) << 17) |
                           ((uint32_t)(kRows >> 4) << 24);
    for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      const int tiles = list ? (int)((min((long long)kListItem, mm.n_valid - item * kListItem) + SPT - 1) / SPT)
                             : item_tiles(a, item, SPT);
      for (int ti = 0; ti < tiles && ok; ++ti, ++i) {
        const int b = (int)(i % kABufs);
        const uint32_t use = (uint32_t)(i / kABufs);
        if (!__all_sync(0xffffffffu, mbar_wait(&bar_afull[b], use & 1, abortp, mm.timeout))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_base = su32(sA + (size_t)b * mm.KA * kAtomBytes);
        for (int c = 0; c < mm.n_chunk; ++c, ++chunk_ctr) {
          const int s = (int)(chunk_ctr & 1);
          const uint32_t su = (uint32_t)(chunk_ctr >> 1);
          if (!__all_sync(0xffffffffu, mbar_wait(&bar_accempty[s], (su & 1) ^ 1, abortp, mm.timeout))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (lane == 0) {
            const uint32_t d_tmem = tmem + (uint32_t)(s * mm.NC);
            for (int kk = 0; kk < mm.kk_steps; ++kk) {
              const uint32_t koff = (uint32_t)((kk >> 2) * kAtomBytes + (kk & 3) * 32);
              const uint64_t ad = desc_sw128(a_base + koff);
              const uint64_t bd = desc_sw128(su32(sB) + (uint32_t)((kk >> 2) * mm.b_atom_bytes) +
                                             (uint32_t)(c * mm.NC * 128) + (uint32_t)((kk & 3) * 32));
              const uint32_t accum = kk > 0 ? 1u : 0u;
              if (kFp8)
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
              else
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(su32(&bar_accfull[s])) : "memory");
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(su32(&bar_aempty[b])) : "memory");
        __syncwarp();
      }
    }
    if (!ok) *abortp = 1;
    // drain: a last commit lands only when every MMA this thread issued has completed,
    // so tensor memory is never freed under an MMA in flight (bounded, ignores the abort flag)
    if (lane == 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(su32(&bar_drain)) : "memory");
    __syncwarp();
    if (!__all_sync(0xffffffffu, mbar_wait(&bar_drain, 0, nullptr, mm.drain_timeout))) *abortp = 1;
  } else {
    // ================= epilogue: |G|^2 and the grid maximum =================
    const int ew = warp - kEpiWarp0;           // 0..7
    const int quarter = warp & 3;              // TMEM lanes 32 * quarter ..
    const int part = 0;                        // all columns of the quarter
    const int etid = tid - kEpiWarp0 * 32;
    const int row = quarter * 32 + lane;       // tile row
    const int sl = row / Ls, m = row - sl * Ls;
    const int half = mm.NC >> 1;               // q values per chunk
    const int qpart = half;                    // q values this warp reads per chunk (>= 16)
    ItemTab &tab = tabs[kGroups];
    long long chunk_ctr = 0, ie = 0;  // ie: CTA-local tile number, as the producers count
    bool ok = true;
    for (long long item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
      if (etid == 0) {
        if (list) {
          tab.nseg = (int)min((long long)kListItem, mm.n_valid - item * kListItem);
          tab.tiles = (tab.nseg + SPT - 1) / SPT;
        } else {
          item_table(a, item, SPT, tab);
        }
      }
      named_sync(kBarEpi, kEpiWarps * 32);
      const int tiles = tab.tiles, nseg = tab.nseg;
      for (int ti = 0; ti < tiles; ++ti, ++ie) {
        float bp = -1.f;
        int bq = 0;
        for (int c = 0; c < mm.n_chunk; ++c, ++chunk_ctr) {
          const int s = (int)(chunk_ctr & 1);
          const uint32_t su = (uint32_t)(chunk_ctr >> 1);
          if (ok && !mbar_wait(&bar_accfull[s], su & 1, abortp, mm.timeout)) ok = false;
          if (!__all_sync(0xffffffffu, ok)) ok = false;  // tcgen05.ld below is warp-collective
          if (!ok) continue;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t t_row = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * mm.NC);
          for (int p0 = part * qpart; p0 < (part + 1) * qpart; p0 += 16) {
            uint32_t re[16], im[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
                           "=r"(re[7]), "=r"(re[8]), "=r"(re[9]), "=r"(re[10]), "=r"(re[11]), "=r"(re[12]), "=r"(re[13]),
                           "=r"(re[14]), "=r"(re[15])
                         : "r"(t_row + (uint32_t)p0));
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
                           "=r"(im[7]), "=r"(im[8]), "=r"(im[9]), "=r"(im[10]), "=r"(im[11]), "=r"(im[12]), "=r"(im[13]),
                           "=r"(im[14]), "=r"(im[15])
                         : "r"(t_row + (uint32_t)(half + p0)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            unsigned key = 0u;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float gr = __uint_as_float(re[j]), gi = __uint_as_float(im[j]);
              const float pw = fmaf(gr, gr, gi * gi);
              key = max(key, (__float_as_uint(pw) & ~31u) | (unsigned)(16 - j));
            }
            const int q = c * half + p0 + 16 - (int)(key & 31u);
            const float pk = __uint_as_float(key & ~31u);
            if (pk > bp || (pk == bp && q < bq)) {
              bp = pk;
              bq = q;
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&bar_accempty[s]);
        }
        // reduce over the rows of each segment of the tile (both column halves)
        float rp = bp;
        int ri = m * Lm + bq;
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const float p2 = __shfl_xor_sync(0xffffffffu, rp, off);
          const int i2 = __shfl_xor_sync(0xffffffffu, ri, off);
          better(rp, ri, p2, i2);
        }
        if (lane == 0) {
          red_p[ew] = rp;
          red_i[ew] = ri;
        }
        if (named_sync_or(kBarEpi, kEpiWarps * 32, !ok)) {
          ok = false;
          break;
        }
        const int wps = Ls / 32;  // lane quarters per segment
        if (lane == 0 && part == 0 && (quarter % wps) == 0) {
          float fp = red_p[quarter];
          int fi = red_i[quarter];
          for (int k = 1; k < wps; ++k) better(fp, fi, red_p[quarter + k], red_i[quarter + k]);
          const int k = ti * SPT + sl;
          if (k < nseg) {
            long long out;
            if (list) {
              out = item * kListItem + k;
            } else {
              int l, k0;
              item_segment(a, tab, k, a.n_win, l, k0, out);
            }
            if (kFp8) {  // undo the segment's scale (its tag proves the entry is this tile's)
              const volatile long long *tag = sc_tag + ie % kScaleRing;
              const long long t0 = clock64();
              while (*tag != ie && clock64() - t0 < mm.timeout) {
              }
              if (*tag != ie) *abortp = 1;
              fp *= sc_inv2[ie % kScaleRing][sl];
            }
            frbx_seg r;
            r.amp = sqrtf(fp);
            r.sbd_idx = (uint16_t)(fi >> a.log2Lm);
            r.mbd_idx = (uint16_t)(fi & (Lm - 1));
            a.out[out] = r;
          }
        }
        named_sync(kBarEpi, kEpiWarps * 32);
      }
    }
    if (!ok) *abortp = 1;
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(mm.tmem_cols) : "memory");
  if (tid == 0 && abort_flag) atomicExch(mm.err, FRBX_ETIMEOUT);
}

__global__ void k_fill_invalid(frbx_seg *out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    frbx_seg r;
    r.amp = -1.f;
    r.sbd_idx = 0;
    r.mbd_idx = 0;
    out[i] = r;
  }
}

void set_mma_constants() { upload_w32(); }

bool mma_supported(int Ls, int Lm, int N, int J) {
  const int KA = (2 * N + 63) / 64;
  const size_t b_bytes = (size_t)KA * 2 * Lm * 128;
  return (Ls == 64 || Ls == 128) && J <= Ls && 2 * Lm >= 32 && (2 * Lm) % 32 == 0 && KA <= 2 &&
         b_bytes <= 144 * 1024;
}

cudaError_t launch_fit_mma(const FitArgs &a, const MmaArgs &mm, int n_bl, bool list_mode, cudaStream_t st,
                           int64_t *launches) {
  (void)n_bl;
  if (!mma_supported(a.Ls, a.Lm, a.N, a.J)) return cudaErrorInvalidConfiguration;
  const MmaLayout L = mma_layout(mm, a.N, a.Ls, a.J1);
  if (L.bytes > max_smem_optin()) return cudaErrorInvalidConfiguration;
  if (!list_mode) {
    const long long n = (long long)n_bl * a.n_dm * a.S_tot;
    if (n > 0) {
      k_fill_invalid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.out, n);
      ++*launches;
    }
  }
  if (mm.n_valid == 0) return cudaGetLastError();
  if ((long long)a.T * a.C >= (1LL << 31)) return cudaErrorInvalidConfiguration;  // 32-bit gather offsets
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long units = list_mode ? (mm.n_valid + kListItem - 1) / kListItem : mm.n_items;
  const unsigned grid = (unsigned)(units < sms ? units : sms);
  auto kern = mm.fp8 ? k_fit_mma<true> : k_fit_mma<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, kMmaThreads, L.bytes, st>>>(a, mm, list_mode ? 1 : 0);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
