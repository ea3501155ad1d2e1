// Window-tree fit with the MBD transform on the tcgen05 tensor cores.
//
// Same method as k_tree_mbd (kernels_tree.cu): the one-AP delay-resolution matrix G_1(k) is
// formed once per AP and every window 2l is G_l(k0) + G_l(k0 + l) (Sec. 5.1 additivity).  Here
// the MBD transform of Eq. 5 is a dense DFT-GEMM on the tensor cores,
//     [Re G | Im G](m, q) = sum_k A[m][k] B[q'][k],   A[m][n] = Re Y(n, m), A[m][N + n] = Im Y(n, m),
// with B the cos / sin rows of the exact phase index g_n q mod Lm, in FP32-equivalent
// precision from three BF16 products: every operand x is split as x_hi = bf16(x),
// x_lo = bf16(x - x_hi), and D = A_hi B_hi + A_hi B_lo + A_lo B_hi accumulates in FP32 in tensor
// memory (the dropped A_lo B_lo term is below 2^-16 of each product).
//
// One CTA owns all Ls = 128 SBD rows of one block of 32 MBD columns q of one (baseline, DM)
// series and walks a time tile AP by AP (10 warps):
//   warp 9 (one lane) copies each AP's split A tiles (written by k_tree_sbd in their
//          shared-memory image) into a ring with cp.async.bulk;
//   warp 8 allocates tensor memory and one lane issues the 3 x K/16 MMAs of an AP into one
//          of three accumulator slots (so it runs up to two APs ahead);
//   warps 0-7 (row quarter w % 4, q half w / 4) read G_1(k) and, from the previous slot,
//          G_1(k - 1), walk their 16 cells through the window tree (deeper anchors held in
//          tensor memory), and reduce every emitted segment's maximum, merged across blocks
//          by a 64-bit atomicMax as in k_tree_mbd.
// Every wait is bounded: on timeout the kernel records FRBX_ETIMEOUT, drains and frees its
// tensor memory.
#include <cuda_bf16.h>

#include "fit_common.cuh"
#include "tc_common.cuh"

namespace frbx {

namespace {

constexpr int kTmNQ = 32;                   // complex MBD columns per CTA
constexpr int kTmCols = 2 * kTmNQ;          // GEMM N: Re G of the 32 q, then Im G
constexpr int kTmABufs = 3;                 // ring of one-AP A tiles
constexpr int kTmEpiWarps = 8;
constexpr int kTmMmaWarp = 8, kTmLoadWarp = 9;
constexpr int kTmThreads = 320;
constexpr int kTmBarEpi = 1;                // named barrier of the epilogue warps
constexpr int kTmSlots = 3;                 // accumulator slots: the MMA runs up to two APs ahead
constexpr int kTmTmemCols = 512;            // slots at 0, 64, 128; anchors at 192 + 64 j
constexpr int kTmMaxLev = 6;
constexpr int kTmWAtom = kTmCols * 128;     // one 64-wide K atom of a W block (8 KB)

__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
               : "memory");
}
__device__ __forceinline__ bool named_sync_or_epi(bool p) { return tc::named_sync_or(kTmBarEpi, kTmEpiWarps * 32, p); }
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace

__global__ void __launch_bounds__(kTmThreads, 1) k_tree_mma(const __grid_constant__ TreeArgs t) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_afull[kTmABufs], bar_aempty[kTmABufs], bar_accfull[kTmSlots], bar_accempty[kTmSlots],
      bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ uint2 red[2][kTmMaxLev + 1][kTmEpiWarps];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // MBD column blocks vary fastest, so the CTAs sharing one series' A tiles run together (L2)
  int item = blockIdx.x;
  const int qb = item % t.n_qb;
  item /= t.n_qb;
  const int tt = item % t.n_tt, s = item / t.n_tt;
  const int2 sd = t.series[s];
  const int kd = t.T - t.dk_max[sd.y];
  const int kb = tt * t.TT;
  if (kb >= kd) return;  // every segment starting here runs past the scan (uniform)
  const int ke = min(kd, kb + t.TT + (1 << t.nlev) - 1);
  const int n_ap = ke - kb;

  unsigned char *sW = smem;                                   // hi atoms | lo atoms
  unsigned char *sA = smem + ((t.w_bytes + 1023) & ~1023);    // ring of one-AP tiles
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(t.wimg + (size_t)qb * t.w_bytes);
    uint4 *dst = reinterpret_cast<uint4 *>(sW);
    for (int i = tid; i < t.w_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (tid == 0) {
    for (int i = 0; i < kTmABufs; ++i) {
      tc::mbar_init(&bar_afull[i], 1);
      tc::mbar_init(&bar_aempty[i], 1);
    }
    for (int i = 0; i < kTmSlots; ++i) {
      tc::mbar_init(&bar_accfull[i], 1);
      tc::mbar_init(&bar_accempty[i], kTmEpiWarps * 32);
    }
    tc::mbar_init(&bar_drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTmMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_base)),
                 "r"(kTmTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int *abortp = &abort_flag;

  if (warp == kTmLoadWarp) {
    // ================= loader: one bulk copy of the split A tiles per AP =================
    if (lane == 0) {
      const unsigned char *src = t.Yt + (size_t)s * t.yt_series + (size_t)kb * t.tile_bytes;
      int issued = 0;
      for (int i = 0; i < n_ap; ++i) {
        const int b = i % kTmABufs;
        const uint32_t use = (uint32_t)(i / kTmABufs);
        if (!tc::mbar_wait(&bar_aempty[b], (use & 1) ^ 1, abortp, t.timeout)) {
          *abortp = 1;
          break;
        }
        tc::mbar_expect_tx(&bar_afull[b], (uint32_t)t.tile_bytes);
        tc::bulk_g2s(sA + (size_t)b * t.tile_bytes, src + (size_t)i * t.tile_bytes, (uint32_t)t.tile_bytes,
                     &bar_afull[b]);
        ++issued;
      }
      // every copy issued has landed before the CTA can leave (bounded; ignores the abort flag)
      for (int i = max(0, issued - kTmABufs); i < issued; ++i)
        if (!tc::mbar_wait(&bar_afull[i % kTmABufs], (uint32_t)(i / kTmABufs) & 1, nullptr, t.timeout)) *abortp = 1;
    }
    __syncwarp();
  } else if (warp == kTmMmaWarp) {
    // ================= MMA issuer: D = A_hi B_hi + A_hi B_lo + A_lo B_hi per AP =================
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTmCols >> 3) << 17) |
                           ((uint32_t)(tc::kRows >> 4) << 24);
    const int kk_steps = t.KA * 4;  // K = 16 per instruction, 4 per 64-wide atom
    const uint32_t a_half = (uint32_t)(t.KA * tc::kAtomBytes), w_half = (uint32_t)(t.KA * kTmWAtom);
    bool ok = true;
    for (int i = 0; i < n_ap && ok; ++i) {
      const int b = i % kTmABufs;
      const uint32_t use = (uint32_t)(i / kTmABufs);
      const int slot = i % kTmSlots;
      const uint32_t su = (uint32_t)(i / kTmSlots);
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_afull[b], use & 1, abortp, t.timeout))) {
        ok = false;
        break;
      }
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_accempty[slot], (su & 1) ^ 1, abortp, t.timeout))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        const uint32_t a_base = tc::su32(sA + (size_t)b * t.tile_bytes), w_base = tc::su32(sW);
        const uint32_t d_tmem = tmem + (uint32_t)(slot * kTmCols);
#pragma unroll
        for (int term = 0; term < 3; ++term) {  // (hi, hi), (hi, lo), (lo, hi)
          const uint32_t ao = term == 2 ? a_half : 0u, wo = term == 1 ? w_half : 0u;
          for (int kk = 0; kk < kk_steps; ++kk) {
            const uint64_t ad = tc::desc_sw128(a_base + ao + (uint32_t)((kk >> 2) * tc::kAtomBytes + (kk & 3) * 32));
            const uint64_t bd = tc::desc_sw128(w_base + wo + (uint32_t)((kk >> 2) * kTmWAtom + (kk & 3) * 32));
            const uint32_t accum = (term > 0 || kk > 0) ? 1u : 0u;
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                         ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tc::su32(&bar_accfull[slot])) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tc::su32(&bar_aempty[b])) : "memory");
      }
      __syncwarp();
    }
    if (!ok) *abortp = 1;
    // drain: a last commit lands only when every MMA this thread issued has completed
    if (lane == 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(tc::su32(&bar_drain)) : "memory");
    __syncwarp();
    if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_drain, 0, nullptr, t.timeout))) *abortp = 1;
  } else {
    // ================= epilogue: window tree and maxima =================
    const int quarter = warp & 3, hh = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t c_re = (uint32_t)(16 * hh), c_im = (uint32_t)(kTmNQ + 16 * hh);
    const int q0 = qb * kTmNQ + 16 * hh;                  // MBD column of cell 0
    unsigned long long *keys = t.keys + ((size_t)sd.x * t.n_dm + sd.y) * t.S_tot;
    {
      float z[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) z[j] = 0.f;
      for (int a = 0; a + 2 <= t.nlev; ++a) {
        const uint32_t ab = lane_base + (uint32_t)((kTmSlots + a) * kTmCols);
        tm_st16(ab + c_re, z);
        tm_st16(ab + c_im, z);
      }
      tm_wait_st();
    }
    bool ok = true;
    for (int i = 0; i < n_ap; ++i) {
      const int k = kb + i, slot = i % kTmSlots, pslot = (i + kTmSlots - 1) % kTmSlots, buf = i & 1;
      const uint32_t su = (uint32_t)(i / kTmSlots);
      if (ok && !tc::mbar_wait(&bar_accfull[slot], su & 1, abortp, t.timeout)) ok = false;
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      const int ctz = __ffs(k + 1) - 1;
      const int E = t.nlev == 0 ? 0 : min(t.nlev, ctz + 1);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float cre[16], cim[16], pre[16], pim[16];
        const uint32_t cur = lane_base + (uint32_t)(slot * kTmCols), prv = lane_base + (uint32_t)(pslot * kTmCols);
        tm_ld16(cur + c_re, cre);
        tm_ld16(cur + c_im, cim);
        if (i > 0) {
          tm_ld16(prv + c_re, pre);
          tm_ld16(prv + c_im, pim);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) pre[j] = pim[j] = 0.f;
        }
        tm_wait_ld();
        if (i > 0) {  // G_1(k - 1) is read: its slot may take AP k + 2
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          tc::mbar_arrive(&bar_accempty[pslot]);
        }
        float are[16], aim[16];
#pragma unroll
        for (int e = 0; e <= kTmMaxLev; ++e) {
          if (e > E) break;
          if (e == 0) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              are[j] = cre[j];
              aim[j] = cim[j];
            }
          } else if (e == 1) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              are[j] = pre[j] + cre[j];
              aim[j] = pim[j] + cim[j];
            }
          } else {
            // anchor of level e - 1: the previous window-2^(e-1) matrix, first half of this one
            const uint32_t ab = lane_base + (uint32_t)((kTmSlots + e - 2) * kTmCols);
            float ore[16], oim[16];
            tm_ld16(ab + c_re, ore);
            tm_ld16(ab + c_im, oim);
            tm_wait_ld();
            tm_st16(ab + c_re, are);
            tm_st16(ab + c_im, aim);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              are[j] += ore[j];
              aim[j] += oim[j];
            }
            tm_wait_st();
          }
          const int w = t.emit_w[e];
          const int k0 = k - (1 << e) + 1;
          if (w >= 0 && k0 >= kb && k0 < kb + t.TT) {  // uniform across the CTA
            // packed key: |G|^2 with its 6 low mantissa bits replaced by 31 - j (lower q wins a tie)
            unsigned kk[16];
#pragma unroll
            for (int j = 0; j < 16; ++j)
              kk[j] = (__float_as_uint(fmaf(are[j], are[j], aim[j] * aim[j])) & ~63u) | (unsigned)(31 - j);
#pragma unroll
            for (int wdt = 8; wdt >= 1; wdt >>= 1) {
#pragma unroll
              for (int j = 0; j < wdt; ++j) kk[j] = max(kk[j], kk[j + wdt]);
            }
            const unsigned wmax = __reduce_max_sync(0xffffffffu, kk[0]);
            const unsigned win = __ballot_sync(0xffffffffu, kk[0] == wmax);
            if (lane == 0) {
              const int L = __ffs(win) - 1;
              const int j = 31 - (int)(wmax & 63u);
              red[buf][e][warp] = make_uint2(wmax & ~63u, (unsigned)((quarter * 32 + L) * t.Lm + q0 + j));
            }
          }
        }
      }
      // one barrier per AP, which also makes a give-up uniform across the epilogue warps
      if (named_sync_or_epi(!ok)) {
        ok = false;
        break;
      }
      // merge the block's maxima of the segments emitted at AP k into the series
      if (tid <= E) {
        const int e = tid, w = t.emit_w[e], k0 = k - (1 << e) + 1;
        if (w >= 0 && k0 >= kb && k0 < kb + t.TT) {
          uint2 best = red[buf][e][0];
          for (int v = 1; v < kTmEpiWarps; ++v) {
            const uint2 r2 = red[buf][e][v];
            if (r2.x > best.x || (r2.x == best.x && r2.y < best.y)) best = r2;
          }
          const int l = 1 << e, step = l > 1 ? l / 2 : 1;
          atomicMax(keys + t.win_off[w] + k0 / step,
                    ((unsigned long long)best.x << 32) | (unsigned long long)(~best.y));
        }
      }
    }
    if (!ok) *abortp = 1;
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kTmMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmTmemCols) : "memory");
  if (tid == 0 && abort_flag) atomicExch(t.err, FRBX_ETIMEOUT);
}

bool tree_mma_supported(int Ls, int Lm, int N, int J) {
  return Ls == tc::kRows && J <= Ls && Lm % kTmNQ == 0 && 2 * N <= 128;
}

static size_t tree_mma_smem(const TreeArgs &t) {
  return (size_t)((t.w_bytes + 1023) & ~1023) + (size_t)kTmABufs * t.tile_bytes + 1024;
}

cudaError_t launch_tree_mma(const TreeArgs &t, cudaStream_t st, int64_t *launches) {
  const size_t smem = tree_mma_smem(t);
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  const long long nb = (long long)t.n_s * t.n_qb * t.n_tt;
  if (nb <= 0) return cudaSuccess;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_tree_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tree_mma<<<(unsigned)nb, kTmThreads, smem, st>>>(t);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
