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
//   warp 8 allocates tensor memory and one lane issues an AP's MMAs into one of kSlots
//          accumulator slots, so it runs up to kSlots - 1 APs ahead.  A tcgen05.mma of
//          M = 128 and K = 16 costs about the same for N = 64 and N = 128, so where tensor
//          memory allows (kCat) the two products of A_hi are one N = 128 MMA against the
//          stacked [W_hi; W_lo], D = [A_hi W_hi | A_hi W_lo + A_lo W_hi], and the epilogue adds
//          the halves: 2 K/16 MMAs per AP instead of 3 K/16;
//   warps 0-7 (row quarter w % 4, q half w / 4) read G_1(k) into registers (freeing its slot
//          at once), keep it there as G_1(k - 1) for the next AP, walk their 16 cells through
//          the window tree with packed FP32x2 arithmetic (deeper anchors held in tensor
//          memory), and merge every emitted segment's warp maximum into the series by a
//          64-bit atomicMax, as k_tree_mbd does per block: the warps never wait for one another.
// Every wait is bounded: on timeout the kernel records FRBX_ETIMEOUT, drains and frees its
// tensor memory.
#include <cuda_bf16.h>

#include "fit_common.cuh"
#include "tc_common.cuh"

namespace frbx {

namespace {

constexpr int kTmNQ = 32;                   // complex MBD columns per CTA
constexpr int kTmCols = 2 * kTmNQ;          // Re G of the 32 q, then Im G
constexpr int kTmABufs = 3;                 // ring of one-AP A tiles
constexpr int kTmEpiWarps = 8;
constexpr int kTmMmaWarp = 8, kTmLoadWarp = 9;
constexpr int kTmThreads = 320;
constexpr int kTmTmemCols = 512;            // kSlots accumulator slots, then the anchors
constexpr int kTmMaxLev = 6;
constexpr int kTmWAtom = kTmCols * 128;     // 64 rows of one 64-wide K atom of W (8 KB)

// 16 consecutive FP32 columns of this thread's tensor-memory lane as 8 packed pairs
__device__ __forceinline__ uint64_t pk(uint32_t lo, uint32_t hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
  return d;
}
__device__ __forceinline__ void upk(uint64_t v, uint32_t &lo, uint32_t &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(v));
}
// element-wise IEEE round-to-nearest on both halves: the same results as two scalar ops
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint64_t (&v)[8]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int p = 0; p < 8; ++p) v[p] = pk(r[2 * p], r[2 * p + 1]);
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const uint64_t (&v)[8]) {
  uint32_t r[16];
#pragma unroll
  for (int p = 0; p < 8; ++p) upk(v[p], r[2 * p], r[2 * p + 1]);
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(tc::kRows >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
}

}  // namespace

// kSlots accumulator slots of kSlotCols columns at 0, kSlotCols, ...; the anchors of levels
// 2..nlev follow at kSlots kSlotCols + 64 j.  kCat: one N = 128 MMA for A_hi [W_hi; W_lo].
template <int kSlots, bool kCat>
__global__ void __launch_bounds__(kTmThreads, 1) k_tree_mma(const __grid_constant__ TreeArgs t) {
  constexpr int kSlotCols = kCat ? 2 * kTmCols : kTmCols;
  constexpr int kAnc = kSlots * kSlotCols;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_afull[kTmABufs], bar_aempty[kTmABufs], bar_accfull[kSlots], bar_accempty[kSlots],
      bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

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

  unsigned char *sW = smem;                                   // per K atom: hi rows | lo rows
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
    for (int i = 0; i < kSlots; ++i) {
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
    // ================= MMA issuer =================
    const uint32_t id64 = idesc_bf16(kTmCols), id128 = idesc_bf16(2 * kTmCols);
    const int kk_steps = t.KA * 4;  // K = 16 per instruction, 4 per 64-wide atom
    // descriptors of the K steps differ only in the start address field (address / 16, in the
    // low 14 bits, which shared-memory offsets below 256 KB never carry out of)
    const uint32_t a_half16 = (uint32_t)(t.KA * tc::kAtomBytes) >> 4, w_lo16 = (uint32_t)kTmWAtom >> 4;
    const uint64_t w0 = tc::desc_sw128(tc::su32(sW));
    bool ok = true;
    for (int i = 0; i < n_ap && ok; ++i) {
      const int b = i % kTmABufs;
      const uint32_t use = (uint32_t)(i / kTmABufs);
      const int slot = i % kSlots;
      const uint32_t su = (uint32_t)(i / kSlots);
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
        const uint64_t a0 = tc::desc_sw128(tc::su32(sA + (size_t)b * t.tile_bytes));
        const uint32_t d_tmem = tmem + (uint32_t)(slot * kSlotCols);
        if (kCat) {
          // D[0:64] = A_hi W_hi, D[64:128] = A_hi W_lo (one N = 128 MMA per K step) + A_lo W_hi
#pragma unroll 4
          for (int kk = 0; kk < kk_steps; ++kk) {
            const uint32_t ao = (uint32_t)(((kk >> 2) * tc::kAtomBytes + (kk & 3) * 32) >> 4);
            const uint32_t bo = (uint32_t)(((kk >> 2) * 2 * kTmWAtom + (kk & 3) * 32) >> 4);
            mma_bf16(d_tmem, a0 + ao, w0 + bo, id128, kk > 0 ? 1u : 0u);
          }
#pragma unroll 4
          for (int kk = 0; kk < kk_steps; ++kk) {
            const uint32_t ao = (uint32_t)(((kk >> 2) * tc::kAtomBytes + (kk & 3) * 32) >> 4);
            const uint32_t bo = (uint32_t)(((kk >> 2) * 2 * kTmWAtom + (kk & 3) * 32) >> 4);
            mma_bf16(d_tmem + (uint32_t)kTmCols, a0 + a_half16 + ao, w0 + bo, id64, 1u);
          }
        } else {
#pragma unroll
          for (int term = 0; term < 3; ++term) {  // (hi, hi), (hi, lo), (lo, hi)
            const uint64_t ab = a0 + (term == 2 ? a_half16 : 0u), bb = w0 + (term == 1 ? w_lo16 : 0u);
#pragma unroll 4
            for (int kk = 0; kk < kk_steps; ++kk) {
              const uint32_t ao = (uint32_t)(((kk >> 2) * tc::kAtomBytes + (kk & 3) * 32) >> 4);
              const uint32_t bo = (uint32_t)(((kk >> 2) * 2 * kTmWAtom + (kk & 3) * 32) >> 4);
              mma_bf16(d_tmem, ab + ao, bb + bo, id64, (term > 0 || kk > 0) ? 1u : 0u);
            }
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
    const unsigned idx0 = (unsigned)((quarter * 32) * t.Lm + qb * kTmNQ + 16 * hh);  // cell 0 of lane 0
    unsigned long long *keys = t.keys + ((size_t)sd.x * t.n_dm + sd.y) * t.S_tot;
    uint64_t pre[8], pim[8];  // G_1(k - 1), carried in registers from the previous AP
#pragma unroll
    for (int p = 0; p < 8; ++p) pre[p] = pim[p] = 0ull;
    for (int a = 0; a + 2 <= t.nlev; ++a) {
      const uint32_t ab = lane_base + (uint32_t)(kAnc + a * kTmCols);
      tm_st16(ab + c_re, pre);
      tm_st16(ab + c_im, pim);
    }
    tm_wait_st();
    bool ok = true;
    for (int i = 0; i < n_ap; ++i) {
      const int k = kb + i, slot = i % kSlots;
      const uint32_t su = (uint32_t)(i / kSlots);
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_accfull[slot], su & 1, abortp, t.timeout))) {
        ok = false;  // uniform within the warp: tcgen05.ld is warp-collective
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      uint64_t cre[8], cim[8];
      const uint32_t cur = lane_base + (uint32_t)(slot * kSlotCols);
      tm_ld16(cur + c_re, cre);
      tm_ld16(cur + c_im, cim);
      if (kCat) {
        uint64_t lre[8], lim[8];
        tm_ld16(cur + kTmCols + c_re, lre);
        tm_ld16(cur + kTmCols + c_im, lim);
        tm_wait_ld();
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          cre[p] = add2(cre[p], lre[p]);
          cim[p] = add2(cim[p], lim[p]);
        }
      } else {
        tm_wait_ld();
      }
      // G_1(k) is in registers: its slot may take AP k + kSlots
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      tc::mbar_arrive(&bar_accempty[slot]);
      const int E = t.nlev == 0 ? 0 : min(t.nlev, __ffs(k + 1));  // levels whose window ends at k
      uint64_t are[8], aim[8];
#pragma unroll
      for (int e = 0; e <= kTmMaxLev; ++e) {
        if (e > E) break;
        if (e == 0) {
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            are[p] = cre[p];
            aim[p] = cim[p];
          }
        } else if (e == 1) {
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            are[p] = add2(pre[p], cre[p]);
            aim[p] = add2(pim[p], cim[p]);
          }
        } else {
          // anchor of level e - 1: the previous window-2^(e-1) matrix, first half of this one
          const uint32_t ab = lane_base + (uint32_t)(kAnc + (e - 2) * kTmCols);
          uint64_t ore[8], oim[8];
          tm_ld16(ab + c_re, ore);
          tm_ld16(ab + c_im, oim);
          tm_wait_ld();
          tm_st16(ab + c_re, are);
          tm_st16(ab + c_im, aim);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            are[p] = add2(are[p], ore[p]);
            aim[p] = add2(aim[p], oim[p]);
          }
          tm_wait_st();
        }
        const int w = t.emit_w[e];
        const int k0 = k - (1 << e) + 1;
        if (w >= 0 && k0 >= kb && k0 < kb + t.TT) {  // uniform across the CTA
          // packed key: |G|^2 with its 6 low mantissa bits replaced by 31 - j (lower q wins a tie)
          unsigned kk[16];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            uint32_t lo, hi;
            upk(fma2(are[p], are[p], mul2(aim[p], aim[p])), lo, hi);
            kk[2 * p] = (lo & ~63u) | (unsigned)(31 - 2 * p);
            kk[2 * p + 1] = (hi & ~63u) | (unsigned)(30 - 2 * p);
          }
#pragma unroll
          for (int wdt = 8; wdt >= 1; wdt >>= 1) {
#pragma unroll
            for (int j = 0; j < wdt; ++j) kk[j] = max(kk[j], kk[j + wdt]);
          }
          const unsigned wmax = __reduce_max_sync(0xffffffffu, kk[0]);
          const unsigned win = __ballot_sync(0xffffffffu, kk[0] == wmax);
          if (lane == 0) {
            const unsigned L = (unsigned)(__ffs(win) - 1), j = 31u - (wmax & 63u);
            const unsigned idx = idx0 + L * (unsigned)t.Lm + j;
            const int l = 1 << e, step = l > 1 ? l / 2 : 1;
            atomicMax(keys + t.win_off[w] + k0 / step, ((unsigned long long)(wmax & ~63u) << 32) | (unsigned long long)(~idx));
          }
        }
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        pre[p] = cre[p];
        pim[p] = cim[p];
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

// Accumulator slots and layout for nlev tree levels: the N = 128 form (slots of 128 columns)
// needs two slots beside the nlev - 1 anchors of 64 columns, so nlev <= 5; level 6 takes the
// three-product form with 64-column slots.
static void tree_mma_layout(int nlev, int *slots, bool *cat) {
  const int anc = kTmCols * max(nlev - 1, 0);
  *cat = kTmTmemCols - anc >= 2 * 2 * kTmCols;
  *slots = *cat ? min(4, (kTmTmemCols - anc) / (2 * kTmCols)) : 3;
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
  if (t.nlev < 0 || t.nlev > kTmMaxLev) return cudaErrorInvalidValue;
  const long long nb = (long long)t.n_s * t.n_qb * t.n_tt;
  if (nb <= 0) return cudaSuccess;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  int slots;
  bool cat;
  tree_mma_layout(t.nlev, &slots, &cat);
  auto kern = !cat ? k_tree_mma<3, false> : slots == 4 ? k_tree_mma<4, true> : slots == 3 ? k_tree_mma<3, true>
                                                                                         : k_tree_mma<2, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)nb, kTmThreads, smem, st>>>(t);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
