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
// series and walks a time tile AP by AP (12 warps in three warpgroups):
//   warp 9 (one lane) copies each AP's split A tiles (written by k_tree_sbd in their
//          shared-memory image) into a ring with cp.async.bulk;
//   warp 8 allocates tensor memory and runs the MMA loop convergently; one elected lane issues
//          an AP's MMAs into one of two accumulator slots of 64 columns, so it runs one AP
//          ahead: per K step three N = 64 MMAs, A_hi W_hi, A_hi W_lo and A_lo W_hi, all
//          accumulating into the same slot (the issue keeps pace with the tensor pipe, and the
//          epilogue reads one 64-column result per AP);
//   warps 10 and 11 have no role: with warps 8 and 9 they form the warpgroup that hands its
//          registers to the epilogue (setmaxnreg), which is bound by each warp's chain of
//          dependent work and gains from keeping more of the tree in registers;
//   warps 0-7 (row quarter w % 4, q half w / 4) read G_1(k) into registers (freeing its slot
//          at once), keep it there as G_1(k - 1) for the next AP, walk their 16 cells through
//          the window tree with packed FP32x2 arithmetic, and merge every emitted segment's
//          warp maximum into the series by a 64-bit atomicMax, as k_tree_mbd does per block:
//          the warps never wait for one another.  The first half of a window of 4 APs (tree
//          level 2) stays in registers; those of windows 8 to 64 (levels 3 to 6) sit in tensor
//          memory after the slots (shared memory takes anchor levels only where tensor memory
//          has no room).
// Two lower-precision forms of the same tree run one product per AP instead of three: kernel 7
// multiplies A_hi by W_hi (BF16, about 4e-3 relative on |G|), kernel 8 multiplies E4M3 operands
// with kind::f8f6f4 (about 6e-2 relative), A scaled per AP by the power of two s with
// s L1 <= 448 (L1 the L1 norm of the AP's dedispersed spectrum, which bounds every |Re Y|,
// |Im Y|); the epilogue multiplies G_1(k) by 1 / s before it enters the tree, so windows sum
// unscaled matrices.
// With delay search windows the SBD pass stores the rows rotated by t.rot (a multiple of 8),
// tile row r = (m - rot) mod Ls, so the searched rows sit in the first row quarters: warps whose
// rows are all outside the SBD window only release their slots, cells outside the windows are
// masked, and CTAs whose 32 q lie outside the MBD window exit at once.  When the searched rows
// fit the first 32 (or 64) tile rows, the SBD pass keeps only those rows of each AP, and one CTA
// stacks the pieces of four (or two) consecutive time tiles into its 128-row A operand: each
// row quarter (pair) of warps walks its own time tile, so no epilogue warp idles.
// Every wait is bounded: on timeout the kernel records FRBX_ETIMEOUT, drains and frees its
// tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fit_common.cuh"
#include "tc_common.cuh"

namespace frbx {

namespace {

constexpr int kTmNQ = 32;                   // complex MBD columns per CTA
constexpr int kTmCols = 2 * kTmNQ;          // Re G of the 32 q, then Im G
constexpr int kTmMaxABufs = 3;              // ring of one-AP A tiles (2 where shared memory is short)
constexpr int kTmTmemCols = 512;            // accumulator slots, then the tensor-memory anchors
constexpr int kTmMaxLev = 6;
constexpr int kTmWAtom = kTmCols * 128;     // 64 rows of one 128-byte K atom of W (8 KB)
constexpr int kTmAncBytes = tc::kRows * kTmCols * 4;  // one anchor level in shared memory (32 KB)
// configuration of the launched instance: epilogue warps (8 or 16) and accumulator slots
constexpr int kTmEpi = 8;
constexpr int kTmSlots = 2;
// Register split.  The block has three warpgroups: the eight epilogue warps (groups 0 and 1) and
// group 2 (the MMA warp, the loader warp and two warps with no role).  Each sub-partition holds one
// warp of every group, so at launch every thread gets 168 registers (16384 per sub-partition over
// three warps).  Group 2 then gives registers back (setmaxnreg.dec to 56) and the epilogue groups
// take them (setmaxnreg.inc to 224): 8 x 32 x 224 + 4 x 32 x 56 = 64512 = 384 x 168, the launch
// allocation exactly, so the increase never waits on registers that do not exist.  The host
// launches the kernel only when it was built with 168 registers per thread.
constexpr int kTmWarps = kTmEpi + 4;
constexpr int kTmLaunchRegs = 168;
constexpr int kTmEpiRegs = 224;
constexpr int kTmAuxRegs = 56;
static_assert(2 * 4 * 32 * kTmEpiRegs + 4 * 32 * kTmAuxRegs == kTmWarps * 32 * kTmLaunchRegs, "register split");
static_assert(kTmEpi == 8, "two epilogue warpgroups");

// forms of the MBD product (TreeArgs::form)
constexpr int kFormSplit = 0;  // A_hi W_hi + A_hi W_lo + A_lo W_hi in BF16 (FP32-equivalent)
constexpr int kFormBf16 = 1;   // A_hi W_hi
constexpr int kFormFp8 = 2;    // E4M3 x E4M3, A scaled per AP

// one accumulator slot: Re G and Im G of the block's 32 q (the split form's three products
// accumulate into it)
__host__ __device__ constexpr int tm_slot_cols(int) { return kTmCols; }
__host__ __device__ constexpr int tm_tmem_anchors(int form, int slots) {
  return (kTmTmemCols - slots * tm_slot_cols(form)) / kTmCols;
}
// K atoms (128 bytes of K per row) of the A tile and of W, and their bytes
__host__ __device__ inline int tm_katoms(int form, int N) { return form == kFormFp8 ? (2 * N + 127) / 128 : (2 * N + 63) / 64; }
__host__ __device__ inline int tm_tile_bytes(int form, int N) {
  return (form == kFormSplit ? 2 : 1) * tm_katoms(form, N) * tc::kAtomBytes;
}
__host__ __device__ inline int tm_w_bytes(int form, int N) {
  return (form == kFormFp8 ? 1 : 2) * tm_katoms(form, N) * kTmWAtom;  // BF16: hi rows then lo rows per atom
}
size_t tm_smem_bytes(int w_bytes, int tile_bytes, int n_abuf, int n_sanc) {
  return (size_t)((w_bytes + 1023) & ~1023) + (size_t)n_abuf * tile_bytes + (size_t)n_sanc * kTmAncBytes + 1024;
}
// Memory plan: the anchor levels go to tensor memory as far as it has room beside the slots (a
// visit moves 64 KB, which shared memory's bandwidth makes slower), the deeper rest to shared
// memory after W and the deepest A-tile ring that fits.  Returns false when nothing fits.
bool tm_plan(int form, int N, int nlev, int *n_abuf, int *n_sanc) {
  const int w_bytes = tm_w_bytes(form, N), tile_bytes = tm_tile_bytes(form, N);
  *n_sanc = max(0, nlev - 1 - tm_tmem_anchors(form, kTmSlots));
  for (int nb = kTmMaxABufs; nb >= 2; --nb)
    if (tm_smem_bytes(w_bytes, tile_bytes, nb, *n_sanc) + 512 <= max_smem_optin()) {  // 512: static
      *n_abuf = nb;
      return true;
    }
  return false;
}

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

// kQ consecutive FP32 columns of this thread's tensor-memory lane, as kQ / 2 packed pairs
template <int kQ>
__device__ __forceinline__ void tm_ld(uint32_t taddr, uint64_t (&v)[kQ / 2]) {
  uint32_t r[kQ];
  if constexpr (kQ == 16) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
  } else {
    static_assert(kQ == 8, "8 or 16 columns");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
#pragma unroll
  for (int p = 0; p < kQ / 2; ++p) v[p] = pk(r[2 * p], r[2 * p + 1]);
}
template <int kQ>
__device__ __forceinline__ void tm_st(uint32_t taddr, const uint64_t (&v)[kQ / 2]) {
  uint32_t r[kQ];
#pragma unroll
  for (int p = 0; p < kQ / 2; ++p) upk(v[p], r[2 * p], r[2 * p + 1]);
  if constexpr (kQ == 16) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                   "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
  } else {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
  }
}
// (v & m) | (c & ~m) in one lop3: the high bits of v with the low bits of the immediate c
__device__ __forceinline__ uint32_t pack_code(uint32_t v, uint32_t c, uint32_t m) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(v), "r"(c), "r"(m));
  return d;
}
// three-input maximum of finite floats (IEEE, subnormals kept)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Placed after tm_wait_ld(): the values a tcgen05.ld wrote pass through this (empty, ordered)
// statement, so no use of them can be scheduled above the wait.
template <int kP>
__device__ __forceinline__ void tm_hold(uint64_t (&v)[kP]) {
  if constexpr (kP == 8) {
    asm volatile("" : "+l"(v[0]), "+l"(v[1]), "+l"(v[2]), "+l"(v[3]), "+l"(v[4]), "+l"(v[5]), "+l"(v[6]), "+l"(v[7]));
  } else {
    static_assert(kP == 4, "4 or 8 packed pairs");
    asm volatile("" : "+l"(v[0]), "+l"(v[1]), "+l"(v[2]), "+l"(v[3]));
  }
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(tc::kRows >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
}
// D = F32, A = B = E4M3 (format code 0), K-major
__device__ __forceinline__ uint32_t idesc_e4m3(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(tc::kRows >> 4) << 24);
}
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
}

}  // namespace

// kEpi epilogue warps, then the MMA warp, the loader warp and two idle warps.  Tensor memory:
// kSlots accumulator slots of 64 columns, then one 64-column block per anchor level e >= 2 at
// block e - 2 (level 2's block is unused: that anchor lives in registers).  Shared memory: W,
// the A-tile ring (t.n_abuf deep), then the t.n_sanc deepest anchor levels as
// [level][16 column quads][128 rows] float4.  kForm: the MBD product (above);
// kFull: the whole delay grid is searched (no windows, no row rotation).
template <int kEpi, int kSlots, int kForm, bool kFull>
__global__ void __launch_bounds__((kEpi + 4) * 32, 1) k_tree_mma(const __grid_constant__ TreeArgs t) {
  constexpr int kMmaWarp = kEpi, kLoadWarp = kEpi + 1;
  constexpr int kQ = kTmNQ / (kEpi / 4);   // MBD columns per epilogue thread (16 or 8)
  constexpr int kP = kQ / 2;               // packed pairs
  constexpr int kSlotCols = tm_slot_cols(kForm);
  constexpr int kAnc = kSlots * kSlotCols;
  static_assert(tm_tmem_anchors(kForm, kSlots) >= 0, "tensor memory");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_afull[kTmMaxABufs], bar_aempty[kTmMaxABufs], bar_accfull[kSlots], bar_accempty[kSlots],
      bar_drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // MBD column blocks vary fastest, so the CTAs sharing one series' A tiles run together (L2)
  int item = blockIdx.x;
  const int qb = item % t.n_qb;
  item /= t.n_qb;
  const int tg = item % t.n_tg, s = item / t.n_tg;
  const int2 sd = t.series[s];
  const int kd = t.T - t.dk_max[sd.y];
  // time tiles tg pack + p (p < pack; pack 1 outside the packed delay-window form), each with
  // its own first AP and AP count; they only get shorter with p
  const int pack = kFull ? 1 : t.pack, lmax = 1 << t.nlev;
  auto tile_kb = [&](int p) { return (tg * pack + p) * t.TT; };
  auto tile_n = [&](int p) { const int b = tile_kb(p); return b < kd ? min(kd, b + t.TT + lmax - 1) - b : 0; };
  const int kb = tile_kb(0);
  if (kb >= kd) return;  // every segment starting here runs past the scan (uniform)
  // searched q of this block (bit j: q = 32 qb + j); none: nothing to do (uniform)
  unsigned qbmask = 0xffffffffu;
  if (!kFull) {
    qbmask = 0u;
    for (int j = 0; j < kTmNQ; ++j)
      if ((((qb * kTmNQ + j) - t.q_lo) & (t.Lm - 1)) < t.q_len) qbmask |= 1u << j;
    if (qbmask == 0u) return;
  }
  const int n_ap = tile_n(0);
  const int nbuf = t.n_abuf, n_tanc = max(t.nlev - 1, 0) - t.n_sanc;  // anchor levels in tensor memory

  unsigned char *sW = smem;                                   // per K atom: hi rows | lo rows
  unsigned char *sA = smem + ((t.w_bytes + 1023) & ~1023);    // ring of one-AP tiles
  ulonglong2 *sAnc = reinterpret_cast<ulonglong2 *>(sA + (size_t)nbuf * t.tile_bytes);
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(t.wimg + (size_t)qb * t.w_bytes);
    uint4 *dst = reinterpret_cast<uint4 *>(sW);
    for (int i = tid; i < t.w_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  if (tid == 0) {
    for (int i = 0; i < nbuf; ++i) {
      tc::mbar_init(&bar_afull[i], 1);
      tc::mbar_init(&bar_aempty[i], 1);
    }
    for (int i = 0; i < kSlots; ++i) {
      tc::mbar_init(&bar_accfull[i], 1);
      tc::mbar_init(&bar_accempty[i], kEpi);  // one arrival per epilogue warp
    }
    tc::mbar_init(&bar_drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
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

  if (warp >= kEpi) {
  // warpgroup 2 (MMA, loader, two idle warps) hands registers to the epilogue warpgroups
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kTmAuxRegs));
  if (warp == kLoadWarp) {
    // ================= loader: one bulk copy of the split A tiles per AP =================
    if (lane == 0) {
      const unsigned char *src = t.Yt + (size_t)s * t.yt_series;
      int issued = 0;
      const int n_load = t.hold ? 0 : n_ap;  // test aid: with hold, no copy is issued
      const int n_sub = t.tile_bytes / tc::kAtomBytes, cut = t.prow * 128;
      // ring position b and the parity of its current use, advanced without a division
      for (int i = 0, b = 0, ph = 0; i < n_load; ++i) {
        if (!tc::mbar_wait(&bar_aempty[b], (uint32_t)ph ^ 1u, abortp, t.timeout)) {
          *abortp = 1;
          break;
        }
        unsigned char *dst = sA + (size_t)b * t.tile_bytes;
        if (pack == 1) {
          tc::mbar_expect_tx(&bar_afull[b], (uint32_t)t.tile_bytes);
          tc::bulk_g2s(dst, src + (size_t)(kb + i) * t.tile_bytes, (uint32_t)t.tile_bytes, &bar_afull[b]);
        } else {
          // the pieces of the tiles still running: piece p fills rows [p prow, (p + 1) prow) of
          // every K atom; rows of finished tiles keep stale values, which only their own
          // (idle) epilogue warps' tensor-memory lanes receive
          int v = 1;
          while (v < pack && i < tile_n(v)) ++v;
          tc::mbar_expect_tx(&bar_afull[b], (uint32_t)(v * t.piece_bytes));
          for (int p = 0; p < v; ++p) {
            const unsigned char *ps = src + (size_t)(tile_kb(p) + i) * t.piece_bytes;
            for (int c = 0; c < n_sub; ++c)
              tc::bulk_g2s(dst + (size_t)c * tc::kAtomBytes + (size_t)p * cut, ps + (size_t)c * cut, (uint32_t)cut,
                           &bar_afull[b]);
          }
        }
        ++issued;
        if (++b == nbuf) {
          b = 0;
          ph ^= 1;
        }
      }
      // every copy issued has landed before the CTA can leave (bounded; ignores the abort flag)
      for (int i = max(0, issued - nbuf); i < issued; ++i)
        if (!tc::mbar_wait(&bar_afull[i % nbuf], (uint32_t)(i / nbuf) & 1, nullptr, t.drain_timeout)) *abortp = 1;
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ================= MMA issuer =================
    // The whole warp runs the loop, so its descriptor arithmetic stays warp-uniform (no
    // per-instruction moves into uniform registers); one elected lane issues the MMAs and
    // commits, which keeps the issue rate at the tensor pipe's pace.
    const bool leader = tc::elect_one();
    const uint32_t id64 = idesc_bf16(kTmCols), id8 = idesc_e4m3(kTmCols);
    // descriptors of the K steps differ only in the start address field (address / 16, in
    // the low 14 bits, which shared-memory offsets below 256 KB never carry out of)
    const uint32_t a_half16 = (uint32_t)(t.KA * tc::kAtomBytes) >> 4;
    const uint64_t w0 = tc::desc_sw128(tc::su32(sW));
    const uint64_t sa0 = tc::desc_sw128(tc::su32(sA));
    const uint32_t tile16 = (uint32_t)t.tile_bytes >> 4;
    bool ok = true;
    for (int i = 0, b = 0, ph = 0, slot = 0, sph = 0; i < n_ap; ++i) {
      const bool got = tc::mbar_wait(&bar_afull[b], (uint32_t)ph, abortp, t.timeout) &&
                       tc::mbar_wait(&bar_accempty[slot], (uint32_t)sph ^ 1u, abortp, t.timeout);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t a0 = sa0 + (uint64_t)(b * tile16);
      const uint32_t d_tmem = tmem + (uint32_t)(slot * kSlotCols);
      if (leader) {
        if constexpr (kForm == kFormSplit) {
          // D = A_hi W_hi + A_hi W_lo + A_lo W_hi, all N = 64 into one accumulator
          for (int ka = 0; ka < t.KA; ++ka) {
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              const uint32_t ao = (uint32_t)((ka * tc::kAtomBytes + k4 * 32) >> 4);
              const uint32_t bo = (uint32_t)((ka * 2 * kTmWAtom + k4 * 32) >> 4);
              mma_bf16(d_tmem, a0 + ao, w0 + bo, id64, (ka | k4) ? 1u : 0u);
              mma_bf16(d_tmem, a0 + ao, w0 + bo + (uint32_t)(kTmWAtom >> 4), id64, 1u);
              mma_bf16(d_tmem, a0 + a_half16 + ao, w0 + bo, id64, 1u);
            }
          }
        } else if constexpr (kForm == kFormBf16) {
          // D = A_hi W_hi (the hi rows of each W atom)
          for (int ka = 0; ka < t.KA; ++ka) {
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              const uint32_t ao = (uint32_t)((ka * tc::kAtomBytes + k4 * 32) >> 4);
              const uint32_t bo = (uint32_t)((ka * 2 * kTmWAtom + k4 * 32) >> 4);
              mma_bf16(d_tmem, a0 + ao, w0 + bo, id64, (ka | k4) ? 1u : 0u);
            }
          }
        } else {
          // D = A8 W8 (E4M3, K = 32 per instruction, 32 bytes of each 128-byte row)
          for (int kk = 0; kk < t.k8_steps; ++kk) {
            const uint32_t ao = (uint32_t)(((kk >> 2) * tc::kAtomBytes + (kk & 3) * 32) >> 4);
            const uint32_t bo = (uint32_t)(((kk >> 2) * kTmWAtom + (kk & 3) * 32) >> 4);
            mma_e4m3(d_tmem, a0 + ao, w0 + bo, id8, kk ? 1u : 0u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tc::su32(&bar_accfull[slot])) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(tc::su32(&bar_aempty[b])) : "memory");
      }
      __syncwarp();
      if (++b == nbuf) {
        b = 0;
        ph ^= 1;
      }
      if (++slot == kSlots) {
        slot = 0;
        sph ^= 1;
      }
    }
    if (!ok && leader) *abortp = 1;
    // drain: a last commit lands only when every MMA the leader issued has completed
    if (leader)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(tc::su32(&bar_drain)) : "memory");
    __syncwarp();
    if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_drain, 0, nullptr, t.drain_timeout)) && leader) *abortp = 1;
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kTmEpiRegs));
    // ================= epilogue: window tree and maxima =================
    const int quarter = warp & 3, part = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t c_re = (uint32_t)(kQ * part), c_im = (uint32_t)(kTmNQ + kQ * part);
    // this warp's time tile (its piece of the packed operand) and its first AP and AP count
    const int qpp = 4 / pack, my_p = quarter / qpp;
    const int kb_me = tile_kb(my_p), n_me = tile_n(my_p);
    // this lane's SBD row m (row (quarter mod qpp) 32 + lane of its piece, rotated by t.rot) and
    // its first cell
    const int m_row = ((quarter % qpp) * 32 + lane + t.rot) & (t.Ls - 1);
    const unsigned idx_base = (unsigned)(m_row * t.Lm + qb * kTmNQ + kQ * part);
    // delay windows: the lane's row is searched, and which of its kQ cells
    const bool row_on = kFull || (((m_row - t.m_lo) & (t.Ls - 1)) < t.m_len);
    const unsigned qmask = kFull ? 0xffffffffu : (qbmask >> (kQ * part)) & ((1u << kQ) - 1u);
    if (!kFull && !__any_sync(0xffffffffu, row_on && qmask != 0u)) {
      // nothing of this warp is searched: it only hands each slot back
      bool ok = true;
      for (int i = 0, slot = 0, sph = 0; i < n_ap && ok; ++i) {
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_accfull[slot], (uint32_t)sph, abortp, t.timeout))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&bar_accempty[slot]);
        if (++slot == kSlots) {
          slot = 0;
          sph ^= 1;
        }
      }
      if (!ok) *abortp = 1;
    } else {
    // this thread's quads of a shared-memory anchor: re at kQ/4 part + u, im at 8 + kQ/4 part + u
    ulonglong2 *my_anc = sAnc + (size_t)(kQ / 4 * part) * tc::kRows + quarter * 32 + lane;
    unsigned long long *keys = t.keys + ((size_t)sd.x * t.n_dm + sd.y) * t.S_tot;
    int woff[kTmMaxLev + 1];  // first slot of the window emitted at each level (-1: none)
#pragma unroll
    for (int e = 0; e <= kTmMaxLev; ++e) woff[e] = t.emit_w[e] >= 0 ? t.win_off[t.emit_w[e]] : -1;
    unsigned wlev = 0;  // levels whose window is searched
#pragma unroll
    for (int e = 0; e <= kTmMaxLev; ++e) wlev |= t.emit_w[e] >= 0 ? 1u << e : 0u;
    uint64_t ga_re[kP], ga_im[kP], gb_re[kP], gb_im[kP];  // G_1 of two consecutive APs, alternating
#pragma unroll
    for (int p = 0; p < kP; ++p) ga_re[p] = ga_im[p] = gb_re[p] = gb_im[p] = 0ull;
    for (int a = 0; a + 2 <= t.nlev; ++a) {
      if (a < n_tanc) {
        const uint32_t ab = lane_base + (uint32_t)(kAnc + a * kTmCols);
        tm_st<kQ>(ab + c_re, ga_re);
        tm_st<kQ>(ab + c_im, ga_im);
      } else {
        ulonglong2 *q = my_anc + (size_t)(a - n_tanc) * 16 * tc::kRows;
#pragma unroll
        for (int u = 0; u < kQ / 4; ++u) {
          q[u * tc::kRows] = make_ulonglong2(0ull, 0ull);
          q[(8 + u) * tc::kRows] = make_ulonglong2(0ull, 0ull);
        }
      }
    }
    tm_wait_st();
    // Maximum of one emitted segment's cells: packed keys (|G|^2 with the 6 low mantissa bits
    // replaced by 31 - j, so the lower q wins a tie), a three-input maximum tree (the keys are
    // non-negative floats, ordered as their bit patterns), the warp maximum, and one 64-bit
    // atomicMax into the series by the lane holding it (tied lanes share j; the atomicMax keeps
    // the lowest of their indices).
    // i0: the segment's first AP, counted from the time tile's first AP kb_me
    const uint32_t kmask = 0xffffffc0u;  // kept in a register: one lop3 per cell packs its code
    // the thread's maximum key over its kQ cells of one segment
    auto seg_top = [&](const uint64_t(&gre)[kP], const uint64_t(&gim)[kP]) -> unsigned {
      float kf[kQ];
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        uint32_t lo, hi;
        upk(fma2(gre[p], gre[p], mul2(gim[p], gim[p])), lo, hi);
        kf[2 * p] = __uint_as_float(pack_code(lo, 31u - 2u * p, kmask));
        kf[2 * p + 1] = __uint_as_float(pack_code(hi, 30u - 2u * p, kmask));
      }
      if (!kFull && qmask != (1u << kQ) - 1u) {  // cells outside the MBD window (uniform per warp)
#pragma unroll
        for (int j = 0; j < kQ; ++j) kf[j] = (qmask >> j) & 1u ? kf[j] : 0.f;
      }
      float top;
      if constexpr (kQ == 16) {
        float m5[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) m5[j] = fmax3(kf[3 * j], kf[3 * j + 1], kf[3 * j + 2]);
        top = fmax3(fmax3(m5[0], m5[1], m5[2]), fmax3(m5[3], m5[4], kf[15]), 0.f);
      } else {
        static_assert(kQ == 8, "8 or 16 cells per thread");
        top = fmax3(fmax3(kf[0], kf[1], kf[2]), fmax3(kf[3], kf[4], kf[5]), fmaxf(kf[6], kf[7]));
      }
      return row_on ? __float_as_uint(top) : 0u;
    };
    // the warp maximum of a segment of level e starting at AP i0 (counted from the time tile's
    // first AP kb_me), merged into the series by the lanes holding it when `on` (uniform)
    // first slot of the tile's segments at levels 0 to 2 (kb_me is a multiple of 64, so a
    // segment starting at tile AP i0 >= 0 sits i0 >> (e - 1) slots further; a merge of a segment
    // starting before the tile is never issued)
    unsigned long long *const base0 = keys + woff[0] + kb_me, *const base1 = keys + woff[1] + kb_me,
                              *const base2 = keys + woff[2] + (kb_me >> 1);
    auto merge = [&](const int e, const int i0, const unsigned tkey, const bool on) {
      const unsigned wmax = __reduce_max_sync(0xffffffffu, tkey);
      // every lane forms the merge; the lanes holding the maximum issue it (predicated, no branch)
      const unsigned idx = idx_base + (31u - (wmax & 63u));
      // slot of the segment: windows of 2^e APs start every 2^(e-1) APs (every AP for e = 0)
      unsigned long long *dst = e == 0   ? base0 + i0
                                : e == 1 ? base1 + i0
                                : e == 2 ? base2 + (i0 >> 1)
                                         : keys + woff[e] + ((kb_me + i0) >> (e - 1));
      const unsigned long long kv = ((unsigned long long)(wmax & ~63u) << 32) | (unsigned long long)(~idx);
      asm volatile("{\n .reg .pred p;\n setp.eq.u32 p, %2, %3;\n setp.ne.and.u32 p, %3, 0, p;\n"
                   " setp.ne.and.u32 p, %4, 0, p;\n @p red.relaxed.gpu.global.max.u64 [%0], %1;\n}\n"
                   ::"l"(dst), "l"(kv), "r"(tkey), "r"(wmax), "r"((unsigned)on) : "memory");
    };
    auto emit = [&](const int e, const int i0, const uint64_t(&gre)[kP], const uint64_t(&gim)[kP]) {
      merge(e, i0, seg_top(gre, gim), true);
    };
    // One AP: cur receives G_1(k); pre holds G_1(k - 1).  odd: k is odd (counted from the tile's
    // first AP, a multiple of 64), so it closes a window of 4 APs: the level-1 sum
    // G_2(k - 1) = G_1(k - 1) + G_1(k) goes to anc_out, and G_4(k - 3) = anc_in + anc_out with
    // anc_in = G_2(k - 3), the previous odd AP's level-1 sum (the level-2 anchor lives in
    // registers; two arrays alternate).  deep: k + 1 is a multiple of 4, so levels 3 and up may
    // close too (anchors in tensor memory).  odd and deep are literals at every call.  Returns
    // false when a wait gave up.
    auto one_ap = [&](const int i, const int slot, const uint32_t sph, const bool odd, const bool deep,
                      const uint64_t(&pre)[kP], const uint64_t(&pim)[kP], uint64_t(&cre)[kP], uint64_t(&cim)[kP],
                      const uint64_t(&ain_re)[kP], const uint64_t(&ain_im)[kP], uint64_t(&aout_re)[kP],
                      uint64_t(&aout_im)[kP]) -> bool {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_accfull[slot], sph, abortp, t.timeout))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t cur = lane_base + (uint32_t)(slot * kSlotCols);
      tm_ld<kQ>(cur + c_re, cre);
      tm_ld<kQ>(cur + c_im, cim);

      float inv_s = 1.f;  // E4M3 form: the AP's A was scaled by s, a power of two
      if constexpr (kForm == kFormFp8) inv_s = __ldg(t.ascale + (size_t)s * t.T + kb_me + i);
      // levels whose window ends at AP kb_me + i, and which of them emit a segment of this time
      // tile (uniform across the warp; kb_me is a multiple of 2^kTmMaxLev, so i's low bits
      // decide)
      // (an even AP closes levels 0 and 1 only, an odd AP that is not deep levels 0 to 2; wlev
      // holds no level above t.nlev)
      const int E = !odd ? min(t.nlev, 1) : !deep ? min(t.nlev, 2) : min(t.nlev, __ffs(i + 1));
      unsigned em = wlev & (!odd ? 3u : !deep ? 7u : (2u << E) - 1u);
      if (i < (1 << kTmMaxLev) - 1 || i >= t.TT) {  // segments starting outside the tile (uniform, rare)
#pragma unroll
        for (int e = 0; e <= kTmMaxLev; ++e) {
          const int i0 = i - (1 << e) + 1;
          if (i0 < 0 || i0 >= t.TT) em &= ~(1u << e);
        }
      }
      tm_wait_ld();
      tm_hold<kP>(cre);
      tm_hold<kP>(cim);
      if constexpr (kForm == kFormFp8) {
        const uint64_t iv = pk(__float_as_uint(inv_s), __float_as_uint(inv_s));
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          cre[p] = mul2(cre[p], iv);
          cim[p] = mul2(cim[p], iv);
        }
      }
      // G_1(k) is in the warp's registers: its slot may take AP k + kSlots.  One arrival per
      // warp: 256 arrivals on one mbarrier serialise as shared-memory atomics.
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_accempty[slot]);
      if (!odd) {
        // levels 0 and 1 as one block without branches (their key trees interleave)
        uint64_t are[kP], aim[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          are[p] = add2(pre[p], cre[p]);
          aim[p] = add2(pim[p], cim[p]);
        }
        const unsigned top0 = seg_top(cre, cim), top1 = seg_top(are, aim);
        merge(0, i, top0, (em & 1u) != 0u);
        merge(1, i - 1, top1, (em & 2u) != 0u);
        return true;
      }
      // odd AP: levels 0, 1 and 2 as one block
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        aout_re[p] = add2(pre[p], cre[p]);
        aout_im[p] = add2(pim[p], cim[p]);
      }
      uint64_t are[kP], aim[kP];
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        are[p] = add2(ain_re[p], aout_re[p]);
        aim[p] = add2(ain_im[p], aout_im[p]);
      }
      const unsigned top0 = seg_top(cre, cim), top1 = seg_top(aout_re, aout_im), top2 = seg_top(are, aim);
      merge(0, i, top0, (em & 1u) != 0u);
      merge(1, i - 1, top1, (em & 2u) != 0u);
      merge(2, i - 3, top2, ((em >> 2) & 1u) != 0u);
      if (!deep || E <= 2) return true;
      // levels 3 and up: anchor e - 2 of tensor memory (or shared memory) holds the first half
#pragma unroll
      for (int e = 3; e <= kTmMaxLev; ++e) {
        if (e > E) break;
        uint64_t ore[kP], oim[kP];
        const bool in_tmem = e - 2 < n_tanc;  // uniform
        if (in_tmem) {
          const uint32_t ab = lane_base + (uint32_t)(kAnc + (e - 2) * kTmCols);
          tm_ld<kQ>(ab + c_re, ore);
          tm_ld<kQ>(ab + c_im, oim);
          tm_wait_ld();
          tm_hold<kP>(ore);
          tm_hold<kP>(oim);
          tm_st<kQ>(ab + c_re, are);
          tm_st<kQ>(ab + c_im, aim);
        } else {
          ulonglong2 *q = my_anc + (size_t)(e - 2 - n_tanc) * 16 * tc::kRows;
#pragma unroll
          for (int u = 0; u < kQ / 4; ++u) {
            const ulonglong2 r = q[u * tc::kRows], m = q[(8 + u) * tc::kRows];
            ore[2 * u] = r.x;
            ore[2 * u + 1] = r.y;
            oim[2 * u] = m.x;
            oim[2 * u + 1] = m.y;
            q[u * tc::kRows] = make_ulonglong2(are[2 * u], are[2 * u + 1]);
            q[(8 + u) * tc::kRows] = make_ulonglong2(aim[2 * u], aim[2 * u + 1]);
          }
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          are[p] = add2(are[p], ore[p]);
          aim[p] = add2(aim[p], oim[p]);
        }
        if (in_tmem) tm_wait_st();
        if ((em >> e) & 1u) emit(e, i - (1 << e) + 1, are, aim);
      }
      return true;
    };
    // AP i uses slot i mod 2 for the (i / 2)-th time, so in every group of four APs starting at
    // a multiple of 4 the slots are 0, 1, 0, 1 and the phase parities 0, 0, 1, 1
    uint64_t ha_re[kP], ha_im[kP], hb_re[kP], hb_im[kP];  // level-2 anchors, alternating
#pragma unroll
    for (int p = 0; p < kP; ++p) ha_re[p] = ha_im[p] = hb_re[p] = hb_im[p] = 0ull;
    bool ok = true;
    int i = 0;
    for (; i + 3 < n_me; i += 4) {
      if (!one_ap(i, 0, 0u, false, false, gb_re, gb_im, ga_re, ga_im, hb_re, hb_im, ha_re, ha_im) ||
          !one_ap(i + 1, 1, 0u, true, false, ga_re, ga_im, gb_re, gb_im, hb_re, hb_im, ha_re, ha_im) ||
          !one_ap(i + 2, 0, 1u, false, false, gb_re, gb_im, ga_re, ga_im, ha_re, ha_im, hb_re, hb_im) ||
          !one_ap(i + 3, 1, 1u, true, true, ga_re, ga_im, gb_re, gb_im, ha_re, ha_im, hb_re, hb_im)) {
        ok = false;
        break;
      }
    }
    // the last one to three APs
    if (ok && i < n_me) {
      ok = one_ap(i, 0, 0u, false, false, gb_re, gb_im, ga_re, ga_im, hb_re, hb_im, ha_re, ha_im);
      ++i;
      if (ok && i < n_me) {
        ok = one_ap(i, 1, 0u, true, false, ga_re, ga_im, gb_re, gb_im, hb_re, hb_im, ha_re, ha_im);
        ++i;
        if (ok && i < n_me) {
          ok = one_ap(i, 0, 1u, false, false, gb_re, gb_im, ga_re, ga_im, ha_re, ha_im, hb_re, hb_im);
          ++i;
        }
      }
    }
    // a packed time tile that ended before the CTA's first one: hand back the slots of the
    // remaining APs
    static_assert(kSlots == 2, "two accumulator slots, used alternately");
    const int n_all = kFull ? n_me : tile_n(0);
    for (; ok && i < n_all; ++i) {
      const int slot = i & 1;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&bar_accfull[slot], (uint32_t)(i >> 1) & 1u, abortp, t.timeout))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bar_accempty[slot]);
    }
    if (!ok) *abortp = 1;
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmTmemCols) : "memory");
  if (tid == 0 && abort_flag) atomicExch(t.err, FRBX_ETIMEOUT);
}

bool tree_mma_supported(int Ls, int Lm, int N, int J) {
  return Ls == tc::kRows && J <= Ls && Lm % kTmNQ == 0 && 2 * N <= 128;
}

bool tree_mma_fits(int form, int N, int nlev) {
  int nb, ns;
  return form >= kFormSplit && form <= kFormFp8 && nlev >= 0 && nlev <= kTmMaxLev && tm_plan(form, N, nlev, &nb, &ns);
}

int tree_mma_tile_bytes(int form, int N) { return tm_tile_bytes(form, N); }
int tree_mma_w_bytes(int form, int N) { return tm_w_bytes(form, N); }

template <int kForm, bool kFull>
static cudaError_t launch_tm_one(const TreeArgs &u, unsigned nb, size_t smem, cudaStream_t st) {
  auto kern = k_tree_mma<kTmEpi, kTmSlots, kForm, kFull>;
  // the register split inside the kernel assumes the launch allocation of kTmLaunchRegs per thread
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kTmLaunchRegs || fa.maxThreadsPerBlock < kTmWarps * 32) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nb, kTmWarps * 32, smem, st>>>(u);
  return cudaGetLastError();
}

cudaError_t launch_tree_mma(const TreeArgs &t, bool full, cudaStream_t st, int64_t *launches) {
  if (t.nlev < 0 || t.nlev > kTmMaxLev || t.form < kFormSplit || t.form > kFormFp8 || t.KA != tm_katoms(t.form, t.N) ||
      t.w_bytes != tm_w_bytes(t.form, t.N) || t.tile_bytes != tm_tile_bytes(t.form, t.N) ||
      (t.form == kFormFp8 && (!t.ascale || t.k8_steps != (2 * t.N + 31) / 32)) || (full && t.rot != 0) ||
      (t.rot & 7) != 0 || !(t.pack == 1 || t.pack == 2 || t.pack == 4) || (full && t.pack != 1) ||
      t.prow * t.pack != tc::kRows || t.piece_bytes * t.pack != t.tile_bytes || t.n_tg * t.pack < t.n_tt ||
      t.TT % (1 << kTmMaxLev) != 0)
    return cudaErrorInvalidValue;
  TreeArgs u = t;
  if (!tm_plan(t.form, t.N, t.nlev, &u.n_abuf, &u.n_sanc)) return cudaErrorInvalidConfiguration;
  const size_t smem = tm_smem_bytes(t.w_bytes, t.tile_bytes, u.n_abuf, u.n_sanc);
  const long long nb = (long long)t.n_s * t.n_qb * t.n_tg;
  if (nb <= 0) return cudaSuccess;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)nb;
  cudaError_t e;
  switch (t.form * 2 + (full ? 1 : 0)) {
    case 0: e = launch_tm_one<kFormSplit, false>(u, g, smem, st); break;
    case 1: e = launch_tm_one<kFormSplit, true>(u, g, smem, st); break;
    case 2: e = launch_tm_one<kFormBf16, false>(u, g, smem, st); break;
    case 3: e = launch_tm_one<kFormBf16, true>(u, g, smem, st); break;
    case 4: e = launch_tm_one<kFormFp8, false>(u, g, smem, st); break;
    default: e = launch_tm_one<kFormFp8, true>(u, g, smem, st); break;
  }
  ++*launches;
  return e;
}

}  // namespace frbx
