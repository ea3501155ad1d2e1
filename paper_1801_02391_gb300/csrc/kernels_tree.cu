// Multi-window segment fit through the additivity of the delay-resolution matrix (Sec. 5.1):
//
//   G_{k0, l1} + G_{k0 + l1, l2} = G_{k0, l1 + l2}
//
// With windows that are powers of two on the half-overlap grid (step l/2, step 1 for l = 1),
// every segment of window 2l is the sum of two segments of window l:
//
//   G_{2l}(k0) = G_l(k0) + G_l(k0 + l),   k0 a multiple of step(2l) = l,
//
// so the 2-D transform (Eq. 5 on the Sec. 5.1 grid) runs once per AP -- on the one-AP
// segment -- and every longer window is built by matrix additions; the Eq. 3 sums over time
// move from the spectra to the delay-resolution matrices.  Two kernels per chunk of
// (baseline, DM) series:
//
//  k_tree_sbd  gathers the dedispersed one-AP spectrum X(n, j) = w c S(n, j, k + dk(n, j)) and
//              applies the SBD transform per channel (32-point register FFTs, as in the
//              segment fit), writing Y[series][k][m][n] to device memory;
//  k_tree_mbd  owns a block of RB SBD rows m of one series and a time tile.  A thread owns 16
//              cells of one row: its rows of Y go to shared memory with channel n in slot
//              (g_n mod 16) + 16 o (o its rank in that class; empty slots zero), and for MBD
//              column class q1 (q = q1 + PM q2) and half h the thread folds the slots (a static
//              loop) into the 16 inputs of one half of a 32-point
//              DIF FFT (even or odd q2), runs a 16-point register FFT and walks the cells
//              through the window tree: the newest matrix of every level is summed with the
//              anchor of that level (the previous segment needed as first half), emitted, and
//              becomes the new anchor.  The level-1 anchor lives in registers, the next three in
//              shared memory, deeper ones in an L2-resident per-CTA slice of device memory.
//              Each emitted segment's maximum over the block's cells is reduced in the CTA and
//              merged across blocks by a 64-bit atomicMax on (|G|^2 bits, ~cell index) in the
//              series buffer, which k_tree_finalize turns into frbx_seg records.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "fit_common.cuh"
#include "fft32.cuh"
#include "tc_common.cuh"

namespace frbx {

constexpr int kTreeThreads = 128;
constexpr int kTreeMaxLev = 6;  // windows up to 64 APs
constexpr int kSbdBatch = 16;   // SBD pass: cube loads in flight per thread

// Anchors of the window tree: level 1 in registers, the next kTreeSmemAnc levels in shared
// memory, deeper ones (touched every 16 APs or less often) in a per-CTA slice of device memory.
constexpr int kTreeSmemAnc = 3;

__host__ __device__ inline int tree_smem_anchors(int nlev) { return nlev - 1 < kTreeSmemAnc ? (nlev > 1 ? nlev - 1 : 0) : kTreeSmemAnc; }
__host__ __device__ inline int tree_global_anchors(int nlev) { return (nlev > 1 ? nlev - 1 : 0) - tree_smem_anchors(nlev); }

__host__ __device__ inline size_t tree_smem_bytes(int NS, int PM, int RB, int nlev) {
  const size_t tw = sizeof(float2) * (size_t)NS * PM * 2;
  const size_t yb = sizeof(float2) * 2 * (size_t)RB * NS;
  const size_t an = sizeof(float2) * (size_t)tree_smem_anchors(nlev) * 16 * kTreeThreads;
  const size_t red = sizeof(uint2) * 2 * (kTreeMaxLev + 1) * (kTreeThreads / 32);
  return tw + yb + an + red;
}

// ----------------------------------------------------------------------------- SBD pass
// shared -> global bulk copy (16-byte aligned addresses, a multiple of 16 bytes), completion
// tracked by the issuing thread's bulk group
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(tc::su32(src)), "r"(bytes)
               : "memory");
}

// kOut 0: FP32 rows Y[m][n] for k_tree_mbd.  kOut 1..3: each AP's output is the tensor-core A
// operand of k_tree_mma in its shared-memory image, 128 rows x K = 2N (Re Y of the channels, then
// Im Y), 128-byte swizzled K atoms: 1 = A_hi = bf16(Y) then A_lo = bf16(Y - A_hi); 2 = A_hi only;
// 3 = E4M3 of s Y, s the power of two with s L1 <= 448 (L1 = the L1 norm of the AP's dedispersed
// spectrum, which bounds every |Re Y|, |Im Y|), 1 / s stored in t.ascale.  Tile row r holds SBD
// row (r + t.rot) mod Ls (rotation for delay windows; 0 for the whole grid); with t.pack > 1
// only the first t.prow rows of every K atom are stored (t.piece_bytes per AP).
template <int kOut>
__global__ void __launch_bounds__(kTreeThreads, 4)
    k_tree_sbd(const __grid_constant__ FitArgs a, const __grid_constant__ TreeArgs t) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float red_l1[kTreeThreads / 32];
  const int N = a.N, Ls = a.Ls, PS = Ls >> 5, lps = __ffs(PS) - 1;
  const int JP = a.J1 * 32, xs = JP + 1;
  const int stage = kOut ? t.tile_bytes : (int)sizeof(float2) * Ls * N;  // one AP of output
  float2 *Ys = reinterpret_cast<float2 *>(smem);                        // [Ls][N] or the tiles
  unsigned char *Yb = smem;
  float2 *X = reinterpret_cast<float2 *>(smem + stage);  // [N][xs]
  float2 *stw = X + N * xs;                              // [PS][xs]
  for (int i = threadIdx.x; i < N * xs; i += blockDim.x) X[i] = make_float2(0.f, 0.f);
  if (kOut)  // K columns beyond 2N stay zero
    for (int i = threadIdx.x; i < stage / 16; i += blockDim.x) reinterpret_cast<uint4 *>(Yb)[i] = make_uint4(0, 0, 0, 0);
  for (int i = threadIdx.x; i < PS * JP; i += blockDim.x) {
    const int r = i / JP, c = i - r * JP;
    stw[r * xs + c] = a.sbd_tw[i];
  }
  // DM trials vary fastest, so the CTAs resident together read the same stretch of the cube
  const int s = blockIdx.x % t.n_s, tile = blockIdx.x / t.n_s;
  const int2 sd = t.series[s];
  const int kd = a.T - t.dk_max[sd.y];
  const int k_lo = tile * t.k_per_cta, k_hi = min(kd, k_lo + t.k_per_cta);
  const int *dk = a.dk + (size_t)sd.y * a.C;
  float4 *Yout = kOut ? reinterpret_cast<float4 *>(const_cast<unsigned char *>(t.Yt) + (size_t)s * t.yt_series)
                      : reinterpret_cast<float4 *>(t.Y + (size_t)s * t.y_series);
  const int row4 = stage / 16;  // float4 per AP
  const int rot8 = t.rot >> 3;  // rotation in groups of 8 rows
  // this thread's points p = tid + blockDim i: channel n and point j stepped without a division
  const int dn = (int)blockDim.x / a.J, dj = (int)blockDim.x - dn * a.J;
  const int n0 = (int)threadIdx.x / a.J, j0 = (int)threadIdx.x - n0 * a.J;
  __syncthreads();
  // When one batch covers every point, the thread's points and their offsets dk(c) C + c in the
  // cube are fixed for the whole series: kept in registers, so no cube address waits on a
  // shift-table load
  const bool one_batch = a.C <= (int)blockDim.x * kSbdBatch;
  int off[kSbdBatch];
#pragma unroll
  for (int q = 0; q < kSbdBatch; ++q) {
    const int p = (int)threadIdx.x + q * (int)blockDim.x;
    off[q] = one_batch && p < a.C ? __ldg(dk + p) * a.C + p : -1;
  }
  for (int k = k_lo; k < k_hi; ++k) {
    // Eq. 3 with l = 1: the dedispersed spectrum of AP k, weighted and rotated; kSbdBatch
    // independent cube loads in flight per thread (the shift-table row stays in L1)
    const size_t row0 = (size_t)sd.x * a.T + k;
    int n = n0, j = j0;
    float l1 = 0.f;
    for (int p0 = threadIdx.x; p0 < a.C; p0 += blockDim.x * kSbdBatch) {
      float2 v[kSbdBatch];
      if (one_batch) {
        const float2 *rowp = a.vis + row0 * a.C;
#pragma unroll
        for (int q = 0; q < kSbdBatch; ++q) v[q] = off[q] >= 0 ? __ldg(rowp + off[q]) : make_float2(0.f, 0.f);
      } else {
#pragma unroll
        for (int q = 0; q < kSbdBatch; ++q) {
          const int p = p0 + q * (int)blockDim.x;
          v[q] = p < a.C ? __ldg(a.vis + (row0 + __ldg(dk + p)) * a.C + p) : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int q = 0; q < kSbdBatch; ++q) {
        const int p = p0 + q * (int)blockDim.x;
        if (p < a.C) {
          const float2 x = cmul(v[q], __ldg(a.wrot + p));
          X[n * xs + j] = x;
          if (kOut == 3) l1 += fabsf(x.x) + fabsf(x.y);
        }
        n += dn;
        j += dj;
        if (j >= a.J) {
          j -= a.J;
          ++n;
        }
      }
    }
    if (kOut == 3) {
#pragma unroll
      for (int off = 16; off; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
      if ((threadIdx.x & 31) == 0) red_l1[threadIdx.x >> 5] = l1;
    }
    // the bulk copy of the previous AP's output has read the staging buffer
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
    float sc = 1.f;
    if (kOut == 3) {
      float tot = 0.f;
#pragma unroll
      for (int w = 0; w < kTreeThreads / 32; ++w) tot += red_l1[w];
      int ex = 1;
      if (tot > 1e-30f) frexpf(448.f / tot, &ex);
      sc = ldexpf(1.f, max(-100, min(100, ex - 1)));
      if (threadIdx.x == 0) t.ascale[(size_t)s * a.T + k] = 1.f / sc;
    }
    // SBD transform of every channel, task (n, m1); row m = m1 + PS m2 holds the channel slots
    for (int u = threadIdx.x; u < N * PS; u += blockDim.x) {
      const int n = u >> lps, m1 = u & (PS - 1);
      float2 A[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) A[i] = make_float2(0.f, 0.f);
      const float2 *xr = X + n * xs;
      const float2 *wr = stw + m1 * xs;
      for (int j1 = 0; j1 < a.J1; ++j1) {
#pragma unroll
        for (int j2 = 0; j2 < 32; ++j2) A[j2] = cfma(A[j2], xr[j1 * 32 + j2], wr[j1 * 32 + j2]);
      }
      fft32_dif(A);
      if (kOut == 1 || kOut == 2) {
        const int half = t.tile_bytes / 2;
        // Ls = 128 rows (PS = 4): row = m1 + 4 b with b = bitrev5(i), so (row - rot) / 8 = b / 2 - rot / 8
        // and row % 8 = m1 + 4 (b % 2); the swizzled offsets of columns n and N + n for even and
        // odd b are fixed per thread, and each element adds its 1 KB row group
        uint32_t o_re[2] = {0u, 0u}, o_im[2] = {0u, 0u};
        if (PS == 4) {
#pragma unroll
          for (int odd = 0; odd < 2; ++odd) {
            o_re[odd] = tc::a_offset(m1 + 4 * odd, n);
            o_im[odd] = tc::a_offset(m1 + 4 * odd, N + n);
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int b = bitrev5(i), row = (m1 + PS * b - t.rot) & (Ls - 1);
          const __nv_bfloat16 rh = __float2bfloat16_rn(A[i].x), ih = __float2bfloat16_rn(A[i].y);
          const uint32_t grp = (uint32_t)(((b >> 1) - rot8) & 15) * 1024u;
          const uint32_t orr = PS == 4 ? o_re[b & 1] + grp : tc::a_offset(row, n);
          const uint32_t oi = PS == 4 ? o_im[b & 1] + grp : tc::a_offset(row, N + n);
          *reinterpret_cast<__nv_bfloat16 *>(Yb + orr) = rh;
          *reinterpret_cast<__nv_bfloat16 *>(Yb + oi) = ih;
          if (kOut == 1) {
            const __nv_bfloat16 rl = __float2bfloat16_rn(A[i].x - __bfloat162float(rh));
            const __nv_bfloat16 il = __float2bfloat16_rn(A[i].y - __bfloat162float(ih));
            *reinterpret_cast<__nv_bfloat16 *>(Yb + half + orr) = rl;
            *reinterpret_cast<__nv_bfloat16 *>(Yb + half + oi) = il;
          }
        }
      } else if (kOut == 3) {
        uint32_t o_re[2] = {0u, 0u}, o_im[2] = {0u, 0u};
        if (PS == 4) {
#pragma unroll
          for (int odd = 0; odd < 2; ++odd) {
            o_re[odd] = tc::a_offset8(m1 + 4 * odd, n);
            o_im[odd] = tc::a_offset8(m1 + 4 * odd, N + n);
          }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int b = bitrev5(i), row = (m1 + PS * b - t.rot) & (Ls - 1);
          const uint32_t grp = (uint32_t)(((b >> 1) - rot8) & 15) * 1024u;
          const uint32_t orr = PS == 4 ? o_re[b & 1] + grp : tc::a_offset8(row, n);
          const uint32_t oi = PS == 4 ? o_im[b & 1] + grp : tc::a_offset8(row, N + n);
          Yb[orr] = (unsigned char)__nv_cvt_float_to_fp8(A[i].x * sc, __NV_SATFINITE, __NV_E4M3);
          Yb[oi] = (unsigned char)__nv_cvt_float_to_fp8(A[i].y * sc, __NV_SATFINITE, __NV_E4M3);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) Ys[(m1 + PS * bitrev5(i)) * N + n] = A[i];
      }
    }
    // the staged output goes to device memory as bulk copies issued by one thread, which run
    // while the next AP is gathered (the generic-proxy writes are fenced for the async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!kOut || t.pack == 1) {
        bulk_s2g(Yout + (size_t)k * row4, Yb, (uint32_t)stage);
      } else {
        // packed delay-window form: the first prow rows of every K atom
        unsigned char *dst = reinterpret_cast<unsigned char *>(Yout) + (size_t)k * t.piece_bytes;
        const uint32_t per = (uint32_t)t.prow * 128u;
        for (int c = 0; c < stage / tc::kAtomBytes; ++c)
          bulk_s2g(dst + (size_t)c * per, Yb + (size_t)c * tc::kAtomBytes, per);
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  // every copy has landed before the CTA leaves
  if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ----------------------------------------------------------------------------- MBD + tree
// Packed per-thread key of a cell, |G|^2 with its low mantissa bits replaced by a code that
// prefers the lower q2 on equal truncated powers.  Whole grid: 4 bits, 15 - b with b = q2 div 2
// the thread's cell rank (2^-19 relative truncation; between the two threads of a class the
// even half h = 0 wins a tie as the lower lane), merged by one lop3 with m = ~15 kept in a
// register.  Delay windows (fewer registers to spare): 6 bits, 32 - q2 (2^-17).
template <bool kFull>
__device__ __forceinline__ unsigned cell_key(float2 v, int b, int h, unsigned m) {
  const float p = fmaf(v.x, v.x, v.y * v.y);
  if constexpr (!kFull) return (__float_as_uint(p) & ~63u) | (unsigned)(32 - (2 * b + h));
  unsigned d;
  asm("lop3.b32 %0, %1, %2, %3, 0xE4;" : "=r"(d) : "r"(__float_as_uint(p)), "r"(15u - (unsigned)b), "r"(m));
  return d;
}

template <int S16, bool kFull>
__global__ void __launch_bounds__(kTreeThreads, 3) k_tree_mbd(const __grid_constant__ TreeArgs t) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NS = 16 * S16;
  const int PM = t.PM, RB = t.RB, Lm = t.Lm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n_sm = tree_smem_anchors(t.nlev);
  float2 *tw = reinterpret_cast<float2 *>(smem);  // [NS/2][PM][2][2]
  float2 *yb = tw + NS * PM * 2;                   // [2][RB][NS]
  float2 *anc = yb + 2 * RB * NS;                  // [n_sm][16][128]
  uint2 *red = reinterpret_cast<uint2 *>(anc + n_sm * 16 * kTreeThreads);  // [2][7][4]
  float2 *ancg = t.anc_g + (size_t)blockIdx.x * tree_global_anchors(t.nlev) * 16 * kTreeThreads;

  int item = blockIdx.x;
  const int tt = item % t.n_tt;
  item /= t.n_tt;
  const int mb = item % t.n_mb, s = item / t.n_mb;
  // a thread owns 16 cells of one row: classes q1 and half h of the 32-point DIF (tpr = 2 PM
  // threads per row), or with Lm = 16 the whole row (the h = 0 half, q = bitrev4(c)); threads
  // past the block's RB rows (Lm = 16 and Ls < 128) only take part in the barriers
  const bool half = t.half != 0;
  const int tpr = half ? 1 : 2 * PM;
  const int rr0 = tid / tpr, q1 = half ? 0 : (tid >> 1) & (PM - 1), h = half ? 0 : tid & 1;
  const bool row_ok = rr0 < RB;
  const int rr = row_ok ? rr0 : 0;
  const int m = mb * RB + rr;
  const int2 sd = t.series[s];
  const int kd = t.T - t.dk_max[sd.y];
  const int kb = tt * t.TT;
  if (kb >= kd) return;  // every segment starting here runs past the scan
  bool row_in = row_ok;
  if (!kFull) {
    row_in = row_ok && ((m - t.m_lo) & (t.Ls - 1)) < t.m_len;
    if (!__syncthreads_or(row_in)) return;  // no SBD row of this block is searched
  }
  const int lmax = 1 << t.nlev;
  const int ke = min(kd, kb + t.TT + lmax - 1);

  for (int i = tid; i < NS * PM * 2; i += kTreeThreads) tw[i] = t.tw[i];
  for (int i = tid; i < n_sm * 16 * kTreeThreads; i += kTreeThreads) anc[i] = make_float2(0.f, 0.f);
  for (int i = tid; i < tree_global_anchors(t.nlev) * 16 * kTreeThreads; i += kTreeThreads)
    ancg[i] = make_float2(0.f, 0.f);
  // cells this thread may report: c -> q2 = 2 bitrev4(c) + h, q = q1 + PM q2
  unsigned cmask = row_ok ? 0xffffu : 0u;
  if (!kFull) {
    cmask = 0u;
    if (row_in) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int q2 = 2 * (bitrev5(c) >> 1) + h;
        const int q = half ? q2 >> 1 : q1 + PM * q2;
        if (((q - t.q_lo) & (Lm - 1)) < t.q_len) cmask |= 1u << c;
      }
    }
  }
  const int rbn = RB * NS, rbg = RB * t.N;  // the block's rows of one AP: slots / channels
  const float2 *Ysrc = t.Y + (size_t)s * t.y_series + (size_t)mb * rbg;
  const size_t ystep = (size_t)t.Ls * t.N;
  // element i of a row block (row i / N, channel i % N) goes to slot (i / N) NS + slot_of(i % N);
  // a thread moves elements tid + 128 u, the first one prefetched a step ahead
  auto slot_at = [&](int i) { return (i / t.N) * NS + __ldg(t.slot_of + i % t.N); };
  const int dst0 = tid < rbg ? slot_at(tid) : -1;
  for (int i = tid; i < 2 * rbn; i += kTreeThreads) yb[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = tid; i < rbg; i += kTreeThreads) yb[slot_at(i)] = __ldg(Ysrc + (size_t)kb * ystep + i);
  unsigned long long *keys = t.keys + ((size_t)sd.x * t.n_dm + sd.y) * t.S_tot;
  __syncthreads();

  // twiddles of slot pairs: float4 (slot 2p, slot 2p + 1) at [p][q1][h]
  const float4 *tw4 = reinterpret_cast<const float4 *>(tw) + q1 * 2 + h;
  const int twn = PM * 2;

  const unsigned kmask = 0xfffffff0u;
  // One AP: cur receives the one-AP matrix G_1(k) of the thread's cells; prev holds G_1(k - 1)
  // (the level-1 anchor).  Callers alternate the two arrays, so no anchor copy is needed.
  auto ap = [&](const int k, const float2(&prev)[16], float2(&cur)[16]) {
    const int buf = (k - kb) & 1;
    // next AP's rows: the first element per thread into a register while this one is transformed
    const bool more = k + 1 < ke;
    float2 nxt = make_float2(0.f, 0.f);
    if (more && dst0 >= 0) nxt = __ldg(Ysrc + (size_t)(k + 1) * ystep + tid);
    // MBD: the channels of slot (r, o) = r + 16 o fold into input r of half h of the 32-point
    // DIF FFT (empty slots hold zeros), then a 16-point FFT
    const float4 *yr4 = reinterpret_cast<const float4 *>(yb + buf * rbn + rr * NS);
#pragma unroll
    for (int r = 0; r < 16; ++r) cur[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 0; o < S16; ++o) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {  // slots 16 o + 2 j and 16 o + 2 j + 1, with their twiddles
        const float4 y = yr4[8 * o + j], w = tw4[(8 * o + j) * twn];
        cur[2 * j] = cfma(cur[2 * j], make_float2(y.x, y.y), make_float2(w.x, w.y));
        cur[2 * j + 1] = cfma(cur[2 * j + 1], make_float2(y.z, y.w), make_float2(w.z, w.w));
      }
    }
    fft16_dif(cur);
    // window tree: level e holds the segment of 2^e APs ending at AP k
    const int ctz = __ffs(k + 1) - 1;
    const int E = t.nlev == 0 ? 0 : min(t.nlev, ctz + 1);
    float2 acc[16];
#pragma unroll
    for (int e = 0; e <= kTreeMaxLev; ++e) {
      if (e > E) break;
      if (e == 0) {
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = cur[c];
      } else if (e == 1) {
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = make_float2(prev[c].x + cur[c].x, prev[c].y + cur[c].y);
      } else {
        // anchors of levels 1..3 in shared memory, deeper ones in the CTA's device slice
        float2 *an = e - 2 < kTreeSmemAnc ? anc + (e - 2) * 16 * kTreeThreads + tid
                                          : ancg + (e - 2 - kTreeSmemAnc) * 16 * kTreeThreads + tid;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float2 g = acc[c], p = an[c * kTreeThreads];
          acc[c] = make_float2(p.x + g.x, p.y + g.y);
          an[c * kTreeThreads] = g;
        }
      }
      const int w = t.emit_w[e];
      const int k0 = k - (1 << e) + 1;
      if (w >= 0 && k0 >= kb && k0 < kb + t.TT) {  // uniform across the CTA
        unsigned kk[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const unsigned kc = cell_key<kFull>(acc[c], bitrev5(c) >> 1, h, kmask);
          kk[c] = kFull || (cmask >> c) & 1u ? kc : 0u;
        }
#pragma unroll
        for (int wdt = 8; wdt >= 1; wdt >>= 1) {  // pairwise, so the maximum is 4 deep, not 16
#pragma unroll
          for (int c = 0; c < wdt; ++c) kk[c] = max(kk[c], kk[c + wdt]);
        }
        const unsigned key = kFull && !row_ok ? 0u : kk[0];
        const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
        const unsigned win = __ballot_sync(0xffffffffu, key == wmax);
        if (lane == 0) {
          uint2 r2 = make_uint2(0u, 0xffffffffu);
          if (wmax != 0u) {
            const int L = __ffs(win) - 1, tl = warp * 32 + L;
            const int q2 = kFull ? 2 * (15 - (int)(wmax & 15u)) + (half ? 0 : tl & 1) : 32 - (int)(wmax & 63u);
            const int mm = mb * RB + tl / tpr, qq1 = (tl >> 1) & (PM - 1);
            r2 = make_uint2(wmax & (kFull ? ~15u : ~63u), (unsigned)(mm * Lm + (half ? q2 >> 1 : qq1 + PM * q2)));
          }
          red[(buf * (kTreeMaxLev + 1) + e) * 4 + warp] = r2;
        }
      }
    }
    if (more) {
      float2 *yn = yb + (buf ^ 1) * rbn;
      if (dst0 >= 0) yn[dst0] = nxt;
      for (int i = tid + kTreeThreads; i < rbg; i += kTreeThreads) yn[slot_at(i)] = __ldg(Ysrc + (size_t)(k + 1) * ystep + i);
    }
    __syncthreads();
    // merge the block's maxima of the segments emitted at AP k into the series
    if (tid <= E) {
      const int e = tid, w = t.emit_w[e], k0 = k - (1 << e) + 1;
      if (w >= 0 && k0 >= kb && k0 < kb + t.TT) {
        uint2 best = make_uint2(0u, 0xffffffffu);
        for (int v = 0; v < kTreeThreads / 32; ++v) {
          const uint2 r2 = red[(buf * (kTreeMaxLev + 1) + e) * 4 + v];
          if (r2.x > best.x || (r2.x == best.x && r2.y < best.y)) best = r2;
        }
        if (best.x != 0u) {
          // windows of 2^e APs start every 2^(e-1) APs (every AP for e = 0); k0 >= 0
          const unsigned long long kv = ((unsigned long long)best.x << 32) | (unsigned long long)(~best.y);
          atomicMax(keys + t.win_off[w] + (k0 >> (e > 0 ? e - 1 : 0)), kv);
        }
      }
    }
  };

  float2 ga[16], gb[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) ga[c] = make_float2(0.f, 0.f);
  int k = kb;
  for (; k + 1 < ke; k += 2) {
    ap(k, ga, gb);
    ap(k + 1, gb, ga);
  }
  if (k < ke) ap(k, ga, gb);
}

// ----------------------------------------------------------------------------- finalize
// Series element -> frbx_seg: valid slots decode the merged key, the others are empty (-1).
__global__ void k_tree_finalize(frbx_seg *series, long long n_el, int S_tot, int n_dm, int n_win,
                                const int *win_len, const int *win_off, const int *n_valid, int log2Lm, int Lm) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_el) return;
  const int slot = (int)(i % S_tot);
  const int d = (int)((i / S_tot) % n_dm);
  int w = 0;
  while (w + 1 < n_win && slot >= win_off[w + 1]) ++w;
  const bool valid = slot - win_off[w] < n_valid[d * n_win + w];
  unsigned long long *kp = reinterpret_cast<unsigned long long *>(series + i);
  const unsigned long long key = *kp;
  frbx_seg r;
  if (valid && key != 0ull) {
    const unsigned idx = ~(unsigned)(key & 0xffffffffull);
    r.amp = sqrtf(__uint_as_float((unsigned)(key >> 32)));
    r.sbd_idx = (uint16_t)(idx >> log2Lm);
    r.mbd_idx = (uint16_t)(idx & (unsigned)(Lm - 1));
  } else {
    r.amp = -1.f;
    r.sbd_idx = 0;
    r.mbd_idx = 0;
  }
  series[i] = r;
}

// ----------------------------------------------------------------------------- host side
void set_tree_constants() { upload_w32(); }

bool tree_supported(int Ls, int Lm, int N, int J, int s16, const int *windows, int n_win, int *nlev) {
  if (Ls % 32 != 0 || (Lm % 32 != 0 && Lm != 16) || J > Ls || s16 < 1 || s16 > 4) return false;
  const int PM = std::max(1, Lm / 32), NS = 16 * s16;
  if (2 * PM > kTreeThreads || N > NS) return false;
  const int RB = tree_rows_per_block(Ls, Lm);
  if (Ls % RB != 0) return false;
  int lmax = 1;
  for (int w = 0; w < n_win; ++w) {
    const int l = windows[w];
    if (l < 1 || (l & (l - 1)) != 0 || l > (1 << kTreeMaxLev)) return false;
    lmax = std::max(lmax, l);
  }
  *nlev = __builtin_ctz((unsigned)lmax);
  // the SBD pass holds one AP of output (Ls N complex, the same bytes as the split tiles of the
  // tensor-core form), the gathered points and its twiddles
  const int JP = (J + 31) / 32 * 32;
  const size_t sbd = sizeof(float2) * ((size_t)Ls * N + (size_t)N * (JP + 1) + (size_t)(Ls / 32) * (JP + 1));
  return tree_smem_bytes(NS, PM, RB, *nlev) <= max_smem_optin() && sbd <= max_smem_optin();
}

int tree_rows_per_block(int Ls, int Lm) { return Lm == 16 ? std::min(kTreeThreads, Ls) : kTreeThreads / (2 * (Lm / 32)); }

size_t tree_anchor_floats(int nlev) { return (size_t)tree_global_anchors(nlev) * 16 * kTreeThreads; }

size_t tree_sbd_smem(const FitArgs &a, const TreeArgs &t) {
  const int JP = a.J1 * 32;
  const size_t stage = t.mma ? (size_t)t.tile_bytes : sizeof(float2) * (size_t)a.Ls * a.N;
  return stage + sizeof(float2) * ((size_t)a.N * (JP + 1) + (size_t)(a.Ls / 32) * (JP + 1));
}

cudaError_t launch_tree_sbd(const FitArgs &a, const TreeArgs &t, cudaStream_t st, int64_t *launches) {
  const size_t smem = tree_sbd_smem(a, t);
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  const long long nb = (long long)t.n_s * t.n_ktile;
  if (nb <= 0) return cudaSuccess;
  if (!t.mma && t.rot != 0) return cudaErrorInvalidValue;
  if (t.mma && (t.pack < 1 || t.piece_bytes * t.pack != t.tile_bytes || t.prow * t.pack != tc::kRows))
    return cudaErrorInvalidValue;
  auto kern = !t.mma ? k_tree_sbd<0> : t.form == 0 ? k_tree_sbd<1> : t.form == 1 ? k_tree_sbd<2> : k_tree_sbd<3>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)nb, kTreeThreads, smem, st>>>(a, t);
  ++*launches;
  return cudaGetLastError();
}

template <int S16, bool kFull>
static cudaError_t launch_mbd_one(const TreeArgs &t, unsigned nb, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tree_mbd<S16, kFull>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tree_mbd<S16, kFull><<<nb, kTreeThreads, smem, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_tree_mbd(const TreeArgs &t, bool full, cudaStream_t st, int64_t *launches) {
  const size_t smem = tree_smem_bytes(t.NS, t.PM, t.RB, t.nlev);
  if (smem > max_smem_optin()) return cudaErrorInvalidConfiguration;
  const long long nb = (long long)t.n_s * t.n_mb * t.n_tt;
  if (nb <= 0) return cudaSuccess;
  if (nb > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const unsigned g = (unsigned)nb;
  cudaError_t e;
  switch (t.NS / 16) {
    case 1: e = full ? launch_mbd_one<1, true>(t, g, smem, st) : launch_mbd_one<1, false>(t, g, smem, st); break;
    case 2: e = full ? launch_mbd_one<2, true>(t, g, smem, st) : launch_mbd_one<2, false>(t, g, smem, st); break;
    case 3: e = full ? launch_mbd_one<3, true>(t, g, smem, st) : launch_mbd_one<3, false>(t, g, smem, st); break;
    case 4: e = full ? launch_mbd_one<4, true>(t, g, smem, st) : launch_mbd_one<4, false>(t, g, smem, st); break;
    default: return cudaErrorInvalidConfiguration;
  }
  ++*launches;
  return e;
}

cudaError_t launch_tree_finalize(frbx_seg *series, long long n_el, int S_tot, int n_dm, int n_win, const int *win_len,
                                 const int *win_off, const int *n_valid, int log2Lm, int Lm, cudaStream_t st,
                                 int64_t *launches) {
  if (n_el <= 0) return cudaSuccess;
  k_tree_finalize<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(series, n_el, S_tot, n_dm, n_win, win_len, win_off,
                                                                   n_valid, log2Lm, Lm);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace frbx
