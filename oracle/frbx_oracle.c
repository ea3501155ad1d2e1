/*
 * frbx_oracle.c -- plain, slow, FP64 reference of the per-segment fringe fit.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the library never does.  It shares no source with the
 * CUDA path.
 *
 * What it computes, for each requested time segment (bl, dm index d, window l,
 * start AP k0):
 *
 *   Eq. 3   X(n,j) = c(n,j) * sum_{k = k0 + dk(d,n,j)}^{k0 + dk(d,n,j) + l - 1} S(n,j,k)
 *           (c = calibration rotation exp(-i[2 pi (f_j - f_bw/2) dtau0_n + dphi0_n]),
 *            the last two terms of Eq. 5's phase)
 *   Eq. 5   G(m,q) = sum_{n=0}^{N-1} sum_{j=1}^{J-1} X(n,j) exp(-i 2 pi [f_j SBD_m + (f0_n - f0_ref) MBD_q])
 *           on the grid of Sec. 5.1: f_j SBD_m = j m / Ls and (f0_n - f0_ref) MBD_q = g_n q / Lm,
 *           so the phase is 2 pi [ (j m mod Ls)/Ls + (g_n q mod Lm)/Lm ].
 *           The exponential of the sum is the product of the two exponentials; the sum
 *           over j is taken first for every (n, m) and the sum over n second (the
 *           row-column form of the 2-D DFT named in Sec. 5.1).  Points with j = 0 are
 *           outside the sum (Sec. 2.3), flagged points likewise.
 *   Sec 5.1 A = max over the grid of |G|, its (m, q) (first in m-major, then q order,
 *           strict '>' so the lowest linear index wins exact ties), and the
 *           runner-up value A2 (largest |G| over all other cells) for the tie rule.
 *
 * Cells outside the optional delay windows (allow_m / allow_q == 0) are skipped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double re, im;
} cplx;

static void fit_one(const float *vis_bl, int T, int N, int J, const int32_t *dk_d, int k0, int l,
                    const uint8_t *flag, const double *rot_re, const double *rot_im,
                    const int32_t *g, int Ls, int Lm, const double *cs, const double *ss,
                    const double *cm, const double *sm, const uint8_t *allow_m,
                    const uint8_t *allow_q, cplx *X, cplx *Y, double *grid, double *out_amp,
                    int32_t *out_m, int32_t *out_q, double *out_amp2) {
  const int C = N * J;
  (void)T;
  /* Eq. 3: time segment, summed in increasing k. */
  for (int c = 0; c < C; ++c) {
    double sr = 0.0, si = 0.0;
    const int kstart = k0 + dk_d[c];
    for (int i = 0; i < l; ++i) {
      const float *p = vis_bl + 2 * ((size_t)(kstart + i) * C + c);
      sr += (double)p[0];
      si += (double)p[1];
    }
    /* calibration rotation (Eq. 5, last two phase terms) */
    X[c].re = sr * rot_re[c] - si * rot_im[c];
    X[c].im = sr * rot_im[c] + si * rot_re[c];
  }
  /* Eq. 5, sum over j (j = 1 .. J-1, unflagged) for every (n, m). */
  for (int n = 0; n < N; ++n) {
    for (int m = 0; m < Ls; ++m) {
      double yr = 0.0, yi = 0.0;
      for (int j = 1; j < J; ++j) {
        const int c = n * J + j;
        if (flag && flag[c]) continue;
        const int k = (int)(((int64_t)j * m) % Ls);
        /* X * exp(-i 2 pi k / Ls) */
        yr += X[c].re * cs[k] + X[c].im * ss[k];
        yi += X[c].im * cs[k] - X[c].re * ss[k];
      }
      Y[n * Ls + m].re = yr;
      Y[n * Ls + m].im = yi;
    }
  }
  /* Eq. 5, sum over n for every (m, q); amplitude and maximum. */
  double best = -1.0, second = -1.0;
  int bm = -1, bq = -1;
  for (int m = 0; m < Ls; ++m) {
    for (int q = 0; q < Lm; ++q) {
      double gr = 0.0, gi = 0.0;
      for (int n = 0; n < N; ++n) {
        const int k = (int)(((int64_t)g[n] * q) % Lm);
        const cplx y = Y[n * Ls + m];
        gr += y.re * cm[k] + y.im * sm[k];
        gi += y.im * cm[k] - y.re * sm[k];
      }
      const double a = sqrt(gr * gr + gi * gi);
      if (grid) {
        grid[2 * ((size_t)m * Lm + q)] = gr;
        grid[2 * ((size_t)m * Lm + q) + 1] = gi;
      }
      if ((allow_m && !allow_m[m]) || (allow_q && !allow_q[q])) continue;
      if (a > best) {
        second = best;
        best = a;
        bm = m;
        bq = q;
      } else if (a > second) {
        second = a;
      }
    }
  }
  *out_amp = best;
  *out_m = bm;
  *out_q = bq;
  *out_amp2 = second;
}

static void make_tables(int L, double *c, double *s) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int k = 0; k < L; ++k) {
    c[k] = cos(two_pi * (double)k / (double)L);
    s[k] = sin(two_pi * (double)k / (double)L);
  }
}

/*
 * Fit a list of segments.  seg[4*i + {0,1,2,3}] = (bl, d, l, k0).
 * vis: complex64 cube [n_bl][T][N*J] as interleaved floats.
 * dk: int32 [n_dm][N*J] AP offsets (Eq. 2).
 * grid_out (optional): if non-NULL, complex G of every cell for every listed segment,
 *   [n_seg][Ls][Lm] as (re, im) pairs.
 * Returns 0, or -1 if a segment would read outside the cube.
 */
int oracle_fit_list(const float *vis, int n_bl, int T, int N, int J, const int32_t *dk, int n_dm,
                    const uint8_t *flag, const double *rot_re, const double *rot_im,
                    const int32_t *g, int Ls, int Lm, const uint8_t *allow_m,
                    const uint8_t *allow_q, const int32_t *seg, int64_t n_seg, double *amp,
                    int32_t *m_idx, int32_t *q_idx, double *amp2, double *grid_out,
                    int n_threads) {
  const int C = N * J;
  double *cs = malloc(sizeof(double) * Ls), *ss = malloc(sizeof(double) * Ls);
  double *cm = malloc(sizeof(double) * Lm), *sm = malloc(sizeof(double) * Lm);
  make_tables(Ls, cs, ss);
  make_tables(Lm, cm, sm);
  int bad = 0;
  /* bounds check first, so no thread ever reads outside the cube */
  for (int64_t i = 0; i < n_seg; ++i) {
    const int32_t *s = seg + 4 * i;
    if (s[0] < 0 || s[0] >= n_bl || s[1] < 0 || s[1] >= n_dm || s[2] < 1 || s[3] < 0) {
      bad = 1;
      break;
    }
    for (int c = 0; c < C; ++c) {
      const int64_t lo = (int64_t)s[3] + dk[(size_t)s[1] * C + c];
      if (lo < 0 || lo + s[2] > T) {
        bad = 1;
        break;
      }
    }
    if (bad) break;
  }
  if (!bad) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
      cplx *X = malloc(sizeof(cplx) * C);
      cplx *Y = malloc(sizeof(cplx) * (size_t)N * Ls);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
      for (int64_t i = 0; i < n_seg; ++i) {
        const int32_t *s = seg + 4 * i;
        const float *vis_bl = vis + 2 * (size_t)s[0] * T * C;
        fit_one(vis_bl, T, N, J, dk + (size_t)s[1] * C, s[3], s[2], flag, rot_re, rot_im, g, Ls,
                Lm, cs, ss, cm, sm, allow_m, allow_q, X, Y,
                grid_out ? grid_out + 2 * (size_t)i * Ls * Lm : NULL, amp + i, m_idx + i, q_idx + i,
                amp2 + i);
      }
      free(X);
      free(Y);
    }
  }
  free(cs);
  free(ss);
  free(cm);
  free(sm);
  return bad ? -1 : 0;
}

/*
 * Literal triple sum of Eq. 5 for one already-built segment X [N*J] (no factoring,
 * phase from the exact integer index): G(m,q) = sum_n sum_{j>=1} X exp(-2 pi i [jm/Ls + g_n q/Lm]).
 * Used only by pins on tiny inputs to check the factored form above.
 */
void oracle_triple_sum(const double *x_re, const double *x_im, int N, int J, const uint8_t *flag,
                       const int32_t *g, int Ls, int Lm, double *g_re, double *g_im) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int m = 0; m < Ls; ++m)
    for (int q = 0; q < Lm; ++q) {
      double ar = 0.0, ai = 0.0;
      for (int n = 0; n < N; ++n)
        for (int j = 1; j < J; ++j) {
          const int c = n * J + j;
          if (flag && flag[c]) continue;
          const double ph = two_pi * ((double)j * m / Ls + (double)g[n] * q / Lm);
          ar += x_re[c] * cos(ph) + x_im[c] * sin(ph);
          ai += x_im[c] * cos(ph) - x_re[c] * sin(ph);
        }
      g_re[(size_t)m * Lm + q] = ar;
      g_im[(size_t)m * Lm + q] = ai;
    }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
