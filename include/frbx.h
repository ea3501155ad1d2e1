/*
 * frbx.h -- C ABI of the GB300 cross-spectrum FRB search library (libfrbx).
 *
 * Method: Liu, Tong, Zheng, Zhang & Tong, "A Fast Radio Burst Search Method for
 * VLBI Observation" (arxiv 1801.02391).  Cross spectra go in; the DM grid,
 * window set, delay search windows and baseline combinations are parameters;
 * per-baseline single pulses, cross-match groups and combined-baseline pulses
 * come out (the problem statement of Sec. 2).
 *
 * Conventions (all entry points):
 *  - Plain C types only.  Every pointer is a host pointer unless the argument
 *    name ends in "_dev" or a flag says otherwise; device pointers are CUDA
 *    global-memory addresses on the handle's device.
 *  - Return value: FRBX_OK (0) or a negative FRBX_E* code.  No C++ exception
 *    crosses the ABI.  frbx_last_error() gives a message for the last failure
 *    on a handle.
 *  - A handle is not thread-safe; use one handle per host thread.  All device
 *    work of a call is issued on the caller's stream (cudaStream_t passed as
 *    void*, NULL = legacy default stream) and the call returns after that
 *    stream's work for the call has finished.
 *  - The library never frees caller memory.  It owns its own device scratch
 *    (shift table, segment series, event lists) inside the handle and grows
 *    it on demand; frbx_destroy() releases it.
 */
#ifndef FRBX_H
#define FRBX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FRBX_OK 0
#define FRBX_EINVAL (-1)      /* bad argument (message says which) */
#define FRBX_ENOMEM (-2)      /* device or host allocation failed */
#define FRBX_ECUDA (-3)       /* a CUDA runtime call failed */
#define FRBX_ETRUNC (-4)      /* an output array was too small; *_count holds the size needed */
#define FRBX_ETIMEOUT (-5)    /* a bounded device wait gave up */
#define FRBX_EUNSUPPORTED (-6) /* shape outside what the kernels support (message says why) */

typedef struct frbx_handle frbx_handle;

/*
 * Observing setup (Sec. 2.2, Sec. 2.3, Eq. 5).
 *  n_chan        N sky-frequency channels (subbands), 1..64.
 *  n_point       J frequency points per channel, 2..256.  Point j of channel n
 *                sits at f(n,j) = f0_mhz[n] + (j * f_bw_mhz) / J  (USB).
 *  f0_mhz        [n_chan] channel edge frequencies, MHz.  Offsets between channels
 *                must be whole kHz; the MBD grid step df_grid is their GCD.
 *  f_bw_mhz      channel bandwidth, MHz.
 *  t_ap_ms       AP (accumulation period) length, ms.
 *  f_ref_dm_mhz  reference frequency of Eq. 1; 0 = the highest point frequency.
 *  chan_delay_ns optional [n_chan] channel delays dtau0_n (Eq. 5); NULL = 0.
 *  chan_phase_rad optional [n_chan] initial phases dphi0_n (Eq. 5); NULL = 0.
 *  flag          optional [n_chan*n_point], nonzero = point excluded from the fit
 *                (j = 0 is always excluded, Sec. 2.3); NULL = none.
 *  sbd_pad       SBD grid Ls = sbd_pad * J (zero padding of App. B); 0 = 2.
 *  mbd_pad       MBD grid Lm = mbd_pad * nextpow2(max g_n + 1); 0 = 2.
 *                Ls and Lm must be powers of two, Ls <= 1024, Lm <= 4096,
 *                Ls * Lm <= 2^20.
 * The arrays are copied; the caller may free them after frbx_create returns.
 */
typedef struct frbx_setup {
  int32_t n_chan;
  int32_t n_point;
  const double *f0_mhz;
  double f_bw_mhz;
  double t_ap_ms;
  double f_ref_dm_mhz;
  const double *chan_delay_ns;
  const double *chan_phase_rad;
  const uint8_t *flag;
  int32_t sbd_pad;
  int32_t mbd_pad;
} frbx_setup;

/*
 * Search parameters (Sec. 2.4).
 *  threshold     normalised-power threshold, P > threshold (Sec. 2.4.1: 3).
 *  nwin_min      N_win,min of step d (Sec. 3.4.1: 3).
 *  sbd_win_ns    SBD search window [lo, hi] in ns; lo > hi means the whole grid.
 *  mbd_win_ns    MBD search window [lo, hi] in ns; lo > hi means the whole grid.
 *                A cell is searched when lo <= delay <= hi, with
 *                SBD(m) = ((s(m) * J) * 1000) / (Ls * f_bw) and
 *                MBD(q) = (s(q) * 1000) / (Lm * df_grid), s(i) = i if i < L/2 else i - L.
 *  combos        [n_combo] baseline bit masks for the power-summation scheme
 *                (Sec. 2.4.2); bit b = baseline b.  May be NULL when n_combo = 0.
 *  kernel        how Eq. 5 is evaluated on the Sec. 5.1 grid (all give the same results
 *                within FP32 rounding unless stated):
 *                0 = choose automatically: 6 where it applies, else 4, else 2, else 1;
 *                1 = direct DFT per segment;
 *                2 = per-segment four-step FFT (Ls and Lm multiples of 32);
 *                3 = per-segment BF16 tensor-core DFT-GEMM (about 4e-3 relative error;
 *                    Ls 64 or 128, whole grid);
 *                4 = window tree: power-of-two windows built from one-AP matrices by the
 *                    additivity of Sec. 5.1, FP32 on the CUDA cores (windows <= 64 APs;
 *                    Ls a multiple of 32, Lm 16 or a multiple of 32);
 *                5 = as 3 with FP8 E4M3 operands (about 6e-2 relative error);
 *                6 = window tree with the MBD transform as a three-term split-BF16
 *                    tensor-core GEMM, FP32 accumulation (about 1e-5 relative; Ls 128,
 *                    n_chan <= 64, Lm a multiple of 32; delay windows allowed);
 *                7 = as 6 with one BF16 product per AP (about 3e-3 relative);
 *                8 = as 6 with E4M3 operands, A scaled per AP by a power of two (about 4e-2
 *                    relative).
 *                frbx_fit_segments treats 4, 6, 7 and 8 as 0 (a list has no window structure).
 */
typedef struct frbx_params {
  float threshold;
  int32_t nwin_min;
  double sbd_win_ns[2];
  double mbd_win_ns[2];
  const uint64_t *combos;
  int32_t n_combo;
  int32_t kernel;
} frbx_params;

/* One fitted time segment (Sec. 5.1): max |G| over the searched grid and its cell. */
typedef struct frbx_seg {
  float amp;
  uint16_t sbd_idx; /* m */
  uint16_t mbd_idx; /* q */
} frbx_seg;

/* A threshold crossing, "candidate signal" of Sec. 2.4.1 step a. */
typedef struct frbx_event {
  int32_t series; /* baseline index, or combination index for combined series */
  int32_t dm_idx;
  int32_t win_idx; /* index into the caller's window list */
  int32_t k0;      /* start AP of the segment (at the DM reference frequency) */
  float amp;       /* |G| (combined series: summed amplitude) */
  float pnorm;     /* normalised power, Eq. 6 */
  uint16_t sbd_idx, mbd_idx; /* 0 for combined series */
} frbx_event;

/* A single pulse (Sec. 2.4.1 step d; Sec. 2.4.2 step d) after the DM merge of Sec. 5.3. */
typedef struct frbx_cand {
  int32_t series;  /* baseline index, or combination index */
  int32_t dm_idx;  /* DM trial of highest power */
  int32_t win_idx;
  int32_t width;   /* window length in APs (characteristic width) */
  int32_t k0;
  int32_t sbd_idx, mbd_idx;
  int32_t n_win;   /* distinct windows that saw it (step d) */
  int32_t group;   /* cross-match group, or -1 (combined pulses, pre-merge lists) */
  float amp;
  float pnorm;     /* characteristic power */
  int32_t reserved;
  double t_s;      /* k0 * t_ap, seconds from the first AP */
  double sbd_ns, mbd_ns;
  double dm;
} frbx_cand;

/* A cross-matching group (Sec. 2.4.1): pulses of different baselines overlapping in time. */
typedef struct frbx_group {
  uint64_t bl_mask;
  int32_t n_baselines;
  int32_t n_pulses;
} frbx_group;

/*
 * Outputs of frbx_search.  Each array is caller-owned with capacity *_cap
 * elements (0 = not wanted; the pointer may then be NULL).  Every *_count is
 * always set to the number of elements the full result has; if a count exceeds
 * its capacity the first *_cap elements are written and frbx_search returns
 * FRBX_ETRUNC after finishing everything else.
 *
 *  pulses      per-baseline single pulses after the DM merge, baseline ascending,
 *              then in order of discovery; .group indexes groups[].
 *  groups      cross-match groups in creation order.
 *  combined    pulses of the power-summation scheme, combination ascending.
 *  pulses_dm   optional: per-(baseline, DM) pulses before the DM merge.
 *  events      optional: all threshold crossings of baselines then combinations,
 *              ordered by (series, dm, window, k0).
 *  series      optional per-segment fits, frbx_seg[n_bl][n_dm][S_tot] (layout from
 *              frbx_series_layout; unused slots hold amp = -1).  Host or device
 *              memory per series_on_device.
 *  pnorm       optional normalised power, float[n_bl][n_dm][S_tot] (unused slots 0),
 *              same memory kind as series.
 */
typedef struct frbx_results {
  frbx_cand *pulses;
  int64_t pulses_cap, pulses_count;
  frbx_group *groups;
  int64_t groups_cap, groups_count;
  frbx_cand *combined;
  int64_t combined_cap, combined_count;
  frbx_cand *pulses_dm;
  int64_t pulses_dm_cap, pulses_dm_count;
  frbx_event *events;
  int64_t events_cap, events_count;
  frbx_seg *series;
  float *pnorm;
  int32_t series_on_device;
  int32_t reserved;
  int64_t series_cap, series_count;
  int64_t events_baseline_count; /* out: the first this-many events are the baselines' */
} frbx_results;

/* Fill *p with the paper's defaults (threshold 3, N_win,min 3, whole grids, no combos). */
void frbx_default_params(frbx_params *p);

/*
 * Create a handle for one setup on the current CUDA device.  Validates the
 * setup, builds the frequency, MBD-grid, rotation and twiddle tables (FP64 on
 * the host, rounded to FP32 once) and uploads them.
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA.  *out is NULL on error.
 */
int frbx_create(const frbx_setup *setup, frbx_handle **out);

/* Release the handle and its device memory.  NULL is ignored. */
void frbx_destroy(frbx_handle *h);

/* Message of the last failed call on h (never NULL; "" if none). */
const char *frbx_last_error(const frbx_handle *h);

/* Grid sizes chosen at create time: Ls, Lm, df_grid (MHz) and g_n ([n_chan], may be NULL). */
int frbx_grid_info(const frbx_handle *h, int32_t *Ls, int32_t *Lm, double *df_grid_mhz,
                   int32_t *g_out);

/*
 * Eq. 1-2: dk[d][c] = floor(0.5 + 4.15e6 * DM_d * (f_c^-2 - f_ref^-2) / t_ap), computed on
 * the device in FP64 in the order a = 4.15e6*DM; b = 1/(f*f) - 1/(fref*fref); dt = a*b;
 * x = dt/t_ap; floor(0.5 + x), each step correctly rounded (no contraction).
 *  dm       [n_dm] host, pc cm^-3, >= 0.
 *  dk_out   [n_dm][n_chan*n_point] int32, host.
 * Errors: FRBX_EINVAL, FRBX_ECUDA.
 */
int frbx_shift_table(frbx_handle *h, const double *dm, int32_t n_dm, int32_t *dk_out,
                     void *cuda_stream);

/*
 * Series layout for T APs and a window list: for window w, segment s starts at
 * k0 = s * step(l_w), step(l) = max(1, l/2) (half overlap, Sec. 2.4.1), and sits
 * at slot offset[w] + s of a (baseline, DM) series of S_tot slots.
 *  offset   [n_win] out (may be NULL); returns S_tot (or a negative error).
 */
int64_t frbx_series_layout(int32_t T, const int32_t *windows, int32_t n_win, int64_t *offset);

/*
 * The whole hot path (Sec. 2.2 - 2.4, Sec. 5.1, Sec. 5.3):
 *  1. dispersion shift table for the DM grid (Eq. 1-2);
 *  2. every valid half-overlapped segment of every window, baseline and DM:
 *     dedispersed sum (Eq. 3), calibration rotation, 2-D delay transform on the
 *     SBD x MBD grid (Eq. 5, Sec. 5.1) and its maximum;  a segment is valid when
 *     k0 + max_c dk(d, c) + l <= T;
 *  3. normalised power per (baseline, DM, window) over the valid segments (Eq. 6)
 *     and the threshold;
 *  4. steps b-d per (baseline, DM), the DM merge, cross-matching (Sec. 2.4.1);
 *  5. for each baseline combination, summed amplitudes, Eq. 6, threshold, steps b
 *     and d (no MBD step) and the DM merge (Sec. 2.4.2).
 *
 *  vis      complex64 cross spectra [n_bl][T][n_chan*n_point] (interleaved re, im
 *           floats, row-major, 8-byte aligned).  If vis_on_device is nonzero it
 *           is a device pointer, else a host pointer (copied to the device inside
 *           the call, one baseline after another on a library stream that follows
 *           cuda_stream, so the window-tree fit of the first baselines overlaps the
 *           copy of the rest; pinned memory is fastest; the buffer is no longer read
 *           once the call returns).
 *  n_bl     1..64 baselines;  T  APs (>= 1).
 *  dm       [n_dm] host, DM trials (pc cm^-3), >= 0.
 *  windows  [n_win] host, distinct window lengths in APs (>= 1), 1..16 of them.
 *  params   search parameters (NULL = defaults).
 *  res      outputs, see frbx_results.
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA, FRBX_ETRUNC, FRBX_EUNSUPPORTED.
 */
int frbx_search(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl, int32_t T,
                const double *dm, int32_t n_dm, const int32_t *windows, int32_t n_win,
                const frbx_params *params, frbx_results *res, void *cuda_stream);

/*
 * Stage entry point: fit an explicit list of segments (Eq. 3, Eq. 5, Sec. 5.1) with the
 * kernels frbx_search uses, e.g. to check sampled segments of a large run.
 *  vis, vis_on_device, n_bl, T, dm, n_dm   as in frbx_search.
 *  segs     host int32 [n_seg][4] rows (bl, dm_idx, l, k0); each must satisfy
 *           0 <= bl < n_bl, 0 <= dm_idx < n_dm, l >= 1, k0 >= 0 and
 *           k0 + max_c dk(dm_idx, c) + l <= T (checked; FRBX_EINVAL otherwise).
 *  out      host frbx_seg [n_seg].
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA, FRBX_EUNSUPPORTED.
 */
int frbx_fit_segments(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl,
                      int32_t T, const double *dm, int32_t n_dm, const int32_t *segs,
                      int64_t n_seg, const frbx_params *params, frbx_seg *out, void *cuda_stream);

/*
 * Host stage entry point (no GPU needed): single-pulse extraction from a list of
 * threshold crossings, i.e. steps b-d of Sec. 2.4.1 per (series, DM), the DM merge of
 * Sec. 5.3 per series and, if cross_match is nonzero, cross-matching of the series
 * as baselines (Sec. 2.4.1).  frbx_search runs exactly this code on its events.
 *  events     [n_events] ordered by (series, dm_idx, win_idx, k0) ascending (checked).
 *  n_series   number of series (baselines or combinations); series < n_series < 64.
 *  T, n_dm    scan length in APs and DM-trial count (event indices must be below them).
 *  windows    [n_win] distinct window lengths (the events' win_idx index them).
 *  Lm         MBD grid size for step c (angle 2 pi mbd_idx / Lm); 0 skips step c (the
 *             power-summation scheme, Sec. 2.4.2).
 *  nwin_min   N_win,min of step d.
 *  pulses     out, DM-merged pulses (cap / *count as in frbx_results); the double fields
 *             (t_s, sbd_ns, mbd_ns, dm) are left 0.
 *  groups     out, cross-match groups (ignored when cross_match is 0).
 *  pre_merge  out, per-(series, DM) pulses before the merge.
 * Errors: FRBX_EINVAL, FRBX_ETRUNC.
 */
int frbx_extract_events(const frbx_event *events, int64_t n_events, int32_t n_series, int32_t T,
                        int32_t n_dm, const int32_t *windows, int32_t n_win, int32_t Lm,
                        int32_t nwin_min, int32_t cross_match, frbx_cand *pulses,
                        int64_t pulses_cap, int64_t *pulses_count, frbx_group *groups,
                        int64_t groups_cap, int64_t *groups_count, frbx_cand *pre_merge,
                        int64_t pre_cap, int64_t *pre_count);

/*
 * Stage times of the last frbx_search on h, from CUDA events recorded on the call's
 * stream (device time between the events) and, for the host stage, the host clock:
 *  [0] shift table (Eq. 1-2)        [1] segment fit kernel (Eq. 3, Eq. 5, Sec. 5.1)
 *  [2] baselines: Eq. 6 + threshold  [3] combinations: sum + Eq. 6 + threshold
 *  [4] host extraction (Sec. 2.4.1 b-d, Sec. 5.3 merge, cross-matching, Sec. 2.4.2)
 *  [5] window-tree fit: device time of its SBD-pass kernels, summed over its chunks
 *  [6] window-tree fit: device time of its MBD-pass kernels (k_tree_mbd or k_tree_mma), summed
 *  [7] window-tree fit: number of chunks (= launches of each of the two kernels)
 *  [8] window-tree fit: 1 if its MBD pass ran on the tensor cores (k_tree_mma), else 0
 *  ms_out  [n] out, milliseconds (stages that did not run report 0).
 * Stages [5] and [6] are bracketed by events on the library's own streams (SBD passes on
 * one, MBD passes on the other); the SBD pass of a chunk overlaps the MBD pass of the
 * previous one, so [5] + [6] can exceed [1].
 * Returns the number of values written (min(n, 9)) or FRBX_EINVAL.
 */
int frbx_last_stage_times(const frbx_handle *h, double *ms_out, int32_t n);

/*
 * Allocation-free segment fit.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate device memory at the point of the call -- for example a
 * real-time back end that reserves all device memory at start-up, code running under a
 * framework's caching allocator that must not see foreign cudaMalloc calls, or code that
 * cannot afford the device-wide synchronisation cudaMalloc / cudaFree may imply.  It
 * computes what frbx_fit_segments computes with the direct-DFT kernel (kernel 1), but
 * needs no handle and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *  setup    observing setup as for frbx_create (read during the call only).
 *  vis_dev  device cube [n_bl][T][n_chan*n_point] complex64, 8-byte aligned.
 *  dm       host [n_dm] DM trials;  segs  host [n_seg][4] rows (bl, dm_idx, l, k0).
 *  out_dev  device frbx_seg [n_seg], 8-byte aligned.
 * Scratch: one fixed array of 16 MiB inside the library, in device memory of every GPU
 * that loads it, held until the process exits.  A call needs, rounded up to 256 bytes per
 * piece, about 4 n_dm n_chan n_point + 16 n_seg + 17 n_chan n_point + 8 (Ls + Lm) bytes;
 * a call that would need more returns FRBX_EINVAL without running anything.
 * Every call looks the array's device address up (cudaGetSymbolAddress) with the caller's
 * device current.  The first call on a device also makes the CUDA driver load the library's
 * device code there (lazy module loading, the default), and that load backs the 16 MiB array
 * with device memory: a caller that reserves device memory up front should make one call at
 * start-up (n_seg = 0 is enough) and should make it before any stream capture.  Later calls
 * allocate nothing.  Every call on a device shares the array and it keeps the last call's
 * contents (each call rewrites what it reads): calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Returns after the work on cuda_stream has finished.
 * Errors: FRBX_EINVAL (bad argument, a row reading outside the cube, scratch too small),
 * FRBX_EUNSUPPORTED, FRBX_ECUDA.
 */
int frbx_fit_segments_noalloc(const frbx_setup *setup, const void *vis_dev, int32_t n_bl, int32_t T,
                              const double *dm, int32_t n_dm, const int32_t *segs, int64_t n_seg,
                              frbx_seg *out_dev, void *cuda_stream);

/*
 * Candidate refinement below the grid spacing (Eq. 4 with its delay-rate term kept; the fine
 * DM search of Sec. 5.3).  For each candidate, the coherent power summed over baselines,
 *   P = sum_b |G_b|^2,  G_b = sum_{n, j>=1} c(n,j) sum_{i<l} X_b(n, j, u(n,j) + i) exp(-i Phi),
 *   u(n,j) = t0 + 4.15e6 DM (f^-2 - f_ref^-2) / t_ap   (continuous, no rounding),
 *   X_b(.., x) = cubic Catmull-Rom interpolation of the cube along time at x,
 *   Phi = 2 pi [(f_j tau_s + (f0_n - min f0) tau_m) 1e-3 + f0_n rho t_ap x 1e-6],
 * with the argument of Phi and u in FP64 and the rest in FP32.
 *  vis_dev    device cube [n_bl][T][n_chan*n_point] complex64.
 *  params_dev device double [n_cand][2 + 3 n_bl]: DM (pc cm^-3), t0 (APs, window start at the
 *             DM reference frequency), then per baseline tau_s (ns), tau_m (ns), rho (ns/s).
 *  width_dev  device int32 [n_cand] window lengths l (APs, >= 1).
 *  power_dev  device float [n_cand] out P;  g_dev device float [n_cand][n_bl][2] out G_b
 *             (keep it for frbx_refine_adjoint).
 *  status_dev device int32 [n_cand] out: 1 if some interpolation taps fell outside the cube
 *             (those samples count as zero), else 0.
 * Errors: FRBX_EINVAL, FRBX_ECUDA.
 */
int frbx_refine_power(frbx_handle *h, const void *vis_dev, int32_t n_bl, int32_t T, const double *params_dev,
                      const int32_t *width_dev, int32_t n_cand, float *power_dev, float *g_dev,
                      int32_t *status_dev, void *cuda_stream);

/*
 * Adjoint of frbx_refine_power: dparams[c][k] = dpower[c] * dP_c / dparams[c][k], from the G_b
 * that frbx_refine_power returned for the same parameters.
 *  dpower_dev  device float [n_cand] upstream gradient;  dparams_dev device float [n_cand][2 + 3 n_bl].
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA.
 */
int frbx_refine_adjoint(frbx_handle *h, const void *vis_dev, int32_t n_bl, int32_t T, const double *params_dev,
                        const int32_t *width_dev, int32_t n_cand, const float *g_dev, const float *dpower_dev,
                        float *dparams_dev, void *cuda_stream);

/*
 * Initial phases and channel delays from a calibrator scan (Appendix A): the segment of APs
 * [k0, k0 + l) at DM 0 is fringe-fitted on the grid (no calibration applied) for the common
 * SBD and MBD; per channel, the delay maximising the channel power after removing the common
 * SBD (grid of 8 J delays, parabolic start, Newton steps), then the residual phase.  The
 * outputs plug into frbx_setup.chan_delay_ns / chan_phase_rad (Eq. 5) of a new handle.
 *  vis, vis_on_device, n_bl, T  as in frbx_search.
 *  sbd_ns, mbd_ns      host [n_bl] out;  delay_ns, phase_rad  host [n_bl][n_chan] out.
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA, FRBX_EUNSUPPORTED.
 */
int frbx_calibrate(frbx_handle *h, const void *vis, int32_t vis_on_device, int32_t n_bl, int32_t T, int32_t k0,
                   int32_t l, double *sbd_ns, double *mbd_ns, double *delay_ns, double *phase_rad,
                   void *cuda_stream);

/*
 * Batched search: many scans, of uneven length and on several observing setups, in one pass.
 * Every scan gets exactly what frbx_search would give it (same kernels, same arithmetic).
 * The device work of the fit -- the dominant stage -- is one persistent launch per setup (and
 * per distinct window layout), whose CTAs claim (scan, baseline, time tile, DM trial) work
 * items from a device counter, so uneven scans load-balance; these launches are captured once
 * into a CUDA graph and replayed while the scans' shapes and buffers stay the same; setups
 * that take the window-tree fit add its two passes per chunk of series to the graph.  The time
 * tile of each setup is chosen by timing candidates on a sample the first time a setup shape
 * is seen by the batch object: 32, 64, 128 APs for the per-segment fit (a stretch of its work
 * items), 512, 1024, 2048 APs for the window tree (one chunk of the setup's longest scan).
 * The window tree's results do not depend on its tile.
 * Normalisation, threshold and extraction then run per scan as in frbx_search.
 */
typedef struct frbx_batch frbx_batch;

typedef struct frbx_scan {
  frbx_handle *setup;    /* handle of the scan's setup; scans may share one */
  const void *vis_dev;   /* device cube [n_bl][T][n_chan*n_point] complex64, 8-byte aligned */
  int32_t n_bl;
  int32_t T;
} frbx_scan;

typedef struct frbx_batch_stats {
  int32_t graph_captures;  /* times the fit graph was (re)captured by this batch object */
  int32_t graph_replays;   /* times it was replayed without capture */
  int32_t n_setups;        /* distinct setups in the last call */
  int32_t time_tile[16];   /* chosen time tile (APs) per setup, in order of first appearance */
  int32_t reserved;
  double fit_ms;           /* device time of the last graph launch (all fits) */
  int64_t launches;        /* kernel launches of the last call (graph kernels counted once) */
} frbx_batch_stats;

int frbx_batch_create(frbx_batch **out);
void frbx_batch_destroy(frbx_batch *b);
const char *frbx_batch_last_error(const frbx_batch *b);
int frbx_batch_info(const frbx_batch *b, frbx_batch_stats *stats);

/*
 *  scans     [n_scans] (1..4096; at most 16 distinct setups).
 *  dm, n_dm, windows, n_win, params  as in frbx_search, shared by all scans (kernel 0, 1, 2,
 *            4 or 6; combination masks must name baselines each scan has).
 *  results   [n_scans] outputs, one frbx_results per scan (series outputs included).
 * Errors: FRBX_EINVAL, FRBX_ENOMEM, FRBX_ECUDA, FRBX_ETRUNC, FRBX_EUNSUPPORTED.
 */
int frbx_search_batch(frbx_batch *b, const frbx_scan *scans, int32_t n_scans, const double *dm, int32_t n_dm,
                      const int32_t *windows, int32_t n_win, const frbx_params *params, frbx_results *results,
                      void *cuda_stream);

/* Number of kernel launches issued by the last frbx_search / frbx_fit_segments call. */
int64_t frbx_last_launch_count(const frbx_handle *h);

/*
 * Per-handle resource and robustness limits.  The paper has no counterpart; these control how
 * the library runs the method, never what it computes.  Zero in a field means its default.
 *  tree_chunk_bytes   window-tree fits (kernels 4, 6, 7, 8; frbx_search): device bytes of one of the
 *                     two scratch sets that the chunked SBD / MBD passes alternate between.
 *                     Default: a quarter of the free device memory, at most 16 GiB.  A small value
 *                     gives more chunks and the same results.
 *  wait_cycles        limit, in SM clock cycles, of every pipeline wait inside the tensor-core
 *                     kernels (kernels 3, 5, 6, 7 and 8).  Default 2e9.  When a wait runs out the call
 *                     returns FRBX_ETIMEOUT.  The waits that drain copies and MMAs still in
 *                     flight before a CTA exits keep the 2e9 limit, so no CTA leaves work behind.
 *  scratch_cap_bytes  cap on the device scratch the handle holds (the buffers it grows on demand;
 *                     the constant tables of frbx_create are not counted).  Default: no cap.  A
 *                     call that would grow the scratch past the cap returns FRBX_ENOMEM.
 *  hold_producers     test aid, 0 = off.  The producer roles of the tensor-core kernels issue
 *                     nothing, so the consumers' bounded waits run out: the call returns
 *                     FRBX_ETIMEOUT without any fault, nothing is left in flight and the handle
 *                     stays usable.  It exists so that tests can exercise the timeout path.
 * A call that fails returns only after the work it queued has finished.
 * frbx_set_limits(h, NULL) restores the defaults.  Errors: FRBX_EINVAL (negative field).
 */
typedef struct frbx_limits {
  int64_t tree_chunk_bytes;
  int64_t wait_cycles;
  int64_t scratch_cap_bytes;
  int32_t hold_producers;
  int32_t reserved;
} frbx_limits;

int frbx_set_limits(frbx_handle *h, const frbx_limits *lim);
int frbx_get_limits(const frbx_handle *h, frbx_limits *lim);

/* Bytes of device scratch the handle holds now (see frbx_limits.scratch_cap_bytes). */
int64_t frbx_scratch_bytes(const frbx_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* FRBX_H */
