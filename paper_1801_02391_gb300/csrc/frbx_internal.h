// Internal declarations shared by the translation units of libfrbx.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/frbx.h"

namespace frbx {

// Largest supported shapes (see frbx_setup in frbx.h).
constexpr int kMaxChan = 64;
constexpr int kMaxPoint = 256;
constexpr int kMaxLs = 1024;
constexpr int kMaxLm = 4096;
constexpr int kMaxWin = 16;
constexpr int kMaxBl = 64;
constexpr int kFitThreads = 256;

// Setup scalars shared by frbx_create and frbx_fit_segments_noalloc (host code, no allocation):
// the checked setup, the reference frequency of Eq. 1 (f_ref), the MBD grid of Eq. 5 (df_grid
// = GCD of the channel offsets in whole kHz, g_n = offset / df_grid) and the grid sizes
// Ls = sbd_pad J, Lm = mbd_pad nextpow2(max g_n + 1).  Point frequencies are
// f0_n + (j f_bw) / J, evaluated in that order.
struct SetupGrid {
  int N, J, C, Ls, Lm;
  double f_ref, df_grid, fmin0;
  int g[kMaxChan];
};
// FRBX_OK, or FRBX_EINVAL / FRBX_EUNSUPPORTED for a setup the library rejects.
int setup_grid(const frbx_setup *s, SetupGrid *out);

// One scan of a batched fit: its cube, output series, valid-segment table and first work item.
struct BatchScan {
  const float2 *vis;       // [n_bl][T][C]
  frbx_seg *out;           // [n_bl][n_dm][S_tot]
  const int *n_valid;      // [n_dm][n_win]
  const int *win_off;      // [n_win] first slot of each window in a series of this scan
  int T, S_tot, n_bl, n_tt;
  long long item0;         // items [item0, item0 + n_bl * n_tt * n_dm) belong to this scan
};

// Segment source of a fit launch: either the implicit half-overlap layout of a
// (baseline, DM) series, or an explicit device list of (bl, d, l, k0) rows.
struct FitArgs {
  const float2 *vis;       // [n_bl][T][C]
  int T, C, N, J;
  int n_dm;
  const int *dk;           // [n_dm][C]
  const float2 *wrot;      // [C]  weight x calibration rotation
  const float2 *tw_s;      // [Ls] exp(-2 pi i k / Ls)
  const float2 *tw_m;      // [Lm] exp(-2 pi i k / Lm)
  const int *g;            // [N]
  int Ls, Lm, log2Lm;
  // delay windows as wrapped index intervals: m searched iff ((m - m_lo) & (Ls-1)) < m_len
  int m_lo, m_len, q_lo, q_len;
  // implicit layout
  int n_win;
  const int *win_len;      // [n_win]
  const int *win_off;      // [n_win] slot offset within a series
  const int *n_valid;      // [n_dm][n_win]
  int S_tot;
  int tile;                // list mode: rows per CTA
  int TT;                  // implicit layout: APs per time tile (one CTA per DM, tile, baseline)
  // explicit list
  const int *seg;          // [n_seg][4]
  long long n_seg;
  frbx_seg *out;           // implicit: [n_bl][n_dm][S_tot]; list: [n_seg]
  // FFT kernel tables
  const int *slot;         // [32][occ] channel with g_n = g2 (mod 32), -1 = empty
  int occ;
  const float2 *sbd_tw;    // [Ls/32][J1*32] exp(-2 pi i (j m1 mod Ls)/Ls), zero for j >= J
  const float2 *mbd_tw;    // [N][Lm/32] exp(-2 pi i (g_n q1 mod Lm)/Lm)
  int J1;                  // ceil(J / 32)
  short slot_n[32][4];     // FFT kernel: channel n with g_n = g2 (mod 32), occupancy o; -1 = none
};

// Launchers (kernels_fit.cu).  Return a cudaError_t.
cudaError_t launch_fit(const FitArgs &a, int n_bl, bool list_mode, int kernel,
                       cudaStream_t st, int64_t *launches);
// Persistent fit over the work items of several scans of one setup (items claimed from *counter,
// which must be zero at launch); ctas_per_sm 0 = as many as fit.
cudaError_t launch_fit_batch(const FitArgs &a, const BatchScan *scans_dev, int n_scans, long long total_items,
                             unsigned int *counter, int kernel, int ctas_per_sm, cudaStream_t st, int64_t *launches);
bool fft_supported(int Ls, int Lm, int J);
void set_fft_constants();
// kernels_mma.cu: tensor-core (tcgen05, BF16) form of the MBD transform
struct MmaArgs {
  const void *bimg;        // constant operand B, already in its shared-memory image (BF16)
  int b_bytes;             // bytes of the image
  int b_atom_bytes;        // bytes of one 64-wide K atom of B (2 Lm rows x 128 B)
  int KA;                  // K atoms (64 BF16 each) per row
  int NC;                  // output columns per MMA chunk (Re G, Im G of NC/2 q values)
  int n_chunk;             // 2 Lm / NC
  int kk_steps;            // K / 16 MMA steps per chunk
  int tmem_cols;           // tensor-memory columns allocated (2 accumulator slots)
  int spt;                 // segments per 128-row tile (128 / Ls)
  long long n_valid;       // segments to fit
  long long n_items;       // implicit layout: n_bl * ceil(T / TT) * n_dm work items
  int *err;                // device flag, set to FRBX_ETIMEOUT when a bounded wait gives up
  long long timeout;       // clock cycles per pipeline wait
  long long drain_timeout; // clock cycles per wait that drains work in flight before exit
  int hold;                // test aid: the producers issue nothing, so the pipeline waits run out
  int fp8;                 // 1: A and B in E4M3 (kind::f8f6f4), A scaled per segment
};
bool mma_supported(int Ls, int Lm, int N, int J);
void set_mma_constants();
cudaError_t launch_fit_mma(const FitArgs &a, const MmaArgs &mm, int n_bl, bool list_mode, cudaStream_t st,
                           int64_t *launches);

// kernels_refine.cu: coherent power of continuous (DM, t0, tau_s, tau_m, rho) and its adjoint
struct RefineArgs {
  const float2 *vis;       // [n_bl][T][C]
  int T, C, J, n_bl, n_cand, n_par;
  const double *f;         // [C] point frequencies
  const double *f0;        // [N] channel edges
  const float2 *wrot;      // [C]
  double f0_min, inv_fref2, f_bw, t_ap;
  const double *params;    // [n_cand][n_par]
  const int *width;        // [n_cand]
  float *g;                // [n_cand][n_bl][2]
  float *power;            // [n_cand]
  int *status;             // [n_cand]
  const float *dpower;     // [n_cand]
  float *dparams;          // [n_cand][n_par]
  float *partial;          // [n_cand][n_bl][2] scratch
};
cudaError_t launch_refine(const RefineArgs &r, bool adjoint, cudaStream_t st, int64_t *launches);

// kernels_calib.cu: Appendix A channel delays and initial phases
cudaError_t launch_cal_sum(const float2 *vis, int T, int C, int n_bl, int k0, int l, const float2 *wrot,
                           double2 *xsum, float2 *xcube, float2 *wunit, cudaStream_t st, int64_t *launches);
cudaError_t launch_cal_channels(const double2 *xsum, const float2 *wrot, int n_bl, int N, int J, double f_bw,
                                const double *f0, double f0_min, const double *sbd_mbd, double *delay_ns,
                                double *phase_rad, cudaStream_t st, int64_t *launches);

// kernels_fft.cu
cudaError_t launch_fit_fft(const FitArgs &a, int n_bl, bool list_mode, cudaStream_t st,
                           int64_t *launches);
cudaError_t launch_fit_fft_batch(const FitArgs &a, const BatchScan *scans_dev, int n_scans, long long total_items,
                                 unsigned int *counter, int ctas_per_sm, cudaStream_t st, int64_t *launches);
size_t max_smem_optin();
bool fit_grid(const FitArgs &a, int n_bl, bool list_mode, dim3 *grid);

// kernels_tree.cu: multi-window fit through the additivity of the delay-resolution matrix
struct TreeArgs {
  // chunk of (baseline, DM) series
  const int2 *series;      // [n_s] (bl, d)
  int n_s;
  const int *dk_max;       // [n_dm]
  int T;
  float2 *Y;               // [n_s][T][Ls][N] SBD-transformed one-AP spectra
  size_t y_series;         // float2 per series in Y
  int n_ktile, k_per_cta;  // SBD pass: APs per CTA
  // merged maxima, in the series buffer viewed as 64-bit keys [n_bl][n_dm][S_tot]
  unsigned long long *keys;
  int n_dm, S_tot;
  const int *win_off;      // [n_win]
  int N, NS, Ls, Lm, PM, RB, n_mb, TT, n_tt, nlev;
  int half;                // k_tree_mbd with Lm = 16: one thread per SBD row, its 16 cells q = 0..15
  int emit_w[8];           // window index of level e (window 2^e), -1 = not searched
  int m_lo, m_len, q_lo, q_len;
  const int *slot_of;      // [N] slot of channel n in a Y row: (g_n mod 16) + 16 rank
  const float2 *tw;        // [NS/2][PM][2][2] MBD twiddles folded with the first DIF stage (0: empty)
  float2 *anc_g;           // deep window-tree anchors, one slice per MBD CTA
  // tensor-core MBD pass (3-term split BF16): Y as per-AP A tiles, W per block of 32 q
  int mma;                 // 1: the SBD pass writes tensor-core A tiles and the MBD pass is k_tree_mma
  const unsigned char *Yt; // split tiles [n_s][T][tile_bytes] (aliases Y)
  size_t yt_series;        // bytes per series in Yt
  int KA;                  // 64-wide K atoms per tile row (K = 2N)
  int tile_bytes;          // one AP: hi tile then lo tile, 2 KA 16 KB
  const unsigned char *wimg;  // [Lm/32][KA][hi | lo][64 rows x 128 B]
  int w_bytes;             // per block of 32 q: 2 KA 8 KB
  int n_qb;                // Lm / 32
  int log2Lm;
  int *err;                // set to FRBX_ETIMEOUT when a bounded wait of k_tree_mma gives up
  long long timeout;       // clock cycles per pipeline wait
  long long drain_timeout; // clock cycles per wait that drains copies / MMAs in flight before exit
  int hold;                // test aid: the loader issues no copies, so the pipeline waits run out
  int form;                // MBD product of k_tree_mma: 0 split BF16 x3, 1 BF16, 2 E4M3
  int k8_steps;            // E4M3 form: K = 32 steps per AP, (2N + 31) / 32
  float *ascale;           // E4M3 form: 1 / s of every AP, [n_s][T] (s: power-of-two scale of A)
  int rot;                 // delay windows: tile row r holds SBD row (r + rot) mod Ls (multiple of 8)
  // delay windows whose rows fit 32 or 64 tile rows: each AP keeps only its first prow rows (a
  // piece of piece_bytes, every K atom cut to prow rows), and k_tree_mma stacks the pieces of
  // pack = 128 / prow time tiles into one 128-row A operand (CTA: pack consecutive time tiles,
  // n_tg groups of them per series); pack 1: whole tiles
  int pack, prow, piece_bytes, n_tg;
  int n_abuf;              // A-tile ring depth of k_tree_mma (set by its launcher)
  int n_sanc;              // window-tree anchor levels of k_tree_mma in shared memory (set by its launcher)
};
bool tree_mma_supported(int Ls, int Lm, int N, int J);
bool tree_mma_fits(int form, int N, int nlev);  // shared memory holds W, the A ring and the deep anchors
int tree_mma_tile_bytes(int form, int N);        // one AP's A operand in its shared-memory image
int tree_mma_w_bytes(int form, int N);           // the DFT operand of one block of 32 q
cudaError_t launch_tree_mma(const TreeArgs &t, bool full, cudaStream_t st, int64_t *launches);
bool tree_supported(int Ls, int Lm, int N, int J, int s16, const int *windows, int n_win, int *nlev);
int tree_rows_per_block(int Ls, int Lm);  // SBD rows per k_tree_mbd CTA
size_t tree_anchor_floats(int nlev);  // float2 per MBD CTA in TreeArgs::anc_g
cudaError_t launch_tree_sbd(const FitArgs &a, const TreeArgs &t, cudaStream_t st, int64_t *launches);
cudaError_t launch_tree_mbd(const TreeArgs &t, bool full, cudaStream_t st, int64_t *launches);
cudaError_t launch_tree_finalize(frbx_seg *series, long long n_el, int S_tot, int n_dm, int n_win, const int *win_len,
                                 const int *win_off, const int *n_valid, int log2Lm, int Lm, cudaStream_t st,
                                 int64_t *launches);
void set_tree_constants();

// kernels_misc.cu
cudaError_t launch_shift_table(const double *f, int C, double fref, const double *dm, int n_dm,
                               double t_ap, int *dk, int *dk_max, cudaStream_t st,
                               int64_t *launches);

struct StatsArgs {
  const frbx_seg *series;  // [n_bl][n_dm][S_tot]
  int n_bl, n_dm, S_tot, n_win;
  const int *win_off;      // [n_win]
  const int *n_valid;      // [n_dm][n_win]
  const int *win_step;     // [n_win]
  const unsigned long long *masks;  // [n_series] baseline masks, or null for plain baselines
  int n_series;
  double threshold;
  double *mean_std;        // [n_series][n_dm][n_win][2]
  int *counts;             // [n_series * n_dm * n_win + 1]
  long long *offsets;      // [n_series * n_dm * n_win + 1]
  frbx_event *events;      // output
  float *pnorm;            // optional [n_series][n_dm][S_tot]
  int series_base;         // value stored in frbx_event.series = series_base + s
};
cudaError_t launch_stats_count(const StatsArgs &a, cudaStream_t st, int64_t *launches);
cudaError_t launch_scan(const StatsArgs &a, cudaStream_t st, int64_t *launches);
cudaError_t launch_events(const StatsArgs &a, cudaStream_t st, int64_t *launches);

// extract.cpp: host steps of Sec. 2.4 and Sec. 5.3
struct ExtractConfig {
  int T, n_dm, n_win, nwin_min, Lm;
  const int *win_len;
};
struct Pulse {
  int series, d, w, l, k0, m, q, n_win, group;
  float amp, p;
};
struct GroupOut {
  uint64_t mask;
  int n_baselines, n_pulses;
};
// events: ordered by (series, d, w, k0).  Outputs per-(series, d) pulses (pre-merge) and
// DM-merged pulses per series.
void extract_pulses(const ExtractConfig &cfg, const frbx_event *ev, int64_t n_ev, int n_series,
                    bool use_mbd, std::vector<Pulse> *pre_merge, std::vector<Pulse> *merged);
void cross_match(int T, std::vector<Pulse> *merged, int n_bl, std::vector<GroupOut> *groups);

}  // namespace frbx

struct frbx_handle {
  int device = 0;
  int N = 0, J = 0, C = 0;
  double f_bw = 0, t_ap = 0, f_ref = 0, df_grid = 0;
  int Ls = 0, Lm = 0, occ = 0, J1 = 0;
  short slot_n[32][4];  // channel of residue class g2 (mod 32), occupancy o; -1 = none
  std::vector<double> f0, f;
  std::vector<int> g;
  std::string err;
  int64_t launches = 0;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double stage_ms[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  // constant device tables
  double *d_f = nullptr, *d_f0 = nullptr;
  float2 *d_wrot = nullptr, *d_tw_s = nullptr, *d_tw_m = nullptr;
  float2 *d_sbd_tw = nullptr, *d_mbd_tw = nullptr;
  float2 *d_tree_tw = nullptr;  // [16 s16][Lm/32][2] MBD twiddles of the window-tree fit
  int *d_tree_slot = nullptr;   // [N] channel slot of the window-tree fit
  int tree_s16 = 0;             // slots per residue class mod 16 (0: no window-tree fit)
  cudaStream_t tree_st[2] = {nullptr, nullptr};  // window-tree fit: SBD passes, MBD passes
  cudaEvent_t tree_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // start, SBD done x2, MBD done x2
  std::vector<cudaEvent_t> tree_kev;  // per window-tree chunk: SBD start / end, MBD start / end
  // host input of a search: the cube is copied one baseline after another on copy_st; vis_ev[b]
  // marks baseline b copied, vis_ev[n_bl] the caller's stream reaching the call
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> vis_ev;
  int tree_chunks = 0;               // chunks of the last window-tree fit (0: another kernel ran)
  int tree_tensor = 0;               // 1: its MBD pass ran on the tensor cores (k_tree_mma)
  void *d_bimg = nullptr;  // BF16 DFT matrix image for the tensor-core fit (if supported)
  void *d_bimg8 = nullptr;  // the same matrix in E4M3
  void *d_wtree = nullptr;  // window-tree tensor-core fit: split-BF16 DFT blocks of 32 q
  void *d_wtree8 = nullptr; // the same blocks in E4M3 (kernel 8)
  int wtree_bytes = 0;      // per block
  int b_bytes = 0, b_bytes8 = 0, b_atom_bytes = 0, KA = 0, NC = 0;
  int *d_g = nullptr, *d_slot = nullptr;
  // scratch, grown on demand
  struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
  };
  frbx_limits lim{};          // frbx_set_limits (all zero = defaults)
  size_t scratch_total = 0;   // bytes held by the Bufs below
  Buf vis, dk, dk_max, series, pnorm, stats, counts, offsets, events, small, seglist, masks, errflag, refine, calib,
      ytree;
};
