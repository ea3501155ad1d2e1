// Host steps of the single-pulse extraction (Sec. 2.4): grouping of candidate signals
// across windows (step b), MBD consistency (step c), window count and best member
// (step d), the DM merge of the coarse DM search (Sec. 5.3) and cross-matching of
// baselines.  Sequential and O(events x window length): each insertion asks "which
// is the first group (in creation order) holding a member whose [k0, k0 + l) overlaps
// mine", answered from a per-AP array of the smallest group id covering that AP.  Series are
// independent until cross-matching, so large event lists are split across host threads.
#include <algorithm>
#include <climits>
#include <cmath>
#include <thread>

#include "frbx_internal.h"

namespace frbx {

namespace {

constexpr double kTwoPi = 6.283185307179586;  // same double as 2 * pi

struct Grouper {
  std::vector<int> min_gid;   // per AP
  std::vector<int> touched;
  int n_groups = 0;

  explicit Grouper(int T) : min_gid((size_t)std::max(T, 1), INT_MAX) {}

  void reset() {
    for (int t : touched) min_gid[(size_t)t] = INT_MAX;
    touched.clear();
    n_groups = 0;
  }
  // Returns the group the range [k0, k0 + l) joins (a new one if none overlaps).
  int insert(int k0, int l) {
    const int T = (int)min_gid.size();
    const int lo = std::max(0, k0), hi = std::min(T, k0 + l);
    int g = INT_MAX;
    for (int t = lo; t < hi; ++t) g = std::min(g, min_gid[(size_t)t]);
    if (g == INT_MAX) g = n_groups++;
    for (int t = lo; t < hi; ++t) {
      if (min_gid[(size_t)t] == INT_MAX) touched.push_back(t);
      min_gid[(size_t)t] = std::min(min_gid[(size_t)t], g);
    }
    return g;
  }
};

// Step c: circular mean of the MBD over the group (period t_ambig; angle 2 pi q / Lm) and
// removal of members at or beyond a quarter period from it.
void mbd_filter(std::vector<const frbx_event *> *grp, int Lm) {
  double sc = 0.0, ss = 0.0;
  for (const frbx_event *e : *grp) {
    const double th = (kTwoPi * (double)e->mbd_idx) / (double)Lm;
    sc += std::cos(th);
    ss += std::sin(th);
  }
  const double mu = std::atan2(ss, sc);
  std::vector<const frbx_event *> keep;
  keep.reserve(grp->size());
  for (const frbx_event *e : *grp) {
    const double th = (kTwoPi * (double)e->mbd_idx) / (double)Lm;
    if (std::fabs(std::remainder(th - mu, kTwoPi)) < M_PI / 2) keep.push_back(e);
  }
  grp->swap(keep);
}

// Series [s_lo, s_hi) whose events are ev[0, n_ev) (sorted by series, DM trial, window, k0).
void extract_range(const ExtractConfig &cfg, const frbx_event *ev, int64_t n_ev, int s_lo, int s_hi,
                   bool use_mbd, std::vector<Pulse> *pre_merge, std::vector<Pulse> *merged) {
  // window visiting order: longest first (step b)
  std::vector<int> order(cfg.n_win);
  for (int w = 0; w < cfg.n_win; ++w) order[w] = w;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return cfg.win_len[x] > cfg.win_len[y]; });
  Grouper gp(cfg.T), gm(cfg.T);
  int64_t pos = 0;
  std::vector<std::vector<const frbx_event *>> groups;
  std::vector<std::pair<int64_t, int64_t>> wr(cfg.n_win);
  for (int s = s_lo; s < s_hi; ++s) {
    std::vector<Pulse> series_pulses;  // DM ascending, discovery order
    for (int d = 0; d < cfg.n_dm; ++d) {
      // the events of (s, d) are contiguous and ordered by window then k0
      for (int w = 0; w < cfg.n_win; ++w) wr[w] = {0, 0};
      while (pos < n_ev && ev[pos].series == s && ev[pos].dm_idx == d) {
        const int w = ev[pos].win_idx;
        int64_t e = pos;
        while (e < n_ev && ev[e].series == s && ev[e].dm_idx == d && ev[e].win_idx == w) ++e;
        wr[w] = {pos, e};
        pos = e;
      }
      gp.reset();
      groups.clear();
      for (int w : order) {
        for (int64_t i = wr[w].first; i < wr[w].second; ++i) {
          const int g = gp.insert(ev[i].k0, cfg.win_len[w]);
          if (g == (int)groups.size()) groups.emplace_back();
          groups[(size_t)g].push_back(&ev[i]);
        }
      }
      for (auto &grp : groups) {
        if (use_mbd) mbd_filter(&grp, cfg.Lm);
        if (grp.empty()) continue;
        // step d: distinct windows, best member (first inserted on ties)
        int wins[kMaxWin];
        int nw = 0;
        for (const frbx_event *e : grp) {
          bool seen = false;
          for (int k = 0; k < nw; ++k) seen |= cfg.win_len[wins[k]] == cfg.win_len[e->win_idx];
          if (!seen) wins[nw++] = e->win_idx;
        }
        if (nw < cfg.nwin_min) continue;
        const frbx_event *best = grp[0];
        for (const frbx_event *e : grp)
          if (e->pnorm > best->pnorm) best = e;
        Pulse p;
        p.series = s;
        p.d = d;
        p.w = best->win_idx;
        p.l = cfg.win_len[best->win_idx];
        p.k0 = best->k0;
        p.m = best->sbd_idx;
        p.q = best->mbd_idx;
        p.n_win = nw;
        p.group = -1;
        p.amp = best->amp;
        p.p = best->pnorm;
        series_pulses.push_back(p);
        if (pre_merge) pre_merge->push_back(p);
      }
    }
    // Sec. 5.3: one pulse per overlap group across DM trials, the one of highest power
    gm.reset();
    std::vector<int> best_of;
    for (size_t i = 0; i < series_pulses.size(); ++i) {
      const int g = gm.insert(series_pulses[i].k0, series_pulses[i].l);
      if (g == (int)best_of.size()) {
        best_of.push_back((int)i);
      } else if (series_pulses[i].p > series_pulses[(size_t)best_of[(size_t)g]].p) {
        best_of[(size_t)g] = (int)i;
      }
    }
    for (int i : best_of) merged->push_back(series_pulses[(size_t)i]);
  }
}

}  // namespace

// The steps above depend only on one series' own events (steps b-d per DM trial, then the DM
// merge of that series), so contiguous runs of series go to host threads, balanced by event
// count, and their pulses are concatenated in series order: the same output as one pass.
void extract_pulses(const ExtractConfig &cfg, const frbx_event *ev, int64_t n_ev, int n_series,
                    bool use_mbd, std::vector<Pulse> *pre_merge, std::vector<Pulse> *merged) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  int n_th = n_ev < 50000 ? 1 : std::min({n_series, hw, 32});
  for (int64_t i = 1; i < n_ev && n_th > 1; ++i)  // split points need events sorted by series
    if (ev[i].series < ev[i - 1].series) n_th = 1;
  if (n_th <= 1) {
    extract_range(cfg, ev, n_ev, 0, n_series, use_mbd, pre_merge, merged);
    return;
  }
  // first event of series s (events are sorted by series)
  auto first_of = [&](int s) -> int64_t {
    return std::lower_bound(ev, ev + n_ev, s, [](const frbx_event &e, int v) { return e.series < v; }) - ev;
  };
  // series cut points: part t ends at the first series whose first event reaches (t + 1) n_ev / n_th
  std::vector<int> cut(n_th + 1, n_series);
  cut[0] = 0;
  for (int t = 1; t < n_th; ++t) {
    const int64_t target = n_ev * t / n_th;
    int s = cut[t - 1];
    while (s < n_series && first_of(s) < target) ++s;
    cut[t] = s;
  }
  std::vector<std::vector<Pulse>> pre_part(n_th), merged_part(n_th);
  std::vector<std::thread> th;
  th.reserve(n_th);
  auto part = [&](int t) {
    const int64_t e0 = first_of(cut[t]), e1 = first_of(cut[t + 1]);
    extract_range(cfg, ev + e0, e1 - e0, cut[t], cut[t + 1], use_mbd, pre_merge ? &pre_part[t] : nullptr,
                  &merged_part[t]);
  };
  for (int t = 0; t < n_th; ++t) {
    if (cut[t] >= cut[t + 1]) continue;
    try {
      th.emplace_back(part, t);
    } catch (...) {  // no thread to be had: this part runs here (no exception crosses the C ABI)
      part(t);
    }
  }
  for (auto &x : th) x.join();
  for (int t = 0; t < n_th; ++t) {
    if (pre_merge) pre_merge->insert(pre_merge->end(), pre_part[t].begin(), pre_part[t].end());
    merged->insert(merged->end(), merged_part[t].begin(), merged_part[t].end());
  }
}

void cross_match(int T, std::vector<Pulse> *merged, int n_bl, std::vector<GroupOut> *groups) {
  // baselines ascending, then pulses by ascending start (stable)
  std::vector<int> idx(merged->size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
    const Pulse &a = (*merged)[(size_t)x], &b = (*merged)[(size_t)y];
    if (a.series != b.series) return a.series < b.series;
    return a.k0 < b.k0;
  });
  (void)n_bl;
  Grouper gp(T);
  groups->clear();
  for (int i : idx) {
    Pulse &p = (*merged)[(size_t)i];
    const int g = gp.insert(p.k0, p.l);
    if (g == (int)groups->size()) groups->push_back(GroupOut{0ull, 0, 0});
    GroupOut &go = (*groups)[(size_t)g];
    go.mask |= 1ull << p.series;
    go.n_pulses += 1;
    p.group = g;
  }
  for (GroupOut &go : *groups) go.n_baselines = __builtin_popcountll(go.mask);
}

}  // namespace frbx
