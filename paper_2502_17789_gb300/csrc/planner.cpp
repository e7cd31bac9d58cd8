// Host partitioner of libidg: splits each baseline's (timestep x channel)
// table into subtables that each fit one L x L subgrid (Section 3.1), with
// the A-term constraint of Section 3.3 applied per segment (or per subgrid
// under IDG_SPLIT_AT_ATERM_INTERVALS).
//
// Must be compiled without floating-point contraction (-ffp-contract=off):
// the decisions depend on pixel coordinates that have to round identically
// on every machine.
//
// Rules (reading of Section 3.1; the paper names the idea, not constants):
//   span S = L - P - 4, growth margin G = max(2, S/4), channel span Sc = S - G
//   1. pending subtables (t_start, c_lo, c_hi) start as (block start, 0, n_ch)
//   2. at t_start, cut [c_lo, c_hi) into maximal runs whose end channels lie
//      within Sc pixels in u and in v (fit with a margin left for time growth)
//   3. extend each run in time while its four corner visibilities stay within
//      S pixels, then shrink while any member falls outside S
//   4. emit it; its later timesteps become a new pending subtable
//   subgrids are ordered by (baseline, block, t_start, c_lo)
//   corner x0 = floor((xi_min + xi_max) / 2) - L/2, likewise y0
//   w check: |w - w0| * max|grad n'| * FOV <= P/2 - 1 (footnote of Section 2.4),
//   i.e. |w - w0| <= w_max.  Without IDG_W_LAYERS w0 = 0 and a larger |w| is
//   an error.  With it (the hybrid with w-stacking of Section 2.4) a row
//   (baseline, timestep) with w < 0 is mirrored -- the visibility V^H of
//   baseline (q, p) at (-u, -v, -w), since V(u,v,w) = V(-u,-v,-w)^H (the
//   footnote's way of halving the layers) -- so every gridded w' >= 0; its
//   layer is k = floor(w' / w_step), w_step = 2 w_max, with w0 = (2k+1) w_max,
//   the set {w_max, 3 w_max, 5 w_max, ...}.  Pixel coordinates of mirrored
//   rows are those of (-u, -v), and every member of a subgrid shares the
//   layer and the side of the run's first visibility (checked on the channel
//   run's ends, the time growth's corners and in the final shrink).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>
#include <thread>

#include "idg_internal.h"

namespace idg {
namespace {

struct Pending {
  int32_t ts, c_lo, c_hi;
};
struct Run {
  int32_t blk, ts, te, c_lo, c_hi, layer;
};

// Pixel coordinates (and w layer keys) of every visibility of one baseline,
// [t][ch].  With w layers the key is 2k + m (k the layer, m = 1 on a
// mirrored row), so equal keys mean one layer and one side.
class BaselinePixels {
 public:
  BaselinePixels(const PlanInput& in, int b, double w_step)
      : n_ch_(in.n_ch), xi_(size_t(in.n_t) * in.n_ch), eta_(xi_.size()), layer_(w_step > 0.0 ? xi_.size() : 0) {
    const double half = double(in.N / 2);
    for (int t = 0; t < in.n_t; ++t) {
      const double* r = in.uvw + (size_t(b) * in.n_t + t) * 3;
      const bool mirror = w_step > 0.0 && r[2] < 0.0;
      const double sgn = mirror ? -1.0 : 1.0;
      for (int c = 0; c < in.n_ch; ++c) {
        const double f = in.freqs[c];
        const double u = (sgn * r[0] * f) / kSpeedOfLight;
        const double v = (sgn * r[1] * f) / kSpeedOfLight;
        xi_[size_t(t) * n_ch_ + c] = u * in.fov + half;
        eta_[size_t(t) * n_ch_ + c] = v * in.fov + half;
        if (w_step > 0.0) {
          const double w = (sgn * r[2] * f) / kSpeedOfLight;
          layer_[size_t(t) * n_ch_ + c] = 2 * int32_t(std::floor(w / w_step)) + (mirror ? 1 : 0);
        }
      }
    }
  }
  double xi(int t, int c) const { return xi_[size_t(t) * n_ch_ + c]; }
  double eta(int t, int c) const { return eta_[size_t(t) * n_ch_ + c]; }
  int32_t layer(int t, int c) const { return layer_.empty() ? 0 : layer_[size_t(t) * n_ch_ + c]; }
  bool same_layer(int ts, int te, int c_lo, int c_hi, int32_t k) const {
    if (layer_.empty()) return true;
    for (int t = ts; t < te; ++t)
      for (int c = c_lo; c < c_hi; ++c)
        if (layer(t, c) != k) return false;
    return true;
  }

  // Extent of a set of (t, c) points along u and v.
  template <size_t K>
  bool within(const int (&ts)[K], const int (&cs)[K], double span) const {
    double xmin = xi(ts[0], cs[0]), xmax = xmin, ymin = eta(ts[0], cs[0]), ymax = ymin;
    for (size_t n = 1; n < K; ++n) {
      const double x = xi(ts[n], cs[n]), y = eta(ts[n], cs[n]);
      xmin = std::min(xmin, x);
      xmax = std::max(xmax, x);
      ymin = std::min(ymin, y);
      ymax = std::max(ymax, y);
    }
    return (xmax - xmin) <= span && (ymax - ymin) <= span;
  }

  struct Box {
    double xmin, xmax, ymin, ymax;
  };
  Box box(int ts, int te, int c_lo, int c_hi) const {
    Box bx{xi(ts, c_lo), xi(ts, c_lo), eta(ts, c_lo), eta(ts, c_lo)};
    for (int t = ts; t < te; ++t)
      for (int c = c_lo; c < c_hi; ++c) {
        bx.xmin = std::min(bx.xmin, xi(t, c));
        bx.xmax = std::max(bx.xmax, xi(t, c));
        bx.ymin = std::min(bx.ymin, eta(t, c));
        bx.ymax = std::max(bx.ymax, eta(t, c));
      }
    return bx;
  }

 private:
  int n_ch_;
  std::vector<double> xi_, eta_;
  std::vector<int32_t> layer_;
};

// Host threads for one partition: up to IDG_PLANNER_THREADS (default: the
// hardware's, at most 16), fewer for small observations.
int planner_threads(int n_bl, size_t n_vis) {
  int hw = int(std::thread::hardware_concurrency());
  if (const char* e = std::getenv("IDG_PLANNER_THREADS")) {
    const int v = std::atoi(e);
    if (v >= 1) hw = v;
  } else {
    hw = std::min(hw, 16);
  }
  const int by_work = int(std::min<size_t>(n_vis / 200000 + 1, size_t(n_bl)));
  return std::max(1, std::min(hw, by_work));
}

}  // namespace

idg_status partition(const PlanInput& in, Partition* out, std::string* err) {
  char msg[256];
  auto fail = [&](idg_status st, const char* what) {
    *err = what;
    return st;
  };
  if (in.N <= 0 || in.N % 2 || in.L <= 0 || in.L % 2 || in.L > in.N || in.P < 0 || in.P % 2)
    return fail(IDG_ERR_INVALID_ARG, "grid_size and subgrid_size must be even with 0 < L <= N; padding even, >= 0");
  if (!(in.fov > 0.0) || !(0.5 * in.fov * in.fov < 1.0))
    return fail(IDG_ERR_INVALID_ARG, "image_size must satisfy 0 < FOV and FOV^2/2 < 1");
  if (in.n_st < 0 || in.n_bl < 0 || in.n_t < 0 || in.n_ch < 0 || in.n_int < 1)
    return fail(IDG_ERR_INVALID_ARG, "negative sizes or no A-term interval");
  if (in.aterm_offsets[0] != 0 || in.aterm_offsets[in.n_int] != in.n_t)
    return fail(IDG_ERR_INVALID_ARG, "aterm_offsets must start at 0 and end at n_timesteps");
  for (int a = 0; a < in.n_int; ++a)
    if (in.aterm_offsets[a + 1] < in.aterm_offsets[a]) return fail(IDG_ERR_INVALID_ARG, "aterm_offsets must ascend");
  for (int c = 1; c < in.n_ch; ++c)
    if (!(in.freqs[c] > in.freqs[c - 1]))
      return fail(IDG_ERR_UNSORTED_FREQ, "channel frequencies must be strictly ascending");
  for (int b = 0; b < in.n_bl; ++b) {
    const int p = in.baselines[2 * b], q = in.baselines[2 * b + 1];
    if (p < 0 || q < 0 || p >= in.n_st || q >= in.n_st) return fail(IDG_ERR_INVALID_ARG, "baseline station out of range");
  }
  const int S = in.L - in.P - 4;
  if (S < 1) return fail(IDG_ERR_INVALID_ARG, "subgrid_size - kernel_padding - 4 must be >= 1");
  const int G = std::max(2, S / 4);
  const int Sc = std::max(0, S - G);

  // w limit: steepest n' gradient is at the subgrid corner l = m = -FOV/2
  const double r2 = 0.5 * in.fov * in.fov;
  const double grad = std::sqrt(r2) / std::sqrt(1.0 - r2);
  const double w_limit = 0.5 * in.P - 1.0;
  const bool layered = (in.flags & IDG_W_LAYERS) != 0;
  const double w_step = 2.0 * (w_limit / (grad * in.fov));
  if (layered && !(w_step > 0.0)) return fail(IDG_ERR_INVALID_ARG, "w layers need kernel_padding > 2");
  out->w_step = layered ? w_step : 0.0;
  // Baselines are partitioned independently (the rules above never look
  // across baselines), so they are planned on a few host threads and the
  // results concatenated in baseline order: the same tables as one thread.
  struct BaselinePlan {
    std::vector<SubgridDesc> sg;   // plan_index and seg_begin relative to the baseline
    std::vector<SegmentDesc> seg;  // subgrid relative to the baseline
    idg_status st = IDG_OK;
    std::string err;
  };
  const bool split = (in.flags & IDG_SPLIT_AT_ATERM_INTERVALS) != 0;
  auto plan_baseline = [&](int b, BaselinePlan& bp) {
    char m[256];
    if (!layered) {  // w check of this baseline, in (t, c) order
      for (int t = 0; t < in.n_t; ++t) {
        const double wm = in.uvw[(size_t(b) * in.n_t + t) * 3 + 2];
        for (int c = 0; c < in.n_ch; ++c) {
          const double w = (wm * in.freqs[c]) / kSpeedOfLight;
          if (std::fabs(w) * grad * in.fov > w_limit) {
            std::snprintf(m, sizeof m, "|w| = %.3f wavelengths (baseline %d, t %d, ch %d) exceeds the %.2f-pixel "
                          "w fringe limit", std::fabs(w), b, t, c, w_limit);
            bp.st = IDG_ERR_W_TOO_LARGE;
            bp.err = m;
            return;
          }
        }
      }
    }
    if (in.n_t == 0 || in.n_ch == 0) return;
    const BaselinePixels px(in, b, layered ? w_step : 0.0);
    std::vector<Run> runs;
    std::vector<Pending> todo;
    const int n_blocks = split ? in.n_int : 1;
    for (int blk = 0; blk < n_blocks; ++blk) {
      const int ta = split ? in.aterm_offsets[blk] : 0;
      const int tb = split ? in.aterm_offsets[blk + 1] : in.n_t;
      if (ta >= tb) continue;
      todo.assign(1, Pending{ta, 0, in.n_ch});
      while (!todo.empty()) {
        const Pending cur = todo.back();
        todo.pop_back();
        for (int lo = cur.c_lo; lo < cur.c_hi;) {
          const int32_t k0 = px.layer(cur.ts, lo);
          int hi = lo + 1;
          while (hi < cur.c_hi) {
            const int ts2[2] = {cur.ts, cur.ts}, cs2[2] = {lo, hi};
            if (!px.within(ts2, cs2, double(Sc))) break;
            if (px.layer(cur.ts, hi) != k0) break;
            ++hi;
          }
          int te = cur.ts + 1;
          while (te < tb) {
            const int ts4[4] = {cur.ts, cur.ts, te, te}, cs4[4] = {lo, hi - 1, lo, hi - 1};
            if (!px.within(ts4, cs4, double(S))) break;
            if (px.layer(te, lo) != k0 || px.layer(te, hi - 1) != k0) break;
            ++te;
          }
          while (te > cur.ts + 1) {
            const auto bx = px.box(cur.ts, te, lo, hi);
            if ((bx.xmax - bx.xmin) <= double(S) && (bx.ymax - bx.ymin) <= double(S) &&
                px.same_layer(cur.ts, te, lo, hi, k0))
              break;
            --te;
          }
          runs.push_back(Run{blk, cur.ts, te, lo, hi, k0});
          if (te < tb) todo.push_back(Pending{te, lo, hi});
          lo = hi;
        }
      }
    }
    std::sort(runs.begin(), runs.end(), [](const Run& x, const Run& y) {
      if (x.blk != y.blk) return x.blk < y.blk;
      if (x.ts != y.ts) return x.ts < y.ts;
      return x.c_lo < y.c_lo;
    });
    for (const Run& r : runs) {
      const auto bx = px.box(r.ts, r.te, r.c_lo, r.c_hi);
      SubgridDesc d{};
      const bool mirror = (r.layer & 1) != 0;  // stations swap on the mirror (q, p)
      d.b = b;
      d.p = in.baselines[2 * b + (mirror ? 1 : 0)];
      d.q = in.baselines[2 * b + (mirror ? 0 : 1)];
      d.t0 = r.ts;
      d.t1 = r.te;
      d.c0 = r.c_lo;
      d.c1 = r.c_hi;
      d.x0 = int32_t(std::floor((bx.xmin + bx.xmax) / 2.0)) - in.L / 2;
      d.y0 = int32_t(std::floor((bx.ymin + bx.ymax) / 2.0)) - in.L / 2;
      d.n_vis = (r.te - r.ts) * (r.c_hi - r.c_lo);
      d.layer = r.layer >> 1;
      d.flags = mirror ? kSubgridMirrored : 0;
      d.plan_index = int32_t(bp.sg.size());
      const bool outside = d.x0 < 0 || d.y0 < 0 || d.x0 > in.N - in.L || d.y0 > in.N - in.L;
      if (outside) {
        if (!(in.flags & IDG_DROP_OUT_OF_GRID)) {
          std::snprintf(m, sizeof m, "baseline %d timesteps [%d,%d) channels [%d,%d) need a subgrid at (%d,%d), "
                        "outside the %d-pixel grid", b, r.ts, r.te, r.c_lo, r.c_hi, d.x0, d.y0, in.N);
          bp.st = IDG_ERR_UV_OUT_OF_GRID;
          bp.err = m;
          return;
        }
        d.flags |= kSubgridDropped;
      }
      d.seg_begin = int32_t(bp.seg.size());
      for (int a = 0; a < in.n_int; ++a) {
        const int lo = std::max(in.aterm_offsets[a], r.ts), hi = std::min(in.aterm_offsets[a + 1], r.te);
        if (lo >= hi) continue;
        const int width = r.c_hi - r.c_lo;
        bp.seg.push_back(SegmentDesc{d.plan_index, a, (lo - r.ts) * width, (hi - r.ts) * width});
      }
      d.seg_count = int32_t(bp.seg.size()) - d.seg_begin;
      bp.sg.push_back(d);
    }
  };

  std::vector<BaselinePlan> per(size_t(std::max(0, in.n_bl)));
  const int n_threads = planner_threads(in.n_bl, size_t(in.n_bl) * in.n_t * in.n_ch);
  if (n_threads <= 1) {
    for (int b = 0; b < in.n_bl; ++b) plan_baseline(b, per[b]);
  } else {
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int k = 0; k < n_threads; ++k)
      pool.emplace_back([&] {
        for (int b = next.fetch_add(1); b < in.n_bl; b = next.fetch_add(1)) plan_baseline(b, per[b]);
      });
    for (std::thread& th : pool) th.join();
  }
  // errors as the sequential order would report them: a w error of any
  // baseline first (the w check precedes all partitioning), then the first
  // baseline with a subgrid outside the grid
  for (int b = 0; b < in.n_bl; ++b)
    if (per[b].st == IDG_ERR_W_TOO_LARGE) return fail(per[b].st, per[b].err.c_str());
  for (int b = 0; b < in.n_bl; ++b)
    if (per[b].st != IDG_OK) return fail(per[b].st, per[b].err.c_str());
  out->subgrids.clear();
  out->segments.clear();
  size_t n_sg = 0, n_seg = 0;
  for (const BaselinePlan& bp : per) {
    n_sg += bp.sg.size();
    n_seg += bp.seg.size();
  }
  out->subgrids.reserve(n_sg);
  out->segments.reserve(n_seg);
  for (BaselinePlan& bp : per) {
    const int32_t sg0 = int32_t(out->subgrids.size()), seg0 = int32_t(out->segments.size());
    for (SubgridDesc d : bp.sg) {
      d.plan_index += sg0;
      d.seg_begin += seg0;
      out->subgrids.push_back(d);
    }
    for (SegmentDesc g : bp.seg) {
      g.subgrid += sg0;
      out->segments.push_back(g);
    }
    bp = BaselinePlan{};
  }
  return IDG_OK;
}

std::vector<double> kaiser_bessel_taper(int L, double beta) {
  // T(l) = I0(beta sqrt(1 - x^2)) / I0(beta), x = 2 l / FOV (Section 4.2);
  // the standard library provides I0, as the paper notes.
  std::vector<double> t(L);
  const double norm = std::cyl_bessel_i(0.0, beta);
  for (int i = 0; i < L; ++i) {
    const double x = double(2 * i - L) / double(L);
    const double r = 1.0 - x * x;
    t[i] = (r > 0.0 ? std::cyl_bessel_i(0.0, beta * std::sqrt(r)) : 1.0) / norm;
  }
  return t;
}

}  // namespace idg
