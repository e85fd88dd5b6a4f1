// Choice of the grid parameters c and m for a target recall (the parameter tuning of
// Sec. III-A and the automatic tuning the paper's conclusion asks for): the fewest grids and
// cheapest cell size whose randomly transformed grids report at least the target fraction of
// the r-neighbour pairs, at the least measured build time.
//
// Recall is measured on a prefix sample of the points (at most kSample of them) against the
// sample's exact pair count (device brute force).  For every cell-size factor c/r of a fixed
// ladder the smallest m reaching the target is found by bisection: the transforms are the
// first m of one seeded generation, which is prefix-consistent, and the pair set of a prefix
// of the grids is a subset of the whole set's, so recall never falls as m grows.  Each
// feasible (c, m) is then built at full size and timed on the device; the fastest is kept.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rtg_host.h"

namespace rtghost {

namespace {

constexpr long long kSample = 32768;
constexpr double kFactors[] = {1.0, 1.1, 1.2, 1.3, 1.4, 1.5, 1.75, 2.0};

// Pairs of one count-only build (exact set when m == 0).
rtg_status count_pairs(rtg_ctx* c, const rtg_instance& it, int m, int dtype, int on_device,
                       uint32_t flags, long long* pairs) {
  rtg_csr out;
  std::memset(&out, 0, sizeof(out));
  Request q{&it, 1, m, dtype, on_device, flags, true};
  const rtg_status s = build(c, q, &out);
  if (s == RTG_OK) *pairs = out.nnz;
  release_out(c, &out);
  return s;
}

}  // namespace

rtg_status tune_params(rtg_ctx* c, const void* points, int dtype, int on_device, int64_t n, int d,
                       double r, double target, uint64_t seed, uint32_t flags,
                       rtg_param_choice* out) {
  std::memset(out, 0, sizeof(*out));
  const uint32_t gflags = flags & RTG_FLAG_SHIFT_ONLY;
  const long long S = n < kSample ? n : kSample;
  rtg_instance sample{points, S, d, r, 1.0, nullptr};
  long long exact = 0;
  rtg_status s = count_pairs(c, sample, 0, dtype, on_device, 0, &exact);
  if (s != RTG_OK) return s;
  out->sample_n = S;
  out->sample_exact = exact;
  std::vector<double> T((size_t)RTG_MAX_GRIDS * (d * d + d));
  // the sample's many small shapes take the default sort variant (measuring each would cost
  // more than it saves); full-size builds use the context's setting
  const bool autotune = c->autotune;
  double best_us = -1.0;
  int measured = 0;
  for (double f : kFactors) {
    const double cs = f * r;
    if (rtg_transforms_generate(seed, d, RTG_MAX_GRIDS, cs, gflags, T.data()) != RTG_OK)
      return fail(c, RTG_E_INVALID, "transform generation failed");
    sample.cell_side = cs;
    sample.transforms = T.data();
    auto recall_of = [&](int m, double* rec) -> rtg_status {
      long long p = 0;
      c->autotune = false;
      const rtg_status st = count_pairs(c, sample, m, dtype, on_device, gflags, &p);
      c->autotune = autotune;
      *rec = exact > 0 ? (double)p / (double)exact : 1.0;
      ++measured;
      return st;
    };
    double rec_max = 0.0;
    if ((s = recall_of(RTG_MAX_GRIDS, &rec_max)) != RTG_OK) return s;
    if (rec_max < target) continue;  // this cell size cannot reach the target
    int lo = 1, hi = RTG_MAX_GRIDS;  // recall(hi) >= target
    double rec_hi = rec_max;
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      double rec = 0.0;
      if ((s = recall_of(mid, &rec)) != RTG_OK) return s;
      if (rec >= target) {
        hi = mid;
        rec_hi = rec;
      } else {
        lo = mid + 1;
      }
    }
    // full-size build time: the second of two builds (the first may read the key width back
    // and choose the sort variant for this shape)
    rtg_instance full{points, n, d, r, cs, T.data()};
    double us = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
      rtg_csr o;
      std::memset(&o, 0, sizeof(o));
      Request q{&full, 1, hi, dtype, on_device, gflags | RTG_FLAG_TIMING, false};
      s = build(c, q, &o);
      us = o.stats.phase_us[7];
      release_out(c, &o);
      if (s != RTG_OK) return s;
    }
    if (best_us < 0.0 || us < best_us) {
      best_us = us;
      out->m = hi;
      out->c_factor = f;
      out->cell_side = cs;
      out->recall = rec_hi;
      out->build_us = us;
    }
  }
  out->candidates = measured;
  if (best_us < 0.0)
    return fail(c, RTG_E_INVALID, "no cell size in [r, 2r] reaches the target recall with at "
                                  "most 64 grids");
  return RTG_OK;
}

}  // namespace rtghost
