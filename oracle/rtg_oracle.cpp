// CPU oracle for all-pairs r-nearest-neighbour reporting with randomly transformed grids.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 statement of what the GPU
// library computes.  Only the test suite, the smoke check and the benchmark's CPU-baseline
// leg load it; the library never does, and the two share no code.
//
// Functions and the passages they follow (Kleinbort, Salzman, Halperin, "Efficient
// high-quality motion planning by fast all-pairs r-nearest-neighbors", arXiv:1409.8112):
//   oracle_brute       - the all-pairs r-NN problem of Sec. I: every pair p, q of P with
//                        Euclidean distance at most r, by checking all n(n-1)/2 pairs.
//   oracle_exact_grid  - the same set through a fixed uniform grid of side r, scanning
//                        same and adjacent cells (the Lenhof-Smid idea recalled in Sec. II-B).
//   oracle_cells       - the point-to-cell step of Alg. 1 for each grid: the cell u each
//                        point lies in, for the rotated + shifted grids of Sec. III ("second
//                        algorithm").
//   oracle_rtg_query   - r-NN queries of new points from the m stored grids (Sec. V).
//   oracle_rtg         - Alg. 1 in full (Sec. III): for each of the m grids, associate points
//                        to cells, go over all pairs inside each non-empty cell, report those
//                        at distance at most r; duplicates across grids are removed with the
//                        array of unordered sets of Sec. III-B (slot i holds j > i).
//   oracle_rtg_threads - the same computation on several host threads: the m grids are
//                        independent (each thread takes whole grids), and the merge into the
//                        array of unordered sets is split by row ranges.  Used only for the
//                        all-core CPU baseline; the tests check it equals oracle_rtg.
//
// Arithmetic (the readings of the paper that make the result unique):
//   * FP32 coordinates are widened exactly to FP64; everything is FP64.
//   * Rotated coordinate: acc = s_k; acc = fma(R[k][l], p[l], acc) for l = 0..d-1.
//   * Cell coordinate: q_k = floor(acc / c) with IEEE division (never a reciprocal).
//   * Squared distance on the ORIGINAL coordinates: e = p_a[l] - p_b[l]; s = fma(e, e, s)
//     for l = 0..d-1 starting from s = 0; the pair is kept iff s <= fl(r * r).
//   This file is compiled with -ffp-contract=off so no other contraction happens.
//
// Diagnostics (counted, never used to decide anything):
//   near-wall: (point, grid) with some axis k where fl(|u - rint(u)| * c) <= 1e-12,
//              u = fl(acc / c), i.e. the rotated point lies within 1e-12 of a cell wall.
//   near-r:    distinct pairs placed in one cell by at least one grid with
//              |sqrt(s) - r| <= 1e-12 * r.
//
// Planted mistakes: building with -DORACLE_MUTANT=k changes one step on purpose (see the
// MUTANT(k) sites); the test suite builds these variants to show its pins catch them.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <unordered_map>
#include <unordered_set>
#include <vector>
#include <algorithm>
#include <thread>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

extern "C" {

typedef struct {
  int64_t n;
  int64_t nnz;
  int64_t* row_ptr;  // n + 1 entries, malloc'ed
  int32_t* col;      // nnz entries, malloc'ed; ascending within a row; col > row
} oracle_csr;

typedef struct {
  int64_t candidates;     // sum over non-empty cells of C(size, 2)
  int64_t nonempty_cells;  // |U| for this grid
  int64_t multi_cells;     // cells holding at least two points
  int64_t max_cell;        // largest cell population
  int64_t near_wall;       // points within 1e-12 of a wall of this grid
  int64_t reported;        // pairs with distance <= r found in this grid (before dedupe)
} oracle_grid_stats;

void oracle_free(oracle_csr* c) {
  if (!c) return;
  free(c->row_ptr);
  free(c->col);
  c->row_ptr = nullptr;
  c->col = nullptr;
}

}  // extern "C"

namespace {

// Widen the input to FP64 (exact for FP32 input).
std::vector<double> widen(const void* pts, int dtype, int64_t n, int d) {
  std::vector<double> p((size_t)n * d);
  if (dtype == 0) {
    std::memcpy(p.data(), pts, sizeof(double) * (size_t)n * d);
  } else {
    const float* f = (const float*)pts;
    for (size_t i = 0; i < (size_t)n * d; ++i) p[i] = (double)f[i];
  }
  return p;
}

// Squared Euclidean distance between points a and b in the fixed order stated above.
double dist2(const double* pa, const double* pb, int d) {
  double s = 0.0;
  for (int l = 0; l < d; ++l) {
    double e = pa[l] - pb[l];
    s = std::fma(e, e, s);
  }
#if ORACLE_MUTANT == 4
  // planted mistake: one coordinate dropped from the distance
  s = 0.0;
  for (int l = 0; l + 1 < d; ++l) {
    double e = pa[l] - pb[l];
    s = std::fma(e, e, s);
  }
#endif
  return s;
}

bool within(double s, double rr) {
  if (MUTANT(3)) return s < rr;  // planted mistake: strict instead of "at most r"
  return s <= rr;
}

// Alg. 1 (point-to-cell step) for grid t: the rotated coordinate y = R p + s and the cell index
// q_k = floor(y_k / c).  Writes q (d entries); returns true if the point lies within
// 1e-12 of a cell wall of this grid.
bool cell_of(const double* p, const double* R, const double* s, int d, double c, int64_t* q) {
  bool near = false;
  for (int k = 0; k < d; ++k) {
    double acc = s[k];
    if (MUTANT(2)) acc = 0.0;  // planted mistake: shift ignored
    for (int l = 0; l < d; ++l) {
      double rkl = MUTANT(1) ? R[l * d + k] : R[k * d + l];  // mutant 1: R transposed
      acc = std::fma(rkl, p[l], acc);
    }
    double u = acc / c;
    double f = MUTANT(5) ? std::trunc(u) : std::floor(u);  // mutant 5: truncation
    q[k] = (int64_t)f;
    double w = std::fabs(u - std::rint(u));
    if (w * c <= 1e-12) near = true;
  }
  return near;
}

void to_csr(const std::vector<std::unordered_set<uint32_t>>& sets, oracle_csr* out) {
  int64_t n = (int64_t)sets.size();
  int64_t nnz = 0;
  for (const auto& s : sets) nnz += (int64_t)s.size();
  out->n = n;
  out->nnz = nnz;
  out->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  out->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t pos = 0;
  std::vector<uint32_t> row;
  for (int64_t i = 0; i < n; ++i) {
    out->row_ptr[i] = pos;
    row.assign(sets[i].begin(), sets[i].end());
    std::sort(row.begin(), row.end());
    for (uint32_t j : row) out->col[pos++] = (int32_t)j;
  }
  out->row_ptr[n] = pos;
}

// Insert the unordered pair {i, j}, i != j, into the array of unordered sets: slot min
// holds max (Sec. III-B).
void report(std::vector<std::unordered_set<uint32_t>>& sets, uint32_t i, uint32_t j) {
  if (MUTANT(6)) {  // planted mistake: pair stored under the larger index
    sets[std::max(i, j)].insert(std::min(i, j));
    return;
  }
  sets[std::min(i, j)].insert(std::max(i, j));
}

}  // namespace

extern "C" {

// All pairs i < j with dist2 <= fl(r*r), by checking every pair (Sec. I problem statement).
int oracle_brute(const void* pts, int dtype, int64_t n, int d, double r, oracle_csr* out) {
  if (n < 0 || d < 1 || !out) return -1;
  std::vector<double> p = widen(pts, dtype, n, d);
  const double rr = r * r;
  std::vector<std::unordered_set<uint32_t>> sets((size_t)n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      if (within(dist2(&p[(size_t)i * d], &p[(size_t)j * d], d), rr))
        sets[(size_t)i].insert((uint32_t)j);
  to_csr(sets, out);
  return 0;
}

// The same set as oracle_brute, through a fixed grid of side r: two points at distance at
// most r lie in the same cell or in adjacent ones (offsets in {-1,0,1}^d).  Each pair of
// cells is visited once (offset lexicographically positive, or the cell with itself).
int oracle_exact_grid(const void* pts, int dtype, int64_t n, int d, double r, oracle_csr* out) {
  if (n < 0 || d < 1 || d > 16 || !out || !(r > 0)) return -1;
  std::vector<double> p = widen(pts, dtype, n, d);
  const double rr = r * r;
  std::map<std::vector<int64_t>, std::vector<uint32_t>> grid;
  std::vector<int64_t> q(d);
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < d; ++k) q[k] = (int64_t)std::floor(p[(size_t)i * d + k] / r);
    grid[q].push_back((uint32_t)i);
  }
  std::vector<std::unordered_set<uint32_t>> sets((size_t)n);
  int64_t noff = 1;
  for (int k = 0; k < d; ++k) noff *= 3;
  std::vector<int64_t> off(d), nb(d);
  for (const auto& cell : grid) {
    const auto& A = cell.second;
    for (size_t a = 0; a < A.size(); ++a)
      for (size_t b = a + 1; b < A.size(); ++b)
        if (within(dist2(&p[(size_t)A[a] * d], &p[(size_t)A[b] * d], d), rr))
          report(sets, A[a], A[b]);
    for (int64_t o = 0; o < noff; ++o) {
      int64_t t = o;
      for (int k = 0; k < d; ++k) {
        off[k] = t % 3 - 1;
        t /= 3;
      }
      // keep offsets whose first non-zero entry (from axis 0) is positive
      int first = 0;
      for (int k = 0; k < d; ++k)
        if (off[k] != 0) {
          first = off[k] > 0 ? 1 : -1;
          break;
        }
      if (first <= 0) continue;
      for (int k = 0; k < d; ++k) nb[k] = cell.first[k] + off[k];
      auto it = grid.find(nb);
      if (it == grid.end()) continue;
      const auto& B = it->second;
      for (uint32_t ia : A)
        for (uint32_t ib : B)
          if (within(dist2(&p[(size_t)ia * d], &p[(size_t)ib * d], d), rr)) report(sets, ia, ib);
    }
  }
  to_csr(sets, out);
  return 0;
}

// The point-to-cell step of Alg. 1 for every grid: q_out[(t*n + i)*d + k] is the cell
// coordinate of point i on axis k in grid t.  near_wall_out (optional, m entries) counts near-wall points.
int oracle_cells(const void* pts, int dtype, int64_t n, int d, const double* T, int m, double c,
                 int64_t* q_out, int64_t* near_wall_out) {
  if (n < 0 || d < 1 || d > 16 || m < 1 || !(c > 0) || !T || !q_out) return -1;
  std::vector<double> p = widen(pts, dtype, n, d);
  const int stride = d * d + d;
  for (int t = 0; t < m; ++t) {
    const double* R = T + (size_t)t * stride;
    const double* s = R + d * d;
    int64_t near = 0;
    for (int64_t i = 0; i < n; ++i)
      near += cell_of(&p[(size_t)i * d], R, s, d, c, &q_out[((size_t)t * n + i) * d]) ? 1 : 0;
    if (near_wall_out) near_wall_out[t] = near;
  }
  return 0;
}

// Alg. 1 (randomly transformed grids), with the array-of-unordered-sets dedupe of
// Sec. III-B.  stats (optional) receives one record per grid; near_r_out (optional) the
// number of distinct co-located pairs with |sqrt(s) - r| <= 1e-12 r.
int oracle_rtg(const void* pts, int dtype, int64_t n, int d, double r, const double* T, int m,
               double c, oracle_csr* out, oracle_grid_stats* stats, int64_t* near_r_out) {
  if (n < 0 || d < 1 || d > 16 || m < 1 || !(c > 0) || !(r > 0) || !T || !out) return -1;
  std::vector<double> p = widen(pts, dtype, n, d);
  const double rr = r * r;
  const int stride = d * d + d;
  std::vector<std::unordered_set<uint32_t>> sets((size_t)n);
  std::vector<std::unordered_set<uint32_t>> colocated;  // for the near-r diagnostic only
  if (near_r_out) colocated.resize((size_t)n);
  int64_t near_r = 0;
  std::vector<int64_t> q(d);
  const int grids = MUTANT(7) ? (m > 1 ? m - 1 : 1) : m;  // mutant 7: last grid skipped
  for (int t = 0; t < grids; ++t) {
    const double* R = T + (size_t)t * stride;
    const double* s = R + d * d;
    // Alg. 1: the set U of non-empty cells and the association of points to cells
    std::map<std::vector<int64_t>, std::vector<uint32_t>> U;
    int64_t near_wall = 0;
    for (int64_t i = 0; i < n; ++i) {
      near_wall += cell_of(&p[(size_t)i * d], R, s, d, c, q.data()) ? 1 : 0;
      U[q].push_back((uint32_t)i);
    }
    // Alg. 1: all pairs inside each non-empty cell, reported if at distance <= r
    int64_t candidates = 0, multi = 0, maxc = 0, reported = 0;
    for (const auto& cell : U) {
      const auto& A = cell.second;
      int64_t sz = (int64_t)A.size();
      candidates += sz * (sz - 1) / 2;
      multi += sz >= 2 ? 1 : 0;
      maxc = std::max(maxc, sz);
      for (int64_t a = 0; a < sz; ++a)
        for (int64_t b = MUTANT(8) ? a : a + 1; b < sz; ++b) {  // mutant 8: self-pairs
          double s2 = dist2(&p[(size_t)A[a] * d], &p[(size_t)A[b] * d], d);
          if (near_r_out) {
            uint32_t lo = std::min(A[a], A[b]), hi = std::max(A[a], A[b]);
            if (colocated[lo].insert(hi).second &&
                std::fabs(std::sqrt(s2) - r) <= 1e-12 * r)
              ++near_r;
          }
          if (within(s2, rr)) {
            ++reported;
            report(sets, A[a], A[b]);
          }
        }
    }
    if (stats) {
      stats[t].candidates = candidates;
      stats[t].nonempty_cells = (int64_t)U.size();
      stats[t].multi_cells = multi;
      stats[t].max_cell = maxc;
      stats[t].near_wall = near_wall;
      stats[t].reported = reported;
    }
  }
  if (near_r_out) *near_r_out = near_r;
  to_csr(sets, out);
  return 0;
}

// Alg. 1 as in oracle_rtg, on `threads` host threads (0: one per hardware thread).  Worker w
// takes grids w, w + threads, ...; each grid's reported pairs (lo << 32 | hi) go to its own
// list.  The lists are then merged into the array of unordered sets by row ranges, worker w
// owning rows [w n / threads, (w + 1) n / threads).  The set of pairs, and so the CSR, is the
// one oracle_rtg returns.
int oracle_rtg_threads(const void* pts, int dtype, int64_t n, int d, double r, const double* T,
                       int m, double c, int threads, oracle_csr* out) {
  if (n < 0 || d < 1 || d > 16 || m < 1 || !(c > 0) || !(r > 0) || !T || !out) return -1;
  if (threads <= 0) threads = (int)std::thread::hardware_concurrency();
  if (threads <= 0) threads = 1;
  std::vector<double> p = widen(pts, dtype, n, d);
  const double rr = r * r;
  const int stride = d * d + d;
  const int grids = MUTANT(7) ? (m > 1 ? m - 1 : 1) : m;
  std::vector<std::vector<uint64_t>> found((size_t)grids);
  auto grid_worker = [&](int w) {
    std::vector<int64_t> q(d);
    for (int t = w; t < grids; t += threads) {
      const double* R = T + (size_t)t * stride;
      const double* s = R + d * d;
      std::map<std::vector<int64_t>, std::vector<uint32_t>> U;
      for (int64_t i = 0; i < n; ++i) {
        cell_of(&p[(size_t)i * d], R, s, d, c, q.data());
        U[q].push_back((uint32_t)i);
      }
      std::vector<uint64_t>& F = found[(size_t)t];
      for (const auto& cell : U) {
        const auto& A = cell.second;
        const size_t sz = A.size();
        for (size_t a = 0; a < sz; ++a)
          for (size_t b = MUTANT(8) ? a : a + 1; b < sz; ++b)
            if (within(dist2(&p[(size_t)A[a] * d], &p[(size_t)A[b] * d], d), rr)) {
              uint32_t lo = std::min(A[a], A[b]), hi = std::max(A[a], A[b]);
              if (MUTANT(6)) std::swap(lo, hi);
              F.push_back(((uint64_t)lo << 32) | hi);
            }
      }
    }
  };
  std::vector<std::unordered_set<uint32_t>> sets((size_t)n);
  auto merge_worker = [&](int w) {
    const uint64_t lo = (uint64_t)((__int128)n * w / threads);
    const uint64_t hi = (uint64_t)((__int128)n * (w + 1) / threads);
    for (const auto& F : found)
      for (uint64_t pr : F) {
        const uint64_t i = pr >> 32;
        if (i >= lo && i < hi) sets[(size_t)i].insert((uint32_t)pr);
      }
  };
  auto run = [&](auto&& fn) {
    std::vector<std::thread> pool;
    for (int w = 1; w < threads; ++w) pool.emplace_back(fn, w);
    fn(0);
    for (auto& th : pool) th.join();
  };
  run(grid_worker);
  run(merge_worker);
  to_csr(sets, out);
  return 0;
}

// An r-NN query of a point x that need not belong to P, answered from the m stored grids
// (the single-query use of the grids in the conclusion, Sec. V): the answer is every point p
// of P with dist2(x, p) <= fl(r*r) that shares a cell with x in at least one grid, the cells
// being those of the point-to-cell step of Alg. 1 for x and for p alike.  Row k of out lists
// the answers to query k, ascending.
int oracle_rtg_query(const void* pts, int dtype, int64_t n, int d, double r, const double* T,
                     int m, double c, const void* queries, int64_t nq, oracle_csr* out) {
  if (n < 0 || nq < 0 || d < 1 || d > 16 || m < 1 || !(c > 0) || !(r > 0) || !T || !out)
    return -1;
  std::vector<double> p = widen(pts, dtype, n, d);
  std::vector<double> x = widen(queries, dtype, nq, d);
  const double rr = r * r;
  const int stride = d * d + d;
  std::vector<std::unordered_set<uint32_t>> sets((size_t)nq);
  std::vector<int64_t> q(d);
  const int grids = MUTANT(9) ? 1 : m;  // mutant 9: a query sees only the first grid
  for (int t = 0; t < grids; ++t) {
    const double* R = T + (size_t)t * stride;
    const double* s = R + d * d;
    std::map<std::vector<int64_t>, std::vector<uint32_t>> U;
    for (int64_t i = 0; i < n; ++i) {
      cell_of(&p[(size_t)i * d], R, s, d, c, q.data());
      U[q].push_back((uint32_t)i);
    }
    for (int64_t k = 0; k < nq; ++k) {
      cell_of(&x[(size_t)k * d], R, s, d, c, q.data());
      const auto it = U.find(q);
      if (it == U.end()) continue;
      for (uint32_t j : it->second)
        if (within(dist2(&x[(size_t)k * d], &p[(size_t)j * d], d), rr)) sets[(size_t)k].insert(j);
    }
  }
  to_csr(sets, out);
  return 0;
}

int oracle_mutant(void) { return ORACLE_MUTANT; }

}  // extern "C"
