// r-nearest-neighbour queries of new points from the m stored grids: the single-query use of
// randomly transformed grids that Sec. V of arXiv:1409.8112 describes (keep all m grids; for
// a query point, examine the m cells that contain it and report the points among them that lie
// within r).
//
// An index keeps what a build of Alg. 1 leaves on the device: the composite cell keys of every
// (point, grid) sorted with their point indices, the per-point key rows, the FP32 rows, the
// FP64 points and the plan (FP32 rotations, error bounds, key ranges and strides, distance
// band).  A query takes the same steps as the build for one more point:
//   * its cell in grid t: the FP32 rotation with the proven bound E, the FP64 reference
//     sequence where the bound leaves the cell open (or for every axis when the query lies
//     outside the indexed points' bounding box, where E does not hold); a cell outside the
//     planned key range holds no point;
//   * the cell's run in the sorted keys, from a per-grid open-addressing hash table built with
//     the index (cell key -> first position and length of its run; one or two probes);
//   * each candidate j: FP32 squared distance outside the band decides, else the FP64 sequence
//     on the original coordinates (the band likewise only inside the bounding box);
//   * j is reported by the first grid that puts it in the query's cell (the dedupe of
//     Sec. III-B by key rows), so every answer appears once.
// One thread per query for indexes of light cells, one warp per query (32 candidates at a time)
// for dense ones.  Two passes: count the answers, scan the counts into row pointers, write the
// answers, then sort each row (the pair path's row sort).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "rtg_host.h"

struct rtg_index {
  const rtg_ctx* owner = nullptr;  // the context that made it (its pool holds the memory)
  int64_t n = 0;
  int d = 0, m = 0, dtype = 0, dpad = 4;
  bool key64 = false;
  long long N = 0;
  void* mem = nullptr;  // one allocation from the context's pool, carved below
  size_t bytes = 0;
  uint64_t handle = 0;
  void* pts = nullptr;
  float* pf = nullptr;
  void* key_mat = nullptr;
  void* skeys = nullptr;
  uint32_t* svals = nullptr;
  rtg::Inst* inst = nullptr;
  rtg::InstPlan* iplan = nullptr;
  rtg::GridPlan* gplan = nullptr;
  double* T64 = nullptr;
  unsigned long long* table = nullptr;  // m open-addressing tables of table_cap slots
  long long table_cap = 0;              // slots per grid (a power of two, at least 2 n)
  bool thread_queries = true;  // light cells: one thread per query, else one warp per query
  double box_lo[rtg::kMaxDim] = {}, box_hi[rtg::kMaxDim] = {};
};

namespace rtg {

namespace {

constexpr int kIndexThreads = 256;

// Bounding box of the indexed points (inside it the FP32 bounds of the plan hold).
struct QueryBox {
  double lo[kMaxDim], hi[kMaxDim];
};

__device__ __forceinline__ double coord(const void* p, int dtype, long long i, int d, int l) {
  return dtype == 0 ? __ldg((const double*)p + i * d + l)
                    : (double)__ldg((const float*)p + i * d + l);
}

// Cell index of the query on axis k of grid t by the FP64 reference sequence (fixed order,
// fused multiply-add, IEEE division), as for the indexed points; false when the index does not
// fit 62 bits (far from every indexed cell).
__device__ bool exact_axis(const void* q, int dtype, long long k_query, int d, const double* Tt,
                           int k, double c, long long* cell) {
  double acc = Tt[d * d + k];
  for (int l = 0; l < d; ++l) acc = __fma_rn(Tt[k * d + l], coord(q, dtype, k_query, d, l), acc);
  const double f = floor(__ddiv_rn(acc, c));
  if (!(fabs(f) < 0x1.0p62)) return false;
  *cell = (long long)f;
  return true;
}

// Composite key of the query's cell in grid t; false when the cell lies outside the planned
// key range (no indexed point is there).
template <typename K, int DPAD>
__device__ bool query_key(const float* qf, bool in_box, const void* q, int dtype, long long kq,
                          const Inst& I, const GridPlan& G, const double* Tt, K* key) {
  const int d = I.d;
  K acc = (K)G.base;
  bool ok = true;
  for (int k = 0; k < d; ++k) {
    long long cell;
    bool certain = false;
    if (in_box) {
      float y = G.sf[k];
#pragma unroll
      for (int l = 0; l < DPAD; ++l) y = fmaf(G.Rf[k * kMaxDim + l], qf[l], y);
      const float u = y * I.inv_cf;
      const float f = floorf(u);
      certain = __fsub_rd(u, G.E[k]) >= f && __fadd_ru(u, G.E[k]) < f + 1.0f;
      cell = (long long)(int)f;
    }
    if (!certain && !exact_axis(q, dtype, kq, d, Tt, k, I.c, &cell)) {
      ok = false;
      continue;
    }
    const long long off = cell - G.qlo[k];
    if ((unsigned long long)off >= G.ext[k]) ok = false;
    else acc += (K)off * (K)G.stride[k];
  }
  *key = acc;
  return ok;
}

constexpr unsigned long long kEmptySlot = ~0ull;

// Slot of a cell key in its grid's table (the splitmix64 finalizer as the mixing function).
__device__ __forceinline__ unsigned long long key_hash(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// One thread per sorted position: the head of every run of equal keys enters its grid's table
// as (first position << 32) | length.  Grid t of the single indexed instance owns positions
// [t n, (t + 1) n) of the sort.
template <typename K>
__global__ void __launch_bounds__(256) k_index_table(const K* __restrict__ skeys, long long n,
                                                     int m, unsigned long long* table,
                                                     long long cap, unsigned int* errors) {
  const long long N = n * m;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    const long long t = p / n, g0 = t * n, g1 = g0 + n;
    const K key = skeys[p];
    if (p > g0 && skeys[p - 1] == key) continue;  // not a run head
    // run end: galloping, then bisection (runs of a large cell can be long)
    long long lo = p + 1, step = 1, hi = lo;
    while (true) {
      hi = lo + step;
      if (hi >= g1) {
        hi = g1;
        break;
      }
      if (skeys[hi] != key) break;
      lo = hi + 1;
      step <<= 1;
    }
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (skeys[mid] == key) lo = mid + 1; else hi = mid;
    }
    const unsigned long long word = ((unsigned long long)p << 32) | (unsigned long long)(lo - p);
    unsigned long long* tab = table + t * cap;
    unsigned long long slot = key_hash((unsigned long long)key) & (unsigned long long)(cap - 1);
    bool placed = false;
    for (long long probe = 0; probe < cap; ++probe) {  // at most half full: ends early
      if (atomicCAS(tab + slot, kEmptySlot, word) == kEmptySlot) {
        placed = true;
        break;
      }
      slot = (slot + 1) & (unsigned long long)(cap - 1);
    }
    if (!placed) atomicOr(errors, kErrLargeOverflow);
  }
}

// [first, end) of the run of `key` in grid t's part of the sort, or an empty range.
template <typename K>
__device__ __forceinline__ void find_run(const K* __restrict__ skeys,
                                         const unsigned long long* __restrict__ tab,
                                         long long cap, K key, long long* lo, long long* hi) {
  unsigned long long slot = key_hash((unsigned long long)key) & (unsigned long long)(cap - 1);
  *lo = *hi = 0;
  for (long long probe = 0; probe < cap; ++probe) {
    const unsigned long long w = __ldg(tab + slot);
    if (w == kEmptySlot) return;
    const long long first = (long long)(w >> 32);
    if (skeys[first] == key) {
      *lo = first;
      *hi = first + (long long)(w & 0xffffffffull);
      return;
    }
    slot = (slot + 1) & (unsigned long long)(cap - 1);
  }
}

// WRITE = false: row_cnt[k] = number of answers of query k.  WRITE = true: the answers go to
// row k in the order found (the row sort orders them).
template <typename K, int DPAD, bool WRITE>
__global__ void __launch_bounds__(kIndexThreads) k_index_query(
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const GridPlan* __restrict__ gplan, const double* __restrict__ T64,
    const K* __restrict__ skeys, const uint32_t* __restrict__ svals,
    const unsigned long long* __restrict__ table, long long cap,
    const K* __restrict__ key_mat, int m, const float* __restrict__ pf,
    const void* __restrict__ queries, int dtype, long long nq, QueryBox box,
    unsigned int* row_cnt, const OutSlot* out, Status* st) {
  const unsigned int full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const Inst I = inst[0];
  const InstPlan IP = iplan[0];
  const int d = I.d;
  const long long warps = (long long)gridDim.x * (kIndexThreads / 32);
  unsigned int rechecks = 0;
  for (long long kq = blockIdx.x * (long long)(kIndexThreads / 32) + (threadIdx.x >> 5); kq < nq;
       kq += warps) {
    // the query: FP32 row (as the build rounds the points), finiteness, inside the box
    float qf[DPAD];
    bool in_box = true, finite = true;
#pragma unroll
    for (int l = 0; l < DPAD; ++l) {
      qf[l] = 0.0f;
      if (l < d) {
        const double x = coord(queries, dtype, kq, d, l);
        finite &= isfinite(x);
        in_box &= x >= box.lo[l] && x <= box.hi[l];
        qf[l] = dtype == 0 ? __double2float_rn(x) : (float)x;
        finite &= isfinite(qf[l]);
      }
    }
    if (!finite) {
      if (lane == 0) {
        atomicOr(&st->errors, kErrNonFinite);
        if (!WRITE) row_cnt[kq] = 0u;
      }
      continue;
    }
    // grids t = lane and lane + 32: the query's key, and the run of that key in the sort
    K key0 = 0, key1 = 0;
    bool has0 = false, has1 = false;
    long long lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
    const int tstride = d * d + d;
    if (lane < m) {
      has0 = query_key<K, DPAD>(qf, in_box, queries, dtype, kq, I, gplan[lane],
                                T64 + I.T0 + (size_t)lane * tstride, &key0);
      if (has0) find_run(skeys, table + (long long)lane * cap, cap, key0, &lo0, &hi0);
    }
    if (lane + 32 < m) {
      has1 = query_key<K, DPAD>(qf, in_box, queries, dtype, kq, I, gplan[lane + 32],
                                T64 + I.T0 + (size_t)(lane + 32) * tstride, &key1);
      if (has1) find_run(skeys, table + (long long)(lane + 32) * cap, cap, key1, &lo1, &hi1);
    }
    const float2 band = IP.filter_on && in_box ? make_float2(IP.s_lo, IP.s_hi)
                                               : make_float2(-1.0f, __int_as_float(0x7f800000));
    unsigned int found = 0;  // answers so far (warp-uniform)
    long long obase = 0;
    if (WRITE) obase = out->row_ptr[kq];
    for (int t = 0; t < m; ++t) {
      const int src = t & 31;
      const long long lo = __shfl_sync(full, t < 32 ? lo0 : lo1, src);
      const long long hi = __shfl_sync(full, t < 32 ? hi0 : hi1, src);
      for (long long p0 = lo; p0 < hi; p0 += 32) {
        const long long pos = p0 + lane;
        bool keep = false;
        unsigned int j = 0;
        if (pos < hi) {
          j = svals[pos];
          // distance: FP32 outside the band, else the FP64 reference sequence
          float sf = 0.0f;
          const float4* pj = reinterpret_cast<const float4*>(pf + (size_t)j * DPAD);
#pragma unroll
          for (int v = 0; v < DPAD / 4; ++v) {
            const float4 y = __ldg(pj + v);
            float e = qf[4 * v] - y.x;
            sf = fmaf(e, e, sf);
            e = qf[4 * v + 1] - y.y;
            sf = fmaf(e, e, sf);
            e = qf[4 * v + 2] - y.z;
            sf = fmaf(e, e, sf);
            e = qf[4 * v + 3] - y.w;
            sf = fmaf(e, e, sf);
          }
          if (sf <= band.y) {
            if (sf < band.x) {
              keep = true;
            } else {
              double s = 0.0;
              for (int l = 0; l < d; ++l) {
                const double e = __dsub_rn(coord(queries, dtype, kq, d, l),
                                           coord(I.pts, dtype, (long long)j, d, l));
                s = __fma_rn(e, e, s);
              }
              keep = s <= IP.rr;
              ++rechecks;
            }
          }
        }
        // reported by the first grid that puts j in the query's cell
        for (int u = 0; u < t; ++u) {
          const K ku = __shfl_sync(full, u < 32 ? key0 : key1, u & 31);
          const bool hu = __shfl_sync(full, u < 32 ? has0 : has1, u & 31);
          if (keep && hu && key_mat[(size_t)j * m + u] == ku) keep = false;
        }
        const unsigned int mask = __ballot_sync(full, keep);
        if (WRITE && keep) out->col[obase + found + __popc(mask & ((1u << lane) - 1u))] = (int)j;
        found += (unsigned int)__popc(mask);
      }
    }
    if (!WRITE && lane == 0) row_cnt[kq] = found;
  }
  for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(full, rechecks, o);
  if (lane == 0 && rechecks) atomicAdd(&st->dist_rechecks, (unsigned long long)rechecks);
}

// One thread per query, for indexes whose cells hold few points (a warp per query would leave
// most lanes idle): the thread walks the m grids in order, keeping the query's keys for the
// first-grid rule, and writes its own row.
template <typename K, int DPAD, bool WRITE>
__global__ void __launch_bounds__(kIndexThreads) k_index_query_thread(
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const GridPlan* __restrict__ gplan, const double* __restrict__ T64,
    const K* __restrict__ skeys, const uint32_t* __restrict__ svals,
    const unsigned long long* __restrict__ table, long long cap,
    const K* __restrict__ key_mat, int m, const float* __restrict__ pf,
    const void* __restrict__ queries, int dtype, long long nq, QueryBox box,
    unsigned int* row_cnt, const OutSlot* out, Status* st) {
  const Inst I = inst[0];
  const InstPlan IP = iplan[0];
  const int d = I.d, tstride = d * d + d;
  unsigned int rechecks = 0;
  for (long long kq = blockIdx.x * (long long)blockDim.x + threadIdx.x; kq < nq;
       kq += (long long)gridDim.x * blockDim.x) {
    float qf[DPAD];
    bool in_box = true, finite = true;
#pragma unroll
    for (int l = 0; l < DPAD; ++l) {
      qf[l] = 0.0f;
      if (l < d) {
        const double x = coord(queries, dtype, kq, d, l);
        finite &= isfinite(x);
        in_box &= x >= box.lo[l] && x <= box.hi[l];
        qf[l] = dtype == 0 ? __double2float_rn(x) : (float)x;
        finite &= isfinite(qf[l]);
      }
    }
    if (!finite) {
      atomicOr(&st->errors, kErrNonFinite);
      if (!WRITE) row_cnt[kq] = 0u;
      continue;
    }
    const float2 band = IP.filter_on && in_box ? make_float2(IP.s_lo, IP.s_hi)
                                               : make_float2(-1.0f, __int_as_float(0x7f800000));
    K keyq[kMaxGrids];
    unsigned long long has = 0;  // grids whose planned range holds the query's cell
    unsigned int found = 0;
    long long obase = 0;
    if (WRITE) obase = out->row_ptr[kq];
    for (int t = 0; t < m; ++t) {
      if (!query_key<K, DPAD>(qf, in_box, queries, dtype, kq, I, gplan[t],
                              T64 + I.T0 + (size_t)t * tstride, &keyq[t]))
        continue;
      has |= 1ull << t;
      long long lo, hi;
      find_run(skeys, table + (long long)t * cap, cap, keyq[t], &lo, &hi);
      for (long long pos = lo; pos < hi; ++pos) {
        const unsigned int j = svals[pos];
        float sf = 0.0f;
        const float4* pj = reinterpret_cast<const float4*>(pf + (size_t)j * DPAD);
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) {
          const float4 y = __ldg(pj + v);
          float e = qf[4 * v] - y.x;
          sf = fmaf(e, e, sf);
          e = qf[4 * v + 1] - y.y;
          sf = fmaf(e, e, sf);
          e = qf[4 * v + 2] - y.z;
          sf = fmaf(e, e, sf);
          e = qf[4 * v + 3] - y.w;
          sf = fmaf(e, e, sf);
        }
        if (sf > band.y) continue;
        if (sf >= band.x) {
          double s2 = 0.0;
          for (int l = 0; l < d; ++l) {
            const double e = __dsub_rn(coord(queries, dtype, kq, d, l),
                                       coord(I.pts, dtype, (long long)j, d, l));
            s2 = __fma_rn(e, e, s2);
          }
          ++rechecks;
          if (!(s2 <= IP.rr)) continue;
        }
        // reported by the first grid that puts j in the query's cell
        bool earlier = false;
        for (int u = 0; u < t && !earlier; ++u)
          earlier = ((has >> u) & 1ull) && key_mat[(size_t)j * m + u] == keyq[u];
        if (earlier) continue;
        if (WRITE) out->col[obase + found] = (int)j;
        ++found;
      }
    }
    if (!WRITE) row_cnt[kq] = found;
  }
  for (int o = 16; o > 0; o >>= 1) rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
  if ((threadIdx.x & 31) == 0 && rechecks)
    atomicAdd(&st->dist_rechecks, (unsigned long long)rechecks);
}

template <typename K, int DPAD, bool WRITE>
void query_launch(const rtg_index* ix, const void* q, long long nq, const QueryBox& box,
                  unsigned int* row_cnt, const OutSlot* out, Status* st, int num_sms,
                  cudaStream_t s) {
  if (ix->thread_queries) {
    long long blocks = (nq + kIndexThreads - 1) / kIndexThreads;
    if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
    if (blocks < 1) blocks = 1;
    k_index_query_thread<K, DPAD, WRITE><<<(unsigned)blocks, kIndexThreads, 0, s>>>(
        ix->inst, ix->iplan, ix->gplan, ix->T64, (const K*)ix->skeys, ix->svals, ix->table,
        ix->table_cap, (const K*)ix->key_mat, ix->m, ix->pf, q, ix->dtype, nq, box, row_cnt,
        out, st);
    return;
  }
  long long blocks = (nq + kIndexThreads / 32 - 1) / (kIndexThreads / 32);
  if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
  if (blocks < 1) blocks = 1;
  k_index_query<K, DPAD, WRITE><<<(unsigned)blocks, kIndexThreads, 0, s>>>(
      ix->inst, ix->iplan, ix->gplan, ix->T64, (const K*)ix->skeys, ix->svals, ix->table,
      ix->table_cap,
      (const K*)ix->key_mat, ix->m, ix->pf, q, ix->dtype, nq, box, row_cnt, out, st);
}

template <bool WRITE>
void launch_index_query(const rtg_index* ix, const void* q, long long nq, const QueryBox& box,
                        unsigned int* row_cnt, const OutSlot* out, Status* st, int num_sms,
                        cudaStream_t s) {
#define RTG_IQ(K, P) query_launch<K, P, WRITE>(ix, q, nq, box, row_cnt, out, st, num_sms, s)
  if (ix->key64) {
    if (ix->dpad == 4) RTG_IQ(unsigned long long, 4);
    else if (ix->dpad == 8) RTG_IQ(unsigned long long, 8);
    else RTG_IQ(unsigned long long, 16);
  } else {
    if (ix->dpad == 4) RTG_IQ(uint32_t, 4);
    else if (ix->dpad == 8) RTG_IQ(uint32_t, 8);
    else RTG_IQ(uint32_t, 16);
  }
#undef RTG_IQ
}

}  // namespace

}  // namespace rtg

namespace rtghost {

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

rtg_status cuda_ok(rtg_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RTG_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? RTG_E_NOMEM : RTG_E_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

void free_index(rtg_ctx* c, rtg_index* ix) {
  if (ix->mem) cudaFreeAsync(ix->mem, c->stream);
  if (ix->handle) {
    std::lock_guard<std::mutex> lk(c->live_mu);
    auto it = c->live.find(ix->handle);
    if (it != c->live.end()) {
      c->out_bytes -= it->second;
      c->live.erase(it);
    }
  }
  delete ix;
}

}  // namespace

rtg_status index_create(rtg_ctx* c, const rtg_instance& it, int m, int dtype, int on_device,
                        rtg_index** out) {
  *out = nullptr;
  const cudaStream_t st = c->stream;
  // the grids of Alg. 1 for the points: one count-only build leaves the plan, the key rows and
  // the sorted keys in the context's workspace
  rtg_csr tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  const Request q{&it, 1, m, dtype, on_device, 0u, true, true};  // grid t at [t n, (t + 1) n)
  rtg_status s = build(c, q, &tmp);
  if (s != RTG_OK) return s;
  const int key_bits = tmp.stats.key_bits;
  // candidates per sorted position: about how many points share a cell with a query
  const double cand_per_pos =
      it.n > 0 ? (double)tmp.stats.total_candidates / ((double)it.n * m) : 0.0;
  release_out(c, &tmp);
  rtg_index* ix = new rtg_index();
  ix->owner = c;
  ix->n = it.n;
  ix->d = it.d;
  ix->m = m;
  ix->dtype = dtype;
  ix->dpad = rtg::dpad_for(it.d);
  ix->key64 = key_bits > 32;
  ix->N = (long long)it.n * m;
  ix->thread_queries = cand_per_pos < 4.0;
  if (it.n == 0) {  // nothing was planned: every query has an empty answer
    *out = ix;
    return RTG_OK;
  }
  const size_t esz = dtype == RTG_DTYPE_F64 ? 8 : 4, kb = ix->key64 ? 8 : 4;
  const size_t b_pts = align256((size_t)it.n * it.d * esz),
               b_pf = align256((size_t)it.n * ix->dpad * 4), b_kr = align256((size_t)ix->N * kb),
               b_sk = b_kr, b_sv = align256((size_t)ix->N * 4),
               b_inst = align256(sizeof(rtg::Inst)), b_ip = align256(sizeof(rtg::InstPlan)),
               b_gp = align256(sizeof(rtg::GridPlan) * (size_t)m),
               b_T = align256(sizeof(double) * (size_t)m * (it.d * it.d + it.d));
  long long cap = 1;
  while (cap < 2 * (long long)it.n) cap <<= 1;  // at most half full: short probe runs
  ix->table_cap = cap;
  const size_t b_tab = align256(sizeof(unsigned long long) * (size_t)cap * m);
  const size_t total = b_pts + b_pf + b_kr + b_sk + b_sv + b_inst + b_ip + b_gp + b_T + b_tab;
  if ((s = alloc_out_on(c, c->stream, total, &ix->mem)) != RTG_OK) {
    delete ix;
    return s;
  }
  ix->bytes = total;
  ix->handle = register_out(c, total);
  char* p = (char*)ix->mem;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += bytes;
    return (void*)r;
  };
  ix->pts = take(b_pts);
  ix->pf = (float*)take(b_pf);
  ix->key_mat = take(b_kr);
  ix->skeys = take(b_sk);
  ix->svals = (uint32_t*)take(b_sv);
  ix->inst = (rtg::Inst*)take(b_inst);
  ix->iplan = (rtg::InstPlan*)take(b_ip);
  ix->gplan = (rtg::GridPlan*)take(b_gp);
  ix->T64 = (double*)take(b_T);
  ix->table = (unsigned long long*)take(b_tab);
  rtg::Inst I = c->h_inst[0];
  const void* src_pts = I.pts;
  I.pts = ix->pts;
  I.p0 = 0;
  I.T0 = 0;
  unsigned long long hb[2 * rtg::kMaxDim];
  const int sorted = c->last_sorted;
  auto copy = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    return cuda_ok(c, cudaMemcpyAsync(dst, src, bytes, kind, st), "index copy");
  };
  const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
  if ((s = copy(ix->pts, src_pts, (size_t)it.n * it.d * esz, d2d)) != RTG_OK ||
      (s = copy(ix->pf, c->pf.p, (size_t)it.n * ix->dpad * 4, d2d)) != RTG_OK ||
      (s = copy(ix->key_mat, c->key_mat.p, (size_t)ix->N * kb, d2d)) != RTG_OK ||
      (s = copy(ix->skeys, sorted ? c->keys1.p : c->keys0.p, (size_t)ix->N * kb,
                cudaMemcpyDeviceToDevice)) != RTG_OK ||
      (s = copy(ix->svals, sorted ? c->vals1.p : c->vals0.p, (size_t)ix->N * 4,
                cudaMemcpyDeviceToDevice)) != RTG_OK ||
      (s = copy(ix->iplan, c->iplan.p, sizeof(rtg::InstPlan), d2d)) != RTG_OK ||
      (s = copy(ix->gplan, c->gplan.p, sizeof(rtg::GridPlan) * (size_t)m,
                cudaMemcpyDeviceToDevice)) != RTG_OK ||
      (s = copy(ix->T64, c->T64.p, sizeof(double) * (size_t)m * (it.d * it.d + it.d),
                cudaMemcpyDeviceToDevice)) != RTG_OK ||
      (s = copy(ix->inst, &I, sizeof(I), cudaMemcpyHostToDevice)) != RTG_OK ||
      (s = copy(hb, bbox_of(c), sizeof(hb), cudaMemcpyDeviceToHost)) != RTG_OK ||
      (s = cuda_ok(c, cudaMemsetAsync(ix->table, 0xff, sizeof(unsigned long long) * (size_t)cap * m,
                                      st),
                   "index table")) != RTG_OK ||
      (s = cuda_ok(c, cudaMemsetAsync(&((rtg::Status*)c->status.p)->errors, 0,
                                      sizeof(unsigned int), st),
                   "index table")) != RTG_OK) {
    free_index(c, ix);
    return s;
  }
  {
    long long blocks = (ix->N + 255) / 256;
    if (blocks > 16LL * c->num_sms) blocks = 16LL * c->num_sms;
    unsigned int* errors = &((rtg::Status*)c->status.p)->errors;
    if (ix->key64)
      rtg::k_index_table<unsigned long long><<<(unsigned)blocks, 256, 0, st>>>(
          (const unsigned long long*)ix->skeys, it.n, m, ix->table, cap, errors);
    else
      rtg::k_index_table<uint32_t><<<(unsigned)blocks, 256, 0, st>>>(
          (const uint32_t*)ix->skeys, it.n, m, ix->table, cap, errors);
  }
  if ((s = cuda_ok(c, cudaGetLastError(), "index table")) != RTG_OK ||
      (s = read_status(c)) != RTG_OK || (s = check_errors(c, ~0u)) != RTG_OK) {
    free_index(c, ix);
    return s;
  }
  for (int l = 0; l < rtg::kMaxDim; ++l) {
    ix->box_hi[l] = rtg::dec_double(hb[2 * l]);
    ix->box_lo[l] = rtg::dec_double(~hb[2 * l + 1]);
  }
  *out = ix;
  return RTG_OK;
}

rtg_status index_query(rtg_ctx* c, const rtg_index* ix, const void* queries, int on_device,
                       int64_t nq, rtg_csr* out) {
  const cudaStream_t st = c->stream;
  std::memset(out, 0, sizeof(*out));
  if (ix->owner != c) return fail(c, RTG_E_INVALID, "the index belongs to another context");
  rtg_status s;
  void* rp = nullptr;
  if ((s = alloc_out_on(c, st, sizeof(int64_t) * (size_t)(nq + 1), &rp)) != RTG_OK) return s;
  out->row_ptr = (int64_t*)rp;
  out->handle = register_out(c, sizeof(int64_t) * (size_t)(nq + 1));
  out->n = nq;
  if (nq == 0 || ix->n == 0 || ix->m == 0) {
    if ((s = cuda_ok(c, cudaMemsetAsync(rp, 0, sizeof(int64_t) * (size_t)(nq + 1), st),
                     "cudaMemsetAsync")) != RTG_OK ||
        (s = cuda_ok(c, cudaStreamSynchronize(st), "cudaStreamSynchronize")) != RTG_OK)
      release_out(c, out);
    return s;
  }
  const size_t esz = ix->dtype == RTG_DTYPE_F64 ? 8 : 4;
  const size_t stat_bytes = (sizeof(rtg::Status) + 255) & ~size_t(255);
  if ((s = ensure(c, c->status, stat_bytes)) != RTG_OK ||
      (s = ensure(c, c->row_cnt, (size_t)nq * 4)) != RTG_OK ||
      (s = ensure(c, c->scan_lb, ((size_t)nq / 4096 + 2) * 8)) != RTG_OK ||
      (s = ensure(c, c->out_slot, sizeof(rtg::OutSlot))) != RTG_OK ||
      (!on_device && (s = ensure(c, c->pts, (size_t)nq * ix->d * esz)) != RTG_OK)) {
    release_out(c, out);
    return s;
  }
  const void* q = queries;
  if (!on_device) {
    if ((s = cuda_ok(c, cudaMemcpyAsync(c->pts.p, queries, (size_t)nq * ix->d * esz,
                                        cudaMemcpyHostToDevice, st),
                     "cudaMemcpyAsync")) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    q = c->pts.p;
  }
  rtg::QueryBox box;
  for (int l = 0; l < rtg::kMaxDim; ++l) {
    box.lo[l] = ix->box_lo[l];
    box.hi[l] = ix->box_hi[l];
  }
  rtg::BuildArgs a{};
  a.st = (rtg::Status*)c->status.p;
  a.row_cnt = (unsigned int*)c->row_cnt.p;
  a.scan_lookback = (unsigned long long*)c->scan_lb.p;
  a.out = (const rtg::OutSlot*)c->out_slot.p;
  a.n_total = nq;
  a.num_sms = c->num_sms;
  c->h_slot->row_ptr = (long long*)rp;
  c->h_slot->col = nullptr;
  c->h_slot->col_cap = 0;
  cudaMemsetAsync(a.st, 0, sizeof(rtg::Status), st);
  cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice, st);
  rtg::launch_index_query<false>(ix, q, nq, box, a.row_cnt, a.out, a.st, c->num_sms, st);
  rtg::launch_scan(a, st);
  if ((s = cuda_ok(c, cudaGetLastError(), "index query")) != RTG_OK ||
      (s = read_status(c)) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  if ((s = check_errors(c, ~0u)) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  const long long nnz = (long long)c->h_status->nnz;
  if (nnz > 0) {
    void* cp = nullptr;
    if ((s = alloc_out_on(c, st, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    out->col = (int32_t*)cp;
    {
      std::lock_guard<std::mutex> lk(c->live_mu);
      c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
    }
    c->h_slot->col = (int*)cp;
    c->h_slot->col_cap = nnz;
    cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice, st);
    rtg::launch_index_query<true>(ix, q, nq, box, a.row_cnt, a.out, a.st, c->num_sms, st);
    rtg::launch_rowsort(a, st, ix->n);  // answers are indexed-point indices
  }
  if ((s = cuda_ok(c, cudaGetLastError(), "index query")) != RTG_OK ||
      (s = read_status(c)) != RTG_OK || (s = check_errors(c, ~0u)) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  out->nnz = nnz;
  out->symmetric = 0;
  return RTG_OK;
}

void index_destroy(rtg_ctx* c, rtg_index* ix) {
  if (ix->owner != c) return;  // not this context's: its owner frees it
  free_index(c, ix);
  cudaStreamSynchronize(c->stream);
}

}  // namespace rtghost
