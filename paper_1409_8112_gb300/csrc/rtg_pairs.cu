// In-cell pair enumeration and CSR assembly (Alg. 1 lines 8-9 and the dedupe of Sec. III-B
// of arXiv:1409.8112), for a batch of instances.
//
// After the sort every (instance, grid, cell) is a run of equal keys.  A block owns the cells
// whose first position lies in its slice of kSlice sorted positions: it finds them with
// adjacent key comparisons, stages their points (FP32, padded rows) in shared memory and walks
// all pairs (a < b) of every cell with at most kSmax points as one flat candidate range.  Cells
// with more points go to the tiled large-cell kernel.
//
// Dedupe without an auxiliary set: the distance test does not depend on the grid, so pair
// {i, j} is reported by grid t iff it is within r and shares a cell in t.  The pair is
// therefore emitted only by the first grid that puts i and j in one cell; a candidate in
// grid t is dropped when key_mat[i][t'] == key_mat[j][t'] for some t' < t.  The check runs
// before the distance (the filtering use of the auxiliary structure in Sec. III-B).
//
// Distance: FP32 on the staged rows; a pair is decided in FP32 only when the FP32 squared
// distance is outside [s_lo, s_hi], the proven error band around fl(r*r) (see the plan
// kernel); otherwise the FP64 reference sequence decides.
//
// Modes: EMIT writes reported pairs to a pair buffer (one atomic per warp) and counts rows;
// after the scan, scatter places them.  COUNT then WRITE enumerates twice and needs no pair
// buffer (for outputs too large to hold twice).  Rows are sorted at the end.
#include <cuda_runtime.h>

#include <climits>

#include "rtg_internal.cuh"

namespace rtg {

namespace {

constexpr int kSlice = 512;
constexpr int kSmax = 128;
constexpr int kPairThreads = 256;
constexpr int kStage = kSlice + kSmax;
constexpr int kKeyWin = kSlice + kSmax + 2;
constexpr unsigned int kUnknown = 0xffffffffu;
constexpr int kTL = 128;  // large-cell tile
constexpr unsigned int kSpinLimit = 1u << 22;

__device__ __forceinline__ double load_coord(const void* pts, int dtype, long long i, int d,
                                             int l) {
  return dtype == 0 ? __ldg((const double*)pts + i * d + l)
                    : (double)__ldg((const float*)pts + i * d + l);
}

// FP64 reference squared distance (fixed order, fused multiply-add, original coordinates).
__device__ __noinline__ double exact_dist2(const void* pts, int dtype, long long i, long long j,
                                           int d) {
  double s = 0.0;
  for (int l = 0; l < d; ++l) {
    const double e = __dsub_rn(load_coord(pts, dtype, i, d, l), load_coord(pts, dtype, j, d, l));
    s = __fma_rn(e, e, s);
  }
  return s;
}

__device__ __forceinline__ unsigned int block_excl_scan(unsigned int v, unsigned int* total,
                                                        unsigned int* sbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sbuf[warp] = x;
  __syncthreads();
  unsigned int wpre = 0, tot = 0;
  for (int w = 0; w < nw; ++w) {
    const unsigned int c = sbuf[w];
    if (w < warp) wpre += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return wpre + x - v;
}

__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v,
                                                                unsigned long long* total,
                                                                unsigned long long* sbuf) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sbuf[warp] = x;
  __syncthreads();
  unsigned long long wpre = 0, tot = 0;
  for (int w = 0; w < nw; ++w) {
    const unsigned long long c = sbuf[w];
    if (w < warp) wpre += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return wpre + x - v;
}

// Per-thread tallies.
struct Tally {
  unsigned int owned = 0, rechecks = 0, near_r = 0, pairs = 0;
  bool overflow = false;
};

// Where the pairs go.
struct Sink {
  unsigned int* row_cnt;
  const long long* row_ptr;
  int* col;
  long long col_cap;
  unsigned long long* pair_buf;
  long long pair_cap;
  unsigned long long* emitted;
  int symmetric;
};

// Decide one candidate pair (i < j, global indices) of grid t of instance I; ki and kj are the
// two points' key rows (shared or global memory).
template <typename K, int DPAD, int MODE>
__device__ __forceinline__ bool decide_pair(unsigned int i, unsigned int j, int t, const float* pa,
                                            const float* pb, const K* ki, const K* kj,
                                            const Inst& I, const InstPlan& IP, int dtype,
                                            Tally& tl) {
  bool earlier = false;  // all loads issued before any test
#pragma unroll 8
  for (int u = 0; u < t; ++u) earlier |= ki[u] == kj[u];
  if (earlier) return false;  // an earlier grid owns this pair
  if (MODE != kWrite) ++tl.owned;
  float sf = 0.0f;
#pragma unroll
  for (int v = 0; v < DPAD / 4; ++v) {
    const float4 x = reinterpret_cast<const float4*>(pa)[v];
    const float4 y = reinterpret_cast<const float4*>(pb)[v];
    float e = x.x - y.x;
    sf = fmaf(e, e, sf);
    e = x.y - y.y;
    sf = fmaf(e, e, sf);
    e = x.z - y.z;
    sf = fmaf(e, e, sf);
    e = x.w - y.w;
    sf = fmaf(e, e, sf);
  }
  bool keep;
  if (IP.filter_on && sf < IP.s_lo) {
    keep = true;
  } else if (IP.filter_on && sf > IP.s_hi) {
    keep = false;
  } else {
    const double s = exact_dist2(I.pts, dtype, (long long)i - I.p0, (long long)j - I.p0, I.d);
    keep = s <= IP.rr;
    if (MODE != kWrite) {
      ++tl.rechecks;
      if (fabs(__dsub_rn(__dsqrt_rn(s), I.r)) <= __dmul_rn(1e-12, I.r)) ++tl.near_r;
    }
  }
  if (keep && MODE != kWrite) ++tl.pairs;
  return keep;
}

// Deliver a decided pair.  Called by all 32 lanes of a warp together (keep may be false).
template <int MODE>
__device__ __forceinline__ void deliver(bool keep, unsigned int i, unsigned int j, const Sink& sk,
                                        Tally& tl) {
  if (MODE == kEmit) {
    const unsigned int mask = __ballot_sync(0xffffffffu, keep);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(sk.emitted, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (keep) {
      const unsigned long long slot = base + __popc(mask & ((1u << lane) - 1));
      if ((long long)slot < sk.pair_cap) sk.pair_buf[slot] = ((unsigned long long)i << 32) | j;
      else tl.overflow = true;
      atomicAdd(&sk.row_cnt[i], 1u);
      if (sk.symmetric) atomicAdd(&sk.row_cnt[j], 1u);
    }
  } else if (MODE == kCount) {
    if (keep) {
      atomicAdd(&sk.row_cnt[i], 1u);
      if (sk.symmetric) atomicAdd(&sk.row_cnt[j], 1u);
    }
  } else {
    if (keep) {
      const long long pi = sk.row_ptr[i] + atomicAdd(&sk.row_cnt[i], 1u);
      if (pi < sk.col_cap) sk.col[pi] = (int)j; else tl.overflow = true;
      if (sk.symmetric) {
        const long long pj = sk.row_ptr[j] + atomicAdd(&sk.row_cnt[j], 1u);
        if (pj < sk.col_cap) sk.col[pj] = (int)i; else tl.overflow = true;
      }
    }
  }
}

template <int MODE>
__device__ __forceinline__ void flush_tally(const Tally& tl, Status* st, unsigned int* sbuf) {
  // sbuf: 4 block-wide counters, zeroed by the caller before its last barrier
  unsigned int v[4] = {tl.owned, tl.rechecks, tl.near_r, tl.pairs};
#pragma unroll
  for (int q = 0; q < 4; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (MODE != kWrite && (threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (v[q]) atomicAdd(&sbuf[q], v[q]);
  }
  if (__syncthreads_or(tl.overflow) && threadIdx.x == 0)
    atomicOr(&st->errors, MODE == kEmit ? kErrPairOverflow : kErrColOverflow);
  if (MODE == kWrite || threadIdx.x != 0) return;
  if (sbuf[0]) atomicAdd(&st->owned_candidates, (unsigned long long)sbuf[0]);
  if (sbuf[1]) atomicAdd(&st->dist_rechecks, (unsigned long long)sbuf[1]);
  if (sbuf[2]) atomicAdd(&st->near_r, (unsigned long long)sbuf[2]);
  if (sbuf[3]) atomicAdd(&st->pairs, (unsigned long long)sbuf[3]);
}

// (instance, grid) of a composite key: the last base <= key.
__device__ __forceinline__ int find_bt(unsigned long long key,
                                       const unsigned long long* __restrict__ bases, int nbt) {
  int lo = 0, hi = nbt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(bases + mid) <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Shared-memory key rows are staged when a row (m keys) is at most this many bytes.
constexpr int kMaxStagedRow = 64;

template <typename K, int DPAD, int MODE>
__global__ void __launch_bounds__(kPairThreads) k_pairs_small(
    const K* __restrict__ skeys, const uint32_t* __restrict__ svals, long long N,
    const float* __restrict__ pf, int dtype, const K* __restrict__ key_mat, int m,
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const unsigned long long* __restrict__ bases, int nbt, Status* st, Sink sk,
    LargeCell* large, unsigned int large_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_pt = reinterpret_cast<float*>(smem);                          // kStage * DPAD
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(s_pt + kStage * DPAD);    // kStage
  K* s_key = reinterpret_cast<K*>(s_idx + kStage);                       // kKeyWin
  unsigned int* c_start = reinterpret_cast<unsigned int*>(s_key + kKeyWin);  // kSlice + 1
  unsigned int* c_cand = c_start + kSlice + 1;                               // kSlice + 1
  unsigned int* c_bt = c_cand + kSlice + 1;                                  // kSlice
  K* s_rows = reinterpret_cast<K*>(c_bt + kSlice + (kSlice & 1));            // kStage * m (opt.)
  const bool stage_rows = m * (int)sizeof(K) <= kMaxStagedRow;
  __shared__ unsigned int s_end, s_stage_lo, s_stage_hi, s_total;
  __shared__ unsigned int sbuf[kPairThreads / 32];
  __shared__ unsigned int s_tally[4];
  __shared__ unsigned long long s_gcand[kMaxGrids];
  __shared__ unsigned long long s_maxcell;

  const int tid = threadIdx.x;
  const long long lo = (long long)blockIdx.x * kSlice;
  const long long hi = min(lo + kSlice, N);
  const long long win_end = min(hi + kSmax + 1, N);

  for (long long x = lo - 1 + tid; x < win_end; x += kPairThreads)
    if (x >= 0) s_key[x - lo + 1] = skeys[x];
  if (tid == 0) {
    s_end = kUnknown;
    s_maxcell = 0;
  }
  if (tid < 4) s_tally[tid] = 0;
  if (MODE != kWrite)
    for (int g = tid; g < kMaxGrids; g += kPairThreads) s_gcand[g] = 0;
  __syncthreads();
  auto is_head = [&](long long x) -> bool {
    return x == 0 || s_key[x - lo + 1] != s_key[x - lo];
  };
  for (long long x = hi + tid; x < win_end; x += kPairThreads)
    if (is_head(x)) atomicMin(&s_end, (unsigned int)(x - lo));
  constexpr int kPer = kSlice / kPairThreads;
  unsigned int flags = 0, cnt = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const long long x = lo + tid * kPer + q;
    if (x < hi && is_head(x)) {
      flags |= 1u << q;
      ++cnt;
    }
  }
  unsigned int ncells;
  unsigned int w = block_excl_scan(cnt, &ncells, sbuf);
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (flags & (1u << q)) c_start[w++] = (unsigned int)(tid * kPer + q);
  if (tid == 0) {
    const unsigned int end_rel =
        s_end != kUnknown ? s_end : (win_end == N ? (unsigned int)(N - lo) : kUnknown);
    c_start[ncells] = end_rel;
  }
  __syncthreads();
  if (ncells == 0) return;
  for (unsigned int e = tid; e < ncells; e += kPairThreads) {
    const unsigned int st_rel = c_start[e], en = c_start[e + 1];
    const K key = s_key[st_rel + 1];
    const int bt = find_bt((unsigned long long)key, bases, nbt);
    const int g = bt % m;
    c_bt[e] = (unsigned int)bt;
    unsigned long long size = en == kUnknown ? 0ull : (unsigned long long)(en - st_rel);
    unsigned int cand = 0;
    if (en == kUnknown || size > (unsigned long long)kSmax) {
      if (MODE != kWrite) {
        if (en == kUnknown) {
          long long a = win_end, b = N;  // the run continues past the window
          while (a < b) {
            const long long mid = (a + b) >> 1;
            if (skeys[mid] == key) a = mid + 1; else b = mid;
          }
          size = (unsigned long long)(a - (lo + st_rel));
        }
        const unsigned long long slot = atomicAdd(&st->large_cells, 1ull);
        if (slot < large_cap) {
          large[slot].start = (unsigned long long)(lo + st_rel);
          large[slot].size = (unsigned int)size;
          large[slot].grid = (unsigned short)g;
          large[slot].inst = (unsigned short)(bt / m);
        } else {
          atomicOr(&st->errors, kErrLargeOverflow);
        }
        atomicAdd(&s_gcand[g], size * (size - 1) / 2);
        atomicMax(&s_maxcell, size);
      }
    } else {
      cand = (unsigned int)(size * (size - 1) / 2);
      if (MODE != kWrite) {
        if (cand) atomicAdd(&s_gcand[g], (unsigned long long)cand);
        atomicMax(&s_maxcell, size);
      }
    }
    c_cand[e] = cand;
  }
  __syncthreads();
  {
    unsigned int v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const unsigned int e = tid * kPer + q;
      v[q] = e < ncells ? c_cand[e] : 0u;
      sum += v[q];
    }
    unsigned int total;
    unsigned int run = block_excl_scan(sum, &total, sbuf);
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const unsigned int e = tid * kPer + q;
      if (e < ncells) c_cand[e] = run;
      run += v[q];
    }
    if (tid == 0) {
      c_cand[ncells] = total;
      s_total = total;
      s_stage_lo = c_start[0];
      const unsigned int last = ncells - 1;
      const unsigned int en = c_start[ncells];
      const bool last_small = en != kUnknown && en - c_start[last] <= (unsigned int)kSmax;
      unsigned int shi = last_small ? en : c_start[last];
      if (shi > s_stage_lo + kStage) shi = s_stage_lo + kStage;
      s_stage_hi = shi;
    }
  }
  __syncthreads();
  if (MODE != kWrite) {
    if (tid < m && s_gcand[tid]) atomicAdd(&st->candidates[tid], s_gcand[tid]);
    if (tid == 0 && s_maxcell) atomicMax(&st->max_cell, s_maxcell);
  }
  const unsigned int T = s_total;
  Tally tl;
  if (T > 0) {
    const unsigned int stage_lo = s_stage_lo, nstage = s_stage_hi - s_stage_lo;
    for (unsigned int x = tid; x < nstage; x += kPairThreads) {
      const uint32_t idx = svals[lo + stage_lo + x];
      s_idx[x] = idx;
      const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
      float4* dst = reinterpret_cast<float4*>(s_pt + (size_t)x * DPAD);
#pragma unroll
      for (int v = 0; v < DPAD / 4; ++v) dst[v] = __ldg(src + v);
      if (stage_rows) {
        const K* kr = key_mat + (size_t)idx * m;
        for (int u = 0; u < m; ++u) s_rows[(size_t)x * m + u] = __ldg(kr + u);
      }
    }
    __syncthreads();
    // Each thread walks a contiguous run of `per` candidates, advancing (cell, a, b)
    // incrementally; all lanes of a warp make the same number of steps so that EMIT can
    // aggregate with ballots.
    const unsigned int per = (T + kPairThreads - 1) / kPairThreads;
    const unsigned int c0 = min(T, (unsigned int)tid * per), c1 = min(T, c0 + per);
    int el = 0;
    unsigned int a = 0, b = 1;
    if (c0 < c1) {
      int eh = (int)ncells - 1;
      while (el < eh) {
        const int mid = (el + eh + 1) >> 1;
        if (c_cand[mid] <= c0) el = mid; else eh = mid - 1;
      }
      const unsigned int l = c0 - c_cand[el];
      b = (unsigned int)((1.0f + sqrtf(8.0f * (float)l + 1.0f)) * 0.5f);
      while (b * (b - 1) / 2 > l) --b;
      while ((b + 1) * b / 2 <= l) ++b;
      a = l - b * (b - 1) / 2;
    }
    for (unsigned int step = 0; step < per; ++step) {
      const unsigned int c = c0 + step;
      bool keep = false;
      unsigned int i = 0, j = 0;
      if (c < c1) {
        while (c >= c_cand[el + 1]) {  // next cell with candidates
          ++el;
          a = 0;
          b = 1;
        }
        const unsigned int xa = c_start[el] + a - stage_lo, xb = c_start[el] + b - stage_lo;
        const unsigned int ia = s_idx[xa], ib = s_idx[xb];
        i = min(ia, ib);
        j = max(ia, ib);
        const unsigned int bt = c_bt[el];
        const int inst_b = (int)(bt / m);
        const K* ka = stage_rows ? s_rows + (size_t)xa * m : key_mat + (size_t)ia * m;
        const K* kb = stage_rows ? s_rows + (size_t)xb * m : key_mat + (size_t)ib * m;
        keep = decide_pair<K, DPAD, MODE>(i, j, (int)(bt % m), s_pt + (size_t)xa * DPAD,
                                          s_pt + (size_t)xb * DPAD, ka, kb, inst[inst_b],
                                          iplan[inst_b], dtype, tl);
        if (++a == b) {  // next pair of the cell in (b, a) order
          a = 0;
          ++b;
        }
      }
      deliver<MODE>(keep, i, j, sk, tl);
    }
  }
  flush_tally<MODE>(tl, st, s_tally);
}

// Job offsets for the large cells: cell e has ceil(size / kTL) row tiles.
__global__ void __launch_bounds__(1024) k_large_setup(const LargeCell* __restrict__ large,
                                                      unsigned int cap, Status* st,
                                                      unsigned long long* job_off) {
  __shared__ unsigned long long sbuf[32];
  __shared__ unsigned long long carry;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (unsigned long long base = 0; base < L; base += blockDim.x) {
    const unsigned long long e = base + threadIdx.x;
    const unsigned long long v = e < L ? (large[e].size + kTL - 1) / kTL : 0;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan64(v, &tot, sbuf);
    if (e < L) job_off[e] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    job_off[L] = carry;
    st->large_jobs = carry;
  }
}

template <typename K, int DPAD, int MODE>
__global__ void __launch_bounds__(kPairThreads) k_pairs_large(
    const uint32_t* __restrict__ svals, const float* __restrict__ pf, int dtype,
    const K* __restrict__ key_mat, int m, const Inst* __restrict__ inst,
    const InstPlan* __restrict__ iplan, Status* st, const LargeCell* __restrict__ large,
    unsigned int cap, const unsigned long long* job_off, Sink sk) {
  __shared__ __align__(16) float sa[kTL * DPAD];
  __shared__ __align__(16) float sb[kTL * DPAD];
  __shared__ uint32_t ia[kTL], ib[kTL];
  __shared__ unsigned int s_tally[4];
  if (threadIdx.x < 4) s_tally[threadIdx.x] = 0;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  const unsigned long long J = L ? job_off[L] : 0;
  const int lane = threadIdx.x & 31;
  Tally tl;
  for (unsigned long long job = blockIdx.x; job < J; job += gridDim.x) {
    long long el = 0, eh = (long long)L - 1;
    while (el < eh) {
      const long long mid = (el + eh + 1) >> 1;
      if (job_off[mid] <= job) el = mid; else eh = mid - 1;
    }
    const LargeCell cell = large[el];
    const Inst I = inst[cell.inst];
    const InstPlan IP = iplan[cell.inst];
    const unsigned int s = cell.size;
    const unsigned int a0 = (unsigned int)(job - job_off[el]) * kTL;
    const unsigned int na = min((unsigned int)kTL, s - a0);
    __syncthreads();
    for (unsigned int x = threadIdx.x; x < na; x += blockDim.x) {
      const uint32_t idx = svals[cell.start + a0 + x];
      ia[x] = idx;
      const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
      float4* dst = reinterpret_cast<float4*>(sa + x * DPAD);
#pragma unroll
      for (int v = 0; v < DPAD / 4; ++v) dst[v] = __ldg(src + v);
    }
    for (unsigned int b0 = a0; b0 < s; b0 += kTL) {
      const unsigned int nb = min((unsigned int)kTL, s - b0);
      __syncthreads();
      for (unsigned int x = threadIdx.x; x < nb; x += blockDim.x) {
        const uint32_t idx = svals[cell.start + b0 + x];
        ib[x] = idx;
        const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
        float4* dst = reinterpret_cast<float4*>(sb + x * DPAD);
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) dst[v] = __ldg(src + v);
      }
      __syncthreads();
      const unsigned int total = na * nb;
      for (unsigned int qb = threadIdx.x & ~31u; qb < total; qb += blockDim.x) {
        const unsigned int q = qb + lane;
        bool keep = false;
        unsigned int i = 0, j = 0;
        if (q < total) {
          const unsigned int x = q / nb, y = q % nb;
          if (a0 + x < b0 + y) {
            i = min(ia[x], ib[y]);
            j = max(ia[x], ib[y]);
            keep = decide_pair<K, DPAD, MODE>(i, j, (int)cell.grid, sa + x * DPAD, sb + y * DPAD,
                                              key_mat + (size_t)ia[x] * m,
                                              key_mat + (size_t)ib[y] * m, I, IP, dtype, tl);
          }
        }
        deliver<MODE>(keep, i, j, sk, tl);
      }
    }
  }
  __syncthreads();
  flush_tally<MODE>(tl, st, s_tally);
}

// Exact set of Sec. I: every pair (i < j) of one instance checked, in 128 x 128 tiles
// (bi <= bj), with the same FP32 filter and FP64 recheck as the in-cell path.
constexpr int kBT = 128;

template <int DPAD, int MODE>
__global__ void __launch_bounds__(kPairThreads) k_brute(const float* __restrict__ pf, int dtype,
                                                        const Inst* __restrict__ inst,
                                                        const InstPlan* __restrict__ iplan,
                                                        Status* st, Sink sk) {
  __shared__ __align__(16) float sa[kBT * DPAD];
  __shared__ __align__(16) float sb[kBT * DPAD];
  __shared__ unsigned int s_tally[4];
  if (threadIdx.x < 4) s_tally[threadIdx.x] = 0;
  const Inst I = inst[0];
  const InstPlan IP = iplan[0];
  const long long n = I.n;
  const long long nt = (n + kBT - 1) / kBT;
  const long long jobs = nt * (nt + 1) / 2;
  Tally tl;
  for (long long job = blockIdx.x; job < jobs; job += gridDim.x) {
    long long bj = (long long)((sqrt(8.0 * (double)job + 1.0) - 1.0) * 0.5);
    while (bj * (bj + 1) / 2 > job) --bj;
    while ((bj + 1) * (bj + 2) / 2 <= job) ++bj;
    const long long bi = job - bj * (bj + 1) / 2;
    const long long i0 = bi * kBT, j0 = bj * kBT;
    const int na = (int)min((long long)kBT, n - i0), nb = (int)min((long long)kBT, n - j0);
    __syncthreads();
    for (int x = threadIdx.x; x < 2 * kBT; x += blockDim.x) {
      const bool first = x < kBT;
      const int xx = first ? x : x - kBT;
      const int cnt = first ? na : nb;
      float* dst = (first ? sa : sb) + xx * DPAD;
      if (xx < cnt) {
        const float4* src =
            reinterpret_cast<const float4*>(pf + (size_t)(I.p0 + (first ? i0 : j0) + xx) * DPAD);
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) reinterpret_cast<float4*>(dst)[v] = __ldg(src + v);
      }
    }
    __syncthreads();
    const int y = threadIdx.x % kBT;
    for (int x = threadIdx.x / kBT; x < na; x += kPairThreads / kBT) {
      const long long li = i0 + x, lj = j0 + y;
      const bool valid = y < nb && li < lj;
      bool keep = false;
      const unsigned int i = (unsigned int)(I.p0 + li), j = (unsigned int)(I.p0 + lj);
      if (valid)
        keep = decide_pair<uint32_t, DPAD, MODE>(i, j, 0, sa + x * DPAD, sb + y * DPAD, nullptr,
                                                 nullptr, I, IP, dtype, tl);
      deliver<MODE>(keep, i, j, sk, tl);
    }
  }
  __syncthreads();
  flush_tally<MODE>(tl, st, s_tally);
}

// Row counts -> row pointers (exclusive scan, single pass with decoupled look-back); the
// counts are reset to zero so that the scatter or WRITE pass can use them as fill cursors.
constexpr int kScanItems = 16;
constexpr int kScanTile = 256 * kScanItems;

__global__ void __launch_bounds__(256) k_scan(unsigned int* row_cnt, long long* row_ptr,
                                              long long n, unsigned long long* lookback,
                                              unsigned int* tile_counter, Status* st,
                                              unsigned int tiles) {
  __shared__ unsigned long long sbuf[8];
  __shared__ unsigned long long s_base;
  __shared__ unsigned int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const unsigned int tile = s_tile;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  unsigned int v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = base + q < n ? row_cnt[base + q] : 0u;
    sum += v[q];
  }
  unsigned long long total;
  const unsigned long long ex = block_excl_scan64(sum, &total, sbuf);
  if (threadIdx.x == 0) {
    const unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kMask = (1ull << 62) - 1;
    unsigned long long excl = 0;
    if (tile == 0) {
      *reinterpret_cast<volatile unsigned long long*>(lookback) = kPre | total;
    } else {
      *reinterpret_cast<volatile unsigned long long*>(lookback + tile) = kAgg | total;
      long long p = (long long)tile - 1;
      unsigned int spins = 0;
      while (p >= 0) {
        const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(lookback + p);
        if ((w >> 62) == 0) {
          if (++spins > kSpinLimit) {
            atomicOr(&st->errors, kErrTimeout);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += w & kMask;
        if ((w >> 62) == 2) break;
        --p;
      }
      *reinterpret_cast<volatile unsigned long long*>(lookback + tile) = kPre | (excl + total);
    }
    s_base = excl;
    if (tile == tiles - 1) {
      row_ptr[n] = (long long)(excl + total);
      st->nnz = excl + total;
    }
  }
  __syncthreads();
  unsigned long long run = s_base + ex;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < n) {
      row_ptr[base + q] = (long long)run;
      row_cnt[base + q] = 0u;
    }
    run += v[q];
  }
}

// Pair buffer -> columns in their rows (row order fixed later by the row sort).
__global__ void __launch_bounds__(256) k_scatter(const unsigned long long* __restrict__ pairs,
                                                 long long cap, const Status* st,
                                                 unsigned int* row_cnt,
                                                 const long long* __restrict__ row_ptr, int* col,
                                                 long long col_cap, int symmetric,
                                                 unsigned int* errors) {
  const long long cnt = min((long long)st->emitted, cap);
  bool overflow = false;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < cnt;
       k += (long long)gridDim.x * blockDim.x) {
    const unsigned long long p = pairs[k];
    const unsigned int i = (unsigned int)(p >> 32), j = (unsigned int)p;
    const long long pi = row_ptr[i] + atomicAdd(&row_cnt[i], 1u);
    if (pi < col_cap) col[pi] = (int)j; else overflow = true;
    if (symmetric) {
      const long long pj = row_ptr[j] + atomicAdd(&row_cnt[j], 1u);
      if (pj < col_cap) col[pj] = (int)i; else overflow = true;
    }
  }
  if (overflow) atomicOr(errors, kErrColOverflow);
}

template <int L>
__device__ __forceinline__ void bitonic_regs(int* v) {
#pragma unroll
  for (int k = 2; k <= L; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int x = 0; x < L; ++x) {
        const int y = x ^ j;
        if (y > x) {
          const bool asc = (x & k) == 0;
          if (asc ? v[x] > v[y] : v[x] < v[y]) {
            const int t = v[x];
            v[x] = v[y];
            v[y] = t;
          }
        }
      }
}

// One thread per row: rows of at most 32 entries are sorted in registers (bitonic network
// with +infinity padding); longer rows are queued for the block kernel.  Rows that reach past
// col_cap (only when an undersized buffer overflowed and the build will be re-run) are left
// alone.
__global__ void __launch_bounds__(256) k_rowsort_thread(const long long* __restrict__ row_ptr,
                                                        int* col, long long n, long long col_cap,
                                                        unsigned int* long_rows,
                                                        unsigned int* long_count) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (row >= n) return;
  const long long b = row_ptr[row], len = row_ptr[row + 1] - b;
  if (len <= 1 || b + len > col_cap) return;
  if (len > 32) {
    long_rows[atomicAdd(long_count, 1u)] = (unsigned int)row;
    return;
  }
  if (len <= 16) {
    int v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = q < len ? col[b + q] : INT_MAX;
    if (len <= 4) bitonic_regs<4>(v);
    else if (len <= 8) bitonic_regs<8>(v);
    else bitonic_regs<16>(v);
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (q < len) col[b + q] = v[q];
  } else {
    int v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = q < len ? col[b + q] : INT_MAX;
    bitonic_regs<32>(v);
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q < len) col[b + q] = v[q];
  }
}

constexpr int kRowSmem = 8192;

__global__ void __launch_bounds__(256) k_rowsort_long(const long long* __restrict__ row_ptr,
                                                      int* col, long long col_cap,
                                                      const unsigned int* __restrict__ long_rows,
                                                      const unsigned int* long_count) {
  __shared__ int buf[kRowSmem];
  const unsigned int cnt = *long_count;
  for (unsigned int k = blockIdx.x; k < cnt; k += gridDim.x) {
    const unsigned int row = long_rows[k];
    const long long b = row_ptr[row], len = row_ptr[row + 1] - b;
    if (b + len > col_cap) continue;  // uniform across the block: same row for all threads
    long long L = 1;
    while (L < len) L <<= 1;
    __syncthreads();
    if (L <= kRowSmem) {
      for (long long x = threadIdx.x; x < L; x += blockDim.x) buf[x] = x < len ? col[b + x] : INT_MAX;
      __syncthreads();
      for (long long kk = 2; kk <= L; kk <<= 1) {
        for (long long j = kk >> 1; j > 0; j >>= 1) {
          for (long long x = threadIdx.x; x < L; x += blockDim.x) {
            const long long y = x ^ j;
            if (y > x) {
              const bool asc = (x & kk) == 0;
              const int u = buf[x], w = buf[y];
              if (asc ? (u > w) : (u < w)) {
                buf[x] = w;
                buf[y] = u;
              }
            }
          }
          __syncthreads();
        }
      }
      for (long long x = threadIdx.x; x < len; x += blockDim.x) col[b + x] = buf[x];
    } else {
      // Sorting network whose every comparator puts the smaller value at the lower index,
      // so positions at or past len behave as +infinity without being stored.
      int* a = col + b;
      for (long long kk = 2; kk <= L; kk <<= 1) {
        for (long long j = kk >> 1; j > 0; j >>= 1) {
          for (long long x = threadIdx.x; x < L; x += blockDim.x) {
            const long long y = (j == (kk >> 1)) ? (x ^ (kk - 1)) : (x ^ j);
            if (y > x && y < len) {
              const int u = a[x], w = a[y];
              if (u > w) {
                a[x] = w;
                a[y] = u;
              }
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

Sink make_sink(const BuildArgs& a) {
  Sink sk;
  sk.row_cnt = a.row_cnt;
  sk.row_ptr = a.row_ptr;
  sk.col = a.col;
  sk.col_cap = a.col_cap;
  sk.pair_buf = a.pair_buf;
  sk.pair_cap = a.pair_cap;
  sk.emitted = &a.st->emitted;
  sk.symmetric = a.symmetric;
  return sk;
}

template <int DPAD, int MODE>
void brute_impl(const BuildArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(8 * a.num_sms);
  k_brute<DPAD, MODE><<<blocks, kPairThreads, 0, s>>>(a.pf, a.dtype, a.inst, a.iplan, a.st,
                                                      make_sink(a));
}

template <typename K, int DPAD, int MODE>
void pairs_mode(const BuildArgs& a, int sorted_buf, cudaStream_t s) {
  const long long N = a.n_total * a.m;
  const unsigned blocks = (unsigned)((N + kSlice - 1) / kSlice);
  const bool stage_rows = a.m * (int)sizeof(K) <= kMaxStagedRow;
  const size_t smem = (size_t)kStage * DPAD * 4 + (size_t)kStage * 4 + (size_t)kKeyWin * sizeof(K) +
                      (size_t)(kSlice + 1) * 8 + (size_t)(kSlice + (kSlice & 1)) * 4 +
                      (stage_rows ? (size_t)kStage * a.m * sizeof(K) : 0);
  const K* sk = (const K*)a.keys[sorted_buf];
  const uint32_t* sv = a.vals[sorted_buf];
  static size_t attr_smem[64] = {};  // largest size granted so far, per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || smem > attr_smem[dev]) {
    cudaFuncSetAttribute(k_pairs_small<K, DPAD, MODE>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < 64) attr_smem[dev] = smem;
  }
  k_pairs_small<K, DPAD, MODE><<<blocks, kPairThreads, smem, s>>>(
      sk, sv, N, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.bases, a.B * a.m,
      a.st, make_sink(a), a.large, a.large_cap);
  if (MODE != kWrite) k_large_setup<<<1, 1024, 0, s>>>(a.large, a.large_cap, a.st, a.large_job_off);
  k_pairs_large<K, DPAD, MODE><<<(unsigned)(4 * a.num_sms), kPairThreads, 0, s>>>(
      sv, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.st, a.large, a.large_cap,
      a.large_job_off, make_sink(a));
}

template <typename K, int DPAD>
int pairs_impl(const BuildArgs& a, int sorted_buf, Mode mode, cudaStream_t s) {
  switch (mode) {
    case kCount: pairs_mode<K, DPAD, kCount>(a, sorted_buf, s); return 3;
    case kWrite: pairs_mode<K, DPAD, kWrite>(a, sorted_buf, s); return 2;
    default: pairs_mode<K, DPAD, kEmit>(a, sorted_buf, s); return 3;
  }
}

}  // namespace

int launch_pairs(const BuildArgs& a, int sorted_buf, Mode mode, cudaStream_t s) {
  if (a.key64) {
    switch (a.dpad) {
      case 4: return pairs_impl<unsigned long long, 4>(a, sorted_buf, mode, s);
      case 8: return pairs_impl<unsigned long long, 8>(a, sorted_buf, mode, s);
      default: return pairs_impl<unsigned long long, 16>(a, sorted_buf, mode, s);
    }
  }
  switch (a.dpad) {
    case 4: return pairs_impl<uint32_t, 4>(a, sorted_buf, mode, s);
    case 8: return pairs_impl<uint32_t, 8>(a, sorted_buf, mode, s);
    default: return pairs_impl<uint32_t, 16>(a, sorted_buf, mode, s);
  }
}

int launch_brute(const BuildArgs& a, Mode mode, cudaStream_t s) {
  switch (a.dpad) {
    case 4:
      if (mode == kCount) brute_impl<4, kCount>(a, s);
      else if (mode == kWrite) brute_impl<4, kWrite>(a, s);
      else brute_impl<4, kEmit>(a, s);
      break;
    case 8:
      if (mode == kCount) brute_impl<8, kCount>(a, s);
      else if (mode == kWrite) brute_impl<8, kWrite>(a, s);
      else brute_impl<8, kEmit>(a, s);
      break;
    default:
      if (mode == kCount) brute_impl<16, kCount>(a, s);
      else if (mode == kWrite) brute_impl<16, kWrite>(a, s);
      else brute_impl<16, kEmit>(a, s);
      break;
  }
  return 1;
}

void launch_scan(const BuildArgs& a, cudaStream_t s) {
  const unsigned tiles = (unsigned)((a.n_total + kScanTile - 1) / kScanTile);
  cudaMemsetAsync(a.scan_lookback, 0, (size_t)tiles * 8, s);
  k_scan<<<tiles, 256, 0, s>>>(a.row_cnt, a.row_ptr, a.n_total, a.scan_lookback,
                               &a.st->scan_tiles, a.st, tiles);
}

int launch_scatter(const BuildArgs& a, cudaStream_t s) {
  k_scatter<<<(unsigned)(8 * a.num_sms), 256, 0, s>>>(a.pair_buf, a.pair_cap, a.st, a.row_cnt,
                                                      a.row_ptr, a.col, a.col_cap, a.symmetric,
                                                      &a.st->errors);
  return 1;
}

int launch_rowsort(const BuildArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)((a.n_total + 255) / 256);
  unsigned int* long_count = &a.st->long_rows;
  k_rowsort_thread<<<blocks, 256, 0, s>>>(a.row_ptr, a.col, a.n_total, a.col_cap, a.row_cnt,
                                          long_count);
  k_rowsort_long<<<(unsigned)(2 * a.num_sms), 256, 0, s>>>(a.row_ptr, a.col, a.col_cap, a.row_cnt,
                                                           long_count);
  return 2;
}

}  // namespace rtg
