// In-cell pair enumeration and CSR assembly (the in-cell pair reporting of Alg. 1 and the
// dedupe of Sec. III-B of arXiv:1409.8112), for a batch of instances.
//
// After the sort every (instance, grid, cell) is a run of equal keys.  A warp owns the cells
// whose first position lies in its span of sorted positions: it finds them with adjacent key
// comparisons (ballots), stages their points (FP32, padded rows) in a per-warp shared-memory
// ring and tests every pair (a < b) of every cell with at most kSmallCell points.  Cells with
// more points go to the tiled large-cell kernel.
//
// Dedupe without an auxiliary set: the distance test does not depend on the grid, so pair
// {i, j} is reported by grid t iff it is within r and shares a cell in t.  The pair is
// therefore emitted only by the first grid that puts i and j in one cell; a candidate in
// grid t is dropped when key_mat[i][t'] == key_mat[j][t'] for some t' < t (the filtering use
// of the auxiliary structure in Sec. III-B).  It runs after the FP32 distance has ruled out
// the pairs that are certainly beyond r, so far pairs cost no key-row loads.
//
// Distance: FP32 on the staged rows; a pair is decided in FP32 only when the FP32 squared
// distance is outside [s_lo, s_hi], the proven error band around fl(r*r) (see the plan
// kernel); otherwise the FP64 reference sequence decides.
//
// Modes: EMIT writes reported pairs to a pair buffer (buffered per warp, one reservation per
// flush) and counts rows;
// after the scan, scatter places them.  COUNT then WRITE enumerates twice and needs no pair
// buffer (for outputs too large to hold twice).  Rows are sorted at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "rtg_internal.cuh"
#include "rtg_tc.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace rtg {

namespace {

constexpr int kPairThreads = 256;
constexpr int kRing = 64;  // staged positions per warp: covers the 31 partners behind a chunk
static_assert(kRing >= kSmallCell - 1 + 32 && (kRing & (kRing - 1)) == 0, "ring too small");
constexpr int kWarpEmit = 128;             // EMIT: reported pairs buffered per warp
constexpr int kWarpFlush = kWarpEmit - 32;  // written out once more than this many are held
constexpr int kTL = 128;                   // large-cell tile
constexpr int kMediumMax = 256;            // large cells up to this size: one warp per cell
constexpr int kMediumWarps = 4;            // warps per block of the medium-cell kernel
constexpr int kMediumKeyBytes = 8192;      // per warp: staged key rows of a medium cell

__device__ __forceinline__ double load_coord(const void* pts, int dtype, long long i, int d,
                                             int l) {
  return dtype == 0 ? __ldg((const double*)pts + i * d + l)
                    : (double)__ldg((const float*)pts + i * d + l);
}

// FP64 reference squared distance (fixed order, fused multiply-add, original coordinates).
__device__ __forceinline__ double exact_dist2(const void* pts, int dtype, long long i, long long j,
                                           int d) {
  double s = 0.0;
  for (int l = 0; l < d; ++l) {
    const double e = __dsub_rn(load_coord(pts, dtype, i, d, l), load_coord(pts, dtype, j, d, l));
    s = __fma_rn(e, e, s);
  }
  return s;
}

// Exclusive scan of one value per thread over the block (a multiple of 32 threads, at most
// 1024); sbuf holds one word per warp.
__device__ __forceinline__ unsigned int block_excl_scan_any(unsigned int v, unsigned int* total,
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

// Per-thread tallies (the rare events, near-r pairs and buffer overflow, go straight to the
// status).
struct Tally {
  unsigned int owned = 0, rechecks = 0, pairs = 0;
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
  unsigned int* errors;
  unsigned long long* near_r;
  unsigned int* bits;
  int symmetric;
};

// Bit-matrix dedupe: set bit (i, j) (and (j, i) for symmetric output) of the instance's matrix.
__device__ __forceinline__ void deliver_bits(bool keep, unsigned int i, unsigned int j,
                                             const Inst* __restrict__ Ip, const Sink& sk) {
  if (!keep) return;
  const Inst& I = *Ip;
  const long long li = (long long)i - I.p0, lj = (long long)j - I.p0;
  atomicOr(&sk.bits[I.bits_off + li * I.bits_w + (lj >> 5)], 1u << (lj & 31));
  if (sk.symmetric) atomicOr(&sk.bits[I.bits_off + lj * I.bits_w + (li >> 5)], 1u << (li & 31));
}

// FP32 band of an instance as (lo, hi): FP32 decides below lo and above hi.  With the filter
// off every candidate falls inside.
__device__ __forceinline__ float2 band_of(const InstPlan& IP) {
  return IP.filter_on ? make_float2(IP.s_lo, IP.s_hi) : make_float2(-1.0f, __int_as_float(0x7f800000));
}

// Decide one candidate pair (i < j, global indices) of grid t of instance I; ki and kj are the
// two points' key rows (shared or global memory); band is band_of(IP).
template <typename K, int DPAD, int MODE, bool VEC = false>
__device__ __forceinline__ bool decide_pair(unsigned int i, unsigned int j, int t, const float* pa,
                                            const float* pb, const K* ki, const K* kj,
                                            const Inst* __restrict__ Ip,
                                            const InstPlan* __restrict__ IPp, float2 band,
                                            int dtype, Tally& tl, unsigned long long* near_r) {
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
  if (sf > band.y) return false;  // beyond r for certain: no ownership test needed
  // an earlier grid owns the pair if it co-locates it; grids in batches of four (the loads of
  // a batch issued together), stopping at the first batch with a match: a close pair usually
  // shares a cell in one of the first grids
  if (MODE != kBits) {
    if (VEC) {
      // rows 16-byte aligned: 16 bytes of each row per load
      constexpr int kpv = 16 / (int)sizeof(K);
      for (int u0 = 0; u0 < t; u0 += kpv) {
        const uint4 va = *reinterpret_cast<const uint4*>(ki + u0);
        const uint4 vb = *reinterpret_cast<const uint4*>(kj + u0);
        const K* xa = reinterpret_cast<const K*>(&va);
        const K* xb = reinterpret_cast<const K*>(&vb);
        bool earlier = false;
#pragma unroll
        for (int q = 0; q < kpv; ++q)
          if (u0 + q < t) earlier |= xa[q] == xb[q];
        if (earlier) return false;
      }
    } else {
      for (int u0 = 0; u0 < t; u0 += 4) {
        bool earlier = false;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (u0 + q < t) earlier |= ki[u0 + q] == kj[u0 + q];
        if (earlier) return false;
      }
    }
  }
  if (MODE != kWrite && MODE != kBits) ++tl.owned;
  bool keep;
  if (sf < band.x) {
    keep = true;
  } else {
    const Inst& I = *Ip;
    const double s = exact_dist2(I.pts, dtype, (long long)i - I.p0, (long long)j - I.p0, I.d);
    keep = s <= IPp->rr;
    if (MODE != kWrite) {
      ++tl.rechecks;
      if (MODE != kBits && fabs(__dsub_rn(__dsqrt_rn(s), I.r)) <= __dmul_rn(1e-12, I.r))
        atomicAdd(near_r, 1ull);
    }
  }
  if (keep && MODE != kWrite) ++tl.pairs;
  return keep;
}

// A candidate that a tensor-core tile proved to be within r (its tile d^2 is below the band
// minus the tile error bound): only the ownership test remains (as in decide_pair).
template <typename K, int MODE>
__device__ __forceinline__ bool decide_inside(int t, const K* ki, const K* kj, Tally& tl) {
  if (MODE != kBits) {
    for (int u0 = 0; u0 < t; u0 += 4) {
      bool earlier = false;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (u0 + q < t) earlier |= ki[u0 + q] == kj[u0 + q];
      if (earlier) return false;
    }
  }
  if (MODE != kWrite && MODE != kBits) ++tl.owned;
  if (MODE != kWrite) ++tl.pairs;
  return true;
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
      else atomicOr(sk.errors, kErrPairOverflow);
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
      if (pi < sk.col_cap) sk.col[pi] = (int)j; else atomicOr(sk.errors, kErrColOverflow);
      if (sk.symmetric) {
        const long long pj = sk.row_ptr[j] + atomicAdd(&sk.row_cnt[j], 1u);
        if (pj < sk.col_cap) sk.col[pj] = (int)i; else atomicOr(sk.errors, kErrColOverflow);
      }
    }
  }
}

// EMIT through a per-warp shared-memory buffer of kWarpEmit pairs: one reservation in the
// pair buffer per flush instead of one per warp step.  Called by all 32 lanes together;
// `ecnt` (the pairs held) is the same in every lane.
__device__ __forceinline__ void warp_flush(unsigned long long* wbuf, unsigned int ecnt,
                                           const Sink& sk) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  unsigned long long b0 = 0;
  if (lane == 0) b0 = atomicAdd(sk.emitted, (unsigned long long)ecnt);
  b0 = __shfl_sync(0xffffffffu, b0, 0);
  for (unsigned int x = lane; x < ecnt; x += 32) {
    if ((long long)(b0 + x) < sk.pair_cap) sk.pair_buf[b0 + x] = wbuf[x];
    else atomicOr(sk.errors, kErrPairOverflow);
  }
  __syncwarp();
}

__device__ __forceinline__ void warp_emit(bool keep, unsigned int i, unsigned int j,
                                          unsigned long long* wbuf, unsigned int& ecnt,
                                          const Sink& sk) {
  const unsigned int mask = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31;
  if (keep) {
    wbuf[ecnt + __popc(mask & ((1u << lane) - 1))] = ((unsigned long long)i << 32) | j;
    atomicAdd(&sk.row_cnt[i], 1u);
    if (sk.symmetric) atomicAdd(&sk.row_cnt[j], 1u);
  }
  ecnt += (unsigned int)__popc(mask);
  if (ecnt > (unsigned int)kWarpFlush) {
    warp_flush(wbuf, ecnt, sk);
    ecnt = 0;
  }
}

template <int MODE>
__device__ __forceinline__ void flush_tally(const Tally& tl, Status* st, unsigned int* sbuf) {
  // sbuf: 3 block-wide counters, zeroed by the caller before its last barrier
  unsigned int v[3] = {tl.owned, tl.rechecks, tl.pairs};
#pragma unroll
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (MODE != kWrite && (threadIdx.x & 31) == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (v[q]) atomicAdd(&sbuf[q], v[q]);
  }
  __syncthreads();
  if (MODE == kWrite || threadIdx.x != 0) return;
  if (sbuf[0]) atomicAdd(&st->owned_candidates, (unsigned long long)sbuf[0]);
  if (sbuf[1]) atomicAdd(&st->dist_rechecks, (unsigned long long)sbuf[1]);
  if (sbuf[2]) atomicAdd(&st->pairs, (unsigned long long)sbuf[2]);
}

// (instance, grid) of a composite key: the last base <= key, searched in [lo, hi].
__device__ __forceinline__ int find_bt(unsigned long long key,
                                       const unsigned long long* __restrict__ bases, int lo,
                                       int hi) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(bases + mid) <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Key rows are staged in shared memory when a row (m keys) is at most this many bytes.
constexpr int kMaxStagedRow = 128;

// Keys between staged key rows in k_pairs_warp: a multiple of 16 bytes (the ownership test
// reads four 32-bit or two 64-bit keys per load), plus 16 bytes when the row would otherwise
// be a multiple of 128 bytes, so that neighbouring rows start in different banks.
template <typename K>
__host__ __device__ inline int staged_row_stride(int m) {
  constexpr int kpv = 16 / (int)sizeof(K);
  int st = (m + kpv - 1) / kpv * kpv;
  if ((st * (int)sizeof(K)) % 128 == 0) st += kpv;
  return st;
}

// Bytes of one warp's shared-memory region in k_pairs_warp (the staged key rows first, so
// that they are 16-byte aligned).
template <typename K, int DPAD>
__host__ __device__ inline int warp_region_bytes(int m, bool stage_rows) {
  const int b = kWarpEmit * 8 + kRing * DPAD * 4 +
                (stage_rows ? kRing * staged_row_stride<K>(m) * (int)sizeof(K) : 0) + kRing * 4 +
                3 * 32 * 4;
  return (b + 15) & ~15;
}

// End of the run of keys equal to `key` that is known to reach position `from`: galloping
// search, then bisection (the run may be long).
template <typename K>
__device__ long long run_end(const K* __restrict__ skeys, long long N, long long from, K key) {
  long long lo = from + 1, step = 64, hi = lo;
  while (true) {  // find hi with skeys[hi] != key (or hi = N)
    hi = lo + step;
    if (hi >= N) {
      hi = N;
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
  return lo;
}

// Segment detection and in-cell enumeration for cells of at most kSmallCell points.
//
// Each warp owns the cells whose first sorted position lies in its span of positions and walks
// the span in chunks of 32 positions, one per lane, with the next chunk's keys and indices
// loaded one chunk ahead.  Cell heads are adjacent-key changes (warp ballot); a head is a large
// cell when the key 32 positions on is still the same, and large cells are queued for
// k_pairs_large and skipped.  Every position of a small cell is staged in the warp's ring of
// kRing slots (FP32 row, index, the first t keys of its key row), so the partners of a position
// (the earlier positions of its cell, at most 31 back) are always in the ring.  The pairs of a
// chunk are (position, earlier position of its cell); a warp scan spreads them over the lanes
// 32 at a time, so the work is balanced whatever the cell sizes.  Only warp-level
// synchronisation is used.
#ifndef RTG_PAIRS_MIN_BLOCKS
#define RTG_PAIRS_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for
#endif
// STAGE: 0 key rows read in place, 1 staged key by key, 2 staged in 16-byte blocks (key rows
// of a multiple of 16 bytes).
template <typename K, int DPAD, int MODE, int STAGE>
__global__ void __launch_bounds__(kPairThreads, RTG_PAIRS_MIN_BLOCKS) k_pairs_warp(
    const K* __restrict__ skeys, const uint32_t* __restrict__ svals, long long N, long long span,
    const float* __restrict__ pf, int dtype, const K* __restrict__ key_mat, int m,
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const unsigned long long* __restrict__ bases, int nbt, Status* st, Sink sk,
    LargeCell* large, unsigned int large_cap, int warp_bytes, unsigned int* span_next,
    int skip_dense, int cell_major) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_gcand[kMaxGrids];
  __shared__ unsigned int s_maxcell;
  __shared__ unsigned int s_tally[4];
  // a sort that gave up (a bounded wait ran out) or flagged an offset may have left stale
  // point indices behind: nothing is read through them (the build reports the error)
  if (st->errors & (kErrTimeout | kErrSortRange)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* ws = smem + (size_t)wib * warp_bytes;
  unsigned long long* w_emit = reinterpret_cast<unsigned long long*>(ws);
  float* w_pt = reinterpret_cast<float*>(ws + kWarpEmit * 8);
  K* w_rows = reinterpret_cast<K*>(w_pt + kRing * DPAD);
  const int rstride = staged_row_stride<K>(m);
  uint32_t* w_idx = reinterpret_cast<uint32_t*>(w_rows + (STAGE != 0 ? kRing * rstride : 0));
  int* w_excl = reinterpret_cast<int*>(w_idx + kRing);  // per lane: first pair of the lane
  int* w_hrel = w_excl + 32;                             // per lane: cell head - chunk start
  unsigned int* w_cell = reinterpret_cast<unsigned int*>(w_hrel + 32);  // (instance << 8) | grid
  for (int g = threadIdx.x; g < kMaxGrids; g += blockDim.x) s_gcand[g] = 0;
  if (threadIdx.x < 4) s_tally[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_maxcell = 0;
  __syncthreads();

  const unsigned int full = 0xffffffffu;
  const unsigned int le = lane == 31 ? full : ((2u << lane) - 1u);
  const long long nspans = (N + span - 1) / span;
  Tally tl;
  unsigned int cand_acc = 0;  // at most 31 per position of the span
  int cand_g = -1;
  unsigned int maxcell = 0;
  unsigned int ecnt = 0;  // pairs in w_emit (warp-uniform)

  // the first span of a warp is its own; when there are more spans than warps the rest are
  // claimed one at a time from a counter, so that a warp whose spans held few pairs takes
  // more of them (cell sizes, and so the work per span, vary)
  const long long launched = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long sp = (long long)blockIdx.x * (blockDim.x >> 5) + wib; sp < nspans;) {
    // Positions inside the span loop are offsets from P0 (int): the warp leaves the span once
    // it passes its end, so every offset it keeps is below span + 32.
    const long long P0 = sp * span;
    const int len = (int)(min(P0 + span, N) - P0);  // owned heads lie in [0, len)
    const int lim = (int)(min(P0 + span + 64, N) - P0);  // positions read lie in [0, lim)
    // (instance, grid) range of every cell this span can own (a cell-major sort leaves the
    // keys in (cell, grid) order, so a span may hold any grid)
    int bt_lo = 0, bt_hi = nbt - 1;
    if (!cell_major) {
      const long long q = lane == 0 ? P0 : P0 + min(len + 32, lim) - 1;
      int v = 0;
      if (lane < 2) v = find_bt((unsigned long long)skeys[q], bases, 0, nbt - 1);
      bt_lo = __shfl_sync(full, v, 0);
      bt_hi = __shfl_sync(full, v, 1);
    }
    // one instance in the span (the usual case): its FP32 band stays in registers
    const int inst_lo = bt_lo / m;
    const bool one_inst = inst_lo == bt_hi / m;
    const float2 span_band = band_of(iplan[inst_lo]);
    const K* kspan = skeys + P0;
    const uint32_t* vspan = svals + P0;
    int P = 0;
    K key_prev = P0 > 0 ? skeys[P0 - 1] : (K)0;
    int ch = -1;              // head of the cell holding position P - 1, -1 if not ours
    unsigned int ccell = 0;   // its (instance << 8) | grid
    K kc = lane < lim ? kspan[lane] : (K)0;
    uint32_t vc = lane < lim ? vspan[lane] : 0u;
    while (true) {
      const int p = P + lane;
      const bool valid = p < lim;
      const int pn = P + 32 + lane;
      const K kn = pn < lim ? kspan[pn] : (K)0;
      const uint32_t vn = pn < lim ? vspan[pn] : 0u;
      K kprev = __shfl_up_sync(full, kc, 1);
      if (lane == 0) kprev = key_prev;
      const bool head = valid && ((P0 == 0 && p == 0) || kc != kprev);
      const unsigned int hmask = __ballot_sync(full, head);
      if (hmask == 0 && ch < 0) {
        // the whole chunk continues a cell that starts before this span: skip past it
        if (P + 32 >= lim) break;
        const K k31 = __shfl_sync(full, kc, 31);
        long long e = 0;
        if (lane == 0) e = run_end(skeys, N, P0 + P + 31, k31);
        e = __shfl_sync(full, e, 0) - P0;
        if (e >= len) break;
        P = (int)e;
        key_prev = k31;
        kc = P + lane < lim ? kspan[P + lane] : (K)0;
        vc = P + lane < lim ? vspan[P + lane] : 0u;
        continue;
      }
      // head lanes: large test, (instance, grid), and a large cell's end (offset, clamped)
      bool lg = false;
      unsigned int cell = 0;
      int lend = 0;
      if (head && p < len) {
        lg = pn < lim && kn == kc;  // lim reaches 32 past every owned head unless N does not
        const int bt = find_bt((unsigned long long)kc, bases, bt_lo, bt_hi);
        const int bi = one_inst ? inst_lo : bt / m;
        cell = ((unsigned int)bi << 8) | (unsigned int)(bt - bi * m);
        if (lg) {
          const long long e = run_end(skeys, N, P0 + pn, kc);
          lend = (int)min(e - P0, (long long)INT_MAX);
          if (MODE != kWrite) {
            // the dense-cell kernels were left out of this launch: the host runs it again
            if (skip_dense) atomicOr(&st->errors, kErrTailSkipped);
            const unsigned long long size = (unsigned long long)(e - (P0 + p));
            const unsigned long long slot = atomicAdd(&st->large_cells, 1ull);
            if (slot < large_cap) {
              large[slot].start = (unsigned long long)(P0 + p);
              large[slot].size = (unsigned int)size;
              large[slot].grid = (unsigned short)(cell & 0xffu);
              large[slot].inst = (unsigned short)(cell >> 8);
            } else {
              atomicOr(&st->errors, kErrLargeOverflow);
            }
            atomicAdd(&s_gcand[cell & 0xffu], size * (size - 1) / 2);
            maxcell = max(maxcell, (unsigned int)min(size, 0xffffffffull));
          }
        }
      }
      const unsigned int hm = hmask & le;
      const int hl = hm ? 31 - __clz(hm) : lane;
      const bool lg_h = __shfl_sync(full, lg, hl);
      const unsigned int cell_h = __shfl_sync(full, cell, hl);
      const int h = hm ? P + hl : ch;
      const bool big = hm ? lg_h : false;
      const unsigned int mycell = hm ? cell_h : ccell;
      const bool owned = valid && h >= 0 && h < len;
      const bool active = owned && !big;
      const int np = active ? p - h : 0;
      // stage this position in the ring
      if (active) {
        const int slot = (int)((P0 + p) & (kRing - 1));
        w_idx[slot] = vc;
        // the FP32 row and the first t keys of the key row, copied asynchronously (all of a
        // lane's gathers in flight at once; waited for below)
        const float* src = pf + (size_t)vc * DPAD;
        float* dst = w_pt + slot * DPAD;
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) cp_async16(dst + 4 * v, src + 4 * v);
        if (STAGE == 2) {
          // 16-byte copies covering the first t keys (key rows and staged rows start on 16-byte
          // boundaries and hold a multiple of 16 bytes, so the copies stay inside both)
          const int t = (int)(mycell & 0xffu);
          const K* kr = key_mat + (size_t)vc * m;
          K* kd = w_rows + slot * rstride;
          constexpr int kpv = 16 / (int)sizeof(K);
          for (int u = 0; u < t; u += kpv) cp_async16(kd + u, kr + u);
        } else if (STAGE == 1) {
          const int t = (int)(mycell & 0xffu);
          const K* kr = key_mat + (size_t)vc * m;
          K* kd = w_rows + slot * rstride;
          for (int u = 0; u < t; ++u) cp_async_small<(int)sizeof(K)>(kd + u, kr + u);
        }
        if (MODE != kWrite) {
          const int g = (int)(mycell & 0xffu);
          if (g != cand_g) {
            if (cand_acc) atomicAdd(&s_gcand[cand_g], (unsigned long long)cand_acc);
            cand_g = g;
            cand_acc = 0;
          }
          cand_acc += (unsigned int)np;
          maxcell = max(maxcell, (unsigned int)np + 1u);
        }
      }
      cp_async_wait_all();  // this lane's staged rows have landed (visible to the warp at
                            // the __syncwarp below)
      // pairs of this chunk, spread over the lanes
      int incl = np;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
      }
      const int total = __shfl_sync(full, incl, 31);
      if (total > 0) {
        w_excl[lane] = incl - np;
        w_hrel[lane] = h - P;
        w_cell[lane] = mycell;
        __syncwarp();
        const int pbase = (int)((P0 + P) & (kRing - 1));
        for (int base = 0; base < total; base += 32) {
          const int k = base + lane;
          bool keep = false;
          unsigned int i = 0, j = 0;
          int pinst = 0;
          if (k < total) {
            int o = 0;
#pragma unroll
            for (int st2 = 16; st2 > 0; st2 >>= 1)
              if (w_excl[o + st2] <= k) o += st2;
            const int sa = (pbase + o) & (kRing - 1);
            const int sb = (pbase + w_hrel[o] + (k - w_excl[o])) & (kRing - 1);
            const unsigned int ia = w_idx[sa], ib = w_idx[sb];
            i = min(ia, ib);
            j = max(ia, ib);
            const unsigned int cl = w_cell[o];
            const int t = (int)(cl & 0xffu), ib_ = (int)(cl >> 8);
            pinst = ib_;
            const K* ka = STAGE != 0 ? w_rows + sa * rstride : key_mat + (size_t)ia * m;
            const K* kb = STAGE != 0 ? w_rows + sb * rstride : key_mat + (size_t)ib * m;
            const float2 band = one_inst ? span_band : band_of(iplan[ib_]);
            keep = decide_pair<K, DPAD, MODE, STAGE != 0>(i, j, t, w_pt + sa * DPAD,
                                                          w_pt + sb * DPAD, ka, kb, inst + ib_,
                                                          iplan + ib_, band, dtype, tl,
                                                          sk.near_r);
          }
          if (MODE == kBits) {
            deliver_bits(keep, i, j, inst + pinst, sk);
          } else if (MODE == kEmit) {
            warp_emit(keep, i, j, w_emit, ecnt, sk);
          } else {
            deliver<MODE>(keep, i, j, sk, tl);
          }
        }
        __syncwarp();
      }
      // next chunk
      const bool own31 = __shfl_sync(full, owned, 31);
      const bool big31 = __shfl_sync(full, big, 31);
      const int h31 = __shfl_sync(full, h, 31);
      const unsigned int cell31 = __shfl_sync(full, mycell, 31);
      const K k31 = __shfl_sync(full, kc, 31);
      if (own31 && big31) {  // jump past the large cell (its head is in this chunk)
        const int hl31 = __shfl_sync(full, hl, 31);
        const int e = __shfl_sync(full, lend, hl31);
        if (e >= len) break;
        P = e;
        key_prev = k31;
        ch = -1;
        kc = P + lane < lim ? kspan[P + lane] : (K)0;
        vc = P + lane < lim ? vspan[P + lane] : 0u;
        continue;
      }
      const int nxt = P + 32;
      if (nxt >= lim) break;
      if (nxt >= len) {
        const K k0n = __shfl_sync(full, kn, 0);
        if (!(own31 && k0n == k31)) break;  // no cell of this span continues
      }
      P = nxt;
      key_prev = k31;
      ch = own31 ? h31 : -1;
      ccell = cell31;
      kc = kn;
      vc = vn;
    }
    if (nspans <= launched) break;
    long long nx = 0;
    if (lane == 0) nx = launched + atomicAdd(span_next, 1u);
    sp = __shfl_sync(full, nx, 0);
  }
  if (MODE == kEmit && ecnt) warp_flush(w_emit, ecnt, sk);
  if (MODE != kWrite) {
    if (cand_acc) atomicAdd(&s_gcand[cand_g], (unsigned long long)cand_acc);
    for (int o = 16; o > 0; o >>= 1) maxcell = max(maxcell, __shfl_xor_sync(full, maxcell, o));
    if (lane == 0 && maxcell) atomicMax(&s_maxcell, maxcell);
  }
  __syncthreads();
  if (MODE != kWrite) {
    if (threadIdx.x < m && s_gcand[threadIdx.x])
      atomicAdd(&st->candidates[threadIdx.x], s_gcand[threadIdx.x]);
    if (threadIdx.x == 0 && s_maxcell) atomicMax(&st->max_cell, (unsigned long long)s_maxcell);
  }
  flush_tally<MODE>(tl, st, s_tally);
}

// Job offsets for the tiled kernel: a cell of more than dense_min (<= kMediumMax) points and
// T = ceil(size / kTL) tiles has T (T + 1) / 2 tile pairs; smaller cells have none (the
// medium-cell kernel takes them).
__global__ void __launch_bounds__(1024) k_large_setup(const LargeCell* __restrict__ large,
                                                      unsigned int cap, Status* st,
                                                      unsigned long long* job_off,
                                                      unsigned int dense_min) {
  __shared__ unsigned long long sbuf[32];
  __shared__ unsigned long long carry;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (unsigned long long base = 0; base < L; base += blockDim.x) {
    const unsigned long long e = base + threadIdx.x;
    const unsigned long long T =
        e < L && large[e].size > dense_min ? (large[e].size + kTL - 1) / kTL : 0;
    const unsigned long long v = T * (T + 1) / 2;
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

// Cells of kSmallCell + 1 .. kMediumMax points, one warp per cell: the warp stages the members
// (FP32 rows, indices) in shared memory and walks the cell's s (s - 1) / 2 pairs 32 at a time,
// pair k = b (b - 1) / 2 + a (a < b) advanced incrementally, so that every lane is busy
// whatever the cell size.
template <typename K, int DPAD, int MODE>
__global__ void __launch_bounds__(kMediumWarps * 32) k_pairs_medium(
    const uint32_t* __restrict__ svals, const float* __restrict__ pf, int dtype,
    const K* __restrict__ key_mat, int m, const Inst* __restrict__ inst,
    const InstPlan* __restrict__ iplan, Status* st, const LargeCell* __restrict__ large,
    unsigned int cap, Sink sk, unsigned int dense_min) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_emit[kMediumWarps][kWarpEmit];
  __shared__ unsigned int s_tally[4];
  if (threadIdx.x < 4) s_tally[threadIdx.x] = 0;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* w_pt = reinterpret_cast<float*>(smem) + (size_t)wib * kMediumMax * DPAD;
  uint32_t* w_idx = reinterpret_cast<uint32_t*>(reinterpret_cast<float*>(smem) +
                                                (size_t)kMediumWarps * kMediumMax * DPAD) +
                    wib * kMediumMax;
  K* w_keys = reinterpret_cast<K*>(reinterpret_cast<unsigned char*>(smem) +
                                   (size_t)kMediumWarps * kMediumMax * (DPAD * 4 + 4) +
                                   (size_t)wib * kMediumKeyBytes);
  unsigned long long* w_emit = s_emit[wib];
  unsigned int ecnt = 0;
  Tally tl;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  const unsigned long long W = (unsigned long long)gridDim.x * kMediumWarps;
  for (unsigned long long e = (unsigned long long)blockIdx.x * kMediumWarps + wib; e < L; e += W) {
    const LargeCell cell = large[e];
    const unsigned int s = cell.size;
    if (s > dense_min) continue;  // warp-uniform (the tiled kernels take it)
    const int t = (int)cell.grid, kst = t + 1;  // staged keys per member (odd stride)
    const bool kstage = (size_t)s * kst * sizeof(K) <= (size_t)kMediumKeyBytes;
    for (unsigned int x = lane; x < s; x += 32) {
      const uint32_t idx = svals[cell.start + x];
      w_idx[x] = idx;
      const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
      float4* dst = reinterpret_cast<float4*>(w_pt + x * DPAD);
#pragma unroll
      for (int v = 0; v < DPAD / 4; ++v) dst[v] = __ldg(src + v);
      if (kstage) {
        const K* kr = key_mat + (size_t)idx * m;
        for (int u = 0; u < t; ++u) w_keys[x * kst + u] = __ldg(kr + u);
      }
    }
    __syncwarp();
    const float2 band = band_of(iplan[cell.inst]);
    const unsigned int P = s * (s - 1) / 2;
    // pair `lane`: b from the triangular root, then a
    unsigned int b = (unsigned int)((1.0f + sqrtf(8.0f * (float)lane + 1.0f)) * 0.5f);
    while (b * (b - 1) / 2 > (unsigned int)lane) --b;
    while ((b + 1) * b / 2 <= (unsigned int)lane) ++b;
    unsigned int a = (unsigned int)lane - b * (b - 1) / 2;
    for (unsigned int base = 0; base < P; base += 32) {
      bool keep = false;
      unsigned int i = 0, j = 0;
      if (base + lane < P) {
        const uint32_t ia = w_idx[a], ib = w_idx[b];
        i = min(ia, ib);
        j = max(ia, ib);
        const K* ka = kstage ? w_keys + a * kst : key_mat + (size_t)ia * m;
        const K* kb = kstage ? w_keys + b * kst : key_mat + (size_t)ib * m;
        keep = decide_pair<K, DPAD, MODE>(i, j, t, w_pt + a * DPAD, w_pt + b * DPAD, ka, kb,
                                          inst + cell.inst, iplan + cell.inst, band, dtype, tl,
                                          sk.near_r);
      }
      if (MODE == kBits) deliver_bits(keep, i, j, inst + cell.inst, sk);
      else if (MODE == kEmit) warp_emit(keep, i, j, w_emit, ecnt, sk);
      else deliver<MODE>(keep, i, j, sk, tl);
      a += 32;  // next pair of this lane: 32 on
      while (a >= b) {
        a -= b;
        ++b;
      }
    }
    __syncwarp();
  }
  if (MODE == kEmit && ecnt) warp_flush(w_emit, ecnt, sk);
  __syncthreads();
  flush_tally<MODE>(tl, st, s_tally);
}

// Cells of more than kSmallCell points, as 128 x 128 tiles of member pairs: job = (cell, row
// tile a, column tile b >= a), so every job is one tile pair however large the cell.  Each
// thread keeps one column member (y) and walks the row members (x), which all lanes of a warp
// read at the same address.
template <typename K, int DPAD, int MODE>
__global__ void __launch_bounds__(kPairThreads) k_pairs_large(
    const uint32_t* __restrict__ svals, const float* __restrict__ pf, int dtype,
    const K* __restrict__ key_mat, int m, const Inst* __restrict__ inst,
    const InstPlan* __restrict__ iplan, Status* st, const LargeCell* __restrict__ large,
    unsigned int cap, const unsigned long long* job_off, Sink sk) {
  __shared__ __align__(16) float sa[kTL * DPAD];
  __shared__ __align__(16) float sb[kTL * DPAD];
  __shared__ uint32_t ia[kTL], ib[kTL];
  // the first t keys of each member's key row for the ownership test (64 bytes a row at
  // most; rows kLK + 1 apart so that neighbouring rows fall in different banks)
  constexpr int kLK = 64 / (int)sizeof(K);
  __shared__ K ska[kTL * (kLK + 1)], skb[kTL * (kLK + 1)];
  __shared__ unsigned long long s_emit[kPairThreads / 32][kWarpEmit];
  __shared__ unsigned int s_tally[4];
  if (threadIdx.x < 4) s_tally[threadIdx.x] = 0;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  const unsigned long long J = L ? job_off[L] : 0;
  unsigned long long* w_emit = s_emit[threadIdx.x >> 5];
  unsigned int ecnt = 0;
  Tally tl;
  for (unsigned long long job = blockIdx.x; job < J; job += gridDim.x) {
    long long el = 0, eh = (long long)L - 1;
    while (el < eh) {
      const long long mid = (el + eh + 1) >> 1;
      if (job_off[mid] <= job) el = mid; else eh = mid - 1;
    }
    const LargeCell cell = large[el];
    const float2 band = band_of(iplan[cell.inst]);
    const unsigned int s = cell.size;
    // tile pair (bi <= bj) of this cell
    const long long k = (long long)(job - job_off[el]);
    long long bj = (long long)((sqrt(8.0 * (double)k + 1.0) - 1.0) * 0.5);
    while (bj * (bj + 1) / 2 > k) --bj;
    while ((bj + 1) * (bj + 2) / 2 <= k) ++bj;
    const long long bi = k - bj * (bj + 1) / 2;
    const unsigned int a0 = (unsigned int)bi * kTL, b0 = (unsigned int)bj * kTL;
    const unsigned int na = min((unsigned int)kTL, s - a0), nb = min((unsigned int)kTL, s - b0);
    const int tg = (int)cell.grid;
    const bool kst = tg <= kLK;  // key rows staged (else read from global memory)
    __syncthreads();
    for (unsigned int x = threadIdx.x; x < 2 * kTL; x += blockDim.x) {
      const bool first = x < kTL;
      const unsigned int xx = first ? x : x - kTL;
      if (xx < (first ? na : nb)) {
        const uint32_t idx = svals[cell.start + (first ? a0 : b0) + xx];
        (first ? ia : ib)[xx] = idx;
        const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
        float4* dst = reinterpret_cast<float4*>((first ? sa : sb) + xx * DPAD);
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) dst[v] = __ldg(src + v);
        if (kst) {
          const K* kr = key_mat + (size_t)idx * m;
          K* kd = (first ? ska : skb) + xx * (kLK + 1);
          for (int u = 0; u < tg; ++u) kd[u] = __ldg(kr + u);
        }
      }
    }
    __syncthreads();
    const unsigned int y = threadIdx.x % kTL;
    const uint32_t iy = y < nb ? ib[y] : 0u;
    for (unsigned int x = threadIdx.x / kTL; x < na; x += kPairThreads / kTL) {
      bool keep = false;
      unsigned int i = 0, j = 0;
      if (y < nb && a0 + x < b0 + y) {
        const uint32_t ix = ia[x];
        i = min(ix, iy);
        j = max(ix, iy);
        keep = decide_pair<K, DPAD, MODE>(
            i, j, tg, sa + x * DPAD, sb + y * DPAD,
            kst ? ska + x * (kLK + 1) : key_mat + (size_t)ix * m,
            kst ? skb + y * (kLK + 1) : key_mat + (size_t)iy * m, inst + cell.inst,
            iplan + cell.inst, band, dtype, tl, sk.near_r);
      }
      if (MODE == kBits) deliver_bits(keep, i, j, inst + cell.inst, sk);
      else if (MODE == kEmit) warp_emit(keep, i, j, w_emit, ecnt, sk);
      else deliver<MODE>(keep, i, j, sk, tl);
    }
  }
  if (MODE == kEmit && ecnt) warp_flush(w_emit, ecnt, sk);
  __syncthreads();
  flush_tally<MODE>(tl, st, s_tally);
}

// Dense cells on the tensor cores (the in-cell distance test of Alg. 1 as d^2 = |x|^2 +
// |y|^2 - 2 x.y tiles): the jobs of k_pairs_large, a 128 x 128 pair of member tiles each.
// The members' FP32 rows are centred on the cell's first member and split into half-precision
// hi + lo; three K = 16 tcgen05 MMAs (hi.hi + hi.lo + lo.hi) accumulate x.y in FP32 in tensor
// memory.  A pair is rejected on the tile only when its tile d^2 exceeds the FP32 band's upper
// end plus 1.25 times the tile error bound (tc_error_bound with M the job's largest centred
// coordinate), so the tile is only a filter: every other pair is decided exactly as on the
// CUDA cores (FP32 outside the band, the FP64 sequence inside), then tested for ownership and
// emitted.  The reported set is unchanged.  4 warps, 128 TMEM columns per block.
constexpr int kLTcK = 32;                          // hi (16) + lo (16) halves per member
constexpr int kLTcTileBytes = kTL * kLTcK * 2;     // 8 KB per 128-member tile

template <typename K, int DPAD>
struct LargeTcSmem {
  static constexpr int kLK = 64 / (int)sizeof(K);  // staged keys per member (as k_pairs_large)
  static constexpr size_t kTiles = 2 * (size_t)kLTcTileBytes;
  static constexpr size_t kRows = 2 * (size_t)kTL * DPAD * 4;
  static constexpr size_t kKeys = 2 * (size_t)kTL * (kLK + 1) * sizeof(K);
  static constexpr size_t kBytes = kTiles + kRows + kKeys + 2 * kTL * 4 /*idx*/ +
                                   2 * kTL * 4 /*norms*/ + 4 * kWarpEmit * 8 + 1024 /*align*/;
};

template <typename K, int DPAD, int MODE, bool BF16>
__global__ void __launch_bounds__(128) k_pairs_large_tc(
    const uint32_t* __restrict__ svals, const float* __restrict__ pf, int dtype,
    const K* __restrict__ key_mat, int m, const Inst* __restrict__ inst,
    const InstPlan* __restrict__ iplan, Status* st, const LargeCell* __restrict__ large,
    unsigned int cap, const unsigned long long* job_off, Sink sk, unsigned int wait_limit,
    unsigned int inject) {
  using SM = LargeTcSmem<K, DPAD>;
  constexpr int kLK = SM::kLK;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* ta = smem;
  unsigned char* tb = ta + kLTcTileBytes;
  float* ra = reinterpret_cast<float*>(tb + kLTcTileBytes);
  float* rb = ra + kTL * DPAD;
  K* ska = reinterpret_cast<K*>(rb + kTL * DPAD);
  K* skb = ska + kTL * (kLK + 1);
  uint32_t* ia = reinterpret_cast<uint32_t*>(skb + kTL * (kLK + 1));
  uint32_t* ib = ia + kTL;
  float* na = reinterpret_cast<float*>(ib + kTL);
  float* nb = na + kTL;
  unsigned long long* s_emit = reinterpret_cast<unsigned long long*>(nb + kTL);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t mbar_idle;  // test hook: a barrier nothing arrives on
  __shared__ uint32_t tmem_base;
  __shared__ unsigned int s_tally[4];
  __shared__ float s_thr, s_thr_in;
  __shared__ unsigned int s_mbits[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned long long L = min(st->large_cells, (unsigned long long)cap);
  const unsigned long long J = L ? job_off[L] : 0;
  if ((unsigned long long)blockIdx.x >= J) return;  // no job for this block: no TMEM either
  if (tid < 4) s_tally[tid] = 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_idle)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) |
                         ((128u >> 3) << 17) | ((128u >> 4) << 24);
  unsigned long long* w_emit = s_emit + (size_t)warp * kWarpEmit;
  unsigned int ecnt = 0;
  Tally tl;
  uint32_t phase = 0;
  for (unsigned long long job = blockIdx.x; job < J; job += gridDim.x) {
    long long el = 0, eh = (long long)L - 1;
    while (el < eh) {
      const long long mid = (el + eh + 1) >> 1;
      if (job_off[mid] <= job) el = mid; else eh = mid - 1;
    }
    const LargeCell cell = large[el];
    const Inst& I = inst[cell.inst];
    const int d = I.d;
    const float2 band = band_of(iplan[cell.inst]);
    const unsigned int s = cell.size;
    const long long k = (long long)(job - job_off[el]);
    long long bj = (long long)((sqrt(8.0 * (double)k + 1.0) - 1.0) * 0.5);
    while (bj * (bj + 1) / 2 > k) --bj;
    while ((bj + 1) * (bj + 2) / 2 <= k) ++bj;
    const long long bi = k - bj * (bj + 1) / 2;
    const unsigned int a0 = (unsigned int)bi * kTL, b0 = (unsigned int)bj * kTL;
    const unsigned int nA = min((unsigned int)kTL, s - a0), nB = min((unsigned int)kTL, s - b0);
    const int tg = (int)cell.grid;
    const bool kst = tg <= kLK;
    // stage member tid of each side: index, FP32 row, centred hi/lo halves, norm, key row
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // the previous job's epilogue is done with shared memory and TMEM
    const uint32_t i0 = svals[cell.start];  // the centre: the cell's first member
    float cen[DPAD];
#pragma unroll
    for (int v = 0; v < DPAD / 4; ++v) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(pf + (size_t)i0 * DPAD) + v);
      cen[4 * v] = q.x;
      cen[4 * v + 1] = q.y;
      cen[4 * v + 2] = q.z;
      cen[4 * v + 3] = q.w;
    }
    float mloc = 0.0f;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const unsigned int nn = side ? nB : nA, base = side ? b0 : a0;
      unsigned char* tile = side ? tb : ta;
      float* rows = side ? rb : ra;
      K* keys = side ? skb : ska;
      uint32_t* ids = side ? ib : ia;
      float* norms = side ? nb : na;
      const bool ok = (unsigned int)tid < nn;
      const uint32_t idx = ok ? svals[cell.start + base + tid] : i0;
      ids[tid] = idx;
      float x[DPAD];
      const float4* src = reinterpret_cast<const float4*>(pf + (size_t)idx * DPAD);
#pragma unroll
      for (int v = 0; v < DPAD / 4; ++v) {
        const float4 q = __ldg(src + v);
        reinterpret_cast<float4*>(rows + tid * DPAD)[v] = q;
        x[4 * v] = q.x;
        x[4 * v + 1] = q.y;
        x[4 * v + 2] = q.z;
        x[4 * v + 3] = q.w;
      }
      float nrm = 0.0f;
#pragma unroll
      for (int l = 0; l < 16; ++l) {
        float xc = 0.0f;
        if (l < DPAD && l < d && ok) xc = x[l < DPAD ? l : 0] - cen[l < DPAD ? l : 0];
        mloc = fmaxf(mloc, fabsf(xc));
        nrm = fmaf(xc, xc, nrm);
        if (BF16) {
          const __nv_bfloat16 h = __float2bfloat16_rn(xc);
          const __nv_bfloat16 lo = __float2bfloat16_rn(xc - __bfloat162float(h));
          *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(tid, l)) = h;
          *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(tid, 16 + l)) = lo;
        } else {
          const __half h = __float2half_rn(xc);
          const __half lo = __float2half_rn(xc - __half2float(h));
          *reinterpret_cast<__half*>(tile + tile_off(tid, l)) = h;
          *reinterpret_cast<__half*>(tile + tile_off(tid, 16 + l)) = lo;
        }
      }
      norms[tid] = nrm;
      if (kst && ok) {
        const K* kr = key_mat + (size_t)idx * m;
        K* kd = keys + tid * (kLK + 1);
        for (int u = 0; u < tg; ++u) kd[u] = __ldg(kr + u);
      }
    }
    // the job's largest centred coordinate (a bound for every staged member), and from it
    // the rejection threshold: the band's upper end plus 1.25 times the tile error bound
    float mw = mloc;
    for (int o = 16; o > 0; o >>= 1) mw = fmaxf(mw, __shfl_xor_sync(0xffffffffu, mw, o));
    if (lane == 0) s_mbits[warp] = __float_as_uint(mw);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const float M = fmaxf(fmaxf(__uint_as_float(s_mbits[0]), __uint_as_float(s_mbits[1])),
                            fmaxf(__uint_as_float(s_mbits[2]), __uint_as_float(s_mbits[3]))) *
                      (1.0f + 0x1.0p-20f);
      const double E = tc_error_bound((double)M, d, BF16);
      s_thr = isinf(band.y) ? band.y : __double2float_ru((double)band.y + 1.25 * E);
      // certainly within r below this (the band's lower end less the error bound); with the
      // FP32 filter off (band.x < 0) nothing is
      s_thr_in = band.x < 0.0f ? -1.0f : __double2float_rd((double)band.x - 1.25 * E);
      // hi.hi + hi.lo + lo.hi: A parts (0, 0, 1), B parts (0, 1, 0); 256 bytes per part
      const uint32_t aa = smem_u32(ta), bb = smem_u32(tb);
      const uint32_t asel[3] = {0u, 0u, 256u}, bsel[3] = {0u, 256u, 0u};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const uint64_t ad = make_desc(aa + asel[q]);
        const uint64_t bd = make_desc(bb + bsel[q]);
        const uint32_t acc = q > 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar)));
    }
    const bool done = mbar_wait(
        (inject & kInjectTcWait) ? smem_u32(&mbar_idle) : smem_u32(&mbar), phase, wait_limit);
    if (!__syncthreads_and(done)) {
      // give up: wait (bounded again) for the MMAs in flight before the tensor memory is freed
      mbar_wait(smem_u32(&mbar), phase, wait_limit);
      if (tid == 0) atomicOr(&st->errors, kErrTimeout);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const float thr = s_thr, thr_in = s_thr_in;
    // epilogue: warp w holds rows 32w..32w+31 (members a0 + row); 32 columns at a time
    const int row = warp * 32 + lane;
    const float nrow = na[row];
    const bool row_ok = (unsigned int)row < nA;
#pragma unroll 1
    for (int c0 = 0; c0 < kTL; c0 += 32) {
      uint32_t rr[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, rr);
      uint32_t hits = 0, inside = 0;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float d2 = (nrow + nb[c0 + q]) - 2.0f * __uint_as_float(rr[q]);
        hits |= (d2 > thr ? 0u : 1u) << q;  // NaN (non-finite tiles) is kept
        inside |= (d2 < thr_in ? 1u : 0u) << q;
      }
      // valid columns: members b0 + col < s, and a0 + row < b0 + col
      {
        const long long lo = (long long)a0 + row - (long long)b0 - c0 + 1;  // first valid q
        const long long hi = (long long)nB - c0;                           // q < hi
        const int q0 = (int)max(0LL, min(32LL, lo)), q1 = (int)max(0LL, min(32LL, hi));
        const uint32_t vm = q1 > q0 ? ((q1 - q0 == 32 ? 0xffffffffu : ((1u << (q1 - q0)) - 1u)) << q0)
                                    : 0u;
        hits &= row_ok ? vm : 0u;
      }
      // transpose the warp's 32 x 32 hit block (lane = row -> lane = column), so that the
      // lanes of a step share one row member: the emitted pairs of a step share their row,
      // as in k_pairs_large (the scatter then takes their slots with one atomic)
      inside &= hits;
      uint32_t colmask = 0, colin = 0;  // bit w: row 32 warp + w (not rejected, proved inside)
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const uint32_t b = __ballot_sync(0xffffffffu, (hits >> q) & 1u);
        const uint32_t bi2 = __ballot_sync(0xffffffffu, (inside >> q) & 1u);
        if (lane == q) {
          colmask = b;
          colin = bi2;
        }
      }
      uint32_t any = __reduce_or_sync(0xffffffffu, colmask);
      const int col = c0 + lane;
      const uint32_t iy = ib[col];
      while (any) {  // rows where some column has a pair that the tile did not reject
        const int w = __ffs(any) - 1;
        any &= any - 1;
        const int rw = warp * 32 + w;
        bool keep = false;
        unsigned int i = 0, j = 0;
        if ((colmask >> w) & 1u) {
          const uint32_t ix = ia[rw];
          i = min(ix, iy);
          j = max(ix, iy);
          const K* kx = kst ? ska + rw * (kLK + 1) : key_mat + (size_t)ix * m;
          const K* ky = kst ? skb + col * (kLK + 1) : key_mat + (size_t)iy * m;
          keep = ((colin >> w) & 1u)
                     ? decide_inside<K, MODE>(tg, kx, ky, tl)
                     : decide_pair<K, DPAD, MODE>(i, j, tg, ra + rw * DPAD, rb + col * DPAD, kx,
                                                  ky, inst + cell.inst, iplan + cell.inst, band,
                                                  dtype, tl, sk.near_r);
        }
        if (MODE == kBits) deliver_bits(keep, i, j, inst + cell.inst, sk);
        else if (MODE == kEmit) warp_emit(keep, i, j, w_emit, ecnt, sk);
        else deliver<MODE>(keep, i, j, sk, tl);
      }
    }
  }
  if (MODE == kEmit && ecnt) warp_flush(w_emit, ecnt, sk);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
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
  const float2 band = band_of(iplan[0]);
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
                                                 nullptr, inst, iplan, band, dtype, tl, sk.near_r);
      deliver<MODE>(keep, i, j, sk, tl);
    }
  }
  __syncthreads();
  flush_tally<MODE>(tl, st, s_tally);
}

// Row counts -> row pointers (exclusive scan, single pass with decoupled look-back); the
// counts are reset to zero so that the scatter or WRITE pass can use them as fill cursors.
// Each thread holds 16 consecutive counts (vector loads and stores); the first warp of a tile
// looks back over 32 predecessor tiles at a time, one per lane.
__global__ void __launch_bounds__(256) k_scan(unsigned int* row_cnt, const OutSlot* out,
                                              long long n, unsigned long long* lookback,
                                              unsigned int* tile_counter, Status* st,
                                              unsigned int tiles, unsigned int spin_limit,
                                              unsigned int inject) {
  long long* row_ptr = out->row_ptr;
  __shared__ unsigned long long sbuf[8];
  __shared__ unsigned long long s_base;
  __shared__ unsigned int s_tile;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const unsigned int tile = s_tile;
  const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
  // 16 whole counts, and both arrays 16-byte aligned (always, for device allocations)
  const bool whole = base + kScanItems <= n &&
                     ((reinterpret_cast<uintptr_t>(row_cnt) | reinterpret_cast<uintptr_t>(row_ptr)) &
                      15u) == 0;
  unsigned int v[kScanItems];
  if (whole) {
    const uint4* src = reinterpret_cast<const uint4*>(row_cnt + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) {
      const uint4 x = src[q];
      v[4 * q] = x.x;
      v[4 * q + 1] = x.y;
      v[4 * q + 2] = x.z;
      v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] = base + q < n ? row_cnt[base + q] : 0u;
  }
  unsigned long long sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) sum += v[q];
  unsigned long long total;
  const unsigned long long ex = block_excl_scan64(sum, &total, sbuf);
  if (threadIdx.x < 32) {
    const unsigned long long kAgg = 1ull << 62, kPre = 2ull << 62, kMask = (1ull << 62) - 1;
    const unsigned int full = 0xffffffffu;
    const int lane = threadIdx.x;
    unsigned long long excl = 0;
    if (tile == 0) {
      if (lane == 0) *reinterpret_cast<volatile unsigned long long*>(lookback) = kPre | total;
    } else {
      if (lane == 0)
        *reinterpret_cast<volatile unsigned long long*>(lookback + tile) = kAgg | total;
      long long p = (long long)tile - 1;  // nearest predecessor of the window (lane 0)
      unsigned int spins = 0;
      while (true) {
        const long long q = p - lane;
        // before tile 0 there is nothing: read as an inclusive prefix of zero
        const unsigned long long w =
            q >= 0 ? *reinterpret_cast<const volatile unsigned long long*>(lookback + q) : kPre;
        // (test hook: predecessors read as never published, so the wait runs to its limit)
        const unsigned int flag = (inject & kInjectScanWait) ? 0u : (unsigned int)(w >> 62);
        const unsigned int pre = __ballot_sync(full, flag == 2);
        const unsigned int upto = pre ? (((pre & (0u - pre)) - 1u) << 1 | 1u) : full;
        if (__ballot_sync(full, flag == 0) & upto) {  // a tile that matters has not published
          if (++spins > spin_limit) {
            if (lane == 0) atomicOr(&st->errors, kErrTimeout);
            break;
          }
          __nanosleep(32);
          continue;
        }
        unsigned long long add = ((upto >> lane) & 1u) ? (w & kMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(full, add, o);
        excl += add;
        if (pre) break;
        p -= 32;
      }
      if (lane == 0)
        *reinterpret_cast<volatile unsigned long long*>(lookback + tile) = kPre | (excl + total);
    }
    if (lane == 0) {
      s_base = excl;
      if (tile == tiles - 1) {
        row_ptr[n] = (long long)(excl + total);
        st->nnz = excl + total;
      }
    }
  }
  __syncthreads();
  unsigned long long run = s_base + ex;
  if (whole) {
    longlong2* dst = reinterpret_cast<longlong2*>(row_ptr + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 2; ++q) {
      longlong2 x;
      x.x = (long long)run;
      run += v[2 * q];
      x.y = (long long)run;
      run += v[2 * q + 1];
      dst[q] = x;
    }
    uint4* z = reinterpret_cast<uint4*>(row_cnt + base);
#pragma unroll
    for (int q = 0; q < kScanItems / 4; ++q) z[q] = make_uint4(0u, 0u, 0u, 0u);
  } else {
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      if (base + q < n) {
        row_ptr[base + q] = (long long)run;
        row_cnt[base + q] = 0u;
      }
      run += v[q];
    }
  }
}

// Pair buffer -> columns in their rows (row order fixed later by the row sort).
__global__ void __launch_bounds__(256) k_scatter(const unsigned long long* __restrict__ pairs,
                                                 long long cap, const Status* st,
                                                 unsigned int* row_cnt, const OutSlot* out,
                                                 int symmetric, unsigned int* errors) {
  const long long* __restrict__ row_ptr = out->row_ptr;
  int* col = out->col;
  const long long col_cap = out->col_cap;
  const long long cnt = min((long long)st->emitted, cap);
  bool overflow = false;
  // four independent pairs per thread and step, their row-pointer loads and cursor atomics in
  // flight together; lanes whose pairs share a row (a dense cell emits runs of them) take
  // consecutive slots with one atomic
  constexpr int U = 4;
  const unsigned int full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned int lt = (1u << lane) - 1u;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long w0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31); w0 < cnt;
       w0 += U * stride) {  // warp-uniform
    unsigned long long pr[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long k = w0 + lane + u * stride;
      pr[u] = k < cnt ? pairs[k] : ~0ull;
    }
    for (int side = 0; side < (symmetric ? 2 : 1); ++side) {
      long long base[U];
      unsigned int slot[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool has = pr[u] != ~0ull;
        const unsigned int row =
            has ? (side == 0 ? (unsigned int)(pr[u] >> 32) : (unsigned int)pr[u]) : 0xffffffffu;
        const unsigned int peers = __match_any_sync(full, row);
        const int leader = __ffs(peers) - 1;
        unsigned int b0 = 0;
        if (has && lane == leader) b0 = atomicAdd(&row_cnt[row], (unsigned int)__popc(peers));
        b0 = __shfl_sync(full, b0, leader);
        slot[u] = b0 + (unsigned int)__popc(peers & lt);
        base[u] = has ? row_ptr[row] : 0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (pr[u] != ~0ull) {
          const long long pos = base[u] + slot[u];
          const int v = side == 0 ? (int)(unsigned int)pr[u] : (int)(pr[u] >> 32);
          if (pos < col_cap) col[pos] = v; else overflow = true;
        }
      }
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

constexpr int kWarpRowMax = 256;  // rows up to this length are sorted by one warp

// One thread per row: rows of at most 32 entries are sorted in registers (bitonic network
// with +infinity padding).  Longer rows are queued in row_queue (n entries): rows of up to
// kWarpRowMax entries from the front for the warp kernel, longer ones from the back for the
// block kernel.  Rows that reach past col_cap (only when an undersized buffer overflowed and
// the build will be re-run) are left alone.
__global__ void __launch_bounds__(256) k_rowsort_thread(const OutSlot* out, long long n,
                                                        unsigned int* row_queue,
                                                        unsigned int* mid_count,
                                                        unsigned int* long_count,
                                                        unsigned int* errors, int skip_long,
                                                        unsigned int* rows_over_margin) {
  const long long* __restrict__ row_ptr = out->row_ptr;
  int* col = out->col;
  const long long col_cap = out->col_cap;
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long b = row < n ? row_ptr[row] : 0, len = row < n ? row_ptr[row + 1] - b : 0;
  // a row near the queued sorts' threshold keeps them in the next build of the shape (one
  // atomic for a warp that has one)
  if (__any_sync(0xffffffffu, len > kSkipMargin) && (threadIdx.x & 31) == 0)
    atomicOr(rows_over_margin, 1u);
  if (row >= n) return;
  if (len <= 1 || b + len > col_cap) return;
  // the queued row sorts were left out of this launch: the host runs it again
  if (skip_long && len > 32) atomicOr(errors, kErrTailSkipped);
  if (len > kWarpRowMax) {
    row_queue[n - 1 - atomicAdd(long_count, 1u)] = (unsigned int)row;
    return;
  }
  if (len > 32) {
    row_queue[atomicAdd(mid_count, 1u)] = (unsigned int)row;
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

// One row of at most 32 V entries sorted by one warp: lane l holds entries l V .. l V + V - 1
// in registers (+infinity padding); bitonic network, exchanges across lanes by shuffles.
template <int V>
__device__ __forceinline__ void warp_sort_row(int* a, int len) {
  constexpr int L = 32 * V;
  const int lane = threadIdx.x & 31;
  int v[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const int e = lane * V + q;
    v[q] = e < len ? a[e] : INT_MAX;
  }
#pragma unroll
  for (int k = 2; k <= L; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= V) {
        const int lj = j / V;  // partner lane distance
        const bool low = (lane & lj) == 0;
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int other = __shfl_xor_sync(0xffffffffu, v[q], lj);
          const bool up = ((lane * V + q) & k) == 0;
          v[q] = (up == low) ? min(v[q], other) : max(v[q], other);
        }
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q) {
          const int p = q ^ j;
          if (p > q) {
            const bool up = ((lane * V + q) & k) == 0;
            if (up ? v[q] > v[p] : v[q] < v[p]) {
              const int t = v[q];
              v[q] = v[p];
              v[p] = t;
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const int e = lane * V + q;
    if (e < len) a[e] = v[q];
  }
}

constexpr int kRowSmem = 16384;       // entries of a long row sorted in shared memory (64 KB)
constexpr int kRowSortThreads = 256;  // threads of a block of the queued-row sort
constexpr int kRowRadixMax = kRowSmem;  // longest row of the radix path

// Stable LSD radix sort, 4-bit digits, of one row of len non-negative values below 2^bits:
// the passes alternate between `row` and the buffer sm, and the result ends in `row` (the
// row in global memory with a shared buffer, or two halves of the shared buffer).  Thread t
// owns the contiguous chunk [t C, (t + 1) C); its digit counts sit in column t of cnt
// (16 x blockDim entries, digit major), whose exclusive scan in that order gives every thread
// its output offsets, so equal digits keep their order.
__device__ void block_radix_row(int* row, int* sm, unsigned short* cnt, unsigned int* sbuf,
                                int len, int bits) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int C = (len + T - 1) / T;
  const int beg = min(len, tid * C), end = min(len, beg + C);
  int* src = row;
  int* dst = sm;
  for (int shift = 0; shift < bits; shift += 4) {
#pragma unroll
    for (int dg = 0; dg < 16; ++dg) cnt[dg * T + tid] = 0;
    for (int x = beg; x < end; ++x) ++cnt[((src[x] >> shift) & 15) * T + tid];
    __syncthreads();
    // exclusive scan of the 16 T counts in digit-major order: thread t takes entries
    // [16 t, 16 t + 16) of that order
    unsigned int v[16], sum = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      v[q] = cnt[16 * tid + q];
      sum += v[q];
    }
    unsigned int total;
    unsigned int run = block_excl_scan_any(sum, &total, sbuf);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      cnt[16 * tid + q] = (unsigned short)run;
      run += v[q];
    }
    __syncthreads();
    for (int x = beg; x < end; ++x) {
      const int val = src[x];
      unsigned short& o = cnt[((val >> shift) & 15) * T + tid];
      dst[o] = val;
      ++o;
    }
    __syncthreads();
    int* t = src;
    src = dst;
    dst = t;
  }
  if (src != row) {  // an odd number of passes: the result is in the shared buffer
    for (int x = tid; x < len; x += T) row[x] = src[x];
  }
}

// The queued rows: first one block per row of more than kWarpRowMax entries (bitonic sort in
// shared memory, or in place when the row is longer than the buffer), then one warp per row of
// kSmallCell + 1 .. kWarpRowMax entries (register sort).  Rows of dense clusters run to
// thousands of entries: a 64 KB buffer per block keeps them out of global memory, with three
// blocks per SM working on different rows.
__global__ void __launch_bounds__(kRowSortThreads) k_rowsort_queued(
    const OutSlot* out, long long n, const unsigned int* __restrict__ row_queue,
    const unsigned int* long_count, const unsigned int* mid_count, int bits) {
  const long long* __restrict__ row_ptr = out->row_ptr;
  int* col = out->col;
  const long long col_cap = out->col_cap;
  extern __shared__ int buf[];  // kRowSmem entries, then the radix counts
  unsigned short* rcnt = reinterpret_cast<unsigned short*>(buf + kRowSmem);  // 16 x blockDim
  __shared__ unsigned int rsbuf[kRowSortThreads / 32];
  __shared__ int s_lo, s_hi;
  const unsigned int cnt = *long_count;
  for (unsigned int k = blockIdx.x; k < cnt; k += gridDim.x) {
    const unsigned int row = row_queue[n - 1 - k];
    const long long b = row_ptr[row], len = row_ptr[row + 1] - b;
    if (b + len > col_cap) continue;  // uniform across the block: same row for all threads
    long long L = 1;
    while (L < len) L <<= 1;
    // Dense rows (columns within a span of at most 64 per entry, as in clustered builds): a
    // bit per value of the span in shared memory, set and then read back in order, which
    // costs span / 32 + len steps instead of one radix pass per 4 bits of the columns.
    {
      int lo = INT_MAX, hi = -1;
      for (long long x = threadIdx.x; x < len; x += blockDim.x) {
        const int v = col[b + x];
        lo = min(lo, v);
        hi = max(hi, v);
      }
      for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      __syncthreads();  // the previous row is done with buf, s_lo and s_hi
      if (threadIdx.x == 0) {
        s_lo = INT_MAX;
        s_hi = -1;
      }
      __syncthreads();
      if ((threadIdx.x & 31) == 0) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
      }
      __syncthreads();
      lo = s_lo;
      hi = s_hi;
      const long long span = (long long)hi - lo + 1;
      if (span >= 1 && span <= 32LL * kRowSmem && span <= 64 * len) {
        unsigned int* bm = reinterpret_cast<unsigned int*>(buf);
        const int words = (int)((span + 31) >> 5);
        for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        for (long long x = threadIdx.x; x < len; x += blockDim.x) {
          const int v = col[b + x] - lo;
          atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
        __syncthreads();
        // thread t reads a contiguous stretch of words; a block scan of the bit counts gives
        // each stretch's first output position
        const int per = (words + (int)blockDim.x - 1) / (int)blockDim.x;
        const int w0 = min(words, (int)threadIdx.x * per), w1 = min(words, w0 + per);
        unsigned int c = 0;
        for (int w = w0; w < w1; ++w) c += (unsigned int)__popc(bm[w]);
        unsigned int total;
        long long pos = b + block_excl_scan_any(c, &total, rsbuf);
        for (int w = w0; w < w1; ++w) {
          unsigned int word = bm[w];
          while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1;
            col[pos++] = lo + w * 32 + bit;
          }
        }
        continue;
      }
    }
    if (len <= kRowSmem / 2) {  // both buffers in shared memory
      for (long long x = threadIdx.x; x < len; x += blockDim.x) buf[x] = col[b + x];
      __syncthreads();
      block_radix_row(buf, buf + kRowSmem / 2, rcnt, rsbuf, (int)len, bits);
      for (long long x = threadIdx.x; x < len; x += blockDim.x) col[b + x] = buf[x];
    } else if (len <= kRowRadixMax) {  // passes alternate between the row and the buffer
      block_radix_row(col + b, buf, rcnt, rsbuf, (int)len, bits);
    } else if (L <= kRowSmem) {
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
  // rows of kSmallCell + 1 .. kWarpRowMax entries, one warp each
  const unsigned int mcnt = *mid_count;
  const unsigned int warps = gridDim.x * (blockDim.x >> 5);
  for (unsigned int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < mcnt;
       k += warps) {
    const unsigned int row = row_queue[k];
    const long long b = row_ptr[row];
    const int len = (int)(row_ptr[row + 1] - b);
    if (len <= 64) warp_sort_row<2>(col + b, len);
    else if (len <= 128) warp_sort_row<4>(col + b, len);
    else warp_sort_row<8>(col + b, len);
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
  sk.errors = &a.st->errors;
  sk.near_r = &a.st->near_r;
  sk.bits = a.bits;
  sk.symmetric = a.symmetric;
  return sk;
}

template <int DPAD, int MODE>
void brute_impl(const BuildArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(8 * a.num_sms);
  k_brute<DPAD, MODE><<<blocks, kPairThreads, 0, s>>>(a.pf, a.dtype, a.inst, a.iplan, a.st,
                                                      make_sink(a));
}

// Cells of more points than this go to the tiled kernels (the tuned value, else kMediumMax;
// never above kMediumMax, the medium kernel's staging capacity).
inline unsigned int dense_min_of(const BuildArgs& a) {
  return a.dense_min > 0 && a.dense_min <= kMediumMax ? (unsigned int)a.dense_min
                                                      : (unsigned int)kMediumMax;
}

// The dense-cell jobs on the tensor cores (FP16 or BF16 halves), 4 blocks of 128 threads per
// SM (128 TMEM columns each).
template <typename K, int DPAD, int MODE>
void large_tc_launch(const BuildArgs& a, const uint32_t* sv, cudaStream_t s) {
  using SM = LargeTcSmem<K, DPAD>;
  const bool bf16 = a.tc_cells == 2;
  auto kern = bf16 ? k_pairs_large_tc<K, DPAD, MODE, true> : k_pairs_large_tc<K, DPAD, MODE, false>;
  static bool attr[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(launch_attr_mutex());
    if (dev < 0 || dev >= 64 || !attr[dev][bf16]) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM::kBytes);
      if (dev >= 0 && dev < 64) attr[dev][bf16] = true;
    }
  }
  kern<<<(unsigned)(4 * a.num_sms), 128, SM::kBytes, s>>>(
      sv, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.st, a.large, a.large_cap,
      a.large_job_off, make_sink(a), spin_limit_of(a.spin_limit) * 16u, a.inject);
}

template <typename K, int DPAD, int MODE>
void pairs_mode(const BuildArgs& a, int sorted_buf, cudaStream_t s) {
  const long long N = a.n_total * a.m;
  constexpr int kWarps = kPairThreads / 32;
  const bool stage_rows = a.m * (int)sizeof(K) <= kMaxStagedRow;
  const int wbytes = warp_region_bytes<K, DPAD>(a.m, stage_rows);
  const size_t smem = (size_t)wbytes * kWarps;
  // spans of a multiple of 32 positions (64..1024), about a.spans_per_warp of them per
  // resident warp (more when spans would pass 1024 positions), for one wave of warps
  const long long resident = 4LL * a.num_sms * kWarps;
  long long W = a.spans_per_warp > 0 ? a.spans_per_warp : 1;
  W = std::max(W, (N + 1024 * resident - 1) / (1024 * resident));  // spans of at most 1024
  long long span = (N + W * resident - 1) / (W * resident);
  span = (span + 31) / 32 * 32;
  span = span < 64 ? 64 : (span > 1024 ? 1024 : span);
  const long long nspans = (N + span - 1) / span;
  long long blocks = (nspans + kWarps - 1) / kWarps;
  if (blocks > 4LL * a.num_sms) blocks = 4LL * a.num_sms;
  const K* sk = (const K*)a.keys[sorted_buf];
  const uint32_t* sv = a.vals[sorted_buf];
  static size_t attr_smem[64] = {};  // largest size granted so far, per device
  int dev = 0;
  cudaGetDevice(&dev);
  const bool rows16 = (a.m * (int)sizeof(K)) % 16 == 0;  // key rows of whole 16-byte blocks
  auto kern = !stage_rows ? k_pairs_warp<K, DPAD, MODE, 0>
                          : (rows16 ? k_pairs_warp<K, DPAD, MODE, 2> : k_pairs_warp<K, DPAD, MODE, 1>);
  {
    std::lock_guard<std::mutex> lk(launch_attr_mutex());
    if (dev < 0 || dev >= 64 || smem > attr_smem[dev]) {
      cudaFuncSetAttribute(k_pairs_warp<K, DPAD, MODE, 0>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_pairs_warp<K, DPAD, MODE, 1>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(k_pairs_warp<K, DPAD, MODE, 2>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (dev >= 0 && dev < 64) attr_smem[dev] = smem;
    }
  }
  kern<<<(unsigned)blocks, kPairThreads, smem, s>>>(
      sk, sv, N, span, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.bases,
      a.B * a.m, a.st, make_sink(a), a.large, a.large_cap, wbytes,
      &a.st->span_next[MODE == kWrite ? 1 : 0], (a.skip_tail & kSkipDense) ? 1 : 0,
      a.cell_major);
  if (a.skip_tail & kSkipDense) return;  // (k_pairs_warp flags any dense cell it meets)
  {
    const size_t msmem =
        (size_t)kMediumWarps * kMediumMax * (DPAD * 4 + 4) + (size_t)kMediumWarps * kMediumKeyBytes;
    // one wave of resident blocks (the kernel loops over the cells): a build without medium
    // cells pays for a single wave of blocks that find nothing to do
    static bool mattr[64] = {};
    static int mocc[64] = {};
    int mper = 2;
    {
      std::lock_guard<std::mutex> lk(launch_attr_mutex());
      if (dev >= 0 && dev < 64 && !mattr[dev]) {
        cudaFuncSetAttribute(k_pairs_medium<K, DPAD, MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pairs_medium<K, DPAD, MODE>,
                                                          kMediumWarps * 32,
                                                          msmem) != cudaSuccess)
          occ = 0;
        mocc[dev] = occ;
        mattr[dev] = true;
      }
      if (dev >= 0 && dev < 64 && mocc[dev] > 0) mper = mocc[dev];
    }
    k_pairs_medium<K, DPAD, MODE><<<(unsigned)(mper * a.num_sms), kMediumWarps * 32, msmem, s>>>(
        sv, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.st, a.large, a.large_cap,
        make_sink(a), dense_min_of(a));
  }
  if (MODE != kWrite)
    k_large_setup<<<1, 1024, 0, s>>>(a.large, a.large_cap, a.st, a.large_job_off, dense_min_of(a));
  if constexpr (MODE != kBits) {
    if (a.tc_cells) {
      large_tc_launch<K, DPAD, MODE>(a, sv, s);
      return;
    }
  }
  k_pairs_large<K, DPAD, MODE><<<(unsigned)(4 * a.num_sms), kPairThreads, 0, s>>>(
      sv, a.pf, a.dtype, (const K*)a.key_mat, a.m, a.inst, a.iplan, a.st, a.large, a.large_cap,
      a.large_job_off, make_sink(a));
}

template <typename K, int DPAD>
int pairs_impl(const BuildArgs& a, int sorted_buf, Mode mode, cudaStream_t s) {
  const bool dense = !(a.skip_tail & kSkipDense);
  switch (mode) {
    case kCount: pairs_mode<K, DPAD, kCount>(a, sorted_buf, s); return dense ? 4 : 1;
    case kWrite: pairs_mode<K, DPAD, kWrite>(a, sorted_buf, s); return dense ? 3 : 1;
    case kBits: pairs_mode<K, DPAD, kBits>(a, sorted_buf, s); return dense ? 4 : 1;
    default: pairs_mode<K, DPAD, kEmit>(a, sorted_buf, s); return dense ? 4 : 1;
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

void reset_pairs_state(const BuildArgs& a, cudaStream_t s) {
  cudaMemsetAsync(&a.st->large_cells, 0, sizeof(a.st->large_cells), s);
  cudaMemsetAsync(&a.st->large_jobs, 0, sizeof(a.st->large_jobs), s);
  cudaMemsetAsync(&a.st->span_next[0], 0, sizeof(a.st->span_next), s);
  cudaMemsetAsync(&a.st->emitted, 0, sizeof(a.st->emitted), s);
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
  if (!a.scan_zeroed) cudaMemsetAsync(a.scan_lookback, 0, (size_t)tiles * 8, s);
  k_scan<<<tiles, 256, 0, s>>>(a.row_cnt, a.out, a.n_total, a.scan_lookback,
                               &a.st->scan_tiles, a.st, tiles, spin_limit_of(a.spin_limit),
                               a.inject);
}

namespace {

// Instance of a global point index (the last instance whose first point is at most i).
__device__ __forceinline__ int instance_of(const Inst* __restrict__ inst, int B, long long i) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].p0 <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One warp per row: the row's count is the population of its matrix row.
__global__ void __launch_bounds__(256) k_bits_count(const Inst* __restrict__ inst, int B,
                                                    const unsigned int* __restrict__ bits,
                                                    unsigned int* row_cnt, long long n_total) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n_total;
       i += warps) {
    const Inst& I = inst[instance_of(inst, B, i)];
    const unsigned int* row = bits + I.bits_off + (i - I.p0) * I.bits_w;
    unsigned int c = 0;
    for (int w = lane; w < I.bits_w; w += 32) c += (unsigned int)__popc(row[w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) row_cnt[i] = c;
  }
}

// One warp per row: set bits become the row's columns, in ascending order (32 words at a
// time, a warp scan placing each word's bits).
__global__ void __launch_bounds__(256) k_bits_write(const Inst* __restrict__ inst, int B,
                                                    const unsigned int* __restrict__ bits,
                                                    const OutSlot* out, long long n_total) {
  const long long* __restrict__ row_ptr = out->row_ptr;
  int* col = out->col;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n_total;
       i += warps) {
    const Inst& I = inst[instance_of(inst, B, i)];
    const unsigned int* row = bits + I.bits_off + (i - I.p0) * I.bits_w;
    long long pos = row_ptr[i];
    for (int w0 = 0; w0 < I.bits_w; w0 += 32) {
      const int w = w0 + lane;
      unsigned int word = w < I.bits_w ? row[w] : 0u;
      const unsigned int c = (unsigned int)__popc(word);
      unsigned int incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      long long p = pos + (incl - c);
      while (word) {
        const int b = __ffs(word) - 1;
        word &= word - 1;
        col[p++] = (int)(I.p0 + (long long)w * 32 + b);
      }
      pos += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
}

unsigned bits_blocks(const BuildArgs& a) {
  long long blocks = (a.n_total + 7) / 8;
  if (blocks > 16LL * a.num_sms) blocks = 16LL * a.num_sms;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

}  // namespace

int launch_bits_count(const BuildArgs& a, cudaStream_t s) {
  k_bits_count<<<bits_blocks(a), 256, 0, s>>>(a.inst, a.B, a.bits, a.row_cnt, a.n_total);
  return 1;
}

int launch_bits_write(const BuildArgs& a, cudaStream_t s) {
  k_bits_write<<<bits_blocks(a), 256, 0, s>>>(a.inst, a.B, a.bits, a.out, a.n_total);
  return 1;
}

int launch_scatter(const BuildArgs& a, cudaStream_t s) {
  k_scatter<<<(unsigned)(8 * a.num_sms), 256, 0, s>>>(a.pair_buf, a.pair_cap, a.st, a.row_cnt,
                                                      a.out, a.symmetric, &a.st->errors);
  return 1;
}

int launch_rowsort(const BuildArgs& a, cudaStream_t s, long long col_bound) {
  const unsigned blocks = (unsigned)((a.n_total + 255) / 256);
  unsigned int* long_count = &a.st->long_rows;
  unsigned int* mid_count = &a.st->mid_rows;
  const int skip_long = (a.skip_tail & kSkipLongRows) ? 1 : 0;
  k_rowsort_thread<<<blocks, 256, 0, s>>>(a.out, a.n_total, a.row_cnt, mid_count, long_count,
                                          &a.st->errors, skip_long, &a.st->rows_over_margin);
  if (skip_long) return 1;
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::unique_lock<std::mutex> lk(launch_attr_mutex());
  const size_t smem =
      (size_t)kRowSmem * sizeof(int) + 16 * kRowSortThreads * sizeof(unsigned short);
  const long long bound = col_bound >= 0 ? col_bound : a.n_total;  // columns lie below it
  int bits = 1;
  while (bits < 31 && (1LL << bits) < bound) ++bits;
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaFuncSetAttribute(k_rowsort_queued, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  lk.unlock();
  k_rowsort_queued<<<(unsigned)(3 * a.num_sms), kRowSortThreads, smem, s>>>(a.out, a.n_total,
                                                                            a.row_cnt,
                                                              long_count, mid_count, bits);
  return 2;
}

}  // namespace rtg
