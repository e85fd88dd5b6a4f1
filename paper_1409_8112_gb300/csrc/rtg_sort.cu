// LSD radix sort of (key, point index) pairs: groups the points of every grid by cell
// (Alg. 1 of arXiv:1409.8112 associates each point with its cell; the sort makes every cell
// a contiguous run).  Stable.
//
// Compile-time variants: digit width BITS (8, 9, 10 or 11 bits per pass, so a key of b bits takes
// ceil(b / BITS) passes) and ITEMS keys per thread (tiles of 256 * ITEMS keys).  The
// autotuner in the host code picks one variant and one pass strategy per shape.
//
// One kernel counts the digits of every pass in a single read of the keys (global digit
// offsets).  A pass is then either
//   * look-back: one kernel; tiles take their index from an atomic counter, publish their
//     digit counts and find their offsets by decoupled look-back over earlier tiles (bounded
//     waits), or
//   * reduce-then-scan: an upsweep counts the digits of every tile, a scan turns the
//     per-(digit, tile) counts into output offsets, and a downsweep places the keys.
// Both rank each tile's keys with a warp-level multisplit (peer masks from one ballot per
// digit bit, per-warp 16-bit digit counters), reorder the tile in shared memory and write each
// digit's run contiguously.
#include <cuda_runtime.h>

#include "rtg_internal.cuh"

#include <mutex>
#include <type_traits>

namespace rtg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

template <int BITS>
struct Digits {
  static constexpr int kCount = 1 << BITS;
  static constexpr int kPerThread = kCount / kSortThreads;
  static_assert(kCount % kSortThreads == 0, "digit count must be a multiple of the block");
};

template <typename K, int BITS, int ITEMS>
struct SortShape {
  static constexpr int kTile = kSortThreads * ITEMS;
  static constexpr int kDigits = 1 << BITS;
  // keys, values, tile digit starts, global digit starts, per-warp 16-bit counters
  static constexpr size_t kSmem = (size_t)kTile * (sizeof(K) + 4) + (size_t)kDigits * 8 +
                                  (size_t)kSortWarps * kDigits * 2;
};

#ifndef RTG_SORT_WIN
#define RTG_SORT_WIN 4  // look-back window: predecessors read per round
#endif
constexpr unsigned long long kFlagAgg = 1ull, kFlagPrefix = 2ull;

__device__ __forceinline__ unsigned long long pack_lb(unsigned long long flag, unsigned int epoch,
                                                      unsigned int value) {
  return (flag << 62) | ((unsigned long long)(epoch & 0x3fffffffu) << 32) | value;
}
__device__ __forceinline__ void st_volatile(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Lanes of the warp whose digit equals this lane's (BITS ballots).  `valid` lanes only; an
// invalid lane gets an arbitrary mask.
template <int BITS>
__device__ __forceinline__ unsigned int peer_mask(unsigned int dg, bool valid) {
  unsigned int peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < BITS; ++b) {
    const bool bit = (dg >> b) & 1u;
    const unsigned int m = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? m : ~m;
  }
  return peers;
}

// Exclusive scan of one value per thread over a 256-thread block; returns the block total
// through *total.
__device__ __forceinline__ unsigned int block_excl_scan_256(unsigned int v, unsigned int* total,
                                                            unsigned int* sbuf /*8*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sbuf[warp] = x;
  __syncthreads();
  unsigned int wpre = 0, tot = 0;
  for (int w = 0; w < kSortWarps; ++w) {
    const unsigned int c = sbuf[w];
    if (w < warp) wpre += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return wpre + x - v;
}

// Adds one to the digit counter of every valid lane; a warp whose lanes share one digit
// (the high digits of neighbouring keys) makes a single add.
__device__ __forceinline__ void count_digit(unsigned int* sh, unsigned int dg, bool valid,
                                            unsigned int vmask) {
  const unsigned int d0 = __shfl_sync(0xffffffffu, dg, 0);
  if (__all_sync(0xffffffffu, !valid || dg == d0)) {
    if ((threadIdx.x & 31) == 0 && vmask) atomicAdd(&sh[d0], (unsigned int)__popc(vmask));
  } else if (valid) {
    atomicAdd(&sh[dg], 1u);
  }
}

// Digit counts of every pass in one read; the last block turns them into exclusive digit
// offsets (digit_off[p * D + digit]) and clears the counts for the next sort.
template <typename K, int BITS>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K* __restrict__ keys,
                                                            long long N, int passes,
                                                            unsigned int* hist,
                                                            unsigned int* digit_off,
                                                            unsigned int* ticket,
                                                            unsigned int* epoch) {
  constexpr int D = Digits<BITS>::kCount, PT = Digits<BITS>::kPerThread;
  extern __shared__ unsigned int sh[];  // passes * D
  __shared__ unsigned int sbuf[kSortWarps];
  __shared__ bool last;
  for (int x = threadIdx.x; x < passes * D; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long step = (long long)gridDim.x * blockDim.x;
  // warp-uniform loop so that the warp votes see every lane
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < N;
       base += step) {
    const long long x = base + lane;
    const bool valid = x < N;
    const K k = valid ? keys[x] : (K)0;
    const unsigned int vmask = __ballot_sync(0xffffffffu, valid);
    for (int p = 0; p < passes; ++p)
      count_digit(sh + p * D, (unsigned int)(k >> (p * BITS)) & (D - 1), valid, vmask);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < passes * D; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int p = 0; p < passes; ++p) {
    unsigned int v[PT], sum = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      v[q] = __ldcg(&hist[p * D + threadIdx.x * PT + q]);
      sum += v[q];
    }
    unsigned int tot;
    unsigned int run = block_excl_scan_256(sum, &tot, sbuf);
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      digit_off[p * D + threadIdx.x * PT + q] = run;
      run += v[q];
      hist[p * D + threadIdx.x * PT + q] = 0;  // ready for the next sort
    }
  }
  if (threadIdx.x == 0) {
    *ticket = 0;
    // a fresh look-back epoch for this sort's passes (never 0: zeroed words are never valid)
    unsigned int e = *epoch + kMaxPasses;
    if ((e & 0x3fffffffu) < (unsigned int)kMaxPasses) e = 1;
    *epoch = e;
  }
}

// Digit counts of every tile of this pass, stored digit-major: counts[digit * tiles + tile].
template <typename K, int BITS, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_sort_upsweep(const K* __restrict__ kin,
                                                               long long N, int shift,
                                                               unsigned int* counts,
                                                               unsigned int tiles) {
  constexpr int D = Digits<BITS>::kCount;
  constexpr int kTile = kSortThreads * ITEMS;
  __shared__ unsigned int sh[D];
  for (int x = threadIdx.x; x < D; x += kSortThreads) sh[x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const long long pos = base + j * kSortThreads + threadIdx.x;
    const bool valid = pos < N;
    const unsigned int dg = valid ? (unsigned int)(kin[pos] >> shift) & (D - 1) : 0u;
    count_digit(sh, dg, valid, __ballot_sync(0xffffffffu, valid));
  }
  __syncthreads();
  for (int x = threadIdx.x; x < D; x += kSortThreads)
    counts[(size_t)x * tiles + blockIdx.x] = sh[x];
}

// One block per digit: exclusive scan of its per-tile counts, offset by the digit's global
// start, in place.
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned int* counts, unsigned int tiles,
                                                    const unsigned int* __restrict__ digit_off) {
  __shared__ unsigned int sbuf[32];
  __shared__ unsigned int carry;
  unsigned int* row = counts + (size_t)blockIdx.x * tiles;
  if (threadIdx.x == 0) carry = digit_off[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned int b = 0; b < tiles; b += blockDim.x) {
    const unsigned int t = b + threadIdx.x;
    const unsigned int v = t < tiles ? row[t] : 0u;
    unsigned int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sbuf[warp] = x;
    __syncthreads();
    unsigned int wpre = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) wpre += sbuf[w];
      tot += sbuf[w];
    }
    if (t < tiles) row[t] = carry + wpre + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
}

// Shared work of the two pass kernels: load a tile, rank its keys (stable), reorder it in
// shared memory.  Afterwards s_tdig[d] is the tile-local start of digit d and tcount[q] the
// tile's count of digit tid * PT + q; the caller fills s_gbase and writes the tile out.
template <typename K, int BITS, int ITEMS>
struct TileRank {
  static constexpr int D = Digits<BITS>::kCount, PT = Digits<BITS>::kPerThread;
  static constexpr int kTile = kSortThreads * ITEMS;
  K* s_keys;
  uint32_t* s_vals;
  unsigned int* s_tdig;     // D
  unsigned int* s_gbase;    // D
  unsigned short* s_whist;  // kSortWarps * D

  __device__ explicit TileRank(unsigned char* smem) {
    s_keys = reinterpret_cast<K*>(smem);
    s_vals = reinterpret_cast<uint32_t*>(s_keys + kTile);
    s_tdig = s_vals + kTile;
    s_gbase = s_tdig + D;
    s_whist = reinterpret_cast<unsigned short*>(s_gbase + D);
  }

  // vin == nullptr: the input is the point-major key-row array, whose position pos holds
  // point pos / m (vdiv = ceil(2^64 / m), exact for pos < 2^31; m = 1 passes vdiv = 0).
  // FULL: every position of the tile is below N (all tiles but the last), so no lane tests it.
  template <bool FULL>
  __device__ void rank(const K* __restrict__ kin, const uint32_t* __restrict__ vin, long long N,
                       long long tile_base, int shift, unsigned int (&tcount)[PT],
                       unsigned int* sbuf, unsigned long long vdiv) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned int* wz = reinterpret_cast<unsigned int*>(s_whist);
    for (int x = tid; x < kSortWarps * D / 2; x += kSortThreads) wz[x] = 0;
    __syncthreads();
    const long long wbase = tile_base + (long long)warp * 32 * ITEMS;
    K key[ITEMS];
    uint32_t val[ITEMS];
    unsigned int rk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const long long pos = wbase + j * 32 + lane;
      if (FULL || pos < N) {
        key[j] = kin[pos];
        val[j] = vin ? vin[pos]
                     : (vdiv ? (uint32_t)__umul64hi((unsigned long long)pos, vdiv) : (uint32_t)pos);
      } else {
        key[j] = (K)0;
        val[j] = 0;
      }
    }
    unsigned short* wh = s_whist + warp * D;
    const unsigned int lt = (1u << lane) - 1;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const bool valid = FULL || wbase + j * 32 + lane < N;
      const unsigned int dg = (unsigned int)(key[j] >> shift) & (D - 1);
      const unsigned int peers = peer_mask<BITS>(dg, valid);
      const unsigned int before = valid ? wh[dg] : 0u;
      __syncwarp();
      if (valid && (peers & lt) == 0) wh[dg] = (unsigned short)(before + __popc(peers));
      __syncwarp();
      rk[j] = before + (unsigned int)__popc(peers & lt);
    }
    __syncthreads();
    // thread tid owns digits tid * PT .. tid * PT + PT - 1: warp-exclusive offsets, tile counts
    unsigned int sum = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int d = tid * PT + q;
      unsigned int run = 0;
      for (int w = 0; w < kSortWarps; ++w) {
        const unsigned int c = s_whist[w * D + d];
        s_whist[w * D + d] = (unsigned short)run;
        run += c;
      }
      tcount[q] = run;
      sum += run;
    }
    unsigned int tot;
    unsigned int start = block_excl_scan_256(sum, &tot, sbuf);
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      s_tdig[tid * PT + q] = start;
      start += tcount[q];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const bool valid = FULL || wbase + j * 32 + lane < N;
      if (valid) {
        const unsigned int dg = (unsigned int)(key[j] >> shift) & (D - 1);
        const unsigned int local = s_tdig[dg] + s_whist[warp * D + dg] + rk[j];
        s_keys[local] = key[j];
        s_vals[local] = val[j];
      }
    }
  }

  // Writes the reordered tile (after a barrier that publishes s_gbase and the tile).  Offsets
  // outside [0, N) (digit counts that do not belong to these keys) are dropped and flagged.
  // REB (last pass of a cell-major sort): the values are grid-major positions q = g n + i;
  // the key written is the cell index plus grid g's base and the value is the point i
  // (g = floor(q / n) by a multiply-high with rdiv = ceil(2^64 / n), exact for q, n < 2^31).
  template <bool FULL, bool REB>
  __device__ void write(K* __restrict__ kout, uint32_t* __restrict__ vout, long long N,
                        long long tile_base, int shift, unsigned int* errors,
                        const unsigned long long* __restrict__ rbases, unsigned int rn,
                        unsigned long long rdiv) {
    const long long rem = N - tile_base;
    const int tvalid = FULL ? kTile : (rem < kTile ? (int)rem : kTile);
    const unsigned int nu = (unsigned int)N;  // the host keeps N below 2^31
    bool bad = false;
#pragma unroll 4
    for (int x = threadIdx.x; x < tvalid; x += kSortThreads) {
      const K k = s_keys[x];
      const unsigned int dg = (unsigned int)(k >> shift) & (D - 1);
      const unsigned int dst = s_gbase[dg] + (unsigned int)x - s_tdig[dg];
      if (dst < nu) {
        if (REB) {
          const uint32_t q = s_vals[x];
          const uint32_t g = (uint32_t)__umul64hi((unsigned long long)q, rdiv);
          kout[dst] = k + (K)__ldg(rbases + g);
          vout[dst] = q - g * rn;
        } else {
          kout[dst] = k;
          vout[dst] = s_vals[x];
        }
      } else {
        bad = true;
      }
    }
    if (bad) atomicOr(errors, kErrSortRange);
  }
};

template <typename K, int BITS, int ITEMS, bool REB>
__global__ void __launch_bounds__(kSortThreads) k_sort_downsweep(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, long long N, int shift, const unsigned int* __restrict__ offs,
    unsigned int tiles, unsigned int* errors, unsigned long long vdiv,
    const unsigned long long* __restrict__ rbases, unsigned int rn, unsigned long long rdiv) {
  using TR = TileRank<K, BITS, ITEMS>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int sbuf[kSortWarps];
  TR tr(smem);
  for (int x = threadIdx.x; x < TR::D; x += kSortThreads)
    tr.s_gbase[x] = offs[(size_t)x * tiles + blockIdx.x];
  const long long tile_base = (long long)blockIdx.x * TR::kTile;
  unsigned int tcount[TR::PT];
  const bool full = tile_base + TR::kTile <= N;
  if (full) tr.template rank<true>(kin, vin, N, tile_base, shift, tcount, sbuf, vdiv);
  else tr.template rank<false>(kin, vin, N, tile_base, shift, tcount, sbuf, vdiv);
  __syncthreads();
  if (full) tr.template write<true, REB>(kout, vout, N, tile_base, shift, errors, rbases, rn, rdiv);
  else tr.template write<false, REB>(kout, vout, N, tile_base, shift, errors, rbases, rn, rdiv);
}

// Single-kernel pass with decoupled look-back (tiles take their index from an atomic
// counter, so a tile waits only on tiles already running; each wait is bounded).  Cheaper
// than reduce-then-scan while all tiles fit in about one wave.
template <typename K, int BITS, int ITEMS, bool REB>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, long long N, int shift, const unsigned int* __restrict__ digit_off,
    unsigned long long* lookback, unsigned int* tile_counter, const unsigned int* epoch_base,
    int pass, unsigned int* errors, unsigned int spin_limit, unsigned int inject,
    unsigned long long vdiv, const unsigned long long* __restrict__ rbases, unsigned int rn,
    unsigned long long rdiv) {
  using TR = TileRank<K, BITS, ITEMS>;
  constexpr int D = TR::D, PT = TR::PT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int sbuf[kSortWarps];
  __shared__ unsigned int s_tile;
  TR tr(smem);
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  __syncthreads();
  const unsigned int tile = s_tile;
  // one index per launched tile (the counter starts at zero); anything else is flagged
  if ((long long)tile * TR::kTile >= N) {
    if (tid == 0) atomicOr(errors, kErrSortRange);
    return;
  }
  const unsigned int epoch = *epoch_base + (unsigned int)pass;
  const long long tile_base = (long long)tile * TR::kTile;
  unsigned int tcount[PT];
  const bool full = tile_base + TR::kTile <= N;
  if (full) tr.template rank<true>(kin, vin, N, tile_base, shift, tcount, sbuf, vdiv);
  else tr.template rank<false>(kin, vin, N, tile_base, shift, tcount, sbuf, vdiv);
  // publish this tile's counts, then look back digit by digit
  unsigned long long* lb_tile = lookback + (size_t)tile * D;
#pragma unroll
  for (int q = 0; q < PT; ++q)
    st_volatile(lb_tile + tid * PT + q,
                pack_lb(tile == 0 ? kFlagPrefix : kFlagAgg, epoch, tcount[q]));
  // (test hook: an epoch no tile publishes, so every wait runs to its limit)
  const unsigned int ep_want = (epoch ^ ((inject & kInjectSortWait) ? 0x20000000u : 0u)) & 0x3fffffffu;
#pragma unroll
  for (int q = 0; q < PT; ++q) {
    const int d = tid * PT + q;
    unsigned int excl = 0;
    if (tile > 0) {
      // a window of kWin predecessors at a time (independent loads), adding aggregates until
      // an inclusive prefix is found
      constexpr int kWin = RTG_SORT_WIN;
      long long p = (long long)tile - 1;
      unsigned int spins = 0;
      while (p >= 0) {
        unsigned long long w[kWin];
#pragma unroll
        for (int u = 0; u < kWin; ++u)
          w[u] = p - u >= 0 ? ld_volatile(lookback + (size_t)(p - u) * D + d) : 0ull;
        int u = 0;
        bool done = false;
        for (; u < kWin && p - u >= 0; ++u) {
          const unsigned long long flag = w[u] >> 62;
          const unsigned int ep = (unsigned int)(w[u] >> 32) & 0x3fffffffu;
          if (flag == 0 || ep != ep_want) break;
          excl += (unsigned int)w[u];
          if (flag == kFlagPrefix) {
            done = true;
            break;
          }
        }
        if (done) break;
        p -= u;
        if (u == 0 || (u < kWin && p >= 0)) {
          if (++spins > spin_limit) {
            atomicOr(errors, kErrTimeout);
            break;
          }
          if (spins > 4) __nanosleep(32);
        }
      }
      st_volatile(lb_tile + d, pack_lb(kFlagPrefix, epoch, excl + tcount[q]));
    }
    tr.s_gbase[d] = digit_off[d] + excl;
  }
  __syncthreads();
  if (full) tr.template write<true, REB>(kout, vout, N, tile_base, shift, errors, rbases, rn, rdiv);
  else tr.template write<false, REB>(kout, vout, N, tile_base, shift, errors, rbases, rn, rdiv);
}

// Grid-wide barrier of a cooperative launch (every block resident), bounded: false when the
// other blocks did not all arrive within `limit` polls (the caller then leaves; kErrTimeout).
__device__ __forceinline__ bool coop_grid_sync(unsigned int* count, unsigned int* gen,
                                               unsigned int limit, unsigned int* errors) {
  __shared__ bool s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = *reinterpret_cast<volatile unsigned int*>(gen);
    __threadfence();
    bool ok = true;
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *reinterpret_cast<volatile unsigned int*>(count) = 0u;  // every block has arrived
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned int spins = 0;
      while (*reinterpret_cast<volatile unsigned int*>(gen) == g) {
        if (++spins > limit) {
          ok = false;
          atomicOr(errors, kErrTimeout);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok;
}

// Every pass in one launch, one tile per block (the host launches it cooperatively, so all
// tiles are resident): a block ranks its tile into shared memory and publishes the tile's digit
// counts (counts[digit * tiles + tile]); after a grid barrier the blocks turn the count
// columns into output offsets (one digit column per block at a time, a block-wide scan over
// the tiles, plus the digit's global start); after a second barrier every block writes its
// ranked tile; a third barrier ends the pass.  No look-back chains, no per-pass launches.
template <typename K, int BITS, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_sort_coop(
    const K* __restrict__ key_rows, K* kbuf0, K* kbuf1, uint32_t* vbuf0, uint32_t* vbuf1,
    long long N, int passes, const unsigned int* __restrict__ digit_off, unsigned int* counts,
    unsigned int tiles, Status* st, unsigned int spin_limit, unsigned long long vdiv) {
  using TR = TileRank<K, BITS, ITEMS>;
  constexpr int D = TR::D, PT = TR::PT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int sbuf[kSortWarps];
  TR tr(smem);
  const unsigned int tile = blockIdx.x;
  const long long tile_base = (long long)tile * TR::kTile;
  const int tid = threadIdx.x;
  unsigned int* errors = &st->errors;
  const bool full = tile_base + TR::kTile <= N;
  for (int p = 0; p < passes; ++p) {
    const K* kin = p == 0 ? key_rows : ((p - 1) & 1 ? kbuf1 : kbuf0);
    const uint32_t* vin = p == 0 ? nullptr : ((p - 1) & 1 ? vbuf1 : vbuf0);
    K* kout = p & 1 ? kbuf1 : kbuf0;
    uint32_t* vout = p & 1 ? vbuf1 : vbuf0;
    const int shift = p * BITS;
    unsigned int tcount[PT];
    const unsigned long long vd = p == 0 ? vdiv : 0ull;
    if (full) tr.template rank<true>(kin, vin, N, tile_base, shift, tcount, sbuf, vd);
    else tr.template rank<false>(kin, vin, N, tile_base, shift, tcount, sbuf, vd);
#pragma unroll
    for (int q = 0; q < PT; ++q) counts[(size_t)(tid * PT + q) * tiles + tile] = tcount[q];
    if (!coop_grid_sync(&st->coop_count, &st->coop_gen, spin_limit, errors)) return;
    // digit columns: exclusive scan over the tiles, offset by the digit's start
    for (int d = blockIdx.x; d < D; d += gridDim.x) {
      unsigned int* col = counts + (size_t)d * tiles;
      unsigned int carry = digit_off[p * D + d];
      for (unsigned int b = 0; b < tiles; b += kSortThreads) {
        const unsigned int t = b + tid;
        const unsigned int v = t < tiles ? col[t] : 0u;
        unsigned int tot;
        const unsigned int ex = block_excl_scan_256(v, &tot, sbuf);
        if (t < tiles) col[t] = carry + ex;
        carry += tot;
      }
    }
    if (!coop_grid_sync(&st->coop_count, &st->coop_gen, spin_limit, errors)) return;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
      const int d = tid * PT + q;
      tr.s_gbase[d] = __ldcg(counts + (size_t)d * tiles + tile);
    }
    __syncthreads();
    if (full) tr.template write<true, false>(kout, vout, N, tile_base, shift, errors, nullptr, 0u, 0ull);
    else tr.template write<false, false>(kout, vout, N, tile_base, shift, errors, nullptr, 0u, 0ull);
    if (!coop_grid_sync(&st->coop_count, &st->coop_gen, spin_limit, errors)) return;
  }
}

// Sets a kernel's dynamic shared-memory limit once per device (static shared memory adds to
// the dynamic part, so the limit is raised whatever the size).
template <typename F>
void set_smem_once(F* kern, size_t smem, bool* done /*64*/) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(launch_attr_mutex());
  if (dev >= 0 && dev < 64 && done[dev]) return;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (dev >= 0 && dev < 64) done[dev] = true;
}

// Identity "sort" (no key bits to sort): the key rows as they are, with their point indices.
template <typename K>
__global__ void __launch_bounds__(256) k_sort_identity(const K* __restrict__ kin, long long N,
                                                       unsigned long long vdiv,
                                                       K* __restrict__ kout,
                                                       uint32_t* __restrict__ vout) {
  for (long long pos = blockIdx.x * 256LL + threadIdx.x; pos < N; pos += 256LL * gridDim.x) {
    kout[pos] = kin[pos];
    vout[pos] = vdiv ? (uint32_t)__umul64hi((unsigned long long)pos, vdiv) : (uint32_t)pos;
  }
}

// The first pass reads the point-major key rows (indices implicit) and writes buffer 0; pass
// p > 0 reads buffer (p - 1) & 1 and writes p & 1.  Returns the buffer holding the result.
template <typename K, int BITS, int ITEMS>
int sort_impl(const BuildArgs& a, cudaStream_t s) {
  using SS = SortShape<K, BITS, ITEMS>;
  constexpr int D = SS::kDigits;
  const long long N = a.n_total * a.m;
  const int passes = a.passes;
  const unsigned long long vdiv = a.m > 1 ? ~0ull / (unsigned long long)a.m + 1ull : 0ull;
  if (N <= 0) return 0;
  if (passes <= 0 || N <= 1) {
    long long blocks = (N + 255) / 256;
    if (blocks > 8LL * a.num_sms) blocks = 8LL * a.num_sms;
    k_sort_identity<K><<<(unsigned)blocks, 256, 0, s>>>((const K*)a.key_mat, N, vdiv,
                                                        (K*)a.keys[0], a.vals[0]);
    return 0;
  }
  long long hb = (N + kSortThreads - 1) / kSortThreads;
  if (hb > 4LL * a.num_sms) hb = 4LL * a.num_sms;
  if (!hist_in_keys(a)) {  // else the key kernel has counted the digits
    static bool hist_attr[64] = {};
    set_smem_once(k_sort_hist<K, BITS>, (size_t)kSortCountWords * 4, hist_attr);
    k_sort_hist<K, BITS><<<(unsigned)hb, kSortThreads, (size_t)passes * D * 4, s>>>(
        (const K*)a.key_mat, N, passes, a.hist, a.digit_off, &a.st->hist_ticket, a.sort_epoch);
  }
  const unsigned tiles = (unsigned)((N + SS::kTile - 1) / SS::kTile);
  // (a single-launch choice whose tiles cannot all be resident runs as reduce-then-scan, which
  // uses the same scratch)
  if (a.sort_mode == kSortCoop && !a.cell_major &&
      sort_coop_fits(N, BITS, ITEMS, a.num_sms, sizeof(K) == 8)) {
    static bool attr[64] = {};
    set_smem_once(k_sort_coop<K, BITS, ITEMS>, SS::kSmem, attr);
    void* args[] = {(void*)&a.key_mat, (void*)&a.keys[0], (void*)&a.keys[1], (void*)&a.vals[0],
                    (void*)&a.vals[1], (void*)&N, (void*)&passes, (void*)&a.digit_off,
                    (void*)&a.lookback, (void*)&tiles, (void*)&a.st, nullptr, (void*)&vdiv};
    const unsigned int limit = spin_limit_of(a.spin_limit);
    args[11] = (void*)&limit;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(kSortThreads);
    cfg.dynamicSmemBytes = SS::kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr_coop[1];
    attr_coop[0].id = cudaLaunchAttributeCooperative;
    attr_coop[0].val.cooperative = 1;
    cfg.attrs = attr_coop;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, (const void*)k_sort_coop<K, BITS, ITEMS>, args);
    return (passes - 1) & 1;
  }
  // cell-major: the first pass reads the grid-major cell indices (keys[1], consumed before the
  // second pass overwrites it) with the positions themselves as values, and the last pass
  // rebases them
  const K* first = a.cell_major ? (const K*)a.keys[1] : (const K*)a.key_mat;
  auto src_k = [&](int p) { return p == 0 ? first : (const K*)a.keys[(p - 1) & 1]; };
  auto src_v = [&](int p) { return p == 0 ? (const uint32_t*)nullptr : a.vals[(p - 1) & 1]; };
  const unsigned long long vd0 = a.cell_major ? 0ull : vdiv;
  const unsigned int rn = a.cell_major ? (unsigned int)a.n_total : 0u;
  const unsigned long long rdiv = a.cell_major ? ~0ull / (unsigned long long)a.n_total + 1ull : 0ull;
  auto rn_of = [&](int p) { return p == passes - 1 ? rn : 0u; };
  // the rebasing last pass is compiled for 8-bit digits over 32-bit keys only, the one form
  // the host chooses a cell-major sort with
  constexpr bool kReb = BITS == 8 && std::is_same<K, uint32_t>::value;
  if (a.sort_mode == kSortLookback) {
    static bool attr[64] = {}, attr_reb[64] = {};
    set_smem_once(k_sort_pass<K, BITS, ITEMS, false>, SS::kSmem, attr);
    if constexpr (kReb)
      if (a.cell_major) set_smem_once(k_sort_pass<K, BITS, ITEMS, kReb>, SS::kSmem, attr_reb);
    for (int p = 0; p < passes; ++p) {
      auto kern = (kReb && rn_of(p)) ? k_sort_pass<K, BITS, ITEMS, kReb>
                                     : k_sort_pass<K, BITS, ITEMS, false>;
      kern<<<tiles, kSortThreads, SS::kSmem, s>>>(
          src_k(p), src_v(p), (K*)a.keys[p & 1], a.vals[p & 1], N, p * BITS,
          a.digit_off + p * D, a.lookback, &a.st->sort_tiles[p], a.sort_epoch, p, &a.st->errors,
          spin_limit_of(a.spin_limit), a.inject, vd0, a.bases, rn_of(p), rdiv);
    }
    return (passes - 1) & 1;
  }
  static bool attr[64] = {}, attr_reb[64] = {};
  set_smem_once(k_sort_downsweep<K, BITS, ITEMS, false>, SS::kSmem, attr);
  if constexpr (kReb)
    if (a.cell_major) set_smem_once(k_sort_downsweep<K, BITS, ITEMS, kReb>, SS::kSmem, attr_reb);
  unsigned int* counts = (unsigned int*)a.lookback;  // D * tiles words
  for (int p = 0; p < passes; ++p) {
    const int shift = p * BITS;
    k_sort_upsweep<K, BITS, ITEMS><<<tiles, kSortThreads, 0, s>>>(src_k(p), N, shift, counts,
                                                                  tiles);
    k_sort_scan<<<D, 1024, 0, s>>>(counts, tiles, a.digit_off + p * D);
    auto down = (kReb && rn_of(p)) ? k_sort_downsweep<K, BITS, ITEMS, kReb>
                                   : k_sort_downsweep<K, BITS, ITEMS, false>;
    down<<<tiles, kSortThreads, SS::kSmem, s>>>(
        src_k(p), src_v(p), (K*)a.keys[p & 1], a.vals[p & 1], N, shift, counts, tiles,
        &a.st->errors, vd0, a.bases, rn_of(p), rdiv);
  }
  return (passes - 1) & 1;
}

template <typename K, int BITS>
int sort_items(const BuildArgs& a, cudaStream_t s) {
  switch (a.sort_items) {
    case 12: return sort_impl<K, BITS, 12>(a, s);
    case 16: return sort_impl<K, BITS, 16>(a, s);
    default: return sort_impl<K, BITS, 8>(a, s);
  }
}

template <typename K>
int sort_width(const BuildArgs& a, cudaStream_t s) {
  switch (a.sort_bits) {
    case 9: return sort_items<K, 9>(a, s);
    case 10: return sort_items<K, 10>(a, s);
    case 11: return sort_items<K, 11>(a, s);
    default: return sort_items<K, 8>(a, s);
  }
}

// Blocks of the single-launch sort that can be resident at once (0 if it cannot launch).
template <typename K, int BITS, int ITEMS>
int coop_resident(int num_sms) {
  static int occ[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(launch_attr_mutex());
  if (dev >= 0 && dev < 64 && occ[dev]) return occ[dev] * num_sms;
  using SS = SortShape<K, BITS, ITEMS>;
  cudaFuncSetAttribute(k_sort_coop<K, BITS, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SS::kSmem);
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_sort_coop<K, BITS, ITEMS>, kSortThreads,
                                                    SS::kSmem) != cudaSuccess)
    o = 0;
  cudaGetLastError();
  if (dev >= 0 && dev < 64) occ[dev] = o;
  return o * num_sms;
}

template <typename K, int BITS>
int coop_resident_items(int items, int num_sms) {
  switch (items) {
    case 12: return coop_resident<K, BITS, 12>(num_sms);
    case 16: return coop_resident<K, BITS, 16>(num_sms);
    default: return coop_resident<K, BITS, 8>(num_sms);
  }
}

template <typename K>
int coop_resident_bits(int bits, int items, int num_sms) {
  switch (bits) {
    case 9: return coop_resident_items<K, 9>(items, num_sms);
    case 10: return coop_resident_items<K, 10>(items, num_sms);
    case 11: return coop_resident_items<K, 11>(items, num_sms);
    default: return coop_resident_items<K, 8>(items, num_sms);
  }
}

}  // namespace

bool sort_coop_fits(long long N, int bits, int items, int num_sms, bool key64) {
  const long long tiles = (long long)sort_tiles_for(N, items);
  const int res = key64 ? coop_resident_bits<unsigned long long>(bits, items, num_sms)
                        : coop_resident_bits<uint32_t>(bits, items, num_sms);
  return tiles >= 1 && tiles <= res;
}

size_t sort_tiles_for(long long N, int items) {
  const long long t = (long long)kSortThreads * items;
  return (size_t)((N + t - 1) / t);
}

int launch_sort(const BuildArgs& a, cudaStream_t s) {
  return a.key64 ? sort_width<unsigned long long>(a, s) : sort_width<uint32_t>(a, s);
}

}  // namespace rtg
