// LSD radix sort of (key, point index) pairs: groups the points of every grid by cell
// (Alg. 1 lines 4-7 of arXiv:1409.8112 associate each point with its cell; the sort makes
// every cell a contiguous run).  Stable, 8-bit digits.
//
// One kernel counts the digits of every pass in a single read of the keys (global digit
// offsets).  A pass is either one kernel with decoupled look-back (few tiles) or
// reduce-then-scan: an upsweep counts the digits of every tile, a
// scan turns the per-(digit, tile) counts into output offsets, and a downsweep ranks each
// tile's keys with a warp-level multisplit (peer masks from one ballot per digit bit),
// reorders the tile in shared memory and writes each digit's run contiguously.  No tile waits
// on another, so a pass costs the same however many tiles run at once.
#include <cuda_runtime.h>

#include "rtg_internal.cuh"

namespace rtg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

template <typename K>
struct SortTile;
template <>
struct SortTile<uint32_t> {
  static constexpr int kItems = 8;
};
template <>
struct SortTile<unsigned long long> {
  static constexpr int kItems = 8;
};

template <typename K>
__host__ __device__ constexpr int tile_size() {
  return kSortWarps * 32 * SortTile<K>::kItems;
}

constexpr unsigned long long kFlagAgg = 1ull, kFlagPrefix = 2ull;
constexpr unsigned int kSpinLimit = 1u << 22;

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

// Lanes of the warp whose digit equals this lane's (kRadixBits ballots; no match.any, which
// is slow here).  `valid` lanes only; an invalid lane gets an arbitrary mask.
__device__ __forceinline__ unsigned int peer_mask(unsigned int dg, bool valid) {
  unsigned int peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < kRadixBits; ++b) {
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

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K* __restrict__ keys,
                                                            long long N, int passes,
                                                            unsigned int* hist,
                                                            unsigned int* digit_off,
                                                            unsigned int* ticket) {
  __shared__ unsigned int sh[kMaxPasses * kRadix];
  __shared__ unsigned int sbuf[kSortWarps];
  __shared__ bool last;
  for (int x = threadIdx.x; x < kMaxPasses * kRadix; x += blockDim.x) sh[x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long step = (long long)gridDim.x * blockDim.x;
  // warp-uniform loop so that match.any sees the full warp
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < N;
       base += step) {
    const long long x = base + lane;
    const bool valid = x < N;
    const K k = valid ? keys[x] : (K)0;
    if (valid)
      for (int p = 0; p < passes; ++p)
        atomicAdd(&sh[p * kRadix + ((unsigned int)(k >> (p * kRadixBits)) & (kRadix - 1))], 1u);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < passes * kRadix; x += blockDim.x)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int p = 0; p < passes; ++p) {
    const unsigned int v = __ldcg(&hist[p * kRadix + threadIdx.x]);
    unsigned int tot;
    const unsigned int e = block_excl_scan_256(v, &tot, sbuf);
    digit_off[p * kRadix + threadIdx.x] = e;
    hist[p * kRadix + threadIdx.x] = 0;  // ready for the next sort
  }
  if (threadIdx.x == 0) *ticket = 0;
}

// Digit counts of every tile of this pass, stored digit-major: counts[digit * tiles + tile].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_upsweep(const K* __restrict__ kin,
                                                               long long N, int shift,
                                                               unsigned int* counts,
                                                               unsigned int tiles) {
  constexpr int kTile = tile_size<K>();
  __shared__ unsigned int sh[kRadix];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
#pragma unroll
  for (int j = 0; j < SortTile<K>::kItems; ++j) {
    const long long pos = base + j * kSortThreads + threadIdx.x;
    if (pos < N) atomicAdd(&sh[(unsigned int)(kin[pos] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * tiles + blockIdx.x] = sh[threadIdx.x];
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

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_downsweep(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, long long N, int shift, const unsigned int* __restrict__ offs,
    unsigned int tiles) {
  constexpr int kItems = SortTile<K>::kItems;
  constexpr int kTile = tile_size<K>();
  extern __shared__ __align__(16) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kTile);
  unsigned int* s_whist = s_vals + kTile;  // kSortWarps * kRadix
  __shared__ unsigned int s_tdig[kRadix];
  __shared__ unsigned int s_gbase[kRadix];
  __shared__ unsigned int sbuf[kSortWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int x = tid; x < kSortWarps * kRadix; x += kSortThreads) s_whist[x] = 0;
  s_gbase[tid] = offs[(size_t)tid * tiles + blockIdx.x];
  __syncthreads();
  const long long tile_base = (long long)blockIdx.x * kTile;
  const long long wbase = tile_base + (long long)warp * 32 * kItems;

  K key[kItems];
  uint32_t val[kItems];
  unsigned int rank[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const long long pos = wbase + j * 32 + lane;
    if (pos < N) {
      key[j] = kin[pos];
      val[j] = vin[pos];
    } else {
      key[j] = (K)0;
      val[j] = 0;
    }
  }
  unsigned int* wh = s_whist + warp * kRadix;
  const unsigned int lt = (1u << lane) - 1;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const bool valid = wbase + j * 32 + lane < N;
    const unsigned int dg = (unsigned int)(key[j] >> shift) & (kRadix - 1);
    const unsigned int peers = peer_mask(dg, valid);
    const unsigned int before = valid ? wh[dg] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0) wh[dg] = before + (unsigned int)__popc(peers);
    __syncwarp();
    rank[j] = before + (unsigned int)__popc(peers & lt);
  }
  __syncthreads();
  // thread tid owns digit tid: warp-exclusive offsets and this tile's count
  unsigned int run = 0;
  for (int w = 0; w < kSortWarps; ++w) {
    const unsigned int c = s_whist[w * kRadix + tid];
    s_whist[w * kRadix + tid] = run;
    run += c;
  }
  unsigned int tot;
  s_tdig[tid] = block_excl_scan_256(run, &tot, sbuf);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const bool valid = wbase + j * 32 + lane < N;
    if (valid) {
      const unsigned int dg = (unsigned int)(key[j] >> shift) & (kRadix - 1);
      const unsigned int local = s_tdig[dg] + s_whist[warp * kRadix + dg] + rank[j];
      s_keys[local] = key[j];
      s_vals[local] = val[j];
    }
  }
  __syncthreads();
  const long long rem = N - tile_base;
  const int tvalid = rem < kTile ? (int)rem : kTile;
  for (int x = tid; x < tvalid; x += kSortThreads) {
    const K k = s_keys[x];
    const unsigned int dg = (unsigned int)(k >> shift) & (kRadix - 1);
    const unsigned int dst = s_gbase[dg] + (unsigned int)x - s_tdig[dg];
    kout[dst] = k;
    vout[dst] = s_vals[x];
  }
}

// Single-kernel pass with decoupled look-back (tiles take their index from an atomic
// counter, so a tile waits only on tiles already running; each wait is bounded).  Cheaper
// than reduce-then-scan while all tiles fit in about one wave.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, long long N, int shift, const unsigned int* __restrict__ digit_off,
    unsigned long long* lookback, unsigned int* tile_counter, unsigned int epoch,
    unsigned int* errors) {
  constexpr int kItems = SortTile<K>::kItems;
  constexpr int kTile = tile_size<K>();
  extern __shared__ __align__(16) unsigned char smem[];
  K* s_keys = reinterpret_cast<K*>(smem);
  uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kTile);
  unsigned int* s_whist = s_vals + kTile;  // kSortWarps * kRadix
  __shared__ unsigned int s_tdig[kRadix];
  __shared__ unsigned int s_gbase[kRadix];
  __shared__ unsigned int sbuf[kSortWarps];
  __shared__ unsigned int s_tile;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int x = tid; x < kSortWarps * kRadix; x += kSortThreads) s_whist[x] = 0;
  __syncthreads();
  const unsigned int tile = s_tile;
  const long long tile_base = (long long)tile * kTile;
  const long long wbase = tile_base + (long long)warp * 32 * kItems;

  K key[kItems];
  uint32_t val[kItems];
  unsigned int rank[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const long long pos = wbase + j * 32 + lane;
    if (pos < N) {
      key[j] = kin[pos];
      val[j] = vin[pos];
    } else {
      key[j] = (K)0;
      val[j] = 0;
    }
  }
  unsigned int* wh = s_whist + warp * kRadix;
  const unsigned int lt = (1u << lane) - 1;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const bool valid = wbase + j * 32 + lane < N;
    const unsigned int dg = (unsigned int)(key[j] >> shift) & (kRadix - 1);
    const unsigned int peers = peer_mask(dg, valid);
    const unsigned int before = valid ? wh[dg] : 0u;
    __syncwarp();
    if (valid && (peers & lt) == 0) wh[dg] = before + (unsigned int)__popc(peers);
    __syncwarp();
    rank[j] = before + (unsigned int)__popc(peers & lt);
  }
  __syncthreads();
  // thread tid owns digit tid: warp-exclusive offsets and this tile's count
  unsigned int run = 0;
  for (int w = 0; w < kSortWarps; ++w) {
    const unsigned int c = s_whist[w * kRadix + tid];
    s_whist[w * kRadix + tid] = run;
    run += c;
  }
  const unsigned int tcount = run;
  unsigned long long* lb = lookback + (size_t)tile * kRadix + tid;
  unsigned int excl = 0;
  if (tile == 0) {
    st_volatile(lb, pack_lb(kFlagPrefix, epoch, tcount));
  } else {
    st_volatile(lb, pack_lb(kFlagAgg, epoch, tcount));
    // Look back over a window of kWin predecessors at a time (independent loads), adding
    // aggregates until an inclusive prefix is found.
    constexpr int kWin = 8;
    long long p = (long long)tile - 1;
    unsigned int spins = 0;
    const unsigned int ep_want = epoch & 0x3fffffffu;
    while (p >= 0) {
      unsigned long long w[kWin];
#pragma unroll
      for (int q = 0; q < kWin; ++q)
        w[q] = p - q >= 0 ? ld_volatile(lookback + (size_t)(p - q) * kRadix + tid) : 0ull;
      int q = 0;
      bool done = false;
      for (; q < kWin && p - q >= 0; ++q) {
        const unsigned long long flag = w[q] >> 62;
        const unsigned int ep = (unsigned int)(w[q] >> 32) & 0x3fffffffu;
        if (flag == 0 || ep != ep_want) break;
        excl += (unsigned int)w[q];
        if (flag == kFlagPrefix) {
          done = true;
          break;
        }
      }
      if (done) break;
      p -= q;
      if (q == 0 || (q < kWin && p >= 0)) {
        if (++spins > kSpinLimit) {
          atomicOr(errors, kErrTimeout);
          break;
        }
        if (spins > 4) __nanosleep(32);
      }
    }
    st_volatile(lb, pack_lb(kFlagPrefix, epoch, excl + tcount));
  }
  s_gbase[tid] = digit_off[tid] + excl;
  unsigned int tot;
  s_tdig[tid] = block_excl_scan_256(tcount, &tot, sbuf);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const bool valid = wbase + j * 32 + lane < N;
    if (valid) {
      const unsigned int dg = (unsigned int)(key[j] >> shift) & (kRadix - 1);
      const unsigned int local = s_tdig[dg] + s_whist[warp * kRadix + dg] + rank[j];
      s_keys[local] = key[j];
      s_vals[local] = val[j];
    }
  }
  __syncthreads();
  const long long rem = N - tile_base;
  const int tvalid = rem < kTile ? (int)rem : kTile;
  for (int x = tid; x < tvalid; x += kSortThreads) {
    const K k = s_keys[x];
    const unsigned int dg = (unsigned int)(k >> shift) & (kRadix - 1);
    const unsigned int dst = s_gbase[dg] + (unsigned int)x - s_tdig[dg];
    kout[dst] = k;
    vout[dst] = s_vals[x];
  }
}

template <typename K>
int sort_impl(const BuildArgs& a, cudaStream_t s) {
  const long long N = a.n_total * a.m;
  const int passes = a.passes;
  if (passes <= 0 || N <= 1) return 0;
  long long hb = (N + kSortThreads - 1) / kSortThreads;
  if (hb > 4LL * a.num_sms) hb = 4LL * a.num_sms;
  k_sort_hist<K><<<(unsigned)hb, kSortThreads, 0, s>>>((const K*)a.keys[0], N, passes, a.hist,
                                                        a.digit_off, &a.st->hist_ticket);
  constexpr int kTile = tile_size<K>();
  const unsigned tiles = (unsigned)((N + kTile - 1) / kTile);
  const size_t smem = (size_t)kTile * (sizeof(K) + 4) + (size_t)kSortWarps * kRadix * 4;
  static bool attr_set[64] = {};  // per instantiation and device; the size is fixed
  int dev = 0;
  cudaGetDevice(&dev);
  if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || !attr_set[dev])) {
    cudaFuncSetAttribute(k_sort_downsweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  int cur = 0;
  if (a.sort_mode == kSortLookback) {
    static bool attr_lb[64] = {};
    if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || !attr_lb[dev])) {
      cudaFuncSetAttribute(k_sort_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (dev >= 0 && dev < 64) attr_lb[dev] = true;
    }
    for (int p = 0; p < passes; ++p) {
      k_sort_pass<K><<<tiles, kSortThreads, smem, s>>>(
          (const K*)a.keys[cur], a.vals[cur], (K*)a.keys[1 - cur], a.vals[1 - cur], N,
          p * kRadixBits, a.digit_off + p * kRadix, a.lookback, &a.st->sort_tiles[p],
          a.epoch + (unsigned)p, &a.st->errors);
      cur = 1 - cur;
    }
    return cur;
  }
  unsigned int* counts = (unsigned int*)a.lookback;  // kRadix * tiles words
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kRadixBits;
    k_sort_upsweep<K><<<tiles, kSortThreads, 0, s>>>((const K*)a.keys[cur], N, shift, counts,
                                                     tiles);
    k_sort_scan<<<kRadix, 1024, 0, s>>>(counts, tiles, a.digit_off + p * kRadix);
    k_sort_downsweep<K><<<tiles, kSortThreads, smem, s>>>(
        (const K*)a.keys[cur], a.vals[cur], (K*)a.keys[1 - cur], a.vals[1 - cur], N, shift,
        counts, tiles);
    cur = 1 - cur;
  }
  return cur;
}

}  // namespace

size_t sort_tiles_for(long long N, bool key64) {
  const int t = key64 ? tile_size<unsigned long long>() : tile_size<uint32_t>();
  return (size_t)((N + t - 1) / t);
}

int launch_sort(const BuildArgs& a, cudaStream_t s) {
  return a.key64 ? sort_impl<unsigned long long>(a, s) : sort_impl<uint32_t>(a, s);
}

}  // namespace rtg
