// Internal declarations shared by the CUDA translation units of the RTG library.
//
// One build processes a batch of B >= 1 roadmaps ("instances"), each with its own points,
// radius r, cell side c and m grid transforms (Alg. 1 of arXiv:1409.8112 per instance), in one
// fixed sequence of kernels over the concatenated points:
//   prep    : FP32 copy of the points (padded rows) + per-instance bounding box
//   plan    : per (instance, grid, axis) the cell-index range (mixed-radix key layout) and the
//             FP32 error bound of the cell index; per instance the distance-filter band;
//             composite key bases so that every (instance, grid) owns a disjoint key range
//   keys    : y = R p + s and q = floor(y / c) per point and grid (the point-to-cell step of
//             Alg. 1), packed into base(instance, grid) + mixed-radix cell key
//   sort    : LSD radix sort (onesweep) of the composite keys with global point indices
//   pairs   : per cell, all pairs (the in-cell reporting of Alg. 1); a pair is owned by the
//             first grid that puts both points in one cell (dedupe of Sec. III-B without an
//             auxiliary set); owned pairs at distance <= r are emitted to a pair buffer with row counts
//             (EMIT), or counted and later written in place (COUNT then WRITE)
//   scan    : row counts -> CSR row pointers
//   scatter : pair buffer -> columns in their rows
//   rowsort : each row's columns ascending
// The CSR of a batch is block diagonal over the global point indices.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include <mutex>

namespace rtg {

constexpr int kMaxDim = 16;
constexpr int kMaxGrids = 64;
constexpr int kMaxPasses = 8;  // radix passes of the narrowest digit (8 bits) over a 64-bit key
// Digit widths and tile sizes the radix sort is compiled for.
constexpr int kSortBitsChoices[] = {8, 9, 10, 11};
constexpr int kSortItemsChoices[] = {8, 12, 16};
constexpr int kSortCountWords = 6 * 2048;  // passes * digits, largest over the digit widths
__host__ __device__ inline int sort_passes_for(int key_bits, int radix_bits) {
  return key_bits <= 0 ? 0 : (key_bits + radix_bits - 1) / radix_bits;
}
constexpr int kPointBlock = 128;   // points per block in the per-point kernels
constexpr int kPrepThreads = 256;
constexpr int kPrepPoints = 256;   // points per block in the prep kernel (at least; a multiple)
// Large builds give each prep block more points: fewer blocks adding their bounds to the
// bounding box (1M points: 37 against 47 us); small ones keep one point per thread.
__host__ __device__ inline int prep_points_for(long long n_total) {
  return n_total >= (1LL << 19) ? 4 * kPrepPoints : kPrepPoints;
}

// Bits of Status::errors.
enum : uint32_t {
  kErrKeyOverflow = 1u,     // composite key range needs more than 64 bits
  kErrTimeout = 2u,         // a bounded spin ran out
  kErrColOverflow = 4u,     // more pairs than the output holds (host re-runs bigger)
  kErrNonFinite = 8u,       // a coordinate is NaN or infinite
  kErrKeyBits = 16u,        // key wider than the launch assumed (host re-runs)
  kErrKeyRange = 32u,       // a cell index fell outside the planned range (internal)
  kErrLargeOverflow = 64u,  // large-cell list full (internal)
  kErrPairOverflow = 128u,  // pair buffer too small (host re-runs bigger)
  kErrQueryRange = 256u,    // a neighbour query names a point outside the graph
  kErrSortRange = 512u,     // a sort tile or offset fell outside the keys (internal)
  kErrTailSkipped = 1024u   // work for a kernel left out of the launch (host re-runs with it)
};

// Kernels a build leaves out because the last build of its shape gave them nothing to do
// (BuildArgs::skip_tail); the kernels before them flag kErrTailSkipped if work turns up.
constexpr int kSkipDense = 1;     // the medium-cell, large-cell set-up and large-cell kernels
constexpr int kSkipLongRows = 2;  // the warp and block row sorts
// A shape whose last build had no cell and no row longer than this leaves those kernels (for
// more than 32 points or entries) out of its next builds; the margin keeps new data of the
// same shape from flipping the decision often.
constexpr int kSkipMargin = 24;

// Bounded device waits (look-back chains, tensor-core commits): iterations before a wait
// gives up, sets kErrTimeout and lets its kernel return.  A context may set a smaller limit
// (BuildArgs::spin_limit; 0 takes this one).
constexpr unsigned int kDefaultSpinLimit = 1u << 22;
__host__ __device__ inline unsigned int spin_limit_of(unsigned int v) {
  return v ? v : kDefaultSpinLimit;
}

// Test hooks (BuildArgs::inject): make one kind of bounded wait wait for something that never
// happens, so that its timeout path runs.  Nothing faults: the wait gives up after its limit.
enum : unsigned int {
  kInjectSortWait = 1u,  // look-back sort passes wait for an epoch no tile publishes
  kInjectScanWait = 2u,  // the CSR row scan waits for predecessors that never publish
  kInjectTcWait = 4u     // the tensor-core kernel waits on an mbarrier nothing arrives on
};

// Cells with more points than this are enumerated by the tiled large-cell kernel.
constexpr int kSmallCell = 32;

// Enumeration modes.
// kBits: every reported candidate sets its bit in the instance's bit matrix (no ownership
// test; the matrix makes the union).
enum Mode : int { kCount = 0, kWrite = 1, kEmit = 2, kBits = 3 };

// Largest instance the bit-matrix dedupe takes (n x ceil(n/32) words: 32 MB at this n).
constexpr int kBitsetMaxN = 16384;

// Radix pass strategies.  kSortCoop: every pass in one cooperative launch (one tile per
// block, all blocks resident), the passes' offsets from per-tile counts scanned between
// bounded grid barriers.
enum SortMode : int { kSortLookback = 0, kSortReduceScan = 1, kSortCoop = 2 };

// One compiled variant of the sort and its pass strategy.
struct SortConfig {
  int bits = 8;   // digit width: 8, 9, 10 or 11
  int items = 8;  // keys per thread: 8, 12 or 16 (tiles of 256 * items keys)
  int mode = kSortReduceScan;
};

// Device-side counters; zeroed at the start of every build.
struct Status {
  unsigned int errors;
  unsigned int sort_bits;  // bits of the composite key (set by the plan)
  unsigned int hist_ticket;
  unsigned int prep_ticket;
  unsigned int scan_tiles;
  unsigned long long nnz;      // stored CSR entries (set by the scan)
  unsigned long long pairs;    // reported pairs
  unsigned long long emitted;  // slots claimed in the pair buffer
  unsigned long long candidates[kMaxGrids];
  unsigned long long owned_candidates;
  unsigned long long near_wall;
  unsigned long long near_r;
  unsigned long long key_rechecks;
  unsigned long long dist_rechecks;
  unsigned long long large_cells;
  unsigned long long large_jobs;
  unsigned long long max_cell;
  unsigned int sort_tiles[kMaxPasses];
  unsigned int span_next[2];  // pair enumeration: next unclaimed span (count/emit, write)
  unsigned int coop_count;  // single-launch sort: blocks arrived at the current grid barrier
  unsigned int coop_gen;    // single-launch sort: grid barriers completed
  unsigned int long_rows;  // rows queued for the block row sort
  unsigned int mid_rows;   // rows queued for the warp row sort
  unsigned int rows_over_margin;  // 1 if a row holds more than kSkipMargin entries
  unsigned int cell_bits;  // bits of the widest grid's cell index range (set by the plan)
  unsigned int tc_max_err_bits;  // tensor-core path: max |FP32 d^2 - FP64 d^2| (float bits)
  double tc_band;                // tensor-core path: band used around r^2
};

// Tensor-core brute force: centre of the points, error bound and decision band.
struct TcPlan {
  double center[kMaxDim];
  double band, bound;
  float lo, hi;  // FP32 d^2 below hi goes to the FP64 check; lo bounds the band from below
};

// One roadmap of a batch (filled on the host).
struct Inst {
  const void* pts;  // device, n x d row-major, FP64 or FP32
  long long p0;     // first global point index
  long long T0;     // first double of its m transforms in the packed transform array
  int n, d;
  double r, c;
  double inv_c;   // fl64(1 / c), set by the host
  float inv_cf;   // fl32(1 / c), set by the host
  long long blk0;   // first block of this instance in the per-point kernels
  long long pblk0;  // first block of this instance in the prep kernel
  long long bits_off;  // bit-matrix dedupe: first word of this instance's matrix
  int bits_w;          // words per matrix row (ceil(n / 32))
};

// Per-instance results of the plan.
struct InstPlan {
  double rr;         // fl(r * r), the reporting threshold
  float s_lo, s_hi;  // FP32 squared-distance band (decide in FP32 outside it)
  int filter_on;     // 0: decide every candidate in FP64
  float inv_c;       // fl32(1 / c)
};

// Per (instance, grid) key layout and FP32 rotation.
struct GridPlan {
  float Rf[kMaxDim * kMaxDim];  // rows padded to kMaxDim, zero beyond d
  float sf[kMaxDim];
  float E[kMaxDim];  // bound on |FP32 y/c - FP64 y/c| (rounded up), plus near-wall margin
  long long qlo[kMaxDim];
  unsigned long long ext[kMaxDim];
  unsigned long long stride[kMaxDim];
  unsigned long long base;   // first composite key of this (instance, grid)
  unsigned long long range;  // number of cell keys (product of extents)
};

struct LargeCell {
  unsigned long long start;  // first sorted position
  unsigned int size;
  unsigned short grid;
  unsigned short inst;
};

// ---- sortable encodings of doubles (monotone) --------------------------------------------
__host__ __device__ inline unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ inline double bitsd(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ inline unsigned long long enc_double(double x) {
  unsigned long long b = dbits(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double dec_double(unsigned long long e) {
  return bitsd((e >> 63) ? (e & 0x7fffffffffffffffull) : ~e);
}

inline int dpad_for(int d) { return d <= 4 ? 4 : (d <= 8 ? 8 : 16); }

// Output CSR of the running build, read by the kernels that write it (the host fills it
// before those kernels run, so that one captured launch sequence serves every build).
struct OutSlot {
  long long* row_ptr;  // n_total + 1
  int* col;
  long long col_cap;
  long long reserved;
};

// ---- launch arguments ----------------------------------------------------------------------
struct BuildArgs {
  int spans_per_warp;  // pair enumeration: spans per resident warp (1: static, one each)
  int dense_min;       // cells of more points than this take the tiled kernels (0: 256)
  int B;              // instances
  int m;              // grids per instance (0: brute force)
  int dtype;          // 0 FP64, 1 FP32 (common to the batch)
  int dpad;           // padded row width (common to the batch)
  int d_common;       // d of every instance when they share one, else 0
  int symmetric;
  long long n_total;  // sum of n
  long long blocks;   // per-point kernel blocks (sum of ceil(n / kPointBlock))
  long long pblocks;  // prep blocks (sum of ceil(n / prep_points))
  int prep_points;    // points per prep block: prep_points_for(n_total), a multiple of 256
  const Inst* inst;   // device, B entries
  InstPlan* iplan;    // device, B entries
  GridPlan* gplan;    // device, B * m entries
  unsigned long long* bases;  // device, B * m composite key bases (ascending)
  unsigned long long* bbox;  // device, B * kMaxDim * 2 (max, complement of min)
  const double* T64;         // device, packed transforms
  Status* st;
  float* pf;          // n_total x dpad
  void* key_mat;      // n_total x m keys, point-major: position g m + t holds point g's key
                      // in grid t (also the first sort pass's input; its index is g)
  void* keys[2];      // N composite keys, ping-pong outputs of the sort passes
  uint32_t* vals[2];  // N global point indices, ping-pong outputs of the sort passes
  unsigned long long* lookback;  // sort: look-back words, or per-(digit, tile) counts (u32)
  unsigned int* hist;            // passes * digits counts (kSortCountWords)
  unsigned int* digit_off;       // passes * digits exclusive digit offsets
  unsigned int* row_cnt;         // n_total
  unsigned long long* scan_lookback;
  LargeCell* large;
  unsigned int large_cap;
  unsigned long long* large_job_off;  // large_cap + 1
  unsigned long long* pair_buf;       // EMIT: (i << 32) | j
  long long pair_cap;
  long long* row_ptr;  // n_total + 1 (as in *out; the two-pass write takes it directly)
  int* col;
  long long col_cap;
  const OutSlot* out;  // device copy of the output pointers
  unsigned int* bits;  // bit-matrix dedupe: the instances' matrices
  bool key64;
  int sort_mode;       // SortMode
  int sort_bits;       // digit width
  int sort_items;      // keys per thread in a tile
  int passes;          // radix passes launched
  unsigned int* sort_epoch;  // device counter: look-back epoch base, advanced by every sort
  int num_sms;
  int tc_cells;             // cells of more than 256 points on the tensor cores: 0 off,
                            // 1 FP16 halves, 2 BF16 halves
  unsigned int spin_limit;  // bounded waits: iterations before giving up (0: the default)
  unsigned int inject;      // test hooks (kInject*), 0 in normal use
  int skip_tail;            // kSkipDense | kSkipLongRows: kernels left out of this launch
  int scan_zeroed;          // the scan's look-back words were zeroed with the counters
  // Cell-major sort (one instance): the sort key is the cell index alone, the first pass reads
  // a grid-major copy of the cell indices (keys[1], written by the key kernel) with their
  // grid-major positions as values, and the last pass adds each grid's base back to the key
  // and turns the position into the point index.  LSD passes are stable, so the output is in
  // (cell, grid, point) order with every (grid, cell) run contiguous; the key carries
  // log2(m) bits fewer.
  int cell_major;
};

// Row-count scan: 16 counts per thread, 256 threads per tile, one 8-byte look-back word per
// tile.
constexpr int kScanItems = 16;
constexpr int kScanTile = 256 * kScanItems;
inline size_t scan_lookback_bytes(long long n_total) {
  return (size_t)((n_total + kScanTile - 1) / kScanTile + 1) * 8;
}

// The key kernel with one thread per (point, grid) serves instances that share d <= 6.
inline bool keys_by_lanes(const BuildArgs& a) {
  return a.d_common >= 1 && a.d_common <= 6 && a.m >= 1 && a.m <= 256;
}
// Digit counts kept in shared memory by that kernel (words), at most.
constexpr int kLaneHistWords = 4096;
// The key kernel also counts the digits of every radix pass (the sort then needs no histogram
// kernel): 8-bit digits always, other widths when the lane kernel runs and the counts fit.
inline bool hist_in_keys(const BuildArgs& a) {
  if (a.passes <= 0) return false;
  if (a.sort_bits == 8) return true;
  return keys_by_lanes(a) && a.passes * (1 << a.sort_bits) <= kLaneHistWords;
}

// Radix digit counting shared by the key and histogram kernels (256 digits per pass).  Adds one
// per valid lane; a warp whose lanes share one digit (the high digits of neighbouring keys)
// makes a single add.  Called by all 32 lanes.
__device__ __forceinline__ void count_digit256(unsigned int* sh, unsigned int dg, bool valid,
                                               unsigned int vmask) {
  const unsigned int d0 = __shfl_sync(0xffffffffu, dg, 0);
  if (__all_sync(0xffffffffu, !valid || dg == d0)) {
    if ((threadIdx.x & 31) == 0 && vmask) atomicAdd(&sh[d0], (unsigned int)__popc(vmask));
  } else if (valid) {
    atomicAdd(&sh[dg], 1u);
  }
}

// End of a digit count: the block adds its counts to the global ones; the last block to finish
// turns them into exclusive digit offsets (digit_off[p * 256 + digit]), clears the counts for
// the next sort and advances the look-back epoch.  Any block size that is a multiple of 32 and
// divides 256.
__device__ __forceinline__ void finish_digit_count256(const unsigned int* sh, int passes,
                                                      unsigned int* hist, unsigned int* digit_off,
                                                      unsigned int* ticket, unsigned int* epoch) {
  __shared__ unsigned int s_w[32];
  __shared__ bool s_last;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = tid; x < passes * 256; x += nt)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int per = 256 / nt, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int p = 0; p < passes; ++p) {
    unsigned int v[8], sum = 0;
    for (int q = 0; q < per; ++q) {
      v[q] = __ldcg(&hist[p * 256 + tid * per + q]);
      sum += v[q];
    }
    unsigned int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned int run = x - sum;
    for (int w = 0; w < warp; ++w) run += s_w[w];
    __syncthreads();
    for (int q = 0; q < per; ++q) {
      digit_off[p * 256 + tid * per + q] = run;
      run += v[q];
      hist[p * 256 + tid * per + q] = 0;  // ready for the next sort
    }
    (void)nw;
  }
  if (tid == 0) {
    *ticket = 0;
    unsigned int e = *epoch + kMaxPasses;  // a fresh look-back epoch, never 0
    if ((e & 0x3fffffffu) < (unsigned int)kMaxPasses) e = 1;
    *epoch = e;
  }
}

// finish_digit_count256 for digits of `bits` bits (D = 2^bits per pass, counts sh[p * D + d]);
// a block of 256 threads.
__device__ __forceinline__ void finish_digit_count_bits(const unsigned int* sh, int passes,
                                                        int bits, unsigned int* hist,
                                                        unsigned int* digit_off,
                                                        unsigned int* ticket,
                                                        unsigned int* epoch) {
  __shared__ unsigned int s_w[8];
  __shared__ bool s_last;
  const int tid = threadIdx.x, nt = blockDim.x, D = 1 << bits;
  for (int x = tid; x < passes * D; x += nt)
    if (sh[x]) atomicAdd(&hist[x], sh[x]);
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int per = D / nt, lane = tid & 31, warp = tid >> 5;  // D >= nt = 256
  for (int p = 0; p < passes; ++p) {
    unsigned int sum = 0;
    for (int q = 0; q < per; ++q) sum += __ldcg(&hist[p * D + tid * per + q]);
    unsigned int x = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    unsigned int run = x - sum;
    for (int w = 0; w < warp; ++w) run += s_w[w];
    __syncthreads();
    for (int q = 0; q < per; ++q) {
      const unsigned int v = __ldcg(&hist[p * D + tid * per + q]);
      digit_off[p * D + tid * per + q] = run;
      run += v;
      hist[p * D + tid * per + q] = 0;  // ready for the next sort
    }
  }
  if (tid == 0) {
    *ticket = 0;
    unsigned int e = *epoch + kMaxPasses;  // a fresh look-back epoch, never 0
    if ((e & 0x3fffffffu) < (unsigned int)kMaxPasses) e = 1;
    *epoch = e;
  }
}

// FP32 rows, zeroed row counters, bounding boxes and the plan (in the prep kernel's last block
// for small batches); returns the kernels launched.
int launch_prep_plan(const BuildArgs& a, cudaStream_t s);
void launch_keys(const BuildArgs& a, cudaStream_t s);
// returns the ping-pong buffer (0 or 1) that holds the sorted data
int launch_sort(const BuildArgs& a, cudaStream_t s);
// the launch_* functions returning int return the number of kernels they launched
int launch_pairs(const BuildArgs& a, int sorted_buf, Mode mode, cudaStream_t s);
int launch_brute(const BuildArgs& a, Mode mode, cudaStream_t s);
void launch_scan(const BuildArgs& a, cudaStream_t s);
int launch_scatter(const BuildArgs& a, cudaStream_t s);
// Bit-matrix dedupe: row counts from the matrices, then (after the scan) the columns.
int launch_bits_count(const BuildArgs& a, cudaStream_t s);
int launch_bits_write(const BuildArgs& a, cudaStream_t s);
// Sorts every row of the output CSR; column values lie in [0, col_bound) (-1: a.n_total).
int launch_rowsort(const BuildArgs& a, cudaStream_t s, long long col_bound = -1);
// Status fields the pair kernels accumulate between launches (large-cell list, span counters),
// cleared so that the enumeration can be run again (the autotuner's trials).
void reset_pairs_state(const BuildArgs& a, cudaStream_t s);

// Guards the per-device caches of kernel attributes (shared-memory limits, occupancy) that
// the launch code keeps in statics: builds of several contexts may launch from several host
// threads at once (the serving lanes).
std::mutex& launch_attr_mutex();

size_t sort_tiles_for(long long N, int items);
// Whether the single-launch sort can run this variant: every tile's block resident at once.
bool sort_coop_fits(long long N, int bits, int items, int num_sms, bool key64);
size_t tc_tiles_bytes(long long n);
// tensor-core brute force (instance 0 only); returns kernels launched
int launch_brute_tc(const BuildArgs& a, bool bf16, Mode mode, unsigned char* tiles, float* norms,
                    TcPlan* tp, cudaStream_t s);

// Text returned by rtg_last_error(NULL) on this thread.
void set_last_error(const char* msg);

}  // namespace rtg
