// Internal declarations shared by the CUDA translation units of the RTG library.
//
// Pipeline of one build (Alg. 1 of arXiv:1409.8112 over all m grids at once):
//   prep   : FP32 copy of the points (padded rows) + per-axis bounding box
//   plan   : per grid, the cell-index range over the bounding box (mixed-radix key layout)
//            and the FP32 error bounds that decide when FP64 must be used
//   keys   : y = R p + s and q = floor(y / c) per point and grid (Alg. 1 lines 4-7),
//            packed into an exact integer key; composite (grid, cell) sort keys
//   sort   : LSD radix sort (onesweep: one upfront histogram, one kernel per digit)
//   count  : per cell, all pairs (Alg. 1 lines 8-9); a pair is owned by the first grid
//            that puts both points in one cell, which removes duplicates across grids
//            without an auxiliary set (Sec. III-B); owned pairs at distance <= r are
//            counted per row
//   scan   : row counts -> CSR row pointers
//   write  : the same enumeration, writing columns into their rows
//   rowsort: each row's columns sorted ascending
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace rtg {

constexpr int kMaxDim = 16;
constexpr int kMaxGrids = 64;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kMaxPasses = 8;

// Bits of Status::errors.
enum : uint32_t {
  kErrKeyOverflow = 1u,    // cell index range needs more than 64 bits
  kErrTimeout = 2u,        // a bounded spin ran out
  kErrColOverflow = 4u,    // more pairs than the column buffer holds
  kErrNonFinite = 8u,      // a coordinate is NaN or infinite
  kErrKeyBits = 16u,       // key wider than the launch assumed (host must redo)
  kErrKeyRange = 32u,      // a cell index fell outside the planned range (internal)
  kErrLargeOverflow = 64u  // large-cell list full (internal)
};

// Device-side counters and bounding box; zeroed at the start of every build.
struct Status {
  unsigned long long bbox_max[kMaxDim];   // sortable encoding of the per-axis maximum
  unsigned long long bbox_nmin[kMaxDim];  // complement of the encoding of the minimum
  unsigned int errors;
  unsigned int key_bits;   // widest per-grid cell key (bits)
  unsigned int grid_bits;  // bits for the grid index
  unsigned int hist_ticket;
  unsigned long long nnz;  // stored CSR entries
  unsigned long long pairs;
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
  unsigned int scan_tiles;
  unsigned int long_rows;  // rows queued for the block row sort
};

// Per-build plan written by the plan kernel.
struct Plan {
  int n, d, m, dtype;
  double c, r, rr;           // rr = fl(r * r)
  float inv_c;               // fl32(1 / c)
  float s_lo, s_hi;          // FP32 squared-distance thresholds (accept below, reject above)
  int filter_on;             // 0: every candidate is decided in FP64
  int key_bits, grid_bits;   // B_max, ceil(log2 m)
  long long qlo[kMaxGrids][kMaxDim];
  unsigned long long ext[kMaxGrids][kMaxDim];
  unsigned long long stride[kMaxGrids][kMaxDim];
  float Rf[kMaxGrids][kMaxDim * kMaxDim];  // rows padded to kMaxDim, zero beyond d
  float sf[kMaxGrids][kMaxDim];
  float E[kMaxGrids][kMaxDim];             // key error bound in cell units (rounded up)
};

struct LargeCell {
  unsigned long long start;  // first sorted position
  unsigned int size;
  unsigned int grid;
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

// ---- launch wrappers (defined in the .cu files) -------------------------------------------
struct BuildArgs {
  // inputs
  const void* pts;  // device, n x d, dtype
  int dtype;
  int n, d, m, dpad;
  double r, c;
  const double* T64;  // device, m * (d*d + d)
  uint32_t flags;
  int symmetric;
  // workspace
  Status* st;
  Plan* plan;
  float* pf;            // n x dpad
  void* key_mat;        // n x m keys
  void* keys[2];        // N composite keys, ping-pong
  uint32_t* vals[2];    // N point indices, ping-pong
  unsigned long long* lookback;  // sort look-back words (tiles * 256)
  unsigned int* hist;            // kMaxPasses * 256 digit counts
  unsigned int* digit_off;       // kMaxPasses * 256 exclusive digit offsets
  unsigned int* row_cnt;         // n
  unsigned long long* scan_lookback;
  LargeCell* large;
  unsigned int large_cap;
  unsigned long long* large_job_off;  // large_cap + 1
  // outputs
  long long* row_ptr;  // n + 1
  int* col;
  long long col_cap;
  // launch decisions
  bool key64;
  int sort_bits;       // bits of the composite key
  unsigned int epoch;  // look-back epoch base for this build's sort passes
  int num_sms;
};

void launch_prep(const BuildArgs& a, cudaStream_t s);
void launch_plan(const BuildArgs& a, int assumed_bits, cudaStream_t s);
void launch_keys(const BuildArgs& a, cudaStream_t s);
// returns 0 if the sorted data ended in buffer 0, 1 if in buffer 1
int launch_sort(const BuildArgs& a, cudaStream_t s);
// The launch_* functions that return int return the number of kernels they launched.
int launch_pairs(const BuildArgs& a, int sorted_buf, bool write, cudaStream_t s);
int launch_brute(const BuildArgs& a, bool write, cudaStream_t s);
void launch_scan(const BuildArgs& a, cudaStream_t s);
int launch_rowsort(const BuildArgs& a, cudaStream_t s);

size_t sort_tiles_for(long long N, bool key64);

// Text returned by rtg_last_error(NULL) on this thread.
void set_last_error(const char* msg);

}  // namespace rtg
