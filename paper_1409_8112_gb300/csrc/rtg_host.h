// Host-side internals shared by rtg_api.cu (contexts, builds) and rtg_serve.cu (the request
// server).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "rtg.h"
#include "rtg_internal.cuh"

namespace rtghost {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  unsigned long long gen = 0;  // allocation number (contents are lost when it changes)
};

// Host tables last copied to a device buffer, so that unchanged tables are not sent again.
struct Upload {
  std::vector<unsigned char> bytes;
  unsigned long long gen = 0;  // DevBuf::gen they were copied to
};

// Launch decisions remembered per shape (sum n, instances, grids, dtype, widest d, flags).
using ShapeKey = std::tuple<long long, int, int, int, int, int, int>;
struct ShapeGuess {
  bool key64 = true;
  int key_bits = 64;
  int cell_bits = 0;  // widest grid's cell index range (bits), the key of a cell-major sort
  long long pair_cap = 0;
  bool sorted_cfg = false;  // sort chosen (tuned or default) for this shape
  rtg::SortConfig sort;
  float cand_per_pos = -1.0f;  // in-cell candidates per sorted position at the last build
  bool pairs_tuned = false;    // enumeration knobs measured for this shape
  int spans_per_warp = 0;      // (tuned) spans per resident warp
  int dense_min = 0;           // (tuned) cells of more points take the tiled kernels
  bool no_dense = false;       // the last build had no cell of more than 32 points
  bool no_long_rows = false;   // the last build had no row of more than 32 entries
};

// A build's launch sequence captured once and replayed for later builds of the same shape.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> sig;  // launch arguments it was captured with
  int launches = 0;
};

// Sort variant per (sorted elements, key bits), measured by the autotuner.
using SortKey = std::pair<long long, int>;
struct TuneEntry {
  rtg::SortConfig cfg;
  double us = 0;  // measured time of the sort, microseconds
};

// One build: a batch of instances sharing m, dtype and the points' location.
struct Request {
  const rtg_instance* items;
  int count;
  int m;  // 0: brute force (count must be 1)
  int dtype;
  int points_on_device;
  uint32_t flags;
  bool count_only;
  bool grid_major = false;  // the sorted keys must come out grid by grid (the index reads them so)
};

struct Server;  // request server of a context (rtg_serve.cu)

// Reported pairs per point of recent builds, per d: a decaying maximum (a figure per size
// class of n was measured to correct more first builds, not fewer).
struct PppHints {
  std::map<int, double> h;
  double get(int d) const {
    const auto it = h.find(d);
    return it == h.end() ? 0.0 : it->second;
  }
  void put(int d, double ppp) {
    double& x = h[d];
    x = std::max(0.9 * x, ppp);
  }
  void raise(int d, double ppp) {
    double& x = h[d];
    x = std::max(x, ppp);
  }
};

}  // namespace rtghost

struct rtg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0;
  int num_sms = 0;
  std::mutex mu;       // one build at a time
  std::mutex live_mu;  // output bookkeeping (live, out_bytes)
  std::string err;
  rtghost::DevBuf status, inst, iplan, gplan, bases, T64, pts, pf, key_mat, keys0, keys1,
      vals0, vals1, lookback, hist, digit_off, row_cnt, scan_lb, large, large_job, pair_buf,
      tc_tiles, tc_norms, tc_plan, out_slot, sort_epoch, q_idx, bits;
  rtg::Status* h_status = nullptr;  // pinned
  rtg::OutSlot* h_slot = nullptr;   // pinned; copied to out_slot before the output kernels
  bool use_graphs = true;           // RTG_GRAPHS=0 launches every kernel directly
  bool cell_major = true;           // RTG_CELL_MAJOR=0 keeps the grid in every sort key
  std::map<rtghost::ShapeKey, rtghost::GraphEntry> graphs;
  cudaMemPool_t pool = nullptr;     // output CSRs (stream ordered, kept cached)
  bool own_pool = true;             // false: a serving lane drawing on its owner's pool
  cudaEvent_t ev[8] = {};
  // the output-slot copy runs on a second stream beside the front of the build
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t ws_bytes = 0;
  size_t ws_need = 0;  // workspace bytes the current build asked for (at most ws_bytes)
  size_t out_bytes = 0;
  uint64_t next_handle = 1;
  std::unordered_map<uint64_t, size_t> live;  // CSR handle -> bytes
  std::map<rtghost::ShapeKey, rtghost::ShapeGuess> guesses;
  // Pairs per point of recent builds: the pair-buffer size of a shape built for the first
  // time, so that clustered inputs seldom overflow it.
  rtghost::PppHints ppp_hint;
  std::map<rtghost::SortKey, rtghost::TuneEntry> sort_tune;  // autotuner results
  std::string tune_path;                                     // JSON cache ("" = none)
  std::string device_name;
  bool autotune = true;
  // shapes with more in-cell candidates keep the default enumeration knobs (the trials would
  // each enumerate them all); RTG_TUNE_PAIRS_MAX_CAND
  double tune_pairs_max_cand = 4.0e9;
  bool sort_forced = false;  // RTG_SORT_VARIANT
  rtg::SortConfig sort_force;
  std::vector<rtg::Inst> h_inst;
  std::vector<double> h_T;
  unsigned long long alloc_gen = 0;
  void* h_stage = nullptr;  // pinned staging for the instance and transform tables
  size_t h_stage_cap = 0;
  rtghost::Upload up_inst, up_T;
  rtghost::Server* server = nullptr;  // created by the first rtg_submit
  int last_sorted = 0;  // keys/vals buffer (0 or 1) that holds the last build's sorted keys
  // Failure-path hooks (rtg_set_test_hooks): the bounded device waits' iteration limit (0:
  // the default), waits made to wait for something that never happens (rtg::kInject*), and
  // the number of the device allocation that is made to fail (0: none).
  unsigned int spin_limit = 0;
  unsigned int inject = 0;
  long long fail_alloc_at = 0;
  std::atomic<long long> alloc_calls{0};
};

namespace rtghost {

// The status buffer holds the Status counters, then the bounding boxes of the build's
// instances (zeroed together, by one memset, at the start of every build).
constexpr size_t kStatusBytes = (sizeof(rtg::Status) + 255) & ~size_t(255);
inline unsigned long long* bbox_of(rtg_ctx* c) {
  return reinterpret_cast<unsigned long long*>(static_cast<char*>(c->status.p) + kStatusBytes);
}

rtg_status fail(rtg_ctx* ctx, rtg_status s, const std::string& msg);
std::string& last_error_text();
// Output memory of ctx's pool, ordered on stream s; counted in ctx's out_bytes.
rtg_status alloc_out_on(rtg_ctx* ctx, cudaStream_t s, size_t bytes, void** p);
uint64_t register_out(rtg_ctx* ctx, size_t bytes);
void release_out(rtg_ctx* ctx, rtg_csr* csr);
rtg_status validate_common(int dtype, int64_t n, int d, double r, double c, const void* points);
rtg_status validate_transforms(const double* T, int d, int m);
rtg_status build(rtg_ctx* c, const Request& q, rtg_csr* out);
// A context of the same device with its own stream, workspace and pool (no server).
rtg_status create_ctx(int device, uint64_t budget, void* stream, rtg_ctx** out);
void destroy_ctx(rtg_ctx* c);
// Frees the per-build workspace (points, rows, keys, pair buffer, ...), the captured graphs and
// the output pool's cached blocks; the next build allocates again.  The caller holds c->mu.
void trim_workspace(rtg_ctx* c);
void stop_server(rtg_ctx* c);  // joins the server's threads; frees unclaimed results
void notify_server(rtg_ctx* c);  // memory was released: waiting requests are considered again

// Sort autotuner (rtg_tune.cu).
// The variant used without measurement: 8-bit digits, 2048-key tiles, look-back while the
// tiles fit in about three waves.
rtg::SortConfig sort_default(long long N, int num_sms);
// Sorts the keys of `a` (regenerated by the key kernel before every trial) with every compiled
// variant and strategy, five times, and returns the one with the lowest median time; records
// it in the context's table and JSON cache.  Needs a's buffers sized for any variant.
rtg_status tune_sort(rtg_ctx* c, rtg::BuildArgs& a, long long N, int key_bits,
                     rtg::SortConfig* out);
// Times the in-cell enumeration of a's keys (sorted with cfg) for each (spans per warp,
// dense-cell threshold) candidate and returns the fastest; 0, 0 (the defaults) when a first
// trial takes long.
rtg_status tune_pairs(rtg_ctx* c, rtg::BuildArgs& a, const rtg::SortConfig& cfg, int key_bits,
                      int* spans_per_warp, int* dense_min);
size_t sort_scratch_bytes(long long N, const rtg::SortConfig& cfg);  // look-back / counts
size_t sort_scratch_bytes_max(long long N);
void tune_load(rtg_ctx* c);

// Workspace and status helpers (rtg_api.cu).
rtg_status ensure(rtg_ctx* c, DevBuf& b, size_t bytes, bool zero = false);
rtg_status read_status(rtg_ctx* c);
rtg_status check_errors(rtg_ctx* c, unsigned int mask);
// Grid parameters for a target recall (rtg_params.cu).
rtg_status tune_params(rtg_ctx* c, const void* points, int dtype, int on_device, int64_t n, int d,
                       double r, double target, uint64_t seed, uint32_t flags,
                       rtg_param_choice* out);
// Neighbour lists of a subset of the points from a symmetric CSR (rtg_query.cu).
rtg_status query_neighbors(rtg_ctx* c, const rtg_csr* g, const int32_t* queries, int64_t nq,
                           int queries_on_device, rtg_csr* out);
rtg_status index_create(rtg_ctx* ctx, const rtg_instance& it, int m, int dtype, int on_device,
                        rtg_index** out);
rtg_status index_query(rtg_ctx* ctx, const rtg_index* ix, const void* queries, int on_device,
                       int64_t nq, rtg_csr* out);
void index_destroy(rtg_ctx* ctx, rtg_index* ix);

}  // namespace rtghost
