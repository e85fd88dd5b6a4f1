// Host-side internals shared by rtg_api.cu (contexts, builds) and rtg_serve.cu (the request
// server).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

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
};

// Launch decisions remembered per shape (sum n, instances, grids, dtype, widest d, flags).
using ShapeKey = std::tuple<long long, int, int, int, int, int, int>;
struct ShapeGuess {
  bool key64 = true;
  int passes = rtg::kMaxPasses;
  long long pair_cap = 0;
  int sort_mode = -1;  // rtg::SortMode; -1: not chosen yet
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
};

struct Server;  // request server of a context (rtg_serve.cu)

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
  rtghost::DevBuf status, inst, iplan, gplan, bases, bbox, T64, pts, pf, key_mat, keys0, keys1,
      vals0, vals1, lookback, hist, digit_off, row_cnt, scan_lb, large, large_job, pair_buf,
      tc_tiles, tc_norms, tc_plan;
  rtg::Status* h_status = nullptr;  // pinned
  cudaMemPool_t pool = nullptr;     // output CSRs (stream ordered, kept cached)
  cudaEvent_t ev[8] = {};
  unsigned int epoch = 1;
  size_t ws_bytes = 0;
  size_t out_bytes = 0;
  uint64_t next_handle = 1;
  std::unordered_map<uint64_t, size_t> live;  // CSR handle -> bytes
  std::map<rtghost::ShapeKey, rtghost::ShapeGuess> guesses;
  std::vector<rtg::Inst> h_inst;
  std::vector<double> h_T;
  rtghost::Server* server = nullptr;  // created by the first rtg_submit
};

namespace rtghost {

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
void stop_server(rtg_ctx* c);  // joins the server's threads; frees unclaimed results

}  // namespace rtghost
