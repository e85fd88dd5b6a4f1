// C ABI of the RTG library (declared in include/rtg.h): contexts, workspace, and the
// orchestration of one build of Alg. 1 (arXiv:1409.8112, Sec. III) on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "gen/rtg_gen.h"
#include "rtg.h"
#include "rtg_internal.cuh"

using rtg::BuildArgs;
using rtg::Plan;
using rtg::Status;

namespace {

thread_local std::string g_err;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

void rtg::set_last_error(const char* msg) { g_err = msg; }

struct rtg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t budget = 0;
  int num_sms = 0;
  std::mutex mu;
  std::string err;
  DevBuf status_plan, T64, pts, pf, key_mat, keys0, keys1, vals0, vals1, lookback, hist,
      digit_off, row_cnt, scan_lb, large, large_job;
  Status* h_status = nullptr;  // pinned
  cudaEvent_t ev[8] = {};
  unsigned int epoch = 1;
  size_t ws_bytes = 0;
  size_t out_bytes = 0;
  uint64_t next_handle = 1;
  std::unordered_map<uint64_t, size_t> live;  // CSR handle -> bytes
};

namespace {

rtg_status fail(rtg_ctx* ctx, rtg_status s, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_err = msg;
  return s;
}

#define RTG_CUDA(ctx, call)                                                               \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? RTG_E_NOMEM : RTG_E_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

size_t total_held(const rtg_ctx* c) { return c->ws_bytes + c->out_bytes; }

// Grow a workspace buffer to at least `bytes` (contents are not kept).
rtg_status ensure(rtg_ctx* c, DevBuf& b, size_t bytes, bool zero = false) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (b.cap >= bytes) return RTG_OK;
  if (c->budget && total_held(c) - b.cap + bytes > c->budget)
    return fail(c, RTG_E_BUDGET, "workspace of " + std::to_string(bytes) +
                                     " bytes exceeds the memory budget");
  if (b.p) {
    cudaFree(b.p);
    c->ws_bytes -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  RTG_CUDA(c, cudaMalloc(&b.p, bytes));
  b.cap = bytes;
  c->ws_bytes += bytes;
  if (zero) RTG_CUDA(c, cudaMemsetAsync(b.p, 0, bytes, c->stream));
  return RTG_OK;
}

void free_buf(rtg_ctx* c, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  c->ws_bytes -= b.cap;
  b = DevBuf();
}

rtg_status alloc_out(rtg_ctx* c, size_t bytes, void** p) {
  if (bytes == 0) {
    *p = nullptr;
    return RTG_OK;
  }
  if (c->budget && total_held(c) + bytes > c->budget)
    return fail(c, RTG_E_BUDGET, "CSR of " + std::to_string(bytes) +
                                     " bytes exceeds the memory budget");
  RTG_CUDA(c, cudaMallocAsync(p, bytes, c->stream));
  c->out_bytes += bytes;
  return RTG_OK;
}

rtg_status read_status(rtg_ctx* c) {
  RTG_CUDA(c, cudaMemcpyAsync(c->h_status, c->status_plan.p, sizeof(Status),
                              cudaMemcpyDeviceToHost, c->stream));
  RTG_CUDA(c, cudaStreamSynchronize(c->stream));
  return RTG_OK;
}

rtg_status check_errors(rtg_ctx* c, unsigned int mask) {
  const unsigned int e = c->h_status->errors & mask;
  if (!e) return RTG_OK;
  if (e & rtg::kErrNonFinite) return fail(c, RTG_E_INVALID, "non-finite point coordinate");
  if (e & rtg::kErrKeyOverflow)
    return fail(c, RTG_E_KEY_OVERFLOW, "cell index range of a grid needs more than 64 bits");
  if (e & rtg::kErrTimeout) return fail(c, RTG_E_TIMEOUT, "a bounded device wait ran out");
  if (e & rtg::kErrKeyRange)
    return fail(c, RTG_E_INTERNAL, "a cell index fell outside the planned key range");
  if (e & rtg::kErrLargeOverflow) return fail(c, RTG_E_INTERNAL, "large-cell list overflow");
  if (e & rtg::kErrColOverflow) return fail(c, RTG_E_INTERNAL, "column buffer overflow");
  return fail(c, RTG_E_INTERNAL, "device error flags " + std::to_string(e));
}

void release_out(rtg_ctx* c, rtg_csr* csr) {
  if (csr->row_ptr) cudaFreeAsync(csr->row_ptr, c->stream);
  if (csr->col) cudaFreeAsync(csr->col, c->stream);
  auto it = c->live.find(csr->handle);
  if (it != c->live.end()) {
    c->out_bytes -= it->second;
    c->live.erase(it);
  }
  std::memset(csr, 0, sizeof(*csr));
}

rtg_status validate(int dtype, int64_t n, int d, double r, const double* T, int m, double c,
                    const void* points) {
  if (dtype != RTG_DTYPE_F64 && dtype != RTG_DTYPE_F32)
    return fail(nullptr, RTG_E_INVALID, "dtype must be RTG_DTYPE_F64 or RTG_DTYPE_F32");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(nullptr, RTG_E_INVALID, "n out of range");
  if (d < 1 || d > RTG_MAX_DIM) return fail(nullptr, RTG_E_INVALID, "d must be in [1, 16]");
  if (m < 1 || m > RTG_MAX_GRIDS) return fail(nullptr, RTG_E_INVALID, "m must be in [1, 64]");
  if (!(r > 0.0) || !std::isfinite(r)) return fail(nullptr, RTG_E_INVALID, "r must be > 0");
  if (!(c > 0.0) || !std::isfinite(c)) return fail(nullptr, RTG_E_INVALID, "cell_side must be > 0");
  if (!T) return fail(nullptr, RTG_E_INVALID, "transforms is NULL");
  if (n > 0 && !points) return fail(nullptr, RTG_E_INVALID, "points is NULL");
  const size_t tn = (size_t)m * (d * d + d);
  for (size_t x = 0; x < tn; ++x)
    if (!std::isfinite(T[x])) return fail(nullptr, RTG_E_INVALID, "non-finite transform entry");
  if ((int64_t)n * m >= (int64_t(1) << 31))
    return fail(nullptr, RTG_E_INVALID, "n * m must be below 2^31");
  return RTG_OK;
}

}  // namespace

extern "C" {

const char* rtg_status_string(rtg_status s) {
  switch (s) {
    case RTG_OK: return "RTG_OK";
    case RTG_E_INVALID: return "RTG_E_INVALID";
    case RTG_E_NOMEM: return "RTG_E_NOMEM";
    case RTG_E_BUDGET: return "RTG_E_BUDGET";
    case RTG_E_KEY_OVERFLOW: return "RTG_E_KEY_OVERFLOW";
    case RTG_E_CUDA: return "RTG_E_CUDA";
    case RTG_E_TIMEOUT: return "RTG_E_TIMEOUT";
    case RTG_PENDING: return "RTG_PENDING";
    case RTG_E_UNKNOWN_TICKET: return "RTG_E_UNKNOWN_TICKET";
    case RTG_E_INTERNAL: return "RTG_E_INTERNAL";
  }
  return "RTG_E_UNKNOWN_STATUS";
}

const char* rtg_last_error(const rtg_ctx* ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

rtg_status rtg_transforms_generate(uint64_t seed, int d, int m, double cell_side, uint32_t flags,
                                   double* out) {
  if (d < 1 || d > RTG_MAX_DIM || m < 1 || !(cell_side > 0.0) || !std::isfinite(cell_side) || !out)
    return fail(nullptr, RTG_E_INVALID, "invalid transform arguments");
  const uint32_t gflags = (flags & RTG_FLAG_SHIFT_ONLY) ? RTG_GEN_SHIFT_ONLY : 0u;
  if (rtg_gen_transforms(seed, d, m, cell_side, gflags, out) != 0)
    return fail(nullptr, RTG_E_INVALID, "invalid transform arguments");
  return RTG_OK;
}

rtg_status rtg_create(const rtg_config* cfg, rtg_ctx** out) {
  if (!out) return fail(nullptr, RTG_E_INVALID, "out is NULL");
  *out = nullptr;
  rtg_config def = {0, 0, nullptr, 0};
  if (!cfg) cfg = &def;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, RTG_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (cfg->device < 0 || cfg->device >= ndev)
    return fail(nullptr, RTG_E_INVALID, "device ordinal out of range");
  rtg_ctx* c = new rtg_ctx();
  c->device = cfg->device;
  c->budget = cfg->mem_budget_bytes;
  auto bail = [&](cudaError_t err) {
    std::string msg = std::string("context setup: ") + cudaGetErrorString(err);
    rtg_destroy(c);
    return fail(nullptr, RTG_E_CUDA, msg);
  };
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return bail(e);
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)) !=
      cudaSuccess)
    return bail(e);
  if (cfg->stream) {
    c->stream = (cudaStream_t)cfg->stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(e);
    c->own_stream = true;
  }
  if ((e = cudaMallocHost(&c->h_status, sizeof(Status))) != cudaSuccess) return bail(e);
  for (auto& ev : c->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e);
  rtg_status s =
      ensure(c, c->status_plan, ((sizeof(Status) + 255) & ~size_t(255)) + sizeof(Plan), true);
  if (s != RTG_OK) {
    std::string msg = c->err;
    rtg_destroy(c);
    return fail(nullptr, s, msg);
  }
  *out = c;
  return RTG_OK;
}

void rtg_destroy(rtg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->status_plan, &c->T64,     &c->pts,     &c->pf,      &c->key_mat,
                    &c->keys0,       &c->keys1,   &c->vals0,   &c->vals1,   &c->lookback,
                    &c->hist,        &c->digit_off, &c->row_cnt, &c->scan_lb, &c->large,
                    &c->large_job};
  for (DevBuf* b : bufs) free_buf(c, *b);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

rtg_status rtg_release(rtg_ctx* c, rtg_csr* csr) {
  if (!c || !csr) return fail(c, RTG_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  release_out(c, csr);
  return RTG_OK;
}

rtg_status rtg_csr_download(rtg_ctx* c, const rtg_csr* csr, int64_t* row_ptr, int32_t* col) {
  if (!c || !csr || !row_ptr || (csr->nnz > 0 && !col)) return fail(c, RTG_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  if (csr->row_ptr)
    RTG_CUDA(c, cudaMemcpyAsync(row_ptr, csr->row_ptr, sizeof(int64_t) * (csr->n + 1),
                                cudaMemcpyDeviceToHost, c->stream));
  else
    std::memset(row_ptr, 0, sizeof(int64_t) * (csr->n + 1));
  if (csr->nnz > 0)
    RTG_CUDA(c, cudaMemcpyAsync(col, csr->col, sizeof(int32_t) * csr->nnz, cudaMemcpyDeviceToHost,
                                c->stream));
  RTG_CUDA(c, cudaStreamSynchronize(c->stream));
  return RTG_OK;
}

}  // extern "C"

namespace {

// Validate, copy inputs in, run prep + plan and read the plan's key width back.
// m == 0 prepares a brute-force build (no grids).
rtg_status begin_build(rtg_ctx* c, const void* points, int dtype, int points_on_device, int64_t n,
                       int d, double r, const double* transforms, int m, double cell_side,
                       uint32_t flags, BuildArgs& a, int& launches) {
  cudaStream_t st = c->stream;
  const int dpad = rtg::dpad_for(d);
  const size_t esz = dtype == RTG_DTYPE_F64 ? 8 : 4;
  rtg_status s;
  if (m > 0) {
    const size_t tbytes = sizeof(double) * (size_t)m * (d * d + d);
    if ((s = ensure(c, c->T64, tbytes)) != RTG_OK) return s;
    RTG_CUDA(c, cudaMemcpyAsync(c->T64.p, transforms, tbytes, cudaMemcpyHostToDevice, st));
  }
  if ((s = ensure(c, c->pf, (size_t)n * dpad * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->row_cnt, (size_t)n * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->scan_lb, ((size_t)n / 4096 + 2) * 8)) != RTG_OK) return s;
  const void* dpts = points;
  if (!points_on_device) {
    if ((s = ensure(c, c->pts, (size_t)n * d * esz)) != RTG_OK) return s;
    RTG_CUDA(c, cudaMemcpyAsync(c->pts.p, points, (size_t)n * d * esz, cudaMemcpyHostToDevice, st));
    dpts = c->pts.p;
  }
  a = BuildArgs{};
  a.pts = dpts;
  a.dtype = dtype;
  a.n = (int)n;
  a.d = d;
  a.m = m;
  a.dpad = dpad;
  a.r = r;
  a.c = cell_side;
  a.T64 = (const double*)c->T64.p;
  a.flags = flags;
  a.symmetric = (flags & RTG_FLAG_SYMMETRIC) ? 1 : 0;
  a.st = (Status*)c->status_plan.p;
  a.plan = (Plan*)((char*)c->status_plan.p + ((sizeof(Status) + 255) & ~size_t(255)));
  a.pf = (float*)c->pf.p;
  a.row_cnt = (unsigned int*)c->row_cnt.p;
  a.scan_lookback = (unsigned long long*)c->scan_lb.p;
  a.num_sms = c->num_sms;
  RTG_CUDA(c, cudaMemsetAsync(a.st, 0, sizeof(Status), st));
  RTG_CUDA(c, cudaMemsetAsync(a.row_cnt, 0, (size_t)n * 4, st));
  rtg::launch_prep(a, st);
  rtg::launch_plan(a, 64, st);
  launches += 2;
  RTG_CUDA(c, cudaGetLastError());
  if ((s = read_status(c)) != RTG_OK) return s;
  return check_errors(c, rtg::kErrNonFinite | rtg::kErrKeyOverflow);
}

// After the COUNT pass: scan, allocate the columns, WRITE pass, row sort.
// `write_pass` launches the WRITE enumeration and returns its kernel count.
template <typename WritePass>
rtg_status finish_build(rtg_ctx* c, BuildArgs& a, rtg_csr* out, bool count_only, int& launches,
                        bool timing, WritePass write_pass) {
  cudaStream_t st = c->stream;
  rtg_status s;
  rtg::launch_scan(a, st);
  launches += 1;
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[5], st));
  RTG_CUDA(c, cudaGetLastError());
  if ((s = read_status(c)) != RTG_OK || (s = check_errors(c, ~0u)) != RTG_OK) return s;
  const long long nnz = (long long)c->h_status->nnz;
  out->nnz = nnz;
  if (count_only) {
    if (timing) {
      RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
      RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
    }
    return RTG_OK;
  }
  void* cp = nullptr;
  if ((s = alloc_out(c, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) return s;
  out->col = (int32_t*)cp;
  c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
  a.col = (int*)cp;
  a.col_cap = nnz;
  if (nnz > 0) launches += write_pass(a);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
  if (nnz > 0) launches += rtg::launch_rowsort(a, st);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
  RTG_CUDA(c, cudaGetLastError());
  if ((s = read_status(c)) != RTG_OK) return s;
  return check_errors(c, ~0u);
}

void fill_stats(rtg_ctx* c, const BuildArgs& a, rtg_csr* out, int launches, bool timing) {
  const Status& h = *c->h_status;
  rtg_stats& S = out->stats;
  long long tc = 0;
  for (int t = 0; t < a.m; ++t) {
    S.candidates[t] = (int64_t)h.candidates[t];
    tc += (long long)h.candidates[t];
  }
  S.total_candidates = tc;
  S.owned_candidates = (int64_t)h.owned_candidates;
  S.near_wall = (int64_t)h.near_wall;
  S.near_r = (int64_t)h.near_r;
  S.key_rechecks = (int64_t)h.key_rechecks;
  S.dist_rechecks = (int64_t)h.dist_rechecks;
  S.large_cells = (int64_t)h.large_cells;
  S.max_cell = (int64_t)h.max_cell;
  S.pairs = (int64_t)h.pairs;
  S.key_bits = a.sort_bits;
  S.sort_passes = a.sort_bits <= 0 ? 0 : (a.sort_bits + rtg::kRadixBits - 1) / rtg::kRadixBits;
  S.launches = launches;
  if (timing) {
    float ms;
    const int idx[8][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {0, 7}};
    for (int p = 0; p < 8; ++p) {
      cudaEventElapsedTime(&ms, c->ev[idx[p][0]], c->ev[idx[p][1]]);
      S.phase_us[p] = 1000.0 * ms;
    }
  }
}

rtg_status empty_csr(rtg_ctx* c, int64_t n, rtg_csr* out) {
  void* rp = nullptr;
  rtg_status s;
  if ((s = alloc_out(c, sizeof(int64_t) * (n + 1), &rp)) != RTG_OK) return s;
  RTG_CUDA(c, cudaMemsetAsync(rp, 0, sizeof(int64_t) * (n + 1), c->stream));
  RTG_CUDA(c, cudaStreamSynchronize(c->stream));
  out->row_ptr = (int64_t*)rp;
  out->handle = c->next_handle++;
  c->live[out->handle] = sizeof(int64_t) * (n + 1);
  return RTG_OK;
}

rtg_status alloc_row_ptr(rtg_ctx* c, BuildArgs& a, rtg_csr* out) {
  void* rp = nullptr;
  rtg_status s;
  if ((s = alloc_out(c, sizeof(int64_t) * (a.n + 1), &rp)) != RTG_OK) return s;
  out->row_ptr = (int64_t*)rp;
  out->handle = c->next_handle++;
  c->live[out->handle] = sizeof(int64_t) * (a.n + 1);
  a.row_ptr = (long long*)rp;
  return RTG_OK;
}

rtg_status all_pairs_impl(rtg_ctx* c, const void* points, int dtype, int points_on_device,
                          int64_t n, int d, double r, const double* transforms, int m,
                          double cell_side, uint32_t flags, rtg_csr* out) {
  cudaStream_t st = c->stream;
  const bool timing = (flags & RTG_FLAG_TIMING) != 0;
  out->n = n;
  out->symmetric = (flags & RTG_FLAG_SYMMETRIC) ? 1 : 0;
  if (n == 0) return empty_csr(c, n, out);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[0], st));
  BuildArgs a;
  int launches = 0;
  rtg_status s = begin_build(c, points, dtype, points_on_device, n, d, r, transforms, m, cell_side,
                             flags, a, launches);
  if (s != RTG_OK) return s;
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[1], st));
  const long long N = n * (long long)m;
  a.sort_bits = (int)c->h_status->key_bits + (int)c->h_status->grid_bits;
  a.key64 = a.sort_bits > 32;
  const size_t ksz = a.key64 ? 8 : 4;
  if ((s = ensure(c, c->key_mat, (size_t)N * ksz)) != RTG_OK) return s;
  if ((s = ensure(c, c->keys0, (size_t)N * ksz)) != RTG_OK) return s;
  if ((s = ensure(c, c->keys1, (size_t)N * ksz)) != RTG_OK) return s;
  if ((s = ensure(c, c->vals0, (size_t)N * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->vals1, (size_t)N * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->lookback, rtg::sort_tiles_for(N, a.key64) * rtg::kRadix * 8, true)) !=
      RTG_OK)
    return s;
  if ((s = ensure(c, c->hist, rtg::kMaxPasses * rtg::kRadix * 4, true)) != RTG_OK) return s;
  if ((s = ensure(c, c->digit_off, rtg::kMaxPasses * rtg::kRadix * 4)) != RTG_OK) return s;
  const unsigned int large_cap = (unsigned int)(N / 129 + 1);
  if ((s = ensure(c, c->large, (size_t)large_cap * sizeof(rtg::LargeCell))) != RTG_OK) return s;
  if ((s = ensure(c, c->large_job, ((size_t)large_cap + 1) * 8)) != RTG_OK) return s;
  a.key_mat = c->key_mat.p;
  a.keys[0] = c->keys0.p;
  a.keys[1] = c->keys1.p;
  a.vals[0] = (uint32_t*)c->vals0.p;
  a.vals[1] = (uint32_t*)c->vals1.p;
  a.lookback = (unsigned long long*)c->lookback.p;
  a.hist = (unsigned int*)c->hist.p;
  a.digit_off = (unsigned int*)c->digit_off.p;
  a.large = (rtg::LargeCell*)c->large.p;
  a.large_cap = large_cap;
  a.large_job_off = (unsigned long long*)c->large_job.p;
  a.epoch = c->epoch;
  c->epoch += rtg::kMaxPasses;
  if ((c->epoch & 0x3fffffffu) < rtg::kMaxPasses) c->epoch = 1;
  if ((s = alloc_row_ptr(c, a, out)) != RTG_OK) return s;

  rtg::launch_keys(a, st);
  launches += 1;
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[2], st));
  const int sorted = rtg::launch_sort(a, st);
  launches += a.sort_bits > 0 && N > 1 ? 1 + (a.sort_bits + rtg::kRadixBits - 1) / rtg::kRadixBits : 0;
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[3], st));
  launches += rtg::launch_pairs(a, sorted, false, st);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[4], st));
  s = finish_build(c, a, out, false, launches, timing,
                   [&](BuildArgs& b) { return rtg::launch_pairs(b, sorted, true, st); });
  if (s != RTG_OK) return s;
  fill_stats(c, a, out, launches, timing);
  return RTG_OK;
}

rtg_status brute_impl(rtg_ctx* c, const void* points, int dtype, int points_on_device, int64_t n,
                      int d, double r, uint32_t flags, int count_only, rtg_csr* out) {
  cudaStream_t st = c->stream;
  const bool timing = (flags & RTG_FLAG_TIMING) != 0;
  out->n = n;
  out->symmetric = (flags & RTG_FLAG_SYMMETRIC) ? 1 : 0;
  if (n == 0) return empty_csr(c, n, out);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[0], st));
  BuildArgs a;
  int launches = 0;
  rtg_status s = begin_build(c, points, dtype, points_on_device, n, d, r, nullptr, 0, 1.0, flags,
                             a, launches);
  if (s != RTG_OK) return s;
  if (timing) {
    RTG_CUDA(c, cudaEventRecord(c->ev[1], st));
    RTG_CUDA(c, cudaEventRecord(c->ev[2], st));
    RTG_CUDA(c, cudaEventRecord(c->ev[3], st));
  }
  if ((s = alloc_row_ptr(c, a, out)) != RTG_OK) return s;
  launches += rtg::launch_brute(a, false, st);
  if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[4], st));
  s = finish_build(c, a, out, count_only != 0, launches, timing,
                   [&](BuildArgs& b) { return rtg::launch_brute(b, true, st); });
  if (s != RTG_OK) return s;
  fill_stats(c, a, out, launches, timing);
  return RTG_OK;
}

}  // namespace

extern "C" {

rtg_status rtg_all_pairs(rtg_ctx* c, const void* points, int dtype, int points_on_device, int64_t n,
                         int d, double r, const double* transforms, int m, double cell_side,
                         uint32_t flags, rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  std::memset(out, 0, sizeof(*out));
  rtg_status s = validate(dtype, n, d, r, transforms, m, cell_side, points);
  if (s != RTG_OK) return fail(c, s, g_err);
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  s = all_pairs_impl(c, points, dtype, points_on_device, n, d, r, transforms, m, cell_side, flags,
                     out);
  if (s != RTG_OK) release_out(c, out);
  return s;
}

rtg_status rtg_brute_force(rtg_ctx* c, const void* points, int dtype, int points_on_device,
                           int64_t n, int d, double r, uint32_t flags, int count_only,
                           rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  std::memset(out, 0, sizeof(*out));
  const double T1[2] = {1.0, 0.0};
  rtg_status s = validate(dtype, n, 1, r, T1, 1, 1.0, points);
  if (s == RTG_OK && (d < 1 || d > RTG_MAX_DIM))
    s = fail(nullptr, RTG_E_INVALID, "d must be in [1, 16]");
  if (s != RTG_OK) return fail(c, s, g_err);
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  s = brute_impl(c, points, dtype, points_on_device, n, d, r, flags, count_only, out);
  if (s != RTG_OK) release_out(c, out);
  return s;
}

}  // extern "C"
