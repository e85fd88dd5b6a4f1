// C ABI of the RTG library (declared in include/rtg.h): contexts, workspace, and the
// orchestration of one build of Alg. 1 (arXiv:1409.8112, Sec. III) for a batch of roadmaps.
//
// A build is one fixed sequence of kernels on the context's stream with a single host
// synchronisation at the end.  Three launch decisions depend on the data: the key width
// (32 or 64 bits), the number of radix passes and the size of the pair buffer.  They are
// taken from the last build of the same shape; the device checks them (kErrKeyBits,
// kErrPairOverflow) and on a miss the build is run again with the values the device
// reported.  The first build of a shape reads the key width back once before sorting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "gen/rtg_gen.h"
#include "rtg.h"
#include "rtg_internal.cuh"

using rtg::BuildArgs;
using rtg::GridPlan;
using rtg::Inst;
using rtg::InstPlan;
using rtg::Status;

#include "rtg_host.h"

namespace {
thread_local std::string g_err;
// Sorts of fewer elements take the default variant: a measurement would cost more than the
// best variant could save.
constexpr long long kTuneMinElements = 1LL << 17;
constexpr size_t kMaxGraphs = 32;  // executable graphs kept per context (one per shape)
}  // namespace

void rtg::set_last_error(const char* msg) { g_err = msg; }

std::mutex& rtg::launch_attr_mutex() {
  static std::mutex m;
  return m;
}

namespace rtghost {

std::string& last_error_text() { return g_err; }

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

// Test hook: the fail_alloc_at-th device allocation of the context fails (once).
bool injected_alloc_failure(rtg_ctx* c) {
  return c->fail_alloc_at > 0 && ++c->alloc_calls == c->fail_alloc_at;
}

// Grow a workspace buffer to at least `bytes` (contents are not kept).
rtg_status ensure(rtg_ctx* c, DevBuf& b, size_t bytes, bool zero) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  c->ws_need += bytes;
  if (b.cap >= bytes) return RTG_OK;
  if (c->budget && total_held(c) - b.cap + bytes > c->budget)
    return fail(c, RTG_E_BUDGET, "workspace of " + std::to_string(bytes) +
                                     " bytes exceeds the memory budget");
  if (injected_alloc_failure(c))
    return fail(c, RTG_E_NOMEM, "device allocation failed (injected by rtg_set_test_hooks)");
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    c->ws_bytes -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  RTG_CUDA(c, cudaMalloc(&b.p, bytes));
  b.cap = bytes;
  b.gen = ++c->alloc_gen;
  c->ws_bytes += bytes;
  if (zero) RTG_CUDA(c, cudaMemsetAsync(b.p, 0, bytes, c->stream));
  return RTG_OK;
}

void free_buf(rtg_ctx* c, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  c->ws_bytes -= b.cap;
  b = DevBuf();
}

rtg_status alloc_out_on(rtg_ctx* c, cudaStream_t s, size_t bytes, void** p) {
  if (bytes == 0) {
    *p = nullptr;
    return RTG_OK;
  }
  if (injected_alloc_failure(c))
    return fail(c, RTG_E_NOMEM, "device allocation failed (injected by rtg_set_test_hooks)");
  {
    std::lock_guard<std::mutex> lk(c->live_mu);
    if (c->budget && total_held(c) + bytes > c->budget)
      return fail(c, RTG_E_BUDGET, "CSR of " + std::to_string(bytes) +
                                       " bytes exceeds the memory budget");
    c->out_bytes += bytes;
  }
  const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, c->pool, s);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(c->live_mu);
    c->out_bytes -= bytes;
    return fail(c, e == cudaErrorMemoryAllocation ? RTG_E_NOMEM : RTG_E_CUDA,
                std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
  }
  return RTG_OK;
}

rtg_status alloc_out(rtg_ctx* c, size_t bytes, void** p) {
  return alloc_out_on(c, c->stream, bytes, p);
}

// Register `bytes` (already counted in out_bytes) under a new CSR handle.
uint64_t register_out(rtg_ctx* c, size_t bytes) {
  std::lock_guard<std::mutex> lk(c->live_mu);
  const uint64_t h = c->next_handle++;
  c->live[h] = bytes;
  return h;
}

rtg_status read_status(rtg_ctx* c) {
  RTG_CUDA(c, cudaMemcpyAsync(c->h_status, c->status.p, sizeof(Status), cudaMemcpyDeviceToHost,
                              c->stream));
  RTG_CUDA(c, cudaStreamSynchronize(c->stream));
  return RTG_OK;
}

rtg_status check_errors(rtg_ctx* c, unsigned int mask) {
  const unsigned int e = c->h_status->errors & mask;
  if (!e) return RTG_OK;
  if (e & rtg::kErrNonFinite)
    return fail(c, RTG_E_INVALID, "a point coordinate is not finite");
  if (e & rtg::kErrKeyOverflow)
    return fail(c, RTG_E_KEY_OVERFLOW, "the cell index ranges need more than 64 key bits");
  if (e & rtg::kErrTimeout) return fail(c, RTG_E_TIMEOUT, "a bounded device wait ran out");
  if (e & rtg::kErrKeyRange)
    return fail(c, RTG_E_INTERNAL, "a cell index fell outside the planned key range");
  if (e & rtg::kErrLargeOverflow) return fail(c, RTG_E_INTERNAL, "large-cell list overflow");
  if (e & rtg::kErrSortRange)
    return fail(c, RTG_E_INTERNAL, "a sort tile or offset fell outside the keys");
  if (e & rtg::kErrColOverflow) return fail(c, RTG_E_INTERNAL, "column buffer overflow");
  return fail(c, RTG_E_INTERNAL, "device error flags " + std::to_string(e));
}

void release_out(rtg_ctx* c, rtg_csr* csr) {
  if (csr->row_ptr) cudaFreeAsync(csr->row_ptr, c->stream);
  if (csr->col) cudaFreeAsync(csr->col, c->stream);
  {
    std::lock_guard<std::mutex> lk(c->live_mu);
    auto it = c->live.find(csr->handle);
    if (it != c->live.end()) {
      c->out_bytes -= it->second;
      c->live.erase(it);
    }
  }
  std::memset(csr, 0, sizeof(*csr));
}

rtg_status validate_common(int dtype, int64_t n, int d, double r, double c, const void* points) {
  if (dtype != RTG_DTYPE_F64 && dtype != RTG_DTYPE_F32)
    return fail(nullptr, RTG_E_INVALID, "dtype must be RTG_DTYPE_F64 or RTG_DTYPE_F32");
  if (n < 0 || n >= (int64_t(1) << 31)) return fail(nullptr, RTG_E_INVALID, "n out of range");
  if (d < 1 || d > RTG_MAX_DIM) return fail(nullptr, RTG_E_INVALID, "d must be in [1, 16]");
  if (!(r > 0.0) || !std::isfinite(r)) return fail(nullptr, RTG_E_INVALID, "r must be > 0");
  if (!(c > 0.0) || !std::isfinite(c)) return fail(nullptr, RTG_E_INVALID, "cell_side must be > 0");
  if (n > 0 && !points) return fail(nullptr, RTG_E_INVALID, "points is NULL");
  return RTG_OK;
}

rtg_status validate_transforms(const double* T, int d, int m) {
  if (!T) return fail(nullptr, RTG_E_INVALID, "transforms is NULL");
  const size_t tn = (size_t)m * (d * d + d);
  for (size_t x = 0; x < tn; ++x)
    if (!std::isfinite(T[x])) return fail(nullptr, RTG_E_INVALID, "non-finite transform entry");
  return RTG_OK;
}

// The whole build.  On success *out holds the block-diagonal CSR of the batch.
// Bytes that decide whether a captured launch sequence can be replayed: every launch argument
// except the output pointers (which the kernels read from the device slot), plus the timing
// flag and the stream.
std::vector<unsigned char> graph_signature(const rtg::BuildArgs& a, bool timing, cudaStream_t st) {
  rtg::BuildArgs b = a;
  b.row_ptr = nullptr;
  b.col = nullptr;
  b.col_cap = 0;
  std::vector<unsigned char> sig(sizeof(b) + 2 + sizeof(st));
  std::memcpy(sig.data(), &b, sizeof(b));
  sig[sizeof(b)] = timing ? 1 : 0;
  sig[sizeof(b) + 1] = 0x5a;
  std::memcpy(sig.data() + sizeof(b) + 2, &st, sizeof(st));
  return sig;
}

void drop_graph(rtg_ctx* c, const ShapeKey& key) {
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) return;
  if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
  c->graphs.erase(it);
}

// The executable graph of this shape's launch sequence: replayed when the arguments match,
// else captured again from `enqueue` (which returns its kernel count).  *exec stays null when
// the sequence cannot be captured; the caller then launches directly.
template <typename F>
rtg_status graph_for(rtg_ctx* c, const ShapeKey& key, const rtg::BuildArgs& a, bool timing,
                     F&& enqueue, cudaGraphExec_t* exec, int* launches) {
  *exec = nullptr;
  const std::vector<unsigned char> sig = graph_signature(a, timing, c->stream);
  auto it = c->graphs.find(key);
  if (it != c->graphs.end() && it->second.sig == sig) {
    *exec = it->second.exec;
    *launches = it->second.launches;
    return RTG_OK;
  }
  drop_graph(c, key);
  if (c->graphs.size() >= kMaxGraphs) drop_graph(c, c->graphs.begin()->first);
  cudaGetLastError();
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return RTG_OK;
  }
  const int l = enqueue();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (e != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return RTG_OK;
  }
  cudaGraphExec_t ge = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ge, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return RTG_OK;
  }
  GraphEntry ent;
  ent.exec = ge;
  ent.sig = sig;
  ent.launches = l;
  c->graphs[key] = ent;
  *exec = ge;
  *launches = l;
  return RTG_OK;
}

rtg_status build(rtg_ctx* c, const Request& q, rtg_csr* out) {
  cudaStream_t st = c->stream;
  c->ws_need = 0;
  const bool timing = (q.flags & RTG_FLAG_TIMING) != 0;
  const int sym = (q.flags & RTG_FLAG_SYMMETRIC) ? 1 : 0;
  const int B = q.count, m = q.m;
  const size_t esz = q.dtype == RTG_DTYPE_F64 ? 8 : 4;
  rtg_status s;

  // ---- instance table and packed transforms (host) ----
  c->h_inst.assign(B, Inst{});
  long long p0 = 0, blk0 = 0, pblk0 = 0, T0 = 0, bits_words = 0;
  long long n_sum = 0;
  for (int b = 0; b < B; ++b) n_sum += q.items[b].n;
  const int prep_pts = rtg::prep_points_for(n_sum);
  const bool bitset = (q.flags & RTG_FLAG_BITSET) != 0 && m > 0;
  int maxd = 1, mind = RTG_MAX_DIM;
  for (int b = 0; b < B; ++b) {
    const rtg_instance& it = q.items[b];
    Inst& I = c->h_inst[b];
    I.pts = it.points;
    I.p0 = p0;
    I.T0 = T0;
    I.n = (int)it.n;
    I.d = it.d;
    I.r = it.r;
    I.c = m > 0 ? it.cell_side : 1.0;
    I.inv_c = 1.0 / I.c;
    I.inv_cf = (float)I.inv_c;
    I.blk0 = blk0;
    I.pblk0 = pblk0;
    I.bits_w = (int)((it.n + 31) / 32);
    I.bits_off = bits_words;
    bits_words += it.n * (long long)I.bits_w;
    p0 += it.n;
    blk0 += (it.n + rtg::kPointBlock - 1) / rtg::kPointBlock;
    pblk0 += (it.n + prep_pts - 1) / prep_pts;
    T0 += (long long)m * (it.d * it.d + it.d);
    maxd = std::max(maxd, it.d);
    mind = std::min(mind, it.d);
  }
  const long long n_total = p0;
  out->n = n_total;
  out->symmetric = sym;
  if (n_total * std::max(m, 1) >= (1LL << 31))
    return fail(c, RTG_E_INVALID, "total points times grids must be below 2^31");
  if (m > 0 && B * (long long)m > 65535)
    return fail(c, RTG_E_INVALID, "instances times grids must be at most 65535");
  if (bitset)
    for (int b = 0; b < B; ++b)
      if (q.items[b].n > rtg::kBitsetMaxN)
        return fail(c, RTG_E_INVALID, "RTG_FLAG_BITSET takes instances of at most 16384 points");
  if (n_total == 0) {
    void* rp = nullptr;
    if ((s = alloc_out(c, sizeof(int64_t), &rp)) != RTG_OK) return s;
    RTG_CUDA(c, cudaMemsetAsync(rp, 0, sizeof(int64_t), st));
    RTG_CUDA(c, cudaStreamSynchronize(st));
    out->row_ptr = (int64_t*)rp;
    out->handle = register_out(c, sizeof(int64_t));
    return RTG_OK;
  }
  const int dpad = rtg::dpad_for(maxd);
  const long long N = n_total * m;
  if (m > 0) {
    c->h_T.resize((size_t)T0);
    for (int b = 0; b < B; ++b) {
      const rtg_instance& it = q.items[b];
      std::memcpy(c->h_T.data() + c->h_inst[b].T0, it.transforms,
                  sizeof(double) * (size_t)m * (it.d * it.d + it.d));
    }
  }

  // ---- workspace ----
  const size_t bbox_bytes = sizeof(unsigned long long) * B * rtg::kMaxDim * 2;
  // counters, bounding boxes and the scan's look-back words, zeroed by one memset per build
  const size_t front_bytes = kStatusBytes + bbox_bytes + rtg::scan_lookback_bytes(n_total);
  if ((s = ensure(c, c->status, front_bytes)) != RTG_OK) return s;
  if ((s = ensure(c, c->inst, sizeof(Inst) * B)) != RTG_OK) return s;
  if ((s = ensure(c, c->iplan, sizeof(InstPlan) * B)) != RTG_OK) return s;
  if (m > 0) {
    if ((s = ensure(c, c->gplan, sizeof(GridPlan) * (size_t)B * m)) != RTG_OK) return s;
    if ((s = ensure(c, c->bases, sizeof(unsigned long long) * ((size_t)B * m + 1))) != RTG_OK) return s;
    if ((s = ensure(c, c->T64, sizeof(double) * (size_t)T0)) != RTG_OK) return s;
  }
  if ((s = ensure(c, c->pf, (size_t)n_total * dpad * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->row_cnt, (size_t)n_total * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->out_slot, sizeof(rtg::OutSlot))) != RTG_OK) return s;
  if (bitset && (s = ensure(c, c->bits, (size_t)bits_words * 4)) != RTG_OK) return s;
  if ((s = ensure(c, c->sort_epoch, sizeof(unsigned int), true)) != RTG_OK) return s;
  if (!q.points_on_device) {
    if ((s = ensure(c, c->pts, (size_t)n_total * maxd * esz + 16 * (size_t)B)) != RTG_OK) return s;
    size_t off = 0;
    for (int b = 0; b < B; ++b) {
      const size_t bytes = (size_t)q.items[b].n * q.items[b].d * esz;
      if (bytes)
        RTG_CUDA(c, cudaMemcpyAsync((char*)c->pts.p + off, q.items[b].points, bytes,
                                    cudaMemcpyHostToDevice, st));
      c->h_inst[b].pts = (char*)c->pts.p + off;
      off += (bytes + 15) & ~size_t(15);
    }
  }
  {
    // instance table and transforms: through pinned staging, and only when they changed
    const size_t ib = sizeof(Inst) * B, tb = m > 0 ? sizeof(double) * (size_t)T0 : 0;
    const size_t ib_al = (ib + 255) & ~size_t(255);
    if (c->h_stage_cap < ib_al + tb) {
      if (c->h_stage) cudaFreeHost(c->h_stage);
      c->h_stage = nullptr;
      c->h_stage_cap = 0;
      RTG_CUDA(c, cudaMallocHost(&c->h_stage, ib_al + tb));
      c->h_stage_cap = ib_al + tb;
    }
    auto upload = [&](DevBuf& dst, const void* src, size_t bytes, size_t off,
                      Upload& last) -> rtg_status {
      if (last.gen == dst.gen && last.bytes.size() == bytes &&
          std::memcmp(last.bytes.data(), src, bytes) == 0)
        return RTG_OK;
      std::memcpy((char*)c->h_stage + off, src, bytes);
      RTG_CUDA(c, cudaMemcpyAsync(dst.p, (char*)c->h_stage + off, bytes, cudaMemcpyHostToDevice,
                                  st));
      last.bytes.assign((const unsigned char*)src, (const unsigned char*)src + bytes);
      last.gen = dst.gen;
      return RTG_OK;
    };
    if ((s = upload(c->inst, c->h_inst.data(), ib, 0, c->up_inst)) != RTG_OK) return s;
    if (m > 0 && (s = upload(c->T64, c->h_T.data(), tb, ib_al, c->up_T)) != RTG_OK) return s;
  }

  BuildArgs a{};
  a.B = B;
  a.m = m;
  a.dtype = q.dtype;
  a.dpad = dpad;
  a.d_common = mind == maxd ? maxd : 0;
  a.symmetric = sym;
  a.n_total = n_total;
  a.blocks = blk0;
  a.pblocks = pblk0;
  a.prep_points = prep_pts;
  a.inst = (const Inst*)c->inst.p;
  a.iplan = (InstPlan*)c->iplan.p;
  a.gplan = (GridPlan*)c->gplan.p;
  a.bases = (unsigned long long*)c->bases.p;
  a.bbox = bbox_of(c);
  a.T64 = (const double*)c->T64.p;
  a.st = (Status*)c->status.p;
  a.pf = (float*)c->pf.p;
  a.row_cnt = (unsigned int*)c->row_cnt.p;
  a.scan_lookback =
      reinterpret_cast<unsigned long long*>((char*)c->status.p + kStatusBytes + bbox_bytes);
  a.scan_zeroed = 1;  // every build path zeroes them with the counters and scans once
  a.out = (const rtg::OutSlot*)c->out_slot.p;
  a.bits = bitset ? (unsigned int*)c->bits.p : nullptr;
  a.sort_epoch = (unsigned int*)c->sort_epoch.p;
  a.num_sms = c->num_sms;
  a.spin_limit = c->spin_limit;
  a.inject = c->inject;
  a.tc_cells = m > 0 ? ((q.flags & RTG_FLAG_TC_BF16) ? 2 : ((q.flags & RTG_FLAG_TC_FP16) ? 1 : 0))
                     : 0;

  const ShapeKey key{n_total, B, m, q.dtype, maxd, sym, q.count_only ? 1 : 0};
  auto git = c->guesses.find(key);
  const bool known = git != c->guesses.end();
  ShapeGuess g = known ? git->second : ShapeGuess{};
  const bool two_pass_flag = (q.flags & RTG_FLAG_TWO_PASS) != 0;

  bool tuned_now = false;
  int recovered = 0;  // columns written by a second enumeration after a pair-buffer overflow
  for (int attempt = 0; attempt < 5; ++attempt) {
    int launches = 0;
    a.skip_tail = 0;
    if (m > 0 && !known && attempt == 0) {
      // first build of this shape: read the key width back once
      RTG_CUDA(c, cudaMemsetAsync(a.st, 0, kStatusBytes + bbox_bytes, st));  // and the boxes
      a.passes = rtg::sort_passes_for(64, 8);
      a.sort_bits = 8;
      rtg::launch_prep_plan(a, st);
      if ((s = read_status(c)) != RTG_OK) return s;
      if ((s = check_errors(c, rtg::kErrNonFinite | rtg::kErrKeyOverflow)) != RTG_OK) return s;
      g.key_bits = (int)c->h_status->sort_bits;
      g.cell_bits = (int)c->h_status->cell_bits;
      g.key64 = g.key_bits > 32;
    }
    // Cell-major sort (one instance, the lane key kernel, 32-bit keys) where leaving the grid
    // out of the key saves an 8-bit pass; the sorted bits are then the cell index's.
    const bool cm_ok = c->cell_major && m > 1 && B == 1 && !bitset && !q.grid_major &&
                       n_total >= 2 && !g.key64 && rtg::keys_by_lanes(a) && g.cell_bits > 0 &&
                       rtg::sort_passes_for(g.cell_bits, 8) < rtg::sort_passes_for(g.key_bits, 8);
    const int sort_key_bits = cm_ok ? g.cell_bits : g.key_bits;
    bool tune_now = false;
    if (m > 0 && !g.sorted_cfg) {
      // sort variant: forced, else the autotuner's table, else measure now (large sorts), else
      // the default
      const auto it = c->sort_tune.find(SortKey(N, sort_key_bits));
      if (c->sort_forced) {
        g.sort = c->sort_force;
        g.sorted_cfg = true;
      } else if (it != c->sort_tune.end()) {
        g.sort = it->second.cfg;
        g.sorted_cfg = true;
      } else if (c->autotune && N >= kTuneMinElements) {
        // measured on the second build of a shape (a repeated shape pays for the trials; a
        // stream of distinct shapes, as in serving, is never held up by them); the first
        // build takes the default and leaves the choice open
        if (known) tune_now = true;
        else g.sort = sort_default(N, c->num_sms);
      } else {
        g.sort = sort_default(N, c->num_sms);
        g.sorted_cfg = true;
      }
    }
    a.key64 = g.key64;
    a.sort_bits = g.sort.bits;
    a.sort_items = g.sort.items;
    a.sort_mode = g.sort.mode;
    // (8-bit digits in separate passes only; the tuner times those forms alone)
    a.cell_major = 0;
    if (cm_ok && (tune_now || (g.sort.mode != rtg::kSortCoop && g.sort.bits == 8))) {
      a.cell_major = 1;
      a.passes = rtg::sort_passes_for(g.cell_bits, g.sort.bits);
    }
    if (!a.cell_major) a.passes = rtg::sort_passes_for(g.key_bits, g.sort.bits);
    // pair enumeration: one static span per warp for light cells (fewest span set-ups); more,
    // smaller spans claimed dynamically when the shape's cells held many candidates, so that
    // warps with heavy spans do not trail
    a.spans_per_warp = g.pairs_tuned ? g.spans_per_warp
                                     : (g.cand_per_pos < 0.0f ? 2 : (g.cand_per_pos >= 3.0f ? 4 : 1));
    a.dense_min = g.pairs_tuned ? g.dense_min : 0;
    if (m > 0) {
      const size_t ksz = a.key64 ? 8 : 4;
      if ((s = ensure(c, c->key_mat, (size_t)N * ksz)) != RTG_OK) return s;
      if ((s = ensure(c, c->keys0, (size_t)N * ksz)) != RTG_OK) return s;
      if ((s = ensure(c, c->keys1, (size_t)N * ksz)) != RTG_OK) return s;
      if ((s = ensure(c, c->vals0, (size_t)N * 4)) != RTG_OK) return s;
      if ((s = ensure(c, c->vals1, (size_t)N * 4)) != RTG_OK) return s;
      // look-back words (8 bytes, epoch tagged) need zeroed memory once; counts (4 bytes) are
      // rewritten by every pass
      const size_t scratch = tune_now ? sort_scratch_bytes_max(N) : sort_scratch_bytes(N, g.sort);
      if ((s = ensure(c, c->lookback, scratch, true)) != RTG_OK) return s;
      if ((s = ensure(c, c->hist, rtg::kSortCountWords * 4, true)) != RTG_OK) return s;
      if ((s = ensure(c, c->digit_off, rtg::kSortCountWords * 4)) != RTG_OK) return s;
      const unsigned int large_cap = (unsigned int)(N / (rtg::kSmallCell + 1) + 1);
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
      if (tune_now) {
        // measure every sort variant on this build's keys (the plan of the key-width read-back
        // above is in place), then run the build from the start
        rtg::SortConfig best;
        if ((s = tune_sort(c, a, N, sort_key_bits, &best)) != RTG_OK) return s;
        g.sort = best;
        g.sorted_cfg = true;
        // and the enumeration knobs, on the keys sorted with that variant, unless the shape
        // has so many in-cell candidates (clustered points) that the trials, each of which
        // enumerates every candidate, would cost seconds
        if (g.cand_per_pos >= 0.0f &&
            (double)g.cand_per_pos * (double)N <= c->tune_pairs_max_cand) {
          if ((s = tune_pairs(c, a, best, sort_key_bits, &g.spans_per_warp, &g.dense_min)) !=
              RTG_OK)
            return s;
          g.pairs_tuned = g.spans_per_warp > 0;
        }
        tuned_now = true;
        continue;
      }
    }

    // output row pointers
    void* rp = nullptr;
    if ((s = alloc_out(c, sizeof(int64_t) * (n_total + 1), &rp)) != RTG_OK) return s;
    out->row_ptr = (int64_t*)rp;
    out->col = nullptr;
    out->handle = register_out(c, sizeof(int64_t) * (n_total + 1));
    a.row_ptr = (long long*)rp;
    a.col = nullptr;
    a.col_cap = 0;

    // pair buffer for EMIT; COUNT then WRITE when asked, when only counting, or when the buffer
    // would not fit the budget
    if (g.pair_cap <= 0) {
      g.pair_cap = std::max<long long>(4096, n_total * 16);
      const double h = m > 0 ? c->ppp_hint.get(maxd) : 0.0;
      if (h > 0.0)
        g.pair_cap = std::max(g.pair_cap, (long long)(1.5 * h * (double)n_total) + 4096);
    }
    bool two_pass = two_pass_flag || q.count_only || bitset;
    if (!two_pass) {
      const size_t need = (size_t)g.pair_cap * 8;
      if (c->budget && total_held(c) - c->pair_buf.cap + need + need / (sym ? 1 : 2) > c->budget) {
        two_pass = true;
        // the count-then-write form needs no pair buffer: a large one from an earlier build
        // would only crowd the columns out of the budget
        free_buf(c, c->pair_buf);
      }
    }
    const bool tc = m == 0 && (q.flags & (RTG_FLAG_TC_FP16 | RTG_FLAG_TC_BF16)) != 0;
    if (tc) {
      if ((s = ensure(c, c->tc_tiles, rtg::tc_tiles_bytes(n_total))) != RTG_OK) return s;
      if ((s = ensure(c, c->tc_norms, (size_t)(n_total + 128) * 4)) != RTG_OK) return s;
      if ((s = ensure(c, c->tc_plan, sizeof(rtg::TcPlan))) != RTG_OK) return s;
    }
    int sorted = 0;
    // phase marks: recorded as real event records even inside a captured graph
    auto mark = [&](int i) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(st, &cs);
      if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(c->ev[i], st, cudaEventRecordExternal);
      else
        cudaEventRecord(c->ev[i], st);
    };
    // front of every build: counters, bounding boxes, plan, keys, sort (phases 0-3)
    auto front = [&]() -> int {
      int l = 0;
      if (timing) mark(0);
      cudaMemsetAsync(a.st, 0, front_bytes, st);  // counters, boxes, scan look-back words
      l += rtg::launch_prep_plan(a, st);
      if (timing) mark(1);
      if (m > 0) {
        rtg::launch_keys(a, st);
        l += 1;
        if (timing) mark(2);
        sorted = rtg::launch_sort(a, st);
        l += (a.passes > 0 && N > 1)
                 ? (rtg::hist_in_keys(a) ? 0 : 1) +
                       (a.sort_mode == rtg::kSortCoop
                            ? 1
                            : (a.sort_mode == rtg::kSortLookback ? 1 : 3) * a.passes)
                 : 1;  // the identity copy when there is nothing to sort
      } else if (timing) {
        mark(2);
      }
      if (timing) mark(3);
      return l;
    };
    auto pairs = [&](rtg::Mode mode) {
      if (m > 0) return rtg::launch_pairs(a, sorted, mode, st);
      if (tc)
        return rtg::launch_brute_tc(a, (q.flags & RTG_FLAG_TC_BF16) != 0, mode,
                                    (unsigned char*)c->tc_tiles.p, (float*)c->tc_norms.p,
                                    (rtg::TcPlan*)c->tc_plan.p, st);
      return rtg::launch_brute(a, mode, st);
    };
    // the output pointers the scan, scatter and row sort read (pinned copy -> device slot)
    auto set_slot = [&]() {
      c->h_slot->row_ptr = a.row_ptr;
      c->h_slot->col = a.col;
      c->h_slot->col_cap = a.col_cap;
      cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice, st);
    };
    if (!two_pass) {
      // kernels the last build of this shape gave nothing to do are left out; the kernels
      // before them flag any work that turns up, and the build runs again with them
      if (m > 0 && known)
        a.skip_tail =
            (g.no_dense ? rtg::kSkipDense : 0) | (g.no_long_rows ? rtg::kSkipLongRows : 0);
      if ((s = ensure(c, c->pair_buf, (size_t)g.pair_cap * 8)) != RTG_OK) return s;
      a.pair_buf = (unsigned long long*)c->pair_buf.p;
      a.pair_cap = g.pair_cap;
      const long long ccap = a.pair_cap * (sym ? 2 : 1);
      void* cp = nullptr;
      if ((s = alloc_out(c, sizeof(int32_t) * (size_t)ccap, &cp)) != RTG_OK) {
        release_out(c, out);
        return s;
      }
      out->col = (int32_t*)cp;
      {
        std::lock_guard<std::mutex> lk(c->live_mu);
        c->live[out->handle] += sizeof(int32_t) * (size_t)ccap;
      }
      a.col = (int*)cp;
      a.col_cap = ccap;
      c->h_slot->row_ptr = a.row_ptr;
      c->h_slot->col = a.col;
      c->h_slot->col_cap = a.col_cap;
      // the whole build as one fixed launch sequence, ending with the status copy-back
      auto emit_build = [&]() -> int {
        int l = 0;
        // the scan is the first reader of the output slot: its copy runs on the side stream
        // beside the front and the enumeration, and joins before the scan
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice,
                        c->side);
        cudaEventRecord(c->ev_join, c->side);
        l += front();
        l += pairs(rtg::kEmit);
        if (timing) mark(4);
        cudaStreamWaitEvent(st, c->ev_join, 0);
        rtg::launch_scan(a, st);
        l += 1;
        if (timing) mark(5);
        l += rtg::launch_scatter(a, st);
        if (timing) mark(6);
        l += rtg::launch_rowsort(a, st);
        if (timing) mark(7);
        cudaMemcpyAsync(c->h_status, c->status.p, sizeof(Status), cudaMemcpyDeviceToHost, st);
        return l;
      };
      bool done = false;
      if (m > 0 && known && attempt == 0 && c->use_graphs) {
        cudaGraphExec_t exec = nullptr;
        int gl = 0;
        if ((s = graph_for(c, key, a, timing, emit_build, &exec, &gl)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
        if (exec && cudaGraphLaunch(exec, st) == cudaSuccess) {
          launches += gl;
          done = true;
        } else {
          cudaGetLastError();
          drop_graph(c, key);
        }
      }
      if (!done) launches += emit_build();
      RTG_CUDA(c, cudaGetLastError());
      {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
          release_out(c, out);
          return fail(c, RTG_E_CUDA, std::string("build: ") + cudaGetErrorString(e));
        }
      }
      // An undersized pair buffer (the first build of a shape, or more pairs than its last
      // build): every pair was still counted in its row and the scan has placed the rows, so
      // only the columns are missing.  A second enumeration writes them straight into their
      // rows, as the two-pass form does, instead of running the whole build again.
      const unsigned int ovf = rtg::kErrPairOverflow | rtg::kErrColOverflow;
      const unsigned int herr = c->h_status->errors;
      if ((herr & rtg::kErrPairOverflow) && !(herr & ~ovf)) {
        const long long nnz = (long long)c->h_status->nnz;
        const size_t old_bytes = sizeof(int32_t) * (size_t)a.col_cap;
        cudaFreeAsync(out->col, st);
        {
          std::lock_guard<std::mutex> lk(c->live_mu);
          c->live[out->handle] -= old_bytes;
          c->out_bytes -= old_bytes;
        }
        out->col = nullptr;
        a.col = nullptr;
        a.col_cap = 0;
        // the pair buffer holds nothing the write pass needs
        if (c->budget && total_held(c) + sizeof(int32_t) * (size_t)nnz > c->budget)
          free_buf(c, c->pair_buf);
        a.pair_buf = nullptr;
        a.pair_cap = 0;
        void* cp = nullptr;
        if ((s = alloc_out(c, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
        out->col = (int32_t*)cp;
        {
          std::lock_guard<std::mutex> lk(c->live_mu);
          c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
        }
        a.col = (int*)cp;
        a.col_cap = nnz;
        // the overflow flags go; the fill cursors (used by the scatter, then by the row sort's
        // queues) and the row-sort queue counts start again from zero
        RTG_CUDA(c, cudaMemsetAsync(&a.st->errors, 0, sizeof(a.st->errors), st));
        RTG_CUDA(c, cudaMemsetAsync(a.row_cnt, 0, sizeof(unsigned int) * (size_t)n_total, st));
        RTG_CUDA(c, cudaMemsetAsync(&a.st->long_rows, 0, sizeof(a.st->long_rows), st));
        RTG_CUDA(c, cudaMemsetAsync(&a.st->mid_rows, 0, sizeof(a.st->mid_rows), st));
        set_slot();
        launches += pairs(rtg::kWrite);
        if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
        launches += rtg::launch_rowsort(a, st);
        if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
        RTG_CUDA(c, cudaGetLastError());
        if ((s = read_status(c)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
        ++recovered;
      }
    } else if (bitset) {
      // bit-matrix dedupe (Sec. III-B): every reported candidate sets its bit; rows come out
      // of the matrices already sorted
      RTG_CUDA(c, cudaMemsetAsync(a.bits, 0, (size_t)bits_words * 4, st));
      set_slot();
      launches += front();
      launches += pairs(rtg::kBits);
      if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[4], st));
      launches += rtg::launch_bits_count(a, st);
      rtg::launch_scan(a, st);
      launches += 1;
      if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[5], st));
      RTG_CUDA(c, cudaGetLastError());
      if ((s = read_status(c)) != RTG_OK) {
        release_out(c, out);
        return s;
      }
      const long long nnz = (long long)c->h_status->nnz;
      if (!(c->h_status->errors & rtg::kErrKeyBits) && !q.count_only && nnz > 0) {
        void* cp = nullptr;
        if ((s = alloc_out(c, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
        out->col = (int32_t*)cp;
        {
          std::lock_guard<std::mutex> lk(c->live_mu);
          c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
        }
        a.col = (int*)cp;
        a.col_cap = nnz;
        set_slot();
        launches += rtg::launch_bits_write(a, st);
      }
      if (timing) {
        RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
        RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
      }
      RTG_CUDA(c, cudaGetLastError());
      if ((s = read_status(c)) != RTG_OK) {
        release_out(c, out);
        return s;
      }
      c->h_status->pairs = c->h_status->nnz / (sym ? 2 : 1);
      c->h_status->owned_candidates = 0;
    } else {
      set_slot();
      launches += front();
      launches += pairs(rtg::kCount);
      if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[4], st));
      rtg::launch_scan(a, st);
      launches += 1;
      if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[5], st));
      RTG_CUDA(c, cudaGetLastError());
      if ((s = read_status(c)) != RTG_OK) {
        release_out(c, out);
        return s;
      }
      if (!(c->h_status->errors & rtg::kErrKeyBits) && !q.count_only && c->h_status->nnz > 0) {
        const long long nnz = (long long)c->h_status->nnz;
        void* cp = nullptr;
        if ((s = alloc_out(c, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
        out->col = (int32_t*)cp;
        {
          std::lock_guard<std::mutex> lk(c->live_mu);
          c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
        }
        a.col = (int*)cp;
        a.col_cap = nnz;
        set_slot();
        launches += pairs(rtg::kWrite);
        if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
        launches += rtg::launch_rowsort(a, st);
        if (timing) RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
        RTG_CUDA(c, cudaGetLastError());
        if ((s = read_status(c)) != RTG_OK) {
          release_out(c, out);
          return s;
        }
      } else if (timing) {
        RTG_CUDA(c, cudaEventRecord(c->ev[6], st));
        RTG_CUDA(c, cudaEventRecord(c->ev[7], st));
        RTG_CUDA(c, cudaEventSynchronize(c->ev[7]));
      }
    }
    const Status& h = *c->h_status;
    if (h.errors & rtg::kErrTimeout) {  // whatever else is flagged follows from the timeout
      release_out(c, out);
      return fail(c, RTG_E_TIMEOUT, "a bounded device wait ran out");
    }
    const unsigned int retry = rtg::kErrKeyBits | rtg::kErrPairOverflow | rtg::kErrTailSkipped;
    if (h.errors & retry) {
      // the launch assumptions were too small: take the device's values and run again
      release_out(c, out);
      if (h.errors & rtg::kErrTailSkipped) {
        g.no_dense = false;
        g.no_long_rows = false;
      }
      if (h.errors & rtg::kErrKeyBits) {
        g.key64 = h.sort_bits > 32;
        g.key_bits = (int)h.sort_bits;
        g.cell_bits = (int)h.cell_bits;
      }
      if (h.errors & rtg::kErrPairOverflow)
        g.pair_cap = (long long)((double)h.emitted * 1.05) + 4096;
      continue;
    }
    if ((s = check_errors(c, ~0u)) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    // remember the launch decisions for the next build of this shape
    if (m > 0) {
      g.key64 = h.sort_bits > 32;
      g.key_bits = (int)h.sort_bits;
      g.cell_bits = (int)h.cell_bits;
    }
    if (!two_pass)
      g.pair_cap = std::max<long long>((long long)((double)h.emitted * 1.05) + 4096, 4096);
    if (m > 0 && !bitset) {
      // with a margin, so that new data of the same shape seldom brings such work back
      g.no_dense = h.max_cell <= (unsigned long long)rtg::kSkipMargin;
      g.no_long_rows = h.rows_over_margin == 0;
    }
    if (m > 0 && n_total > 0 && !q.count_only) {
      c->ppp_hint.put(maxd, (double)h.pairs / (double)n_total);
    }
    {
      double cand = 0.0;
      for (int t = 0; t < m && t < RTG_MAX_GRIDS; ++t) cand += (double)h.candidates[t];
      g.cand_per_pos = N > 0 ? (float)(cand / (double)N) : 0.0f;
    }
    c->guesses[key] = g;
    c->last_sorted = sorted;

    out->n = n_total;
    out->symmetric = sym;
    out->nnz = q.count_only ? (long long)h.pairs * (sym ? 2 : 1) : (long long)h.nnz;
    rtg_stats& S = out->stats;
    std::memset(&S, 0, sizeof(S));
    long long total_cand = 0;
    for (int t = 0; t < m && t < RTG_MAX_GRIDS; ++t) {
      S.candidates[t] = (int64_t)h.candidates[t];
      total_cand += (long long)h.candidates[t];
    }
    S.total_candidates = total_cand;
    S.owned_candidates = (int64_t)h.owned_candidates;
    S.near_wall = (int64_t)h.near_wall;
    S.near_r = (int64_t)h.near_r;
    S.key_rechecks = (int64_t)h.key_rechecks;
    S.dist_rechecks = (int64_t)h.dist_rechecks;
    S.large_cells = (int64_t)h.large_cells;
    S.max_cell = (int64_t)h.max_cell;
    S.pairs = (int64_t)h.pairs;
    S.key_bits = (int32_t)h.sort_bits;
    S.sort_passes = m > 0 ? a.passes : 0;
    S.sort_digit_bits = m > 0 ? a.sort_bits : 0;
    S.sort_tile_keys = m > 0 ? 256 * a.sort_items : 0;
    S.sort_lookback =
        m > 0 ? (a.sort_mode == rtg::kSortLookback ? 1 : (a.sort_mode == rtg::kSortCoop ? 2 : 0))
              : 0;
    {
      const auto it = c->sort_tune.find(SortKey(N, sort_key_bits));
      S.sort_tuned = m > 0 && it != c->sort_tune.end() && it->second.cfg.bits == g.sort.bits &&
                     it->second.cfg.items == g.sort.items && it->second.cfg.mode == g.sort.mode;
    }
    S.launches = launches;
    S.attempts = attempt + 1 - (tuned_now ? 1 : 0) + recovered;
    S.pairs_spans_per_warp = m > 0 ? a.spans_per_warp : 0;
    S.dense_cell_min = m > 0 ? (a.dense_min > 0 ? a.dense_min : 256) : 0;
    S.pairs_tuned = m > 0 && g.pairs_tuned ? 1 : 0;
    S.sort_cell_major = m > 0 && a.cell_major ? 1 : 0;
    S.sort_key_bits = m > 0 ? (a.cell_major ? (int32_t)h.cell_bits : (int32_t)h.sort_bits) : 0;
    {
      // bytes each phase reads and writes by its design (phase order of phase_us)
      const double n_ = (double)n_total, N_ = (double)N, kb = a.key64 ? 8.0 : 4.0;
      double in_bytes = 0.0;  // the points, n d S over the instances
      for (int b = 0; b < B; ++b) in_bytes += (double)q.items[b].n * q.items[b].d * (double)esz;
      const double P = (double)h.pairs, stored = (double)h.nnz;
      const double rows = n_ * dpad * 4.0;
      double pb[7] = {};
      pb[0] = in_bytes + rows + 4.0 * n_;  // points in, FP32 rows and zeroed row counts out
      if (m > 0) {
        // FP32 rows in, key rows out (and their grid-major copy for a cell-major sort)
        pb[1] = rows + N_ * kb * (a.cell_major ? 2.0 : 1.0);
        // the first pass reads the key rows (indices implicit); every pass writes keys and
        // indices, and the later ones also read them
        pb[2] = a.passes > 0 ? N_ * kb + N_ * (kb + 4.0) +
                                   (a.passes - 1) * 2.0 * N_ * (kb + 4.0) +
                                   (rtg::hist_in_keys(a) ? 0.0 : N_ * kb)
                             : 0.0;
        pb[3] = N_ * (kb + 4.0) + N_ * dpad * 4.0 + (two_pass ? 0.0 : 8.0 * P);
      } else {
        pb[3] = rows + (two_pass ? 0.0 : 8.0 * P);  // brute force: the rows, the pairs out
      }
      pb[4] = 4.0 * n_ + 8.0 * (n_ + 1.0);  // row counts in, row pointers out
      pb[5] = two_pass ? 4.0 * stored : 8.0 * P + 4.0 * stored;  // pairs in, columns out
      pb[6] = 8.0 * stored;                                      // columns read and written
      double tot = 0.0;
      for (int p = 0; p < 7; ++p) {
        S.phase_bytes[p] = (int64_t)pb[p];
        tot += pb[p];
      }
      S.phase_bytes[7] = (int64_t)tot;
      S.bytes_moved = (int64_t)tot;
    }
    {
      float e;
      std::memcpy(&e, &h.tc_max_err_bits, 4);
      S.max_abs_err_d2 = e;
      S.band = h.tc_band;
    }
    if (timing) {
      float ms;
      // prep+plan, keys, sort, pairs, scan, scatter/write, rowsort, total
      const int idx[8][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {4, 5}, {5, 6}, {6, 7}, {0, 7}};
      for (int p = 0; p < 8; ++p) {
        ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[idx[p][0]], c->ev[idx[p][1]]) != cudaSuccess) {
          cudaGetLastError();
          ms = 0.f;
        }
        S.phase_us[p] = 1000.0 * ms;
      }
    }
    return RTG_OK;
  }
  return fail(c, RTG_E_INTERNAL, "launch assumptions did not converge");
}


rtg_status create_ctx(int device, uint64_t budget, void* stream, rtg_ctx** out) {
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, RTG_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (device < 0 || device >= ndev) return fail(nullptr, RTG_E_INVALID, "device ordinal out of range");
  rtg_ctx* c = new rtg_ctx();
  c->device = device;
  c->budget = budget;
  auto bail = [&](cudaError_t err) {
    std::string msg = std::string("context setup: ") + cudaGetErrorString(err);
    destroy_ctx(c);
    return fail(nullptr, RTG_E_CUDA, msg);
  };
  if ((e = cudaSetDevice(c->device)) != cudaSuccess) return bail(e);
  if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device)) !=
      cudaSuccess)
    return bail(e);
  {
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, c->device)) != cudaSuccess) return bail(e);
    c->device_name = std::string(prop.name) + " sm_" + std::to_string(prop.major) +
                     std::to_string(prop.minor) + " " + std::to_string(prop.multiProcessorCount) +
                     "SM";
  }
  tune_load(c);
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
      return bail(e);
    c->own_stream = true;
  }
  if ((e = cudaMallocHost(&c->h_status, sizeof(Status))) != cudaSuccess) return bail(e);
  if ((e = cudaMallocHost(&c->h_slot, sizeof(rtg::OutSlot))) != cudaSuccess) return bail(e);
  {
    const char* g = std::getenv("RTG_GRAPHS");
    c->use_graphs = !(g && std::strcmp(g, "0") == 0);
    const char* cm = std::getenv("RTG_CELL_MAJOR");
    c->cell_major = !(cm && std::strcmp(cm, "0") == 0);
  }

  {
    // a pool of its own for the output CSRs, so that freed blocks stay cached between builds
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    if ((e = cudaMemPoolCreate(&c->pool, &props)) != cudaSuccess) return bail(e);
    uint64_t keep = ~0ull;
    if ((e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep)) !=
        cudaSuccess)
      return bail(e);
  }
  for (auto& ev : c->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(e);
  if ((e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming)) != cudaSuccess)
    return bail(e);
  rtg_status s = ensure(c, c->status, kStatusBytes, true);
  if (s != RTG_OK) {
    std::string msg = c->err;
    destroy_ctx(c);
    return fail(nullptr, s, msg);
  }
  *out = c;
  return RTG_OK;
}

void trim_workspace(rtg_ctx* c) {
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->pts,      &c->pf,        &c->key_mat, &c->keys0,    &c->keys1,
                    &c->vals0,    &c->vals1,     &c->lookback, &c->row_cnt, &c->scan_lb,
                    &c->large,    &c->large_job, &c->pair_buf, &c->tc_tiles, &c->tc_norms};
  for (DevBuf* b : bufs) free_buf(c, *b);
  // captured graphs name the freed buffers (a replay needs the same pointers, so none would
  // replay; they go now rather than when their shape comes back)
  while (!c->graphs.empty()) drop_graph(c, c->graphs.begin()->first);
  if (c->pool) cudaMemPoolTrimTo(c->pool, 0);
}

void destroy_ctx(rtg_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->status,    &c->inst,      &c->iplan,   &c->gplan,   &c->bases,
                    &c->T64,       &c->pts,       &c->pf,      &c->key_mat,
                    &c->keys0,     &c->keys1,     &c->vals0,   &c->vals1,   &c->lookback,
                    &c->hist,      &c->digit_off, &c->row_cnt, &c->scan_lb, &c->large,
                    &c->large_job, &c->pair_buf,  &c->tc_tiles, &c->tc_norms, &c->tc_plan};
  for (DevBuf* b : bufs) free_buf(c, *b);
  while (!c->graphs.empty()) drop_graph(c, c->graphs.begin()->first);
  free_buf(c, c->out_slot);
  free_buf(c, c->q_idx);
  free_buf(c, c->bits);
  free_buf(c, c->sort_epoch);
  if (c->h_slot) cudaFreeHost(c->h_slot);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->pool && c->own_pool) cudaMemPoolDestroy(c->pool);  // outstanding CSRs go with it
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace rtghost

using namespace rtghost;

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

void* rtg_get_stream(const rtg_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

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
  return create_ctx(cfg->device, cfg->mem_budget_bytes, cfg->stream, out);
}

void rtg_destroy(rtg_ctx* c) {
  if (!c) return;
  stop_server(c);
  destroy_ctx(c);
}

rtg_status rtg_set_test_hooks(rtg_ctx* c, uint32_t inject, uint32_t wait_limit,
                              int64_t fail_alloc_after) {
  if (!c) return fail(nullptr, RTG_E_INVALID, "ctx is NULL");
  if (inject & ~(uint32_t)(RTG_INJECT_SORT_WAIT | RTG_INJECT_SCAN_WAIT | RTG_INJECT_TC_WAIT))
    return fail(c, RTG_E_INVALID, "unknown hook bits");
  if (wait_limit >= (1u << 31)) return fail(c, RTG_E_INVALID, "wait_limit must be below 2^31");
  std::lock_guard<std::mutex> lk(c->mu);
  c->inject = (inject & RTG_INJECT_SORT_WAIT ? rtg::kInjectSortWait : 0u) |
              (inject & RTG_INJECT_SCAN_WAIT ? rtg::kInjectScanWait : 0u) |
              (inject & RTG_INJECT_TC_WAIT ? rtg::kInjectTcWait : 0u);
  c->spin_limit = wait_limit;
  c->fail_alloc_at = fail_alloc_after > 0 ? c->alloc_calls.load() + fail_alloc_after : 0;
  return RTG_OK;
}

rtg_status rtg_release(rtg_ctx* c, rtg_csr* csr) {
  if (!c || !csr) return fail(c, RTG_E_INVALID, "NULL argument");
  {
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    release_out(c, csr);
  }
  // a request waiting for memory may fit now
  notify_server(c);
  return RTG_OK;
}

rtg_status rtg_tune_params(rtg_ctx* c, const void* points, int dtype, int points_on_device,
                           int64_t n, int d, double r, double target_recall, uint64_t seed,
                           uint32_t flags, rtg_param_choice* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  std::memset(out, 0, sizeof(*out));
  rtg_status s = validate_common(dtype, n, d, r, r, points);
  if (s != RTG_OK) return fail(c, s, g_err);
  if (!(target_recall > 0.0 && target_recall <= 1.0))
    return fail(c, RTG_E_INVALID, "target_recall must be in (0, 1]");
  if (n < 2) return fail(c, RTG_E_INVALID, "n must be at least 2");
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  return tune_params(c, points, dtype, points_on_device, n, d, r, target_recall, seed, flags, out);
}

rtg_status rtg_query_neighbors(rtg_ctx* c, const rtg_csr* graph, const int32_t* queries,
                               int64_t nq, int queries_on_device, rtg_csr* out) {
  if (!c || !graph || !out) return fail(c, RTG_E_INVALID, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (!graph->symmetric)
    return fail(c, RTG_E_INVALID, "neighbour queries need a symmetric CSR (RTG_FLAG_SYMMETRIC)");
  if (nq < 0 || nq >= (int64_t(1) << 31) || (nq > 0 && !queries))
    return fail(c, RTG_E_INVALID, "queries: count out of range or NULL");
  if (graph->n > 0 && !graph->row_ptr) return fail(c, RTG_E_INVALID, "graph has no row pointers");
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  return query_neighbors(c, graph, queries, nq, queries_on_device, out);
}

rtg_status rtg_index_create(rtg_ctx* c, const void* points, int dtype, int points_on_device,
                            int64_t n, int d, double r, const double* transforms, int m,
                            double cell_side, rtg_index** out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  *out = nullptr;
  rtg_status s = validate_common(dtype, n, d, r, cell_side, points);
  if (s == RTG_OK && (m < 1 || m > RTG_MAX_GRIDS))
    s = fail(nullptr, RTG_E_INVALID, "m must be in [1, 64]");
  if (s == RTG_OK) s = validate_transforms(transforms, d, m);
  if (s != RTG_OK) return fail(c, s, g_err);
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  rtg_instance it{points, n, d, r, cell_side, transforms};
  return index_create(c, it, m, dtype, points_on_device, out);
}

rtg_status rtg_index_query(rtg_ctx* c, const rtg_index* index, const void* queries,
                           int queries_on_device, int64_t nq, rtg_csr* out) {
  if (!c || !index || !out) return fail(c, RTG_E_INVALID, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (nq < 0 || nq >= (int64_t(1) << 31) || (nq > 0 && !queries))
    return fail(c, RTG_E_INVALID, "queries: count out of range or NULL");
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  return index_query(c, index, queries, queries_on_device, nq, out);
}

void rtg_index_destroy(rtg_ctx* c, rtg_index* index) {
  if (!c || !index) return;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaSetDevice(c->device);
  index_destroy(c, index);
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
  if (csr->nnz > 0 && csr->col)
    RTG_CUDA(c, cudaMemcpyAsync(col, csr->col, sizeof(int32_t) * csr->nnz, cudaMemcpyDeviceToHost,
                                c->stream));
  RTG_CUDA(c, cudaStreamSynchronize(c->stream));
  return RTG_OK;
}

rtg_status rtg_all_pairs(rtg_ctx* c, const void* points, int dtype, int points_on_device, int64_t n,
                         int d, double r, const double* transforms, int m, double cell_side,
                         uint32_t flags, rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  std::memset(out, 0, sizeof(*out));
  rtg_status s = validate_common(dtype, n, d, r, cell_side, points);
  if (s == RTG_OK && (m < 1 || m > RTG_MAX_GRIDS))
    s = fail(nullptr, RTG_E_INVALID, "m must be in [1, 64]");
  if (s == RTG_OK) s = validate_transforms(transforms, d, m);
  if (s != RTG_OK) return fail(c, s, g_err);
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  rtg_instance it{points, n, d, r, cell_side, transforms};
  Request q{&it, 1, m, dtype, points_on_device, flags, false};
  s = build(c, q, out);
  if (s != RTG_OK) release_out(c, out);
  return s;
}

rtg_status rtg_batch_all_pairs(rtg_ctx* c, const rtg_instance* items, int count, int m, int dtype,
                               int points_on_device, uint32_t flags, rtg_csr* out,
                               int64_t* row_offsets) {
  if (!c || !out || (count > 0 && !items)) return fail(c, RTG_E_INVALID, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (count < 1 || count > 65535) return fail(c, RTG_E_INVALID, "count must be in [1, 65535]");
  if (m < 1 || m > RTG_MAX_GRIDS) return fail(c, RTG_E_INVALID, "m must be in [1, 64]");
  long long off = 0;
  for (int b = 0; b < count; ++b) {
    const rtg_instance& it = items[b];
    rtg_status s = validate_common(dtype, it.n, it.d, it.r, it.cell_side, it.points);
    if (s == RTG_OK) s = validate_transforms(it.transforms, it.d, m);
    if (s != RTG_OK) return fail(c, s, "instance " + std::to_string(b) + ": " + g_err);
    if (row_offsets) row_offsets[b] = off;
    off += it.n;
  }
  if (row_offsets) row_offsets[count] = off;
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  Request q{items, count, m, dtype, points_on_device, flags, false};
  rtg_status s = build(c, q, out);
  if (s != RTG_OK) release_out(c, out);
  return s;
}

rtg_status rtg_brute_force(rtg_ctx* c, const void* points, int dtype, int points_on_device,
                           int64_t n, int d, double r, uint32_t flags, int count_only,
                           rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL context or output");
  std::memset(out, 0, sizeof(*out));
  rtg_status s = validate_common(dtype, n, d, r, 1.0, points);
  if (s != RTG_OK) return fail(c, s, g_err);
  std::lock_guard<std::mutex> lk(c->mu);
  RTG_CUDA(c, cudaSetDevice(c->device));
  rtg_instance it{points, n, d, r, 1.0, nullptr};
  Request q{&it, 1, 0, dtype, points_on_device, flags, count_only != 0};
  s = build(c, q, out);
  if (s != RTG_OK) release_out(c, out);
  return s;
}

}  // extern "C"
