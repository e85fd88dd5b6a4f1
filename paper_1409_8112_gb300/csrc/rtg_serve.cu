// Request server of a context: continuous batching of roadmap builds (rtg_submit, rtg_poll,
// rtg_wait).  Each request is one run of Alg. 1 of arXiv:1409.8112 over its own points.
//
// Requests wait in one FIFO queue.  A few lanes (each an internal context with its own stream,
// workspace and pool) take the oldest waiting request and the later waiting requests that share
// its m, dtype, flags and d as one batch, build them together with the batch pipeline, and split
// the block-diagonal result into one device CSR per request.  Lanes run concurrently, so a
// batch formed from requests that arrived while another batch was on the GPU overlaps with it.
//
// Admission by device memory: with a budget B (the context's mem_budget_bytes), a batch starts
// only when its estimated footprint fits next to everything already held (the context's own
// memory, the results not yet released, idle lanes' workspaces and running lanes'
// reservations); the oldest request has priority (nothing overtakes a waiting head; requests
// of its kind may join its batch ahead of older requests of another kind).  A lane
// builds with its reservation as its budget; a batch that does not fit is re-queued at the
// front as single exclusive requests, each of which then runs alone with all free memory, and
// fails with RTG_E_BUDGET if it still does not fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rtg_host.h"

namespace rtghost {

using Clock = std::chrono::steady_clock;

struct Ticket {
  uint64_t id = 0;
  std::vector<unsigned char> pts;
  std::vector<double> T;
  int dtype = 0;
  int64_t n = 0;
  int d = 1;
  double r = 0, c = 0;
  int m = 1;
  uint32_t flags = 0;
  bool exclusive = false;
  enum State { kQueued, kRunning, kDone, kFailed } state = kQueued;
  rtg_status status = RTG_OK;
  std::string err;
  rtg_csr result{};
  Clock::time_point t_submit, t_start, t_done;
};

struct Lane {
  rtg_ctx* ctx = nullptr;
  std::thread th;
  bool busy = false;
  uint64_t reservation = 0;
};

struct Server {
  rtg_ctx* owner = nullptr;
  std::vector<Lane> lanes;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Ticket*> queue;
  std::unordered_map<uint64_t, Ticket*> tickets;
  uint64_t next = 1;
  bool stop = false;
  int max_batch = 256;
  long long max_points = 1LL << 20;
  bool log = false;  // RTG_SERVE_LOG=1: one line per batch on stderr
  // reported pairs per point of finished batches (S->mu)
  PppHints ppp;
};

namespace {

struct SplitItem {
  long long off, n, base, nnz;
  long long* rp;
  int* col;
};

__global__ void k_gather_bases(const long long* __restrict__ row_ptr,
                               const long long* __restrict__ offs, int B, long long* bases) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b <= B) bases[b] = row_ptr[offs[b]];
}

// instance of a global row / entry: the last item whose start is <= x
__device__ __forceinline__ int find_item(const SplitItem* items, int B, long long x, bool by_base) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((by_base ? items[mid].base : items[mid].off) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_split_rows(const long long* __restrict__ row_ptr,
                             const SplitItem* __restrict__ items, int B, long long n_total) {
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < B;
       b += (long long)gridDim.x * blockDim.x)
    items[b].rp[items[b].n] = items[b].nnz;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n_total;
       g += (long long)gridDim.x * blockDim.x) {
    const SplitItem it = items[find_item(items, B, g, false)];
    it.rp[g - it.off] = row_ptr[g] - it.base;
  }
}

__global__ void k_split_cols(const int* __restrict__ col, const SplitItem* __restrict__ items,
                             int B, long long nnz_total) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz_total;
       e += (long long)gridDim.x * blockDim.x) {
    const SplitItem it = items[find_item(items, B, e, true)];
    it.col[e - it.base] = col[e] - (int)it.off;
  }
}

uint64_t held_except(Server* S, int li) {
  uint64_t h;
  {
    std::lock_guard<std::mutex> lk(S->owner->live_mu);
    h = S->owner->ws_bytes + S->owner->out_bytes;
  }
  for (int k = 0; k < (int)S->lanes.size(); ++k) {
    if (k == li) continue;
    const Lane& L = S->lanes[k];
    h += L.busy ? L.reservation : (uint64_t)(L.ctx->ws_bytes + L.ctx->out_bytes);
  }
  return h;
}

// Rough peak footprint of a batch (worst-case 64-bit keys; pairs per point as finished batches
// of the same d reported, at least 16).
uint64_t estimate(long long npts, long long nd, int m, int maxd, int dtype, double ppp) {
  const long long N = npts * m;
  const long long P = (long long)((double)npts * std::max(16.0, 1.25 * ppp));
  const long long dpad = rtg::dpad_for(maxd);
  return (uint64_t)(npts * (dpad * 4 + 4 + 8 + 8) + nd * (dtype == 0 ? 8 : 4) + 33 * N + 16 * P +
                    (1 << 20));
}

double ppp_of(Server* S, int d) { return S->ppp.get(d); }

bool compatible(const Ticket* a, const Ticket* b) {
  return a->m == b->m && a->dtype == b->dtype &&
         ((a->flags ^ b->flags) & RTG_FLAG_SYMMETRIC) == 0;
}

// Workspaces of idle lanes above this size are freed when the oldest request needs the memory.
constexpr uint64_t kTrimFloor = 64ull << 20;
// Requests of at least this many points are built alone.
constexpr long long kAloneMin = 1LL << 17;

// Frees the workspaces of lane li and of the other idle lanes, so that their memory counts as
// free again.  Called with S->mu held (an idle lane's thread holds no lock of its context).
void trim_idle(Server* S, int li) {
  for (int k = 0; k < (int)S->lanes.size(); ++k) {
    Lane& L = S->lanes[k];
    if (k != li && L.busy) continue;
    std::lock_guard<std::mutex> g(L.ctx->mu);
    if (L.ctx->ws_bytes > kTrimFloor) trim_workspace(L.ctx);
  }
}

// Called with S->mu held.  Takes a batch from the front of the queue if one may start on
// lane li now.
bool try_form(Server* S, int li, std::vector<Ticket*>& batch, uint64_t& reservation) {
  const uint64_t total = S->owner->budget;
  Ticket* head = S->queue.front();
  bool others_busy = false;
  for (int k = 0; k < (int)S->lanes.size(); ++k)
    if (k != li && S->lanes[k].busy) others_busy = true;
  uint64_t held = held_except(S, li);
  uint64_t free_mem = total == 0 ? ~0ull : (total > held ? total - held : 0);
  if (total != 0 &&
      (head->exclusive ||
       estimate(head->n, head->n * head->d, head->m, head->d, head->dtype, ppp_of(S, head->d)) >
           free_mem)) {
    // the oldest request does not fit next to what is held: idle lanes give back their
    // workspaces first
    trim_idle(S, li);
    held = held_except(S, li);
    free_mem = total > held ? total - held : 0;
  }
  if (head->exclusive) {
    if (others_busy) return false;
    batch.push_back(head);
    S->queue.pop_front();
    reservation = total == 0 ? 0 : free_mem;
    return true;
  }
  // the head, then later waiting requests of the same kind (m, dtype, flags and d: a batch of
  // one dimension needs no padding to its widest member and keeps the shape's key kernel)
  long long npts = 0, nd = 0;
  int maxd = 1;
  uint64_t est = 0;
  std::vector<size_t> take;
  for (size_t k = 0; k < S->queue.size(); ++k) {
    Ticket* t = S->queue[k];
    if (k > 0 && (t->exclusive || !compatible(t, head) || t->d != head->d)) continue;
    // a request of kAloneMin points or more fills the GPU by itself: it runs alone, and a
    // batch takes none (a batch that does not fit its memory fails after its enumeration)
    if (k > 0 && (head->n >= kAloneMin || t->n >= kAloneMin)) continue;
    if (k > 0 && ((int)take.size() >= S->max_batch || npts + t->n > S->max_points)) break;
    const uint64_t e =
        estimate(npts + t->n, nd + t->n * t->d, t->m, std::max(maxd, t->d), t->dtype,
                 ppp_of(S, head->d));
    if (total != 0 && 2 * e > free_mem && k > 0) break;
    if (total != 0 && e > free_mem) {
      if (k == 0 && !others_busy) {
        // the head cannot fit next to anything: run it alone with all free memory
        head->exclusive = true;
        batch.push_back(head);
        S->queue.pop_front();
        reservation = free_mem;
        return true;
      }
      if (k == 0) return false;  // wait for memory; nothing overtakes the head
      break;
    }
    npts += t->n;
    nd += t->n * t->d;
    maxd = std::max(maxd, t->d);
    est = e;
    take.push_back(k);
  }
  if (take.empty()) return false;
  for (size_t q : take) batch.push_back(S->queue[q]);
  for (auto it = take.rbegin(); it != take.rend(); ++it)
    S->queue.erase(S->queue.begin() + (std::ptrdiff_t)*it);
  // The estimate guesses the pairs (clustered points report hundreds of times more than
  // uniform ones), so a lane reserves an even share of the free memory among the lanes that
  // are idle now (itself included), and at least twice the estimate: a batch whose pair
  // buffer would not fit its reservation enumerates twice (count, then write).
  int idle = 0;
  for (int q = 0; q < (int)S->lanes.size(); ++q)
    if (q == li || !S->lanes[q].busy) ++idle;
  reservation = total == 0 ? 0 : std::min(free_mem, std::max(2 * est, free_mem / (uint64_t)idle));
  return true;
}

void finish(Ticket* t, rtg_status s, const std::string& err) {
  t->status = s;
  t->err = err;
  t->state = s == RTG_OK ? Ticket::kDone : Ticket::kFailed;
  t->t_done = Clock::now();
}

// Build the batch on lane L and hand out one CSR per request.  Returns the build status.
rtg_status run_batch(Server* S, Lane& L, std::vector<Ticket*>& batch, uint64_t reservation) {
  rtg_ctx* lc = L.ctx;
  rtg_ctx* owner = S->owner;
  std::lock_guard<std::mutex> g(lc->mu);
  lc->budget = reservation;
  const int B = (int)batch.size();
  std::vector<rtg_instance> items(B);
  std::vector<long long> offs(B + 1, 0);
  for (int b = 0; b < B; ++b) {
    Ticket* t = batch[b];
    items[b] = rtg_instance{t->pts.data(), t->n, t->d, t->r, t->c, t->T.data()};
    offs[b + 1] = offs[b] + t->n;
  }
  Request q{items.data(), B, batch[0]->m, batch[0]->dtype, 0, batch[0]->flags, false};
  rtg_csr blk{};
  cudaSetDevice(lc->device);
  {
    // the pairs per point every lane has seen for this d size the pair buffer of a new shape
    double ppp = 0.0;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      ppp = ppp_of(S, batch[0]->d);
    }
    lc->ppp_hint.raise(batch[0]->d, ppp);
  }
  rtg_status s = build(lc, q, &blk);
  if (s != RTG_OK) {
    release_out(lc, &blk);
    return s;
  }
  // the admission estimate of this batch against what the batch needed (the workspace its
  // build asked for and the block CSR): the slack of the estimate, reported with every result
  int64_t mem_est = 0, mem_peak = 0;
  {
    long long npts = 0, nd = 0;
    int maxd = 1;
    for (Ticket* t : batch) {
      npts += t->n;
      nd += t->n * t->d;
      maxd = std::max(maxd, t->d);
    }
    double ppp = 0.0;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      ppp = ppp_of(S, batch[0]->d);
    }
    mem_est = (int64_t)estimate(npts, nd, batch[0]->m, maxd, batch[0]->dtype, ppp);
    // what this batch needed: the workspace its build asked for and its block CSR
    mem_peak = (int64_t)lc->ws_need + (int64_t)(sizeof(int64_t) * (blk.n + 1)) +
               (int64_t)(sizeof(int32_t) * blk.nnz);
  }
  if (B == 1) {
    // a batch of one: its block CSR (from the owner's pool) is the request's CSR, handed to the
    // owner as it is (no copy, and never two copies in memory)
    size_t bytes = 0;
    {
      std::lock_guard<std::mutex> lk(lc->live_mu);
      auto it = lc->live.find(blk.handle);
      if (it != lc->live.end()) {
        bytes = it->second;
        lc->out_bytes -= bytes;
        lc->live.erase(it);
      }
    }
    {
      std::lock_guard<std::mutex> lk(owner->live_mu);
      owner->out_bytes += bytes;
    }
    blk.handle = register_out(owner, bytes);
    if (owner->budget && lc->ws_bytes > owner->budget / 4) trim_workspace(lc);
    Ticket* t = batch[0];
    t->result = blk;
    const auto now = Clock::now();
    t->result.stats.phase_us[0] =
        std::chrono::duration<double, std::micro>(t->t_start - t->t_submit).count();
    t->result.stats.phase_us[7] =
        std::chrono::duration<double, std::micro>(now - t->t_submit).count();
    t->result.stats.mem_estimate = mem_est;
    t->result.stats.mem_peak = mem_peak;
    return RTG_OK;
  }
  cudaStream_t st = lc->stream;
  // entry offsets of each request in the block-diagonal CSR
  void* dtmp = nullptr;
  const size_t tmp_bytes = sizeof(long long) * (2 * (size_t)B + 2) + sizeof(SplitItem) * B;
  s = alloc_out_on(lc, st, tmp_bytes, &dtmp);
  if (s != RTG_OK) {
    release_out(lc, &blk);
    return s;
  }
  long long* d_offs = (long long*)dtmp;
  long long* d_bases = d_offs + (B + 1);
  SplitItem* d_items = (SplitItem*)(d_bases + (B + 1));
  std::vector<long long> bases(B + 1, 0);
  cudaMemcpyAsync(d_offs, offs.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, st);
  k_gather_bases<<<(B + 1 + 255) / 256, 256, 0, st>>>((const long long*)blk.row_ptr, d_offs, B,
                                                     d_bases);
  cudaMemcpyAsync(bases.data(), d_bases, sizeof(long long) * (B + 1), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  std::vector<SplitItem> host_items(B);
  std::vector<rtg_csr> outs(B);
  for (int b = 0; b < B && e == cudaSuccess && s == RTG_OK; ++b) {
    const long long nnz = bases[b + 1] - bases[b];
    void *rp = nullptr, *cp = nullptr;
    const size_t rb = sizeof(int64_t) * (batch[b]->n + 1), cb = sizeof(int32_t) * nnz;
    // results are covered by the batch's reservation
    s = alloc_out_on(owner, st, rb, &rp);
    if (s == RTG_OK && cb) s = alloc_out_on(owner, st, cb, &cp);
    outs[b].n = batch[b]->n;
    outs[b].nnz = nnz;
    outs[b].row_ptr = (int64_t*)rp;
    outs[b].col = (int32_t*)cp;
    outs[b].symmetric = blk.symmetric;
    outs[b].handle = register_out(owner, rb + cb);
    outs[b].stats = blk.stats;
    host_items[b] = SplitItem{offs[b], batch[b]->n, bases[b], nnz, (long long*)rp, (int*)cp};
  }
  if (e == cudaSuccess && s == RTG_OK) {
    cudaMemcpyAsync(d_items, host_items.data(), sizeof(SplitItem) * B, cudaMemcpyHostToDevice, st);
    const int grid = 4 * lc->num_sms;
    k_split_rows<<<grid, 256, 0, st>>>((const long long*)blk.row_ptr, d_items, B, offs[B]);
    if (blk.nnz > 0)
      k_split_cols<<<grid, 256, 0, st>>>(blk.col, d_items, B, bases[B]);
    e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(dtmp, st);
  {
    std::lock_guard<std::mutex> lk(lc->live_mu);
    lc->out_bytes -= tmp_bytes;
  }
  release_out(lc, &blk);
  if (e != cudaSuccess) s = fail(lc, RTG_E_CUDA, std::string("split: ") + cudaGetErrorString(e));
  if (s != RTG_OK) {
    for (auto& o : outs) release_out(owner, &o);
    return s;
  }
  // a lane keeps its workspace for the next batch, unless it has grown past a quarter of the
  // budget (a large batch's pair buffer): then the memory goes back to the other lanes
  if (owner->budget && lc->ws_bytes > owner->budget / 4) trim_workspace(lc);
  const auto now = Clock::now();
  for (int b = 0; b < B; ++b) {
    Ticket* t = batch[b];
    t->result = outs[b];
    t->result.stats.phase_us[0] =
        std::chrono::duration<double, std::micro>(t->t_start - t->t_submit).count();
    t->result.stats.phase_us[7] =
        std::chrono::duration<double, std::micro>(now - t->t_submit).count();
    t->result.stats.mem_estimate = mem_est;
    t->result.stats.mem_peak = mem_peak;
  }
  return RTG_OK;
}

void lane_loop(Server* S, int li) {
  for (;;) {
    std::vector<Ticket*> batch;
    uint64_t reservation = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        if (!S->queue.empty() && try_form(S, li, batch, reservation)) break;
        S->cv.wait(lk);
      }
      Lane& L = S->lanes[li];
      L.busy = true;
      L.reservation = reservation;
      const auto now = Clock::now();
      for (Ticket* t : batch) {
        t->state = Ticket::kRunning;
        t->t_start = now;
      }
    }
    const auto t_run = Clock::now();
    const rtg_status s = run_batch(S, S->lanes[li], batch, reservation);
    if (S->log) {
      long long npts = 0;
      for (Ticket* t : batch) npts += t->n;
      std::fprintf(stderr, "serve lane %d: %zu requests, %lld points, d %d%s, %.3f ms, status %d\n",
                   li, batch.size(), npts, batch[0]->d, batch[0]->exclusive ? " (alone)" : "",
                   std::chrono::duration<double, std::milli>(Clock::now() - t_run).count(),
                   (int)s);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      Lane& L = S->lanes[li];
      L.busy = false;
      L.reservation = 0;
      const bool budget = s == RTG_E_BUDGET || s == RTG_E_NOMEM;
      if (s == RTG_OK) {
        long long npts = 0, pairs = 0;
        for (Ticket* t : batch) {  // (a result's stats are its batch's; its nnz is its own)
          npts += t->n;
          pairs += t->result.nnz / (t->result.symmetric ? 2 : 1);
        }
        if (npts > 0) S->ppp.put(batch[0]->d, (double)pairs / (double)npts);
        for (Ticket* t : batch) finish(t, RTG_OK, "");
      } else if (budget && (batch.size() > 1 || !batch[0]->exclusive)) {
        // retry each request alone with all free memory, keeping their order at the front
        for (auto it = batch.rbegin(); it != batch.rend(); ++it) {
          (*it)->exclusive = true;
          (*it)->state = Ticket::kQueued;
          S->queue.push_front(*it);
        }
      } else {
        for (Ticket* t : batch) finish(t, s, L.ctx->err);
      }
    }
    S->cv.notify_all();
  }
}

Server* get_server(rtg_ctx* c) {
  if (c->server) return c->server;
  Server* S = new Server();
  S->owner = c;
  if (const char* v = std::getenv("RTG_SERVE_LOG")) S->log = std::atoi(v) != 0;
  int lanes = 2;
  if (const char* v = std::getenv("RTG_SERVE_LANES")) lanes = std::max(1, std::min(8, std::atoi(v)));
  S->lanes.resize(lanes);
  for (int k = 0; k < lanes; ++k) {
    rtg_ctx* lc = nullptr;
    if (create_ctx(c->device, 0, nullptr, &lc) != RTG_OK) {
      for (int j = 0; j < k; ++j) destroy_ctx(S->lanes[j].ctx);
      delete S;
      return nullptr;
    }
    // the lane's CSRs come from the owner's pool, so that a result handed over as it is
    // (a batch of one) is the owner's memory like any other result
    if (lc->pool) cudaMemPoolDestroy(lc->pool);
    lc->pool = c->pool;
    lc->own_pool = false;
    S->lanes[k].ctx = lc;
  }
  for (int k = 0; k < lanes; ++k) S->lanes[k].th = std::thread(lane_loop, S, k);
  c->server = S;
  return S;
}

rtg_status take(rtg_ctx* c, Server* S, uint64_t ticket, rtg_csr* out, bool* pending) {
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) return fail(c, RTG_E_UNKNOWN_TICKET, "unknown ticket");
  Ticket* t = it->second;
  *pending = false;
  if (t->state == Ticket::kDone) {
    *out = t->result;
    S->tickets.erase(it);
    delete t;
    return RTG_OK;
  }
  if (t->state == Ticket::kFailed) {
    const rtg_status s = t->status;
    c->err = t->err;
    S->tickets.erase(it);
    delete t;
    return s;
  }
  *pending = true;
  return RTG_PENDING;
}

}  // namespace

void notify_server(rtg_ctx* c) {
  Server* S = c->server;
  if (!S) return;
  { std::lock_guard<std::mutex> lk(S->mu); }  // a lane between its check and its wait sees it
  S->cv.notify_all();
}

void stop_server(rtg_ctx* c) {
  Server* S = c->server;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (Lane& L : S->lanes)
    if (L.th.joinable()) L.th.join();
  for (Lane& L : S->lanes) destroy_ctx(L.ctx);
  for (auto& kv : S->tickets) {
    if (kv.second->state == Ticket::kDone) release_out(c, &kv.second->result);
    delete kv.second;
  }
  delete S;
  c->server = nullptr;
}

}  // namespace rtghost

using namespace rtghost;

extern "C" {

rtg_status rtg_submit(rtg_ctx* c, const rtg_request* req, uint64_t* ticket) {
  if (!c || !req || !ticket) return fail(c, RTG_E_INVALID, "NULL argument");
  *ticket = 0;
  rtg_status s = validate_common(req->dtype, req->n, req->d, req->r, req->cell_side, req->points);
  if (s == RTG_OK && (req->m < 1 || req->m > RTG_MAX_GRIDS))
    s = fail(nullptr, RTG_E_INVALID, "m must be in [1, 64]");
  if (s == RTG_OK) s = validate_transforms(req->transforms, req->d, req->m);
  if (s != RTG_OK) return fail(c, s, last_error_text());
  Ticket* t = new Ticket();
  const size_t esz = req->dtype == RTG_DTYPE_F64 ? 8 : 4;
  t->pts.assign((const unsigned char*)req->points,
                (const unsigned char*)req->points + (size_t)req->n * req->d * esz);
  t->T.assign(req->transforms, req->transforms + (size_t)req->m * (req->d * req->d + req->d));
  t->dtype = req->dtype;
  t->n = req->n;
  t->d = req->d;
  t->r = req->r;
  t->c = req->cell_side;
  t->m = req->m;
  t->flags = req->flags & RTG_FLAG_SYMMETRIC;
  t->t_submit = Clock::now();
  Server* S;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    S = get_server(c);
  }
  if (!S) {
    delete t;
    return fail(c, RTG_E_CUDA, "could not start the request server");
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    t->id = S->next++;
    S->tickets[t->id] = t;
    S->queue.push_back(t);
    *ticket = t->id;
  }
  S->cv.notify_all();
  return RTG_OK;
}

rtg_status rtg_poll(rtg_ctx* c, uint64_t ticket, rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL argument");
  Server* S = c->server;
  if (!S) return fail(c, RTG_E_UNKNOWN_TICKET, "unknown ticket");
  std::lock_guard<std::mutex> lk(S->mu);
  bool pending;
  return take(c, S, ticket, out, &pending);
}

rtg_status rtg_wait(rtg_ctx* c, uint64_t ticket, int64_t timeout_us, rtg_csr* out) {
  if (!c || !out) return fail(c, RTG_E_INVALID, "NULL argument");
  Server* S = c->server;
  if (!S) return fail(c, RTG_E_UNKNOWN_TICKET, "unknown ticket");
  std::unique_lock<std::mutex> lk(S->mu);
  auto done = [&] {
    auto it = S->tickets.find(ticket);
    return it == S->tickets.end() || it->second->state == Ticket::kDone ||
           it->second->state == Ticket::kFailed;
  };
  if (timeout_us < 0) S->cv.wait(lk, done);
  else S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  bool pending;
  const rtg_status s = take(c, S, ticket, out, &pending);
  if (pending) return fail(c, RTG_E_TIMEOUT, "the build is not finished");
  return s;
}

}  // extern "C"
