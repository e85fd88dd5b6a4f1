// Multiple r-nearest-neighbour queries (Sec. II of arXiv:1409.8112): the neighbours of a subset
// of the input points, answered from a stored pair set that holds every pair twice (the
// symmetric CSR of Sec. III-B).  Row k of the answer is the neighbour list of query k.
//
// Three kernels: per-query degrees, their exclusive scan (the pair kernels' row scan), and one
// warp per query copying its neighbour list (already ascending) into place.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "rtg_host.h"

namespace rtg {

namespace {

__global__ void __launch_bounds__(256) k_query_count(const long long* __restrict__ row_ptr,
                                                     long long n, const int* __restrict__ q,
                                                     long long nq, unsigned int* cnt,
                                                     unsigned int* errors) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nq;
       k += (long long)gridDim.x * blockDim.x) {
    const int v = q[k];
    if (v < 0 || v >= n) {
      cnt[k] = 0u;
      atomicOr(errors, kErrQueryRange);
    } else {
      cnt[k] = (unsigned int)(row_ptr[v + 1] - row_ptr[v]);
    }
  }
}

__global__ void __launch_bounds__(256) k_query_copy(const long long* __restrict__ row_ptr,
                                                    const int* __restrict__ col,
                                                    const int* __restrict__ q, long long nq,
                                                    const OutSlot* out) {
  const long long* __restrict__ out_ptr = out->row_ptr;
  int* out_col = out->col;
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long k = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); k < nq;
       k += warps) {
    const int v = q[k];
    const long long b = row_ptr[v], len = row_ptr[v + 1] - b, o = out_ptr[k];
    for (long long x = lane; x < len; x += 32) out_col[o + x] = col[b + x];
  }
}

}  // namespace

}  // namespace rtg

namespace rtghost {

rtg_status query_neighbors(rtg_ctx* c, const rtg_csr* g, const int32_t* queries, int64_t nq,
                           int queries_on_device, rtg_csr* out) {
  const cudaStream_t st = c->stream;
  std::memset(out, 0, sizeof(*out));
  rtg_status s;
  auto cuda = [&](cudaError_t e, const char* what) -> rtg_status {
    if (e == cudaSuccess) return RTG_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? RTG_E_NOMEM : RTG_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
  void* rp = nullptr;
  if ((s = alloc_out_on(c, st, sizeof(int64_t) * (size_t)(nq + 1), &rp)) != RTG_OK) return s;
  out->row_ptr = (int64_t*)rp;
  out->handle = register_out(c, sizeof(int64_t) * (size_t)(nq + 1));
  out->n = nq;
  if (nq == 0) {
    if ((s = cuda(cudaMemsetAsync(rp, 0, sizeof(int64_t), st), "cudaMemsetAsync")) != RTG_OK ||
        (s = cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    return RTG_OK;
  }
  const size_t stat_bytes = (sizeof(rtg::Status) + 255) & ~size_t(255);
  if ((s = ensure(c, c->status, stat_bytes)) != RTG_OK ||
      (s = ensure(c, c->row_cnt, (size_t)nq * 4)) != RTG_OK ||
      (s = ensure(c, c->scan_lb, ((size_t)nq / 4096 + 2) * 8)) != RTG_OK ||
      (s = ensure(c, c->out_slot, sizeof(rtg::OutSlot))) != RTG_OK ||
      (!queries_on_device && (s = ensure(c, c->q_idx, (size_t)nq * 4)) != RTG_OK)) {
    release_out(c, out);
    return s;
  }
  const int* q = queries;
  if (!queries_on_device) {
    if ((s = cuda(cudaMemcpyAsync(c->q_idx.p, queries, (size_t)nq * 4, cudaMemcpyHostToDevice, st),
                  "cudaMemcpyAsync")) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    q = (const int*)c->q_idx.p;
  }
  rtg::BuildArgs a{};
  a.st = (rtg::Status*)c->status.p;
  a.row_cnt = (unsigned int*)c->row_cnt.p;
  a.scan_lookback = (unsigned long long*)c->scan_lb.p;
  a.out = (const rtg::OutSlot*)c->out_slot.p;
  a.n_total = nq;
  a.num_sms = c->num_sms;
  c->h_slot->row_ptr = (long long*)rp;
  c->h_slot->col = nullptr;
  c->h_slot->col_cap = 0;
  long long blocks = (nq + 255) / 256;
  if (blocks > 8LL * c->num_sms) blocks = 8LL * c->num_sms;
  cudaMemsetAsync(a.st, 0, sizeof(rtg::Status), st);
  cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice, st);
  rtg::k_query_count<<<(unsigned)blocks, 256, 0, st>>>((const long long*)g->row_ptr, g->n, q, nq,
                                                       a.row_cnt, &a.st->errors);
  rtg::launch_scan(a, st);
  if ((s = cuda(cudaGetLastError(), "query launch")) != RTG_OK ||
      (s = read_status(c)) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  if (c->h_status->errors & rtg::kErrQueryRange) {
    release_out(c, out);
    return fail(c, RTG_E_INVALID, "a query index is outside [0, n) of the graph");
  }
  if ((s = check_errors(c, ~0u)) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  const long long nnz = (long long)c->h_status->nnz;
  if (nnz > 0) {
    void* cp = nullptr;
    if ((s = alloc_out_on(c, st, sizeof(int32_t) * (size_t)nnz, &cp)) != RTG_OK) {
      release_out(c, out);
      return s;
    }
    out->col = (int32_t*)cp;
    {
      std::lock_guard<std::mutex> lk(c->live_mu);
      c->live[out->handle] += sizeof(int32_t) * (size_t)nnz;
    }
    c->h_slot->col = (int*)cp;
    c->h_slot->col_cap = nnz;
    cudaMemcpyAsync(c->out_slot.p, c->h_slot, sizeof(rtg::OutSlot), cudaMemcpyHostToDevice, st);
    long long wblocks = (nq + 7) / 8;
    if (wblocks > 16LL * c->num_sms) wblocks = 16LL * c->num_sms;
    rtg::k_query_copy<<<(unsigned)wblocks, 256, 0, st>>>((const long long*)g->row_ptr,
                                                         (const int*)g->col, q, nq, a.out);
  }
  if ((s = cuda(cudaGetLastError(), "query copy")) != RTG_OK ||
      (s = cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize")) != RTG_OK) {
    release_out(c, out);
    return s;
  }
  out->nnz = nnz;
  out->symmetric = 0;
  return RTG_OK;
}

}  // namespace rtghost
