// Exact pair count for callers that cannot allocate device memory.
//
// A motion-planning control loop that runs under a fixed memory plan or a hard latency
// budget, or a plug-in that lives inside a host application which owns every device
// allocation, cannot call cudaMalloc (nor create an rtg_ctx, which allocates).  For them,
// rtg_brute_count_noalloc counts the pairs at distance <= r with the same kernels as
// rtg_brute_force, but its scratch (status counters, plan, FP32 point rows, row counts) is one
// file-scope device array of fixed size, held by every GPU that loads the library until the
// process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "rtg.h"
#include "rtg_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxPoints = 65536;
constexpr size_t kStatusBytes = (sizeof(rtg::Status) + 255) & ~size_t(255);
constexpr size_t kInstBytes = (sizeof(rtg::Inst) + 255) & ~size_t(255);
constexpr size_t kIPlanBytes = (sizeof(rtg::InstPlan) + 255) & ~size_t(255);
constexpr size_t kBoxBytes = rtg::kMaxDim * 2 * 8;
constexpr size_t kRowsBytes = (size_t)kNoAllocMaxPoints * rtg::kMaxDim * 4;  // FP32 rows, dpad <= 16
constexpr size_t kCountBytes = (size_t)kNoAllocMaxPoints * 4;
constexpr size_t kScratchBytes =
    kStatusBytes + kInstBytes + kIPlanBytes + kBoxBytes + kRowsBytes + kCountBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// the message is readable with rtg_last_error(NULL)
rtg_status fail(rtg_status s, const char* msg) {
  rtg::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" rtg_status rtg_brute_count_noalloc(const void* points, int dtype, int64_t n, int d,
                                              double r, void* stream, uint64_t* count) {
  if (!count) return fail(RTG_E_INVALID, "count is NULL");
  if (dtype != RTG_DTYPE_F64 && dtype != RTG_DTYPE_F32) return fail(RTG_E_INVALID, "bad dtype");
  if (n < 0 || n > kNoAllocMaxPoints)
    return fail(RTG_E_INVALID, "n exceeds the 65536-point limit of the static scratch");
  if (d < 1 || d > RTG_MAX_DIM) return fail(RTG_E_INVALID, "d must be in [1, 16]");
  if (!(r > 0.0) || !std::isfinite(r)) return fail(RTG_E_INVALID, "r must be > 0 and finite");
  if (n > 0 && !points) return fail(RTG_E_INVALID, "points is NULL");
  *count = 0;
  if (n < 2) return RTG_OK;
  {
    // the call synchronises its stream and reads the count back, neither of which a stream
    // capture allows
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone)
      return fail(RTG_E_INVALID, "rtg_brute_count_noalloc cannot run inside a stream capture");
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(RTG_E_CUDA, "no current CUDA device");
  void* base = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return fail(RTG_E_CUDA, cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(RTG_E_CUDA, "cudaDeviceGetAttribute failed");
  cudaStream_t s = (cudaStream_t)stream;

  char* p = (char*)base;
  rtg::BuildArgs a{};
  a.B = 1;
  a.m = 0;
  a.dtype = dtype;
  a.dpad = rtg::dpad_for(d);
  a.n_total = n;
  a.blocks = (n + rtg::kPointBlock - 1) / rtg::kPointBlock;
  a.prep_points = rtg::kPrepPoints;
  a.pblocks = (n + rtg::kPrepPoints - 1) / rtg::kPrepPoints;
  a.st = (rtg::Status*)p;
  a.inst = (const rtg::Inst*)(p + kStatusBytes);
  a.iplan = (rtg::InstPlan*)(p + kStatusBytes + kInstBytes);
  a.bbox = (unsigned long long*)(p + kStatusBytes + kInstBytes + kIPlanBytes);
  a.pf = (float*)(p + kStatusBytes + kInstBytes + kIPlanBytes + kBoxBytes);
  a.row_cnt = (unsigned int*)(p + kStatusBytes + kInstBytes + kIPlanBytes + kBoxBytes + kRowsBytes);
  a.num_sms = sms;
  rtg::Inst I{};
  I.pts = points;
  I.n = (int)n;
  I.d = d;
  I.r = r;
  I.c = 1.0;
  I.inv_c = 1.0;
  I.inv_cf = 1.0f;
  // the counters and the bounding box must start at zero; the instance record is copied in;
  // the plan and the point rows are fully rewritten, and the row counts are zeroed by the
  // prep kernel and then only incremented (the count itself comes from Status.pairs)
  if (cudaMemsetAsync(a.st, 0, sizeof(rtg::Status), s) != cudaSuccess ||
      cudaMemsetAsync(a.bbox, 0, kBoxBytes, s) != cudaSuccess ||
      cudaMemcpyAsync((void*)a.inst, &I, sizeof(I), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(RTG_E_CUDA, "scratch set-up failed");
  rtg::launch_prep_plan(a, s);
  rtg::launch_brute(a, rtg::kCount, s);
  {
    // a launch that failed without a sticky error would otherwise leave Status at zero and
    // report a count of 0
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return fail(RTG_E_CUDA, cudaGetErrorString(le));
  }
  rtg::Status h;
  std::memset(&h, 0, sizeof(h));
  cudaError_t e = cudaMemcpyAsync(&h, a.st, sizeof(rtg::Status), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(RTG_E_CUDA, cudaGetErrorString(e));
  if (h.errors & rtg::kErrNonFinite) return fail(RTG_E_INVALID, "non-finite point coordinate");
  if (h.errors & rtg::kErrTimeout) return fail(RTG_E_TIMEOUT, "a bounded device wait ran out");
  if (h.errors) return fail(RTG_E_INTERNAL, "device error flags set");
  *count = h.pairs;
  return RTG_OK;
}
