// Exact all-pairs r-NN (the problem of Sec. I of arXiv:1409.8112) with the distances taken
// from tensor-core tiles: d^2 = |x|^2 + |y|^2 - 2 x.y with x.y from tcgen05.mma (FP16 or BF16
// inputs, FP32 accumulation in tensor memory), and every pair whose FP32 d^2 lies within a
// band around fl(r^2) decided again with the FP64 reference sequence, so that the reported
// set is the same as the FP64 definition's.
//
// Each coordinate is centred on the bounding box and split as x = hi + lo (both half
// precision); x.y is approximated by hi.hi + hi.lo + lo.hi, three K = 16 MMAs per tile pair
// (d <= 16 padded with zeros).  Operands sit in shared memory in the K-major layout without
// swizzle: core matrices of 8 rows x 16 bytes, 128 bytes apart along K and 512 bytes apart
// along M or N.  A CTA of 4 warps owns a 128 x 128 FP32 accumulator (128 TMEM columns);
// warp w reads lanes 32w..32w+31.  The band is max(1e-3 r^2, E) where E bounds the error of
// the FP32 d^2: the hi/lo representation and dropped lo.lo term, FP32 accumulation of the
// 48 products, the norms, the epilogue and the centring (see tc_plan).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cfloat>

#include "rtg_internal.cuh"
#include "rtg_tc.cuh"

namespace rtg {

namespace {

constexpr int kTcRows = 128;
constexpr int kTcK = 32;                          // hi (16) + lo (16)
constexpr int kTcTileBytes = kTcRows * kTcK * 2;  // 8 KB per 128-point tile
constexpr int kTcThreads = 128;
// MMA completion waits: the context's spin limit times this (a commit takes far longer than
// one look-back step)
constexpr unsigned int kTcWaitScale = 16;

__device__ __forceinline__ double load_coord(const void* pts, int dtype, long long i, int d,
                                             int l) {
  return dtype == 0 ? __ldg((const double*)pts + i * d + l)
                    : (double)__ldg((const float*)pts + i * d + l);
}

// Band, thresholds and centre for instance 0 (one thread).
__global__ void k_tc_plan(const Inst* __restrict__ inst, const unsigned long long* bbox,
                          const InstPlan* __restrict__ iplan, TcPlan* tp, Status* st, int bf16) {
  const Inst I = inst[0];
  const int d = I.d;
  double M = 0.0;
  for (int l = 0; l < d; ++l) {
    const double hi = I.n > 0 ? dec_double(bbox[l * 2 + 0]) : 0.0;
    const double lo = I.n > 0 ? dec_double(~bbox[l * 2 + 1]) : 0.0;
    tp->center[l] = 0.5 * (lo + hi);
    M = fmax(M, 0.5 * (hi - lo) * (1.0 + 1e-12) + 1e-300);
  }
  for (int l = d; l < kMaxDim; ++l) tp->center[l] = 0.0;
  // Error bound of the FP32 d^2 (absolute), with u16 the unit roundoff of the half type:
  //   centring to FP32             8 sqrt(d) 2^-24 M (2 sqrt(d) M)
  //   hi/lo split + dropped lo.lo  2 d M^2 (2 u16^2 + 2^-22) + 2 d 2^-24 M   (x2 for -2x.y)
  //   FP32 accumulation of 48 terms 2 * 48 * 2^-24 * 2 d M^2, times 4 for an unknown order
  //   norms (two sums of d squares) 2 d 2^-24 d M^2
  //   epilogue (two roundings)      3 2^-24 (4 d M^2)
  const double E = tc_error_bound(M, d, bf16 != 0);
  const double rr = iplan[0].rr;
  const double band = fmax(1e-3 * rr, 1.25 * E);
  tp->band = band;
  tp->bound = E;
  st->tc_band = band;
  tp->lo = __double2float_rd(rr - band);
  tp->hi = __double2float_ru(rr + band);
}

// Half-precision hi/lo rows in the tile layout, and FP32 norms of the centred points.
template <bool BF16>
__global__ void __launch_bounds__(256) k_tc_prep(const Inst* __restrict__ inst, int dtype,
                                                 const TcPlan* __restrict__ tp,
                                                 unsigned char* __restrict__ tiles,
                                                 float* __restrict__ norms, long long n_pad) {
  const Inst I = inst[0];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  unsigned char* tile = tiles + (i / kTcRows) * (long long)kTcTileBytes;
  const int m = (int)(i % kTcRows);
  float nrm = 0.0f;
  for (int k = 0; k < 16; ++k) {
    float xc = 0.0f;
    if (i < I.n && k < I.d)
      xc = __double2float_rn(__dsub_rn(load_coord(I.pts, dtype, i, I.d, k), tp->center[k]));
    nrm = fmaf(xc, xc, nrm);
    if (BF16) {
      const __nv_bfloat16 h = __float2bfloat16_rn(xc);
      const __nv_bfloat16 l = __float2bfloat16_rn(xc - __bfloat162float(h));
      *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(m, k)) = h;
      *reinterpret_cast<__nv_bfloat16*>(tile + tile_off(m, 16 + k)) = l;
    } else {
      const __half h = __float2half_rn(xc);
      const __half l = __float2half_rn(xc - __half2float(h));
      *reinterpret_cast<__half*>(tile + tile_off(m, k)) = h;
      *reinterpret_cast<__half*>(tile + tile_off(m, 16 + k)) = l;
    }
  }
  norms[i] = nrm;
}

struct TcSink {
  unsigned int* row_cnt;
  unsigned long long* pair_buf;
  long long pair_cap;
  unsigned long long* emitted;
  int symmetric;
};

__device__ __noinline__ double exact_dist2(const void* pts, int dtype, long long i, long long j,
                                           int d) {
  double s = 0.0;
  for (int l = 0; l < d; ++l) {
    const double e = __dsub_rn(load_coord(pts, dtype, i, d, l), load_coord(pts, dtype, j, d, l));
    s = __fma_rn(e, e, s);
  }
  return s;
}

// A pair the tile did not reject: decided with the FP64 reference sequence (only rejections
// rely on the error bound); [lo, hi] is where the tile alone could not decide.
__device__ __noinline__ void tc_candidate(float d2, long long gi, long long gj, const Inst& I,
                                          const InstPlan& IP, int dtype, float lo_thr,
                                          const TcSink& sk, bool emit, unsigned int& pairs,
                                          unsigned int& rechecks, unsigned int& near_r,
                                          float& max_err, bool& overflow) {
  const double s = exact_dist2(I.pts, dtype, gi, gj, I.d);
  max_err = fmaxf(max_err, (float)fabs((double)d2 - s));
  if (d2 >= lo_thr) ++rechecks;
  if (fabs(__dsub_rn(__dsqrt_rn(s), I.r)) <= __dmul_rn(1e-12, I.r)) ++near_r;
  if (!(s <= IP.rr)) return;
  ++pairs;
  const unsigned int i = (unsigned int)(I.p0 + gi), j = (unsigned int)(I.p0 + gj);
  if (emit) {
    const unsigned long long slot = atomicAdd(sk.emitted, 1ull);
    if ((long long)slot < sk.pair_cap) sk.pair_buf[slot] = ((unsigned long long)i << 32) | j;
    else overflow = true;
  }
  atomicAdd(&sk.row_cnt[i], 1u);
  if (sk.symmetric) atomicAdd(&sk.row_cnt[j], 1u);
}

// Persistent: each CTA walks a contiguous range of tile pairs (bi <= bj) in bi-major order,
// so the A tile is reloaded only when bi changes.
template <bool BF16, bool EMIT>
__global__ void __launch_bounds__(kTcThreads) k_brute_tc(
    const unsigned char* __restrict__ tiles, const float* __restrict__ norms,
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const TcPlan* __restrict__ tp, int dtype, Status* st, TcSink sk, long long nt,
    unsigned int wait_limit, unsigned int inject) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sa = smem;                       // 8 KB
  unsigned char* sb = smem + kTcTileBytes;        // 8 KB
  float* na = reinterpret_cast<float*>(smem + 2 * kTcTileBytes);  // 128
  float* nb = na + kTcRows;                                         // 128
  __shared__ __align__(8) uint64_t mbar;
  __shared__ __align__(8) uint64_t mbar_idle;  // test hook: a barrier nothing arrives on
  __shared__ uint32_t tmem_base;
  __shared__ unsigned int s_cnt[4];
  __shared__ unsigned int s_err;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Inst I = inst[0];
  const InstPlan IP = iplan[0];
  const float lo_thr = tp->lo, hi_thr = tp->hi;
  const long long n = I.n;

  if (tid < 4) s_cnt[tid] = 0;
  if (tid == 0) {
    s_err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_idle)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) |
                         ((128u >> 3) << 17) | ((128u >> 4) << 24);

  const long long jobs = nt * (nt + 1) / 2;
  const long long per = (jobs + gridDim.x - 1) / gridDim.x;
  const long long j0 = (long long)blockIdx.x * per, j1 = min(jobs, j0 + per);
  // first (bi, bj) of this CTA: bi-major order over the upper triangle
  long long bi = 0, bj = 0;
  if (j0 < j1) {
    long long lo = 0, hi = nt - 1;
    while (lo < hi) {  // largest bi whose first job index is <= j0
      const long long mid = (lo + hi + 1) >> 1;
      if (mid * nt - mid * (mid - 1) / 2 <= j0) lo = mid; else hi = mid - 1;
    }
    bi = lo;
    bj = bi + (j0 - (bi * nt - bi * (bi - 1) / 2));
  }
  long long loaded_a = -1;
  uint32_t phase = 0;
  bool timed_out = false;
  unsigned int tl_pairs = 0, tl_rechecks = 0, tl_near = 0;
  bool overflow = false;
  float max_err = 0.0f;
  for (long long job = j0; job < j1 && !timed_out; ++job) {
    // stage the operand tiles (16-byte copies) and norms
    const uint4* gb = reinterpret_cast<const uint4*>(tiles + bj * (long long)kTcTileBytes);
    for (int x = tid; x < kTcTileBytes / 16; x += kTcThreads)
      reinterpret_cast<uint4*>(sb)[x] = __ldg(gb + x);
    nb[tid] = __ldg(norms + bj * kTcRows + tid);
    if (bi != loaded_a) {
      const uint4* ga = reinterpret_cast<const uint4*>(tiles + bi * (long long)kTcTileBytes);
      for (int x = tid; x < kTcTileBytes / 16; x += kTcThreads)
        reinterpret_cast<uint4*>(sa)[x] = __ldg(ga + x);
      na[tid] = __ldg(norms + bi * kTcRows + tid);
      loaded_a = bi;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      // hi.hi + hi.lo + lo.hi: A parts (0, 0, 1), B parts (0, 1, 0); 256 bytes per part
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
      const uint32_t asel[3] = {0u, 0u, 256u}, bsel[3] = {0u, 256u, 0u};
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const uint64_t ad = make_desc(a0 + asel[s]);
        const uint64_t bd = make_desc(b0 + bsel[s]);
        const uint32_t acc = s > 0 ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&mbar)));
    }
    // bounded wait for this job's MMAs (the test hook waits on a barrier nothing arrives on)
    const bool done = mbar_wait(
        (inject & kInjectTcWait) ? smem_u32(&mbar_idle) : smem_u32(&mbar), phase, wait_limit);
    if (!__syncthreads_and(done)) {
      // give up: wait (bounded again) for the MMAs in flight, so that the tensor memory they
      // write is not freed under them, then leave
      mbar_wait(smem_u32(&mbar), phase, wait_limit);
      if (tid == 0) atomicOr(&st->errors, kErrTimeout);
      timed_out = true;
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: row `row` of the tile against its 128 columns.  The fast path only builds a
    // mask of the columns the tile does not reject; those (rare) go to the exact check.
    const int row = warp * 32 + lane;
    const long long gi = bi * kTcRows + row;
    const float nrow = na[row];
#pragma unroll 1
    for (int c = 0; c < 128; c += 32) {
      uint32_t r[32];
      tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, r);
      const long long colbase = bj * kTcRows + c;
      // columns q with gi < colbase + q < n
      const long long qlo = gi - colbase + 1, qhi = n - colbase;
      uint32_t valid = 0;
      if (qlo < 32 && qhi > 0) {
        const int a0 = qlo > 0 ? (int)qlo : 0, a1 = qhi < 32 ? (int)qhi : 32;
        if (a1 > a0) valid = (a1 - a0 == 32 ? 0xffffffffu : ((1u << (a1 - a0)) - 1u)) << a0;
      }
      float d2v[32];
      uint32_t hits = 0;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        d2v[q] = (nrow + nb[c + q]) - 2.0f * __uint_as_float(r[q]);
        hits |= (d2v[q] > hi_thr ? 0u : 1u) << q;  // NaN (overflowed tiles) goes to FP64
      }
      hits &= valid;
      if (hits) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (hits & (1u << q))
            tc_candidate(d2v[q], gi, colbase + q, I, IP, dtype, lo_thr, sk, EMIT, tl_pairs,
                         tl_rechecks, tl_near, max_err, overflow);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();  // TMEM and shared tiles are reused by the next job
    if (++bj == nt) {
      ++bi;
      bj = bi;
    }
  }
  // tallies
  for (int o = 16; o > 0; o >>= 1) {
    tl_pairs += __shfl_xor_sync(0xffffffffu, tl_pairs, o);
    tl_rechecks += __shfl_xor_sync(0xffffffffu, tl_rechecks, o);
    tl_near += __shfl_xor_sync(0xffffffffu, tl_near, o);
    max_err = fmaxf(max_err, __shfl_xor_sync(0xffffffffu, max_err, o));
  }
  if (lane == 0) {
    atomicAdd(&s_cnt[0], tl_pairs);
    atomicAdd(&s_cnt[1], tl_rechecks);
    atomicAdd(&s_cnt[2], tl_near);
    atomicMax(&s_err, __float_as_uint(max_err));
  }
  if (__syncthreads_or(overflow) && tid == 0) atomicOr(&st->errors, kErrPairOverflow);
  if (tid == 0) {
    if (s_cnt[0]) atomicAdd(&st->pairs, (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&st->dist_rechecks, (unsigned long long)s_cnt[1]);
    if (s_cnt[2]) atomicAdd(&st->near_r, (unsigned long long)s_cnt[2]);
    atomicMax(&st->tc_max_err_bits, s_err);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

size_t tc_tiles_bytes(long long n) {
  const long long nt = (n + kTcRows - 1) / kTcRows;
  return (size_t)nt * kTcTileBytes;
}

int launch_brute_tc(const BuildArgs& a, bool bf16, Mode mode, unsigned char* tiles, float* norms,
                    TcPlan* tp, cudaStream_t s) {
  const long long n = a.n_total;
  const long long nt = (n + kTcRows - 1) / kTcRows;
  const long long n_pad = nt * kTcRows;
  k_tc_plan<<<1, 1, 0, s>>>(a.inst, a.bbox, a.iplan, tp, a.st, bf16 ? 1 : 0);
  if (bf16)
    k_tc_prep<true><<<(unsigned)((n_pad + 255) / 256), 256, 0, s>>>(a.inst, a.dtype, tp, tiles,
                                                                    norms, n_pad);
  else
    k_tc_prep<false><<<(unsigned)((n_pad + 255) / 256), 256, 0, s>>>(a.inst, a.dtype, tp, tiles,
                                                                     norms, n_pad);
  TcSink sk{a.row_cnt, a.pair_buf, a.pair_cap, &a.st->emitted, a.symmetric};
  // 4 CTAs per SM at most: 128 TMEM columns each fill the 512 columns of an SM.  The dynamic
  // shared memory (two tiles, norms, padding to 50 KB) enforces that occupancy.
  const size_t smem = 50 * 1024;
  const long long jobs = nt * (nt + 1) / 2;
  const unsigned grid = (unsigned)(jobs < 4LL * a.num_sms ? jobs : 4LL * a.num_sms);
  const bool emit = mode == kEmit;
#define RTG_TC_LAUNCH(B, E)                                                                    \
  do {                                                                                         \
    static size_t attr[64] = {};                                                               \
    int dev = 0;                                                                               \
    cudaGetDevice(&dev);                                                                       \
    if (dev < 0 || dev >= 64 || attr[dev] < smem) {                                            \
      cudaFuncSetAttribute(k_brute_tc<B, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                           (int)smem);                                                         \
      if (dev >= 0 && dev < 64) attr[dev] = smem;                                              \
    }                                                                                          \
    k_brute_tc<B, E><<<grid, kTcThreads, smem, s>>>(tiles, norms, a.inst, a.iplan, tp, a.dtype, \
                                                    a.st, sk, nt,                              \
                                                    spin_limit_of(a.spin_limit) * kTcWaitScale, \
                                                    a.inject);                                 \
  } while (0)
  if (grid > 0) {
    if (bf16 && emit) RTG_TC_LAUNCH(true, true);
    else if (bf16) RTG_TC_LAUNCH(true, false);
    else if (emit) RTG_TC_LAUNCH(false, true);
    else RTG_TC_LAUNCH(false, false);
  }
#undef RTG_TC_LAUNCH
  return grid > 0 ? 3 : 2;
}

}  // namespace rtg
