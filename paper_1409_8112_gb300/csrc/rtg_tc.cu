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
#include <type_traits>

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
                          const InstPlan* __restrict__ iplan, TcPlan* tp, Status* st, int bf16,
                          int fold) {
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
  const double E = fold ? tc_error_bound_folded(M, d, bf16 != 0) : tc_error_bound(M, d, bf16 != 0);
  const double rr = iplan[0].rr;
  const double band = fmax(1e-3 * rr, 1.25 * E);
  tp->band = band;
  tp->bound = E;
  st->tc_band = band;
  tp->lo = __double2float_rd(rr - band);
  tp->hi = __double2float_ru(rr + band);
}

// Half-precision hi/lo rows in the tile layout, and FP32 norms of the centred points.  FOLD
// (d <= 12): the tiles come in two versions, the A operand's ([-2 x, |x|^2 hi, |x|^2 lo, 1, 1]
// in the hi block) and the B operand's ([x, 1, 1, |y|^2 hi, |y|^2 lo]), so that the MMAs
// accumulate |x|^2 + |y|^2 - 2 x.y; the norms array is then not read.
template <bool BF16, bool FOLD>
__global__ void __launch_bounds__(256) k_tc_prep(const Inst* __restrict__ inst, int dtype,
                                                 const TcPlan* __restrict__ tp,
                                                 unsigned char* __restrict__ tiles,
                                                 float* __restrict__ norms, long long n_pad) {
  using H = typename std::conditional<BF16, __nv_bfloat16, __half>::type;
  auto to_h = [](float v) -> H {
    if constexpr (BF16) return __float2bfloat16_rn(v); else return __float2half_rn(v);
  };
  auto to_f = [](H v) -> float {
    if constexpr (BF16) return __bfloat162float(v); else return __half2float(v);
  };
  const Inst I = inst[0];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const long long ntile = n_pad / kTcRows;
  unsigned char* tile = tiles + (i / kTcRows) * (long long)kTcTileBytes;
  unsigned char* tileB = FOLD ? tile + ntile * (long long)kTcTileBytes : tile;
  const int m = (int)(i % kTcRows);
  float nrm = 0.0f;
  for (int k = 0; k < 16; ++k) {
    float xc = 0.0f;
    if (i < I.n && k < I.d)
      xc = __double2float_rn(__dsub_rn(load_coord(I.pts, dtype, i, I.d, k), tp->center[k]));
    nrm = fmaf(xc, xc, nrm);
    const H h = to_h(xc);
    const H l = to_h(xc - to_f(h));
    // A version: -2 x (exact scaling by a power of two)
    *reinterpret_cast<H*>(tile + tile_off(m, k)) = FOLD ? to_h(-2.0f * to_f(h)) : h;
    *reinterpret_cast<H*>(tile + tile_off(m, 16 + k)) = FOLD ? to_h(-2.0f * to_f(l)) : l;
    if (FOLD) {
      *reinterpret_cast<H*>(tileB + tile_off(m, k)) = h;
      *reinterpret_cast<H*>(tileB + tile_off(m, 16 + k)) = l;
    }
  }
  if (FOLD) {
    const int d = I.d;  // slots d .. d + 3 of the hi block are free (d <= 12)
    const H nh = to_h(nrm), nl = to_h(nrm - to_f(nh)), one = to_h(1.0f);
    *reinterpret_cast<H*>(tile + tile_off(m, d)) = nh;
    *reinterpret_cast<H*>(tile + tile_off(m, d + 1)) = nl;
    *reinterpret_cast<H*>(tile + tile_off(m, d + 2)) = one;
    *reinterpret_cast<H*>(tile + tile_off(m, d + 3)) = one;
    *reinterpret_cast<H*>(tileB + tile_off(m, d)) = one;
    *reinterpret_cast<H*>(tileB + tile_off(m, d + 1)) = one;
    *reinterpret_cast<H*>(tileB + tile_off(m, d + 2)) = nh;
    *reinterpret_cast<H*>(tileB + tile_off(m, d + 3)) = nl;
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

// Candidates queued per warp before their exact check.  A chunk with more candidates than this
// (dense inputs: up to 32 x 32) is decided by its lanes directly.
constexpr int kTcQueue = 256 + 32;

// Decides the qn queued candidates of a warp, 32 at a time (one per lane).  Called by all lanes.
__device__ __forceinline__ void tc_drain(const unsigned int* q_i, const unsigned int* q_j,
                                         const float* q_d, unsigned int qn, int lane,
                                         const Inst& I, const InstPlan& IP, int dtype,
                                         float lo_thr, const TcSink& sk, bool emit,
                                         unsigned int& pairs, unsigned int& rechecks,
                                         unsigned int& near_r, float& max_err, bool& overflow) {
  __syncwarp();
  for (unsigned int b = 0; b < qn; b += 32) {
    const unsigned int e = b + lane;
    if (e < qn)
      tc_candidate(q_d[e], (long long)q_i[e], (long long)q_j[e], I, IP, dtype, lo_thr, sk, emit,
                   pairs, rechecks, near_r, max_err, overflow);
  }
  __syncwarp();
}

// Persistent: each CTA walks a contiguous range of tile pairs (bi <= bj) in bi-major order,
// so the A tile is reloaded only when bi changes.
template <bool BF16, bool EMIT, bool FOLD>
__global__ void __launch_bounds__(kTcThreads) k_brute_tc(
    const unsigned char* __restrict__ tiles, const float* __restrict__ norms,
    const Inst* __restrict__ inst, const InstPlan* __restrict__ iplan,
    const TcPlan* __restrict__ tp, int dtype, Status* st, TcSink sk, long long nt,
    unsigned int wait_limit, unsigned int inject) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // double-buffered operand tiles and norms: the next job's are copied in while this job's
  // MMAs and epilogue run
  unsigned char* sa2 = smem;                                         // 2 x 8 KB
  unsigned char* sb2 = smem + 2 * kTcTileBytes;                      // 2 x 8 KB
  float* na2 = reinterpret_cast<float*>(smem + 4 * kTcTileBytes);   // 2 x 128
  float* nb2 = na2 + 2 * kTcRows;                                    // 2 x 128
  const float* nb = nullptr;  // this job's column norms
  // per warp: the candidate queue (rows, columns, tile d^2), after the norms
  unsigned int* q_i = reinterpret_cast<unsigned int*>(nb2 + 2 * kTcRows) +
                      (size_t)(threadIdx.x >> 5) * 3 * kTcQueue;
  unsigned int* q_j = q_i + kTcQueue;
  float* q_d = reinterpret_cast<float*>(q_j + kTcQueue);
  unsigned int qn = 0;  // entries queued (warp-uniform)
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
  uint32_t phase = 0;
  bool timed_out = false;
  unsigned int tl_pairs = 0, tl_rechecks = 0, tl_near = 0;
  bool overflow = false;
  float max_err = 0.0f;
  // asynchronous copy of tile t and its norms into buffer `buf` of a side (16-byte copies)
  // (FOLD: the B operand's tiles follow the A operand's, and the norms are in the tiles)
  const unsigned char* tilesB = FOLD ? tiles + nt * (long long)kTcTileBytes : tiles;
  auto stage = [&](const unsigned char* src, unsigned char* side, float* nside, long long t,
                   int buf) {
    const unsigned char* g = src + t * (long long)kTcTileBytes;
    unsigned char* dst = side + buf * kTcTileBytes;
    for (int x = tid; x < kTcTileBytes / 16; x += kTcThreads) cp_async16(dst + 16 * x, g + 16 * x);
    if (!FOLD) cp_async_small<4>(nside + buf * kTcRows + tid, norms + t * kTcRows + tid);
  };
  int abuf = 0, bbuf = 0;
  if (j0 < j1) {
    stage(tiles, sa2, na2, bi, 0);
    stage(tilesB, sb2, nb2, bj, 0);
  }
  for (long long job = j0; job < j1 && !timed_out; ++job) {
    cp_async_wait_all();  // this job's tiles (copied during the previous job) have landed
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    unsigned char* sa = sa2 + abuf * kTcTileBytes;
    unsigned char* sb = sb2 + bbuf * kTcTileBytes;
    const float* na = na2 + abuf * kTcRows;
    nb = nb2 + bbuf * kTcRows;
    // the next job's tiles go to the other buffers while this job runs
    long long ni = bi, nj = bj + 1;
    if (nj == nt) {
      ++ni;
      nj = ni;
    }
    const bool more = job + 1 < j1;
    const bool new_a = ni != bi;
    if (more) {
      if (new_a) stage(tiles, sa2, na2, ni, abuf ^ 1);
      stage(tilesB, sb2, nb2, nj, bbuf ^ 1);
    }
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
        d2v[q] = FOLD ? __uint_as_float(r[q])
                      : (nrow + nb[c + q]) - 2.0f * __uint_as_float(r[q]);
        hits |= (d2v[q] > hi_thr ? 0u : 1u) << q;  // NaN (overflowed tiles) goes to FP64
      }
      hits &= valid;
      // queue this chunk's candidates (the warp's shared-memory queue, kept across jobs) and
      // decide them 32 at a time, one per lane, so that the FP64 checks and their global
      // loads run in parallel instead of one lane at a time
      const unsigned int nh = (unsigned int)__popc(hits);
      unsigned int incl = nh;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
      if (total > (unsigned int)kTcQueue) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (hits & (1u << q))
            tc_candidate(d2v[q], gi, colbase + q, I, IP, dtype, lo_thr, sk, EMIT, tl_pairs,
                         tl_rechecks, tl_near, max_err, overflow);
      } else if (total) {
        if (qn + total > (unsigned int)kTcQueue) {  // room for the chunk: decide the queue first
          tc_drain(q_i, q_j, q_d, qn, lane, I, IP, dtype, lo_thr, sk, EMIT, tl_pairs,
                   tl_rechecks, tl_near, max_err, overflow);
          qn = 0;
        }
        unsigned int pos = qn + incl - nh;
        if (hits) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            if (hits & (1u << q)) {
              q_i[pos] = (unsigned int)gi;
              q_j[pos] = (unsigned int)(colbase + q);
              q_d[pos] = d2v[q];
              ++pos;
            }
        }
        qn += total;
        __syncwarp();
        while (qn >= 32) {  // the newest 32 entries, one per lane
          const unsigned int e = qn - 32 + lane;
          tc_candidate(q_d[e], (long long)q_i[e], (long long)q_j[e], I, IP, dtype, lo_thr, sk,
                       EMIT, tl_pairs, tl_rechecks, tl_near, max_err, overflow);
          qn -= 32;
          __syncwarp();
        }
      }
            }
    asm volatile("tcgen05.fence::before_thread_sync;");
    // (the barrier at the top of the next job separates this epilogue from its MMAs)
    bi = ni;
    bj = nj;
    if (new_a) abuf ^= 1;
    bbuf ^= 1;
  }
  cp_async_wait_all();  // no copy of this block is left in flight
  if (qn)  // the candidates still queued
    tc_drain(q_i, q_j, q_d, qn, lane, I, IP, dtype, lo_thr, sk, EMIT, tl_pairs, tl_rechecks,
             tl_near, max_err, overflow);
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
  return 2 * (size_t)nt * kTcTileBytes;  // A and B versions (norms folded into the MMA)
}

int launch_brute_tc(const BuildArgs& a, bool bf16, Mode mode, unsigned char* tiles, float* norms,
                    TcPlan* tp, cudaStream_t s) {
  const long long n = a.n_total;
  const long long nt = (n + kTcRows - 1) / kTcRows;
  const long long n_pad = nt * kTcRows;
  // the norms ride in the MMA when 4 slots of the K = 16 hi block are free (d <= 12)
  const bool fold = a.dpad <= 16 && a.d_common >= 1 && a.d_common <= 12;
  k_tc_plan<<<1, 1, 0, s>>>(a.inst, a.bbox, a.iplan, tp, a.st, bf16 ? 1 : 0, fold ? 1 : 0);
  const unsigned pblocks = (unsigned)((n_pad + 255) / 256);
  if (bf16 && fold)
    k_tc_prep<true, true><<<pblocks, 256, 0, s>>>(a.inst, a.dtype, tp, tiles, norms, n_pad);
  else if (bf16)
    k_tc_prep<true, false><<<pblocks, 256, 0, s>>>(a.inst, a.dtype, tp, tiles, norms, n_pad);
  else if (fold)
    k_tc_prep<false, true><<<pblocks, 256, 0, s>>>(a.inst, a.dtype, tp, tiles, norms, n_pad);
  else
    k_tc_prep<false, false><<<pblocks, 256, 0, s>>>(a.inst, a.dtype, tp, tiles, norms, n_pad);
  TcSink sk{a.row_cnt, a.pair_buf, a.pair_cap, &a.st->emitted, a.symmetric};
  // 4 CTAs per SM at most: 128 TMEM columns each fill the 512 columns of an SM.  The dynamic
  // shared memory (two tiles, norms, the warps' candidate queues, padding to 50 KB) enforces
  // that occupancy.
  const size_t smem = 50 * 1024;
  const long long jobs = nt * (nt + 1) / 2;
  const unsigned grid = (unsigned)(jobs < 4LL * a.num_sms ? jobs : 4LL * a.num_sms);
  const bool emit = mode == kEmit;
#define RTG_TC_LAUNCH1(B, E, F)                                                                \
  do {                                                                                         \
    static size_t attr[64] = {};                                                               \
    int dev = 0;                                                                               \
    cudaGetDevice(&dev);                                                                       \
    if (dev < 0 || dev >= 64 || attr[dev] < smem) {                                            \
      cudaFuncSetAttribute(k_brute_tc<B, E, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                           (int)smem);                                                         \
      if (dev >= 0 && dev < 64) attr[dev] = smem;                                              \
    }                                                                                          \
    k_brute_tc<B, E, F><<<grid, kTcThreads, smem, s>>>(tiles, norms, a.inst, a.iplan, tp,       \
                                                       a.dtype,                                \
                                                    a.st, sk, nt,                              \
                                                    spin_limit_of(a.spin_limit) * kTcWaitScale, \
                                                    a.inject);                                 \
  } while (0)
#define RTG_TC_LAUNCH(B, E)             \
  do {                                   \
    if (fold) RTG_TC_LAUNCH1(B, E, true); \
    else RTG_TC_LAUNCH1(B, E, false);     \
  } while (0)
  if (grid > 0) {
    if (bf16 && emit) RTG_TC_LAUNCH(true, true);
    else if (bf16) RTG_TC_LAUNCH(true, false);
    else if (emit) RTG_TC_LAUNCH(false, true);
    else RTG_TC_LAUNCH(false, false);
  }
#undef RTG_TC_LAUNCH
#undef RTG_TC_LAUNCH1
  return grid > 0 ? 3 : 2;
}

}  // namespace rtg
