// Point preparation, per-build plan and the transform+key kernel (the point-to-cell step of
// Alg. 1 of arXiv:1409.8112, for the rotated + shifted grids of Sec. III), for a batch of
// instances.
//
// The cell index of a point in grid t is q_k = floor(y_k / c) with y = R_t p + s_t, where the
// reference value is the FP64 fma chain acc = s_k; acc = fma(R[k][l], p_l, acc) followed by an
// IEEE division.  GB300 runs FP64 at about 1/60 of its FP32 rate, so the kernel evaluates the
// same expression in FP32 and proves, per coordinate, that floor() of the FP64 value equals
// floor() of the FP32 estimate: with A = |s_k| + sum_l |R_kl| max|p_l| the FP32 estimate of
// y_k / c is within E = (d + 6) 2^-24 A / c of the FP64 quotient (rounding of R, s and p to
// FP32, d rounded fmas, the rounded reciprocal and product; the FP64 chain's own error is
// below 2^-29 of that).  When [u - E, u + E] holds no integer the FP32 floor is exact;
// otherwise the coordinate is recomputed with the FP64 sequence.  E is widened by 3e-12 / c
// so every coordinate within 1e-12 of a wall takes the FP64 path, where it is counted.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "rtg_internal.cuh"

namespace rtg {

namespace {

__device__ __forceinline__ double load_coord(const void* pts, int dtype, long long i, int d,
                                             int l) {
  return dtype == 0 ? __ldg((const double*)pts + i * d + l)
                    : (double)__ldg((const float*)pts + i * d + l);
}

// Instance owning block `blk` of a per-point kernel (first-block offsets ascending): binary
// search by one thread, broadcast through shared memory.
template <bool PREP>
__device__ __forceinline__ int block_instance(const Inst* inst, int B, long long blk,
                                              int* s_b) {
  if (threadIdx.x == 0) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((PREP ? inst[mid].pblk0 : inst[mid].blk0) <= blk) lo = mid; else hi = mid - 1;
    }
    *s_b = lo;
  }
  __syncthreads();
  return *s_b;
}

__device__ void plan_axis_item(long long idx, const Inst* __restrict__ inst, int m, int dtype,
                               const double* __restrict__ T64, const unsigned long long* bbox,
                               InstPlan* iplan, GridPlan* gplan);
__device__ void plan_ranges_block(const Inst* __restrict__ inst, int B, int m, GridPlan* gplan,
                                  unsigned long long* bases, Status* st, int passes,
                                  int radix_bits, int key64, int cell_major);

// Plan arguments for the prep kernel's last block (small batches plan there, saving two
// launches on the build's critical path).
struct PlanArgs {
  int fuse;    // 1: the last block to finish runs the plan
  int points;  // points per block (a multiple of the block size)
  int m;
  const double* T64;
  InstPlan* iplan;
  GridPlan* gplan;
  unsigned long long* bases;
  int passes, radix_bits, key64;
  int cell_major;  // the sort keys are cell indices alone (the pass check uses their width)
};

// FP32 rows of the points, zeroed row counters and the per-instance bounding box;
// pa.points points per block (one or four per thread), so that each block adds one bound per
// axis.
template <int DPAD>
__global__ void __launch_bounds__(kPrepThreads) k_prep(const Inst* __restrict__ inst, int B,
                                                       int dtype, float* __restrict__ pf,
                                                       unsigned int* __restrict__ row_cnt,
                                                       unsigned long long* bbox, Status* st,
                                                       PlanArgs pa) {
  // The bounding box only has to contain every coordinate: it is kept in FP32, each value
  // widened by one ulp (the FP32 row is the FP64 value rounded to nearest), so that no FP64
  // arithmetic runs here.  Finiteness of FP64 input is tested on the exponent bits.  A finite
  // FP64 value beyond the FP32 range has an infinite FP32 row entry and goes into the box as
  // the FP64 value itself; the plan's bounds (cell index, distance band) then become infinite
  // or non-finite for its instance, which sends every decision of that instance to the FP64
  // sequences.
  __shared__ int s_b;
  __shared__ float smn[kPrepThreads / 32][DPAD], smx[kPrepThreads / 32][DPAD];
  const int b = block_instance<true>(inst, B, blockIdx.x, &s_b);
  const Inst I = inst[b];
  const int d = I.d;
  float mn[DPAD], mx[DPAD];
  bool bad = false;
#pragma unroll
  for (int l = 0; l < DPAD; ++l) {
    mn[l] = FLT_MAX;
    mx[l] = -FLT_MAX;
  }
  const long long base = (blockIdx.x - I.pblk0) * (long long)pa.points;
  for (int q = 0; q < pa.points / kPrepThreads; ++q) {
    const long long i = base + q * kPrepThreads + threadIdx.x;
    if (i >= I.n) break;
    float row[DPAD];
#pragma unroll
    for (int l = 0; l < DPAD; ++l) {
      row[l] = 0.0f;
      if (l < d) {
        float f;
        if (dtype == 0) {
          const double x = __ldg((const double*)I.pts + i * d + l);
          const bool nonfinite = ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
          bad |= nonfinite;
          f = __double2float_rn(x);
          if (isfinite(f)) {
            mn[l] = fminf(mn[l], nextafterf(f, -FLT_MAX));
            mx[l] = fmaxf(mx[l], nextafterf(f, FLT_MAX));
          } else if (!nonfinite) {  // beyond the FP32 range (rare): the FP64 value itself
            atomicMax(&bbox[((size_t)b * kMaxDim + l) * 2 + 0], enc_double(x));
            atomicMax(&bbox[((size_t)b * kMaxDim + l) * 2 + 1], ~enc_double(x));
          }
        } else {
          f = __ldg((const float*)I.pts + i * d + l);
          mn[l] = fminf(mn[l], f);
          mx[l] = fmaxf(mx[l], f);
          bad |= !isfinite(f);
        }
        row[l] = f;
      }
    }
    float4* dst = reinterpret_cast<float4*>(pf + (I.p0 + i) * DPAD);
#pragma unroll
    for (int v = 0; v < DPAD / 4; ++v)
      dst[v] = make_float4(row[4 * v], row[4 * v + 1], row[4 * v + 2], row[4 * v + 3]);
    row_cnt[I.p0 + i] = 0u;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < DPAD; ++l) {
    float a = mn[l], c = mx[l];
    for (int o = 16; o > 0; o >>= 1) {
      a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
      c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    if (lane == 0) {
      smn[warp][l] = a;
      smx[warp][l] = c;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->errors, kErrNonFinite);
  if (threadIdx.x < d) {
    const int l = threadIdx.x;
    float a = smn[0][l], c = smx[0][l];
    for (int w = 1; w < kPrepThreads / 32; ++w) {
      a = fminf(a, smn[w][l]);
      c = fmaxf(c, smx[w][l]);
    }
    if (a <= c) {
      atomicMax(&bbox[((size_t)b * kMaxDim + l) * 2 + 0], enc_double((double)c));
      atomicMax(&bbox[((size_t)b * kMaxDim + l) * 2 + 1], ~enc_double((double)a));
    }
  }
  if (!pa.fuse) return;
  // the last block to finish plans every (instance, grid, axis), then the key ranges
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&st->prep_ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const long long items = (long long)B * (pa.m > 0 ? pa.m : 1) * kMaxDim;
  for (long long idx = threadIdx.x; idx < items; idx += blockDim.x)
    plan_axis_item(idx, inst, pa.m, dtype, pa.T64, bbox, pa.iplan, pa.gplan);
  if (pa.m == 0) return;
  __syncthreads();
  plan_ranges_block(inst, B, pa.m, pa.gplan, pa.bases, st, pa.passes, pa.radix_bits, pa.key64,
                    pa.cell_major);
}

// Distance band of instance b (one thread).  The bounding box is read from L2 (it was built
// by atomics).
__device__ void plan_band(int b, const Inst& I, int dtype, const unsigned long long* bbox,
                          InstPlan* iplan) {
  const int d = I.d;
  double M[kMaxDim];
  for (int l = 0; l < d; ++l) {
    const double hi = I.n > 0 ? dec_double(__ldcg(bbox + ((size_t)b * kMaxDim + l) * 2 + 0)) : 0.0;
    const double lo = I.n > 0 ? dec_double(~__ldcg(bbox + ((size_t)b * kMaxDim + l) * 2 + 1)) : 0.0;
    M[l] = fmax(fabs(lo), fabs(hi));
  }
  {
    // Distance band.  With S the exact squared distance and e_f the FP32 differences,
    // |fl32-chain(e_f) - S| <= 2|eta| sqrt(S) + |eta|^2 + d 2^-24 (sqrt(S) + |eta|)^2 where
    // eta_l bounds |e_f,l - e_l|: 2^-24 (|p_a,l| + |p_b,l|) from rounding FP64 input to FP32
    // plus 2^-24 |e_l| from the FP32 subtraction.  Evaluated at S <= 2 rr; the FP64
    // reference chain adds (d + 3) 2^-53 S.  The 3e-12 rr term sends every pair within
    // 1e-12 r of r to FP64, where the near-r diagnostic is counted.
    const double r = I.r;
    const double rr = __dmul_rn(r, r);
    const double u32 = 0x1.0p-24, u64 = 0x1.0p-53;
    const double S2 = sqrt(2.0 * rr) * (1.0 + 1e-9);
    double eta2 = 0.0;
    for (int l = 0; l < d; ++l) {
      const double delta = dtype == 0 ? 2.0 * u32 * M[l] * (1.0 + u32) : 0.0;
      const double eta = delta * (1.0 + u32) + u32 * S2 * (1.0 + 1e-6);
      eta2 += eta * eta;
    }
    const double eta = sqrt(eta2) * (1.0 + 1e-9);
    const double E1 = 2.0 * eta * S2 + eta * eta +
                      (double)d * u32 * (S2 + eta) * (S2 + eta) * (1.0 + 1e-3);
    const double Es = (E1 + (double)(d + 3) * u64 * 2.0 * rr + 3e-12 * rr) * 1.01;
    const bool on = isfinite(Es) && eta <= 1e-3 * r && rr > 0.0 && (rr - Es) > 0.0 &&
                    rr + Es < 1e30;
    InstPlan ip;
    ip.rr = rr;
    ip.filter_on = on ? 1 : 0;
    ip.s_lo = on ? __double2float_rd(rr - Es) : 0.0f;
    ip.s_hi = on ? __double2float_ru(rr + Es) : 0.0f;
    ip.inv_c = I.inv_cf;
    iplan[b] = ip;
  }
}

// Item (b, t, k): key layout of axis k of grid t of instance b (the bounding box is read from
// L2).  Without grids (brute force) item (b, 0, 0) sets the instance's distance band; with
// grids the key kernel sets it, off the critical path.
__device__ void plan_axis_item(long long idx, const Inst* __restrict__ inst, int m, int dtype,
                               const double* __restrict__ T64, const unsigned long long* bbox,
                               InstPlan* iplan, GridPlan* gplan) {
  const int mm = m > 0 ? m : 1;
  const int b = (int)(idx / (mm * kMaxDim));
  const int t = (int)(idx / kMaxDim % mm);
  const int k = (int)(idx % kMaxDim);
  const Inst I = inst[b];
  if (m == 0) {
    if (t == 0 && k == 0) plan_band(b, I, dtype, bbox, iplan);
    return;
  }
  const int d = I.d;
  GridPlan& G = gplan[(size_t)b * m + t];
  if (k >= d) {
    for (int l = 0; l < kMaxDim; ++l) G.Rf[k * kMaxDim + l] = 0.0f;
    G.sf[k] = 0.0f;
    G.E[k] = 0.0f;
    G.qlo[k] = 0;
    G.ext[k] = 1;
    return;
  }
  const double* R = T64 + I.T0 + (size_t)t * (d * d + d);
  const double* s = R + d * d;
  double ymin = s[k], ymax = s[k], A = fabs(s[k]);
#pragma unroll 3  // the loads of a few axes in flight together
  for (int l = 0; l < d; ++l) {
    const double hi = I.n > 0 ? dec_double(__ldcg(bbox + ((size_t)b * kMaxDim + l) * 2 + 0)) : 0.0;
    const double lo = I.n > 0 ? dec_double(~__ldcg(bbox + ((size_t)b * kMaxDim + l) * 2 + 1)) : 0.0;
    const double rkl = R[k * d + l];
    const double a = rkl * lo, bb = rkl * hi;
    ymin += fmin(a, bb);
    ymax += fmax(a, bb);
    A += fabs(rkl) * fmax(fabs(lo), fabs(hi));
    G.Rf[k * kMaxDim + l] = __double2float_rn(rkl);
  }
  for (int l = d; l < kMaxDim; ++l) G.Rf[k * kMaxDim + l] = 0.0f;
  G.sf[k] = __double2float_rn(s[k]);
  // The margin absorbs every rounding difference between these sums and the per-point
  // chains: each is within (d + 3) 2^-53 A / c of the exact y / c (d <= 16), so the two
  // together stay below 2^-47 A / c, less than 1 + floor(2^-46 A / c) cells: one cell on
  // each side for every A / c below 2^46, more beyond; 1/c comes from the host.
  const double margin = 1.0 + floor(A * I.inv_c * 0x1.0p-46);
  const double qmin = floor(ymin * I.inv_c) - margin, qmax = floor(ymax * I.inv_c) + margin;
  if (!(qmin > -4.0e18 && qmax < 4.0e18)) {
    G.qlo[k] = 0;
    G.ext[k] = ~0ull;  // flagged as overflow by the range pass
  } else {
    G.qlo[k] = (long long)qmin;
    G.ext[k] = (unsigned long long)((long long)qmax - (long long)qmin + 1);
  }
  const double E = ((double)(d + 6) * 0x1.0p-24 * A + 3e-12) * I.inv_c * (1.0 + 1e-6);
  G.E[k] = __double2float_ru(E);
}

__global__ void __launch_bounds__(128) k_plan_axes(const Inst* __restrict__ inst, int B, int m,
                                                   int dtype, const double* __restrict__ T64,
                                                   const unsigned long long* bbox,
                                                   InstPlan* iplan, GridPlan* gplan) {
  const int mm = m > 0 ? m : 1;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx < (long long)B * mm * kMaxDim) plan_axis_item(idx, inst, m, dtype, T64, bbox, iplan, gplan);
}

// One block: strides and key range of every (instance, grid), their exclusive prefix (the
// composite key bases), and the width of the composite key.  Any block size that is a
// multiple of 32, up to 1024.
__device__ void plan_ranges_block(const Inst* __restrict__ inst, int B, int m, GridPlan* gplan,
                                  unsigned long long* bases, Status* st, int passes,
                                  int radix_bits, int key64, int cell_major) {
  __shared__ unsigned long long sbuf[32];
  __shared__ unsigned long long carry;
  __shared__ int overflow;
  __shared__ unsigned int s_cbits;  // widest cell index range of one grid (bits)
  if (threadIdx.x == 0) {
    carry = 0;
    overflow = 0;
    s_cbits = 0;
  }
  __syncthreads();
  const long long total_bt = (long long)B * m;
  for (long long base = 0; base < total_bt; base += blockDim.x) {
    const long long bt = base + threadIdx.x;
    unsigned long long range = 0;
    if (bt < total_bt) {
      const int d = inst[bt / m].d;
      GridPlan& G = gplan[bt];
      unsigned long long strd = 1;
      bool of = false;
      for (int k = 0; k < kMaxDim; ++k) {
        if (k < d) {
          G.stride[k] = strd;
          const unsigned long long e = G.ext[k];
          if (e == ~0ull || __umul64hi(strd, e) != 0) of = true;
          strd *= e;
        } else {
          G.stride[k] = 0;
        }
      }
      if (of) {
        atomicOr((unsigned int*)&overflow, 1u);
        strd = 1;
      }
      G.range = strd;
      range = strd;
      if (strd > 1) atomicMax(&s_cbits, 64u - (unsigned)__clzll((long long)(strd - 1)));
    }
    // block exclusive scan of the ranges (with a carry across chunks)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x = range;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sbuf[warp] = x;
    __syncthreads();
    unsigned long long wpre = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) wpre += sbuf[w];
      tot += sbuf[w];
    }
    const unsigned long long ex = carry + wpre + x - range;
    if (bt < total_bt) {
      gplan[bt].base = ex;
      bases[bt] = ex;
      if (ex < carry) atomicOr((unsigned int*)&overflow, 1u);  // wrapped
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned long long nc = carry + tot;
      if (nc < carry) overflow = 1;
      carry = nc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = carry;
    const unsigned int bits = total <= 1 ? 0u : 64u - (unsigned)__clzll((long long)(total - 1));
    st->sort_bits = bits;
    st->cell_bits = s_cbits;
    if (overflow) atomicOr(&st->errors, kErrKeyOverflow);
    const unsigned int sorted_bits = cell_major ? s_cbits : bits;
    if (sort_passes_for((int)sorted_bits, radix_bits) > passes || (!key64 && bits > 32))
      atomicOr(&st->errors, kErrKeyBits);
  }
}

__global__ void __launch_bounds__(1024) k_plan_ranges(const Inst* __restrict__ inst, int B, int m,
                                                      GridPlan* gplan,
                                                      unsigned long long* bases, Status* st,
                                                      int passes, int radix_bits, int key64,
                                                      int cell_major) {
  plan_ranges_block(inst, B, m, gplan, bases, st, passes, radix_bits, key64, cell_major);
}

// FP64 reference cell index (the oracle's sequence) for point i, grid data Tt, axis k.
__device__ __noinline__ long long exact_cell(const void* pts, int dtype, long long i, int d,
                                             const double* Tt, int k, double c, bool* near) {
  const double* R = Tt;
  const double* s = Tt + d * d;
  double acc = s[k];
  for (int l = 0; l < d; ++l) acc = __fma_rn(R[k * d + l], load_coord(pts, dtype, i, d, l), acc);
  const double u = __ddiv_rn(acc, c);
  const double w = fabs(__dsub_rn(u, rint(u)));
  if (__dmul_rn(w, c) <= 1e-12) *near = true;
  return (long long)floor(u);
}

// One (grid, axis) row of the key computation, 16-byte aligned in shared memory so that a
// thread reads it with a few vector loads: the FP32 rotation row, the FP32 shift and error
// bound, and the axis's cell range and key stride.
template <int DPAD>
struct __align__(16) AxisRow {
  float R[DPAD];
  float s, E;
  float pad0, pad1;
  long long qlo;
  unsigned long long ext;
  unsigned long long stride;
  unsigned long long pad2;
};

template <int DPAD>
constexpr size_t axis_row_bytes() {
  return sizeof(AxisRow<DPAD>);
}

template <typename K, int DPAD>
__global__ void __launch_bounds__(kPointBlock) k_keys(
    const Inst* __restrict__ inst, int B, int m, int dtype, const float* __restrict__ pf,
    const double* __restrict__ T64, const GridPlan* __restrict__ gplan, InstPlan* iplan,
    const unsigned long long* bbox, Status* st, K* __restrict__ key_mat, int hist_passes,
    unsigned int* hist, unsigned int* digit_off, unsigned int* sort_epoch) {
  __shared__ int s_b;
  __shared__ unsigned int s_hist[kMaxPasses * 256];  // 8-bit digit counts of every pass
  for (int x = threadIdx.x; x < hist_passes * 256; x += blockDim.x) s_hist[x] = 0;
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = block_instance<false>(inst, B, blockIdx.x, &s_b);
  const Inst I = inst[b];
  const int d = I.d;
  // layout: the m*d axis rows (grid-major), the m grid bases, then the block's key rows
  // (kPointBlock rows of m keys, m + 1 apart), written out together at the end
  AxisRow<DPAD>* rows = reinterpret_cast<AxisRow<DPAD>*>(smem);
  unsigned long long* sbase = reinterpret_cast<unsigned long long*>(rows + m * d);
  K* s_krow = reinterpret_cast<K*>(sbase + m);
  const GridPlan* Gb = gplan + (size_t)b * m;
  for (int x = threadIdx.x; x < m * d; x += blockDim.x) {
    const int t = x / d, k = x - t * d;
    AxisRow<DPAD>& A = rows[x];
#pragma unroll
    for (int l = 0; l < DPAD; ++l) A.R[l] = Gb[t].Rf[k * kMaxDim + l];
    A.s = Gb[t].sf[k];
    A.E = Gb[t].E[k];
    A.qlo = Gb[t].qlo[k];
    A.ext = Gb[t].ext[k];
    A.stride = Gb[t].stride[k];
  }
  for (int t = threadIdx.x; t < m; t += blockDim.x) sbase[t] = Gb[t].base;
  __syncthreads();
  const float inv_c = I.inv_cf;
  if (threadIdx.x == 0 && blockIdx.x == I.blk0) plan_band(b, I, dtype, bbox, iplan);
  const double c = I.c;
  const long long i = (blockIdx.x - I.blk0) * (long long)kPointBlock + threadIdx.x;
  unsigned int near_cnt = 0, rechecks = 0;
  bool range_err = false;
  const bool valid = i < I.n;
  const unsigned int vmask = __ballot_sync(0xffffffffu, valid);
  {
    const long long g = I.p0 + (valid ? i : 0);
    float p[DPAD];
    const float4* src = reinterpret_cast<const float4*>(pf + g * DPAD);
#pragma unroll
    for (int v = 0; v < DPAD / 4; ++v) {
      const float4 q = valid ? src[v] : make_float4(0.f, 0.f, 0.f, 0.f);
      p[4 * v] = q.x;
      p[4 * v + 1] = q.y;
      p[4 * v + 2] = q.z;
      p[4 * v + 3] = q.w;
    }
    const int tstride = d * d + d;
    K* krow = s_krow + threadIdx.x * (m + 1);
    const int dv = valid ? d : 0;
    for (int t = 0; t < m; ++t) {  // every lane takes every grid (warp votes below)
      K key = (K)sbase[t];
      bool near = false;
      const AxisRow<DPAD>* A = rows + t * d;
      unsigned int redo = 0;  // axes whose FP32 index is not certain
      for (int k = 0; k < dv; ++k) {
        const float2 se = *reinterpret_cast<const float2*>(&A[k].s);
        float y = se.x;
#pragma unroll
        for (int v = 0; v < DPAD / 4; ++v) {
          const float4 r = reinterpret_cast<const float4*>(A[k].R)[v];
          y = fmaf(r.x, p[4 * v], y);
          y = fmaf(r.y, p[4 * v + 1], y);
          y = fmaf(r.z, p[4 * v + 2], y);
          y = fmaf(r.w, p[4 * v + 3], y);
        }
        const float u = y * inv_c;
        // the FP32 index is certain when [u - E, u + E] holds no cell wall: both ends (rounded
        // outwards) lie in [floor(u), floor(u) + 1).  |u| >= 2^23 always fails (u is then an
        // integer and u - E < u), so floor(u) is exact in 32-bit integers here.
        const float f = floorf(u);
        const bool certain = __fsub_rd(u, se.y) >= f && __fadd_ru(u, se.y) < f + 1.0f;
        const longlong2 qe = *reinterpret_cast<const longlong2*>(&A[k].qlo);
        long long off = (long long)(int)f - qe.x;
        const bool out = (unsigned long long)off >= (unsigned long long)qe.y;
        if (!certain) redo |= 1u << k;
        if (certain && out) range_err = true;
        if (!certain || out) off = 0;
        key += (K)off * (K)A[k].stride;
      }
      while (redo) {  // rare: the FP64 reference sequence decides these axes
        const int k = __ffs(redo) - 1;
        redo &= redo - 1;
        const long long q =
            exact_cell(I.pts, dtype, i, d, T64 + I.T0 + (size_t)t * tstride, k, c, &near);
        ++rechecks;
        long long off = q - A[k].qlo;
        if ((unsigned long long)off >= A[k].ext) {
          range_err = true;
          off = 0;
        }
        key += (K)off * (K)A[k].stride;
      }
      if (valid) {
        krow[t] = key;
        near_cnt += near ? 1u : 0u;
      }
      // digit counts: the low digits of neighbouring points differ, so only the top digit
      // (mostly the grid's base) tries the one-add-per-warp path
      for (int q = 0; q + 1 < hist_passes; ++q)
        if (valid) atomicAdd(&s_hist[q * 256 + ((unsigned int)(key >> (8 * q)) & 255u)], 1u);
      if (hist_passes > 0)
        count_digit256(s_hist + (hist_passes - 1) * 256,
                       (unsigned int)(key >> (8 * (hist_passes - 1))) & 255u, valid, vmask);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    near_cnt += __shfl_xor_sync(0xffffffffu, near_cnt, o);
    rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (near_cnt) atomicAdd(&st->near_wall, (unsigned long long)near_cnt);
    if (rechecks) atomicAdd(&st->key_rechecks, (unsigned long long)rechecks);
  }
  if (range_err) atomicOr(&st->errors, kErrKeyRange);
  __syncthreads();
  {  // the block's key rows are one contiguous stretch of key_mat: coalesced copy-out
    const long long i0 = (blockIdx.x - I.blk0) * (long long)kPointBlock;
    const unsigned int words = (unsigned int)max(0LL, min((long long)kPointBlock, I.n - i0)) * m;
    K* dst = key_mat + (size_t)(I.p0 + i0) * m;
    for (unsigned int w = threadIdx.x; w < words; w += kPointBlock) {
      const unsigned int row = w / (unsigned int)m;
      dst[w] = s_krow[row * (m + 1) + (w - row * m)];
    }
  }
  if (hist_passes > 0) {
    finish_digit_count256(s_hist, hist_passes, hist, digit_off, &st->hist_ticket, sort_epoch);
  }
}

// Batches up to this many (instance, grid, axis) items plan in the prep kernel's last block.
constexpr long long kFusedPlanItems = 4096;

bool plan_fused(const BuildArgs& a) {
  return (long long)a.B * (a.m > 0 ? a.m : 1) * kMaxDim <= kFusedPlanItems;
}

template <int DPAD>
void prep_impl(const BuildArgs& a, cudaStream_t s) {
  PlanArgs pa;
  pa.fuse = plan_fused(a) ? 1 : 0;
  pa.points = a.prep_points > 0 ? a.prep_points : kPrepPoints;
  pa.m = a.m;
  pa.T64 = a.T64;
  pa.iplan = a.iplan;
  pa.gplan = a.gplan;
  pa.bases = a.bases;
  pa.passes = a.passes;
  pa.radix_bits = a.sort_bits;
  pa.key64 = a.key64 ? 1 : 0;
  pa.cell_major = a.cell_major;
  k_prep<DPAD><<<(unsigned)a.pblocks, kPrepThreads, 0, s>>>(a.inst, a.B, a.dtype, a.pf,
                                                             a.row_cnt, a.bbox, a.st, pa);
}

template <typename K, int DPAD>
void keys_impl(const BuildArgs& a, int maxd, cudaStream_t s) {
  const size_t smem = (size_t)a.m * maxd * axis_row_bytes<DPAD>() + (size_t)a.m * 8 +
                      (size_t)kPointBlock * (a.m + 1) * sizeof(K);
  // the 48 KB default covers static and dynamic shared memory together (the digit counts
  // are static), so the limit is raised to every new largest size, not only above 48 KB
  static size_t attr_smem[64] = {};  // largest size granted so far, per device
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(launch_attr_mutex());
    if (dev < 0 || dev >= 64 || smem > attr_smem[dev]) {
      cudaFuncSetAttribute(k_keys<K, DPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      if (dev >= 0 && dev < 64) attr_smem[dev] = smem;
    }
  }
  k_keys<K, DPAD><<<(unsigned)a.blocks, kPointBlock, smem, s>>>(
      a.inst, a.B, a.m, a.dtype, a.pf, a.T64, a.gplan, a.iplan, a.bbox, a.st, (K*)a.key_mat,
      hist_in_keys(a) ? a.passes : 0, a.hist, a.digit_off, a.sort_epoch);
}

// Keys with one thread per (point, grid): for instances that share d <= 6.  Each thread keeps
// its grid's FP32 rotation and shift in registers for the whole block (the grid of a thread
// never changes), so the inner loop is the d x d FMAs and the floor test; the per-axis error
// bound and key layout come from shared memory, stored axis-major so that the different grids
// of a warp read different banks.  A block's threads write consecutive key-row words.  The
// arithmetic, bounds and FP64 fallback are those of k_keys.  With 32-bit keys the cell offsets
// are formed modulo 2^32, which is exact for every index inside the planned range (the range
// check then only guards the plan itself).
constexpr int kKeyLaneThreads = 256;

// Per (axis, grid) record of k_keys_lanes.
template <typename K>
struct __align__(16) LaneAxis {
  float E;
  unsigned int pad;
  K qlo, ext, stride;
};
template <>
struct __align__(16) LaneAxis<uint32_t> {
  float E;
  uint32_t qlo, ext, stride;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Chunk c of the per-point numbering (kPointBlock points, blk0 offsets per instance): its
// instance, first global point and point count.
struct ChunkInfo {
  int b, npts;
  long long g0, i0;
};
__device__ __forceinline__ ChunkInfo chunk_info(const Inst* __restrict__ inst, int B,
                                                long long c) {
  int lo = 0, hi = B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].blk0 <= c) lo = mid; else hi = mid - 1;
  }
  ChunkInfo ci;
  ci.b = lo;
  ci.i0 = (c - inst[lo].blk0) * (long long)kPointBlock;
  ci.g0 = inst[lo].p0 + ci.i0;
  ci.npts = (int)min((long long)kPointBlock, (long long)inst[lo].n - ci.i0);
  return ci;
}

// One thread: start the bulk copy of chunk ci's FP32 rows (contiguous, 16-byte multiples)
// into dst, completing on bar.
__device__ __forceinline__ void stage_rows(const float* pf, int dpad, const ChunkInfo& ci,
                                           float* dst, uint64_t* bar) {
  const unsigned int bytes = (unsigned int)ci.npts * (unsigned int)dpad * 4u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(pf + ci.g0 * dpad), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait for phase `parity` of the mbarrier bar.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned int limit) {
  for (unsigned int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <typename K, int D>
__global__ void __launch_bounds__(kKeyLaneThreads, 2) k_keys_lanes(
    const Inst* __restrict__ inst, int B, int m, int dtype, int dpad,
    const float* __restrict__ pf, const double* __restrict__ T64,
    const GridPlan* __restrict__ gplan, InstPlan* iplan, const unsigned long long* bbox,
    Status* st, K* __restrict__ key_mat, long long chunks, int hist_passes, int hist_bits,
    unsigned int* hist, unsigned int* digit_off, unsigned int* sort_epoch,
    unsigned int wait_limit, K* __restrict__ key_gm, long long gm_n) {
  constexpr int DP = D <= 4 ? 4 : 8;  // padded row width of the FP32 rows
  __shared__ unsigned int s_hist[kLaneHistWords];  // digit counts of every pass
  __shared__ __align__(16) float s_rows[2][kPointBlock * DP];  // double-buffered chunk rows
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ ChunkInfo s_info[2];
  extern __shared__ __align__(16) unsigned char smem[];
  LaneAxis<K>* s_ax = reinterpret_cast<LaneAxis<K>*>(smem);  // [axis][grid]
  for (int x = threadIdx.x; x < hist_passes << hist_bits; x += blockDim.x) s_hist[x] = 0;
  const long long stride_c = gridDim.x;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("fence.proxy.async.shared::cta;");
    if ((long long)blockIdx.x < chunks) {
      s_info[0] = chunk_info(inst, B, blockIdx.x);
      stage_rows(pf, dpad, s_info[0], s_rows[0], &s_bar[0]);
    }
  }
  __syncthreads();
  const int P = kKeyLaneThreads / m;  // points per step of the block
  const int t = (int)threadIdx.x % m, slot = (int)threadIdx.x / m;
  const bool lane_on = slot < P;
  float R[D][D], sf[D];
  K base = 0;
  int cur_b = -1;
  const GridPlan* G = nullptr;
  Inst I;
  // phase: parity to wait for, per buffer; pending (thread 0): copies issued, not yet consumed
  unsigned int near_cnt = 0, rechecks = 0, phase = 0, pending = 1u;
  bool range_err = false, timed_out = false;
  // persistent: the block takes 128-point chunks gridDim apart, their rows staged one chunk
  // ahead by bulk copies, and reloads its plan only when a chunk is of another instance
  int k = 0;
  for (long long chunk = blockIdx.x; chunk < chunks; chunk += stride_c, ++k) {
    const int buf = k & 1;
    const ChunkInfo ci = s_info[buf];
    if (threadIdx.x == 0 && chunk + stride_c < chunks) {
      // the other buffer was last read before the previous iteration's closing barrier
      s_info[buf ^ 1] = chunk_info(inst, B, chunk + stride_c);
      stage_rows(pf, dpad, s_info[buf ^ 1], s_rows[buf ^ 1], &s_bar[buf ^ 1]);
      pending |= 2u >> buf;  // the copy into buffer buf ^ 1 is in flight
    }
    if (ci.b != cur_b) {  // block-uniform
      const GridPlan* Gb = gplan + (size_t)ci.b * m;
      for (int x = threadIdx.x; x < D * m; x += blockDim.x) {
        const int a = x / m, g = x - a * m;
        LaneAxis<K> r;
        r.E = Gb[g].E[a];
        r.qlo = (K)Gb[g].qlo[a];
        r.ext = (K)Gb[g].ext[a];
        r.stride = (K)Gb[g].stride[a];
        s_ax[x] = r;
      }
      I = inst[ci.b];
      G = Gb + t;
#pragma unroll
      for (int a = 0; a < D; ++a) {
#pragma unroll
        for (int l = 0; l < D; ++l) R[a][l] = G->Rf[a * kMaxDim + l];
        sf[a] = G->sf[a];
      }
      base = (K)G->base;
      cur_b = ci.b;
      __syncthreads();
    }
    if (threadIdx.x == 0 && chunk == I.blk0) plan_band(ci.b, I, dtype, bbox, iplan);
    // this chunk's rows
    const bool ok = mbar_wait_bounded(&s_bar[buf], (phase >> buf) & 1u, wait_limit);
    if (!__syncthreads_and(ok)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << buf;
    pending &= ~(1u << buf);
    const float inv_c = I.inv_cf;
    const float* rows = s_rows[buf];
    K* out = key_mat + ci.g0 * m + (long long)(slot * m + t);  // this thread's first word
    for (int p0 = 0; p0 < ci.npts; p0 += P, out += P * m) {  // block-uniform
      const int p = p0 + slot;
      const bool valid = lane_on && p < ci.npts;
      const int pp = valid ? p : 0;
      float x[DP];
#pragma unroll
      for (int v = 0; v < DP / 4; ++v) {
        const float4 q = *reinterpret_cast<const float4*>(rows + pp * dpad + 4 * v);
        x[4 * v] = q.x;
        x[4 * v + 1] = q.y;
        x[4 * v + 2] = q.z;
        x[4 * v + 3] = q.w;
      }
      K key = base;
      unsigned int redo = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        float y = sf[a];
#pragma unroll
        for (int l = 0; l < D; ++l) y = fmaf(R[a][l], x[l], y);
        const LaneAxis<K> ax = s_ax[a * m + t];
        const float u = y * inv_c;
        const float f = floorf(u);
        // certain when [u - E, u + E], rounded outwards, holds no cell wall (as in k_keys)
        const bool certain = __fsub_rd(u, ax.E) >= f && __fadd_ru(u, ax.E) < f + 1.0f;
        const K off = (K)(long long)(int)f - ax.qlo;
        const bool out = off >= ax.ext;
        if (!certain) redo |= 1u << a;
        if (certain && out) range_err = true;
        key += (certain && !out) ? off * ax.stride : (K)0;
      }
      if (!valid) redo = 0;
      bool near = false;
      while (redo) {  // rare: the FP64 reference sequence decides these axes
        const int a = __ffs(redo) - 1;
        redo &= redo - 1;
        const long long q = exact_cell(I.pts, dtype, ci.i0 + pp, D,
                                       T64 + I.T0 + (size_t)t * (D * D + D), a, I.c, &near);
        ++rechecks;
        const long long off = q - G->qlo[a];
        if ((unsigned long long)off >= G->ext[a]) {
          range_err = true;
        } else {
          key += (K)off * (K)G->stride[a];
        }
      }
      if (valid) {
        *out = key;
        near_cnt += near ? 1u : 0u;
        // cell-major sort: the digits are those of the cell index, whose grid-major copy the
        // first pass reads (one instance, so point ci.g0 + p is its own grid-major offset)
        const K hkey = key_gm ? key - base : key;
        if (key_gm) key_gm[(long long)t * gm_n + ci.g0 + p] = hkey;
        if (hist_bits == 8) {
          const unsigned int lo = (unsigned int)hkey,
                             hi = (unsigned int)((unsigned long long)hkey >> 32);
#pragma unroll
          for (int q = 0; q < kMaxPasses; ++q)  // digit q is byte q of the key
            if (q < hist_passes)
              atomicAdd(&s_hist[q * 256 + __byte_perm(q < 4 ? lo : hi, 0u, 0x4440u + (q & 3))],
                        1u);
        } else {
          const unsigned int dm = (1u << hist_bits) - 1u;
#pragma unroll 1
          for (int q = 0; q < hist_passes; ++q)
            atomicAdd(&s_hist[(q << hist_bits) + ((unsigned int)(hkey >> (hist_bits * q)) & dm)],
                      1u);
        }
      }
    }
    __syncthreads();  // rows[buf], s_info[buf] and s_ax are rewritten later
  }
  if (timed_out) {
    // a staged copy may still be in flight: wait for it (bounded) before the block exits
    if (threadIdx.x == 0) {
      atomicOr(&st->errors, kErrTimeout);
      for (int q = 0; q < 2; ++q)
        if ((pending >> q) & 1u) mbar_wait_bounded(&s_bar[q], (phase >> q) & 1u, wait_limit);
    }
    return;  // the digit counts stay incomplete; the build reports the timeout
  }
  for (int o = 16; o > 0; o >>= 1) {
    near_cnt += __shfl_xor_sync(0xffffffffu, near_cnt, o);
    rechecks += __shfl_xor_sync(0xffffffffu, rechecks, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (near_cnt) atomicAdd(&st->near_wall, (unsigned long long)near_cnt);
    if (rechecks) atomicAdd(&st->key_rechecks, (unsigned long long)rechecks);
  }
  if (range_err) atomicOr(&st->errors, kErrKeyRange);
  __syncthreads();
  if (hist_passes > 0)
    finish_digit_count_bits(s_hist, hist_passes, hist_bits, hist, digit_off, &st->hist_ticket,
                            sort_epoch);
}

template <typename K, int D>
void keys_lanes_launch(const BuildArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(LaneAxis<K>) * (size_t)D * a.m;  // at most 16 KB
  // two resident blocks per SM (the register budget), each looping over chunks
  long long grid = 2LL * a.num_sms;
  if (grid > a.blocks) grid = a.blocks;
  k_keys_lanes<K, D><<<(unsigned)grid, kKeyLaneThreads, smem, s>>>(
      a.inst, a.B, a.m, a.dtype, a.dpad, a.pf, a.T64, a.gplan, a.iplan, a.bbox, a.st,
      (K*)a.key_mat, a.blocks, hist_in_keys(a) ? a.passes : 0, a.sort_bits, a.hist,
      a.digit_off, a.sort_epoch, spin_limit_of(a.spin_limit) * 16u,
      a.cell_major ? (K*)a.keys[1] : (K*)nullptr, a.n_total);
}

template <typename K>
bool keys_lanes(const BuildArgs& a, cudaStream_t s) {
  if (!keys_by_lanes(a)) return false;
  switch (a.d_common) {
    case 1: keys_lanes_launch<K, 1>(a, s); return true;
    case 2: keys_lanes_launch<K, 2>(a, s); return true;
    case 3: keys_lanes_launch<K, 3>(a, s); return true;
    case 4: keys_lanes_launch<K, 4>(a, s); return true;
    case 5: keys_lanes_launch<K, 5>(a, s); return true;
    case 6: keys_lanes_launch<K, 6>(a, s); return true;
    default: return false;  // wider rows would not fit the register budget
  }
}

}  // namespace

int launch_prep_plan(const BuildArgs& a, cudaStream_t s) {
  switch (a.dpad) {
    case 4: prep_impl<4>(a, s); break;
    case 8: prep_impl<8>(a, s); break;
    default: prep_impl<16>(a, s); break;
  }
  if (plan_fused(a)) return 1;
  const long long threads = (long long)a.B * (a.m > 0 ? a.m : 1) * kMaxDim;
  k_plan_axes<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(a.inst, a.B, a.m, a.dtype, a.T64,
                                                              a.bbox, a.iplan, a.gplan);
  if (a.m > 0)
    k_plan_ranges<<<1, 1024, 0, s>>>(a.inst, a.B, a.m, a.gplan, a.bases, a.st, a.passes,
                                     a.sort_bits, a.key64 ? 1 : 0, a.cell_major);
  return a.m > 0 ? 3 : 2;
}

void launch_keys(const BuildArgs& a, cudaStream_t s) {
  if (a.key64 ? keys_lanes<unsigned long long>(a, s) : keys_lanes<uint32_t>(a, s)) return;
  const int maxd = a.dpad;  // rows staged per grid never exceed the padded width
  if (a.key64) {
    switch (a.dpad) {
      case 4: keys_impl<unsigned long long, 4>(a, maxd, s); break;
      case 8: keys_impl<unsigned long long, 8>(a, maxd, s); break;
      default: keys_impl<unsigned long long, 16>(a, maxd, s); break;
    }
  } else {
    switch (a.dpad) {
      case 4: keys_impl<uint32_t, 4>(a, maxd, s); break;
      case 8: keys_impl<uint32_t, 8>(a, maxd, s); break;
      default: keys_impl<uint32_t, 16>(a, maxd, s); break;
    }
  }
}

}  // namespace rtg
