// Point preparation, per-build plan and the transform+key kernel (Alg. 1 lines 4-7 of
// arXiv:1409.8112, for the rotated + shifted grids of Sec. III).
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

template <int DPAD>
__global__ void __launch_bounds__(256) k_prep(const void* __restrict__ pts, int dtype, int n,
                                              int d, float* __restrict__ pf, Status* st) {
  double mn[DPAD], mx[DPAD];
#pragma unroll
  for (int l = 0; l < DPAD; ++l) {
    mn[l] = DBL_MAX;
    mx[l] = -DBL_MAX;
  }
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float row[DPAD];
#pragma unroll
    for (int l = 0; l < DPAD; ++l) {
      if (l < d) {
        double x = load_coord(pts, dtype, i, d, l);
        bad |= !isfinite(x);
        mn[l] = fmin(mn[l], x);
        mx[l] = fmax(mx[l], x);
        row[l] = __double2float_rn(x);
      } else {
        row[l] = 0.0f;
      }
    }
    float4* dst = reinterpret_cast<float4*>(pf + i * DPAD);
#pragma unroll
    for (int v = 0; v < DPAD / 4; ++v)
      dst[v] = make_float4(row[4 * v], row[4 * v + 1], row[4 * v + 2], row[4 * v + 3]);
  }
  // block reduction of the bounding box, then one atomic per axis per block
  __shared__ double smn[8][DPAD], smx[8][DPAD];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < DPAD; ++l) {
    double a = mn[l], b = mx[l];
    for (int o = 16; o > 0; o >>= 1) {
      a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if (lane == 0) {
      smn[warp][l] = a;
      smx[warp][l] = b;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&st->errors, kErrNonFinite);
  if (threadIdx.x < d) {
    const int l = threadIdx.x;
    double a = smn[0][l], b = smx[0][l];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = fmin(a, smn[w][l]);
      b = fmax(b, smx[w][l]);
    }
    if (a <= b) {  // the block saw at least one point
      atomicMax(&st->bbox_nmin[l], ~enc_double(a));
      atomicMax(&st->bbox_max[l], enc_double(b));
    }
  }
}

// One block.  Threads (t, k) fill the key layout and the FP32 data of grid t, axis k.
__global__ void __launch_bounds__(1024) k_plan(Plan* P, Status* st, const double* T64, int n,
                                               int d, int m, int dtype, double r, double c,
                                               int assumed_bits) {
  __shared__ double lo[kMaxDim], hi[kMaxDim], M[kMaxDim];
  __shared__ unsigned int bits_t[kMaxGrids];
  const int tid = threadIdx.x;
  if (tid < kMaxDim) {
    double a = 0.0, b = 0.0;
    if (tid < d && n > 0) {
      a = dec_double(~st->bbox_nmin[tid]);
      b = dec_double(st->bbox_max[tid]);
    }
    lo[tid] = a;
    hi[tid] = b;
    M[tid] = fmax(fabs(a), fabs(b));
  }
  __syncthreads();
  const int stride = d * d + d;
  for (int idx = tid; idx < m * kMaxDim; idx += blockDim.x) {
    const int t = idx / kMaxDim, k = idx % kMaxDim;
    if (k >= d) {
      for (int l = 0; l < kMaxDim; ++l) P->Rf[t][k * kMaxDim + l] = 0.0f;
      P->sf[t][k] = 0.0f;
      P->E[t][k] = 0.0f;
      P->qlo[t][k] = 0;
      P->ext[t][k] = 1;
      continue;
    }
    const double* R = T64 + (size_t)t * stride;
    const double* s = R + d * d;
    double ymin = s[k], ymax = s[k], A = fabs(s[k]);
    for (int l = 0; l < kMaxDim; ++l) {
      if (l < d) {
        const double rkl = R[k * d + l];
        const double a = rkl * lo[l], b = rkl * hi[l];
        ymin += fmin(a, b);
        ymax += fmax(a, b);
        A += fabs(rkl) * M[l];
        P->Rf[t][k * kMaxDim + l] = __double2float_rn(rkl);
      } else {
        P->Rf[t][k * kMaxDim + l] = 0.0f;
      }
    }
    P->sf[t][k] = __double2float_rn(s[k]);
    // Two cells of margin on each side absorb every rounding difference between these sums
    // and the per-point fma chains (both are far below one cell).
    const double qmin = floor(ymin / c) - 2.0, qmax = floor(ymax / c) + 2.0;
    if (!(qmin > -4.0e18 && qmax < 4.0e18)) {
      atomicOr(&st->errors, kErrKeyOverflow);
      P->qlo[t][k] = 0;
      P->ext[t][k] = 1;
    } else {
      P->qlo[t][k] = (long long)qmin;
      P->ext[t][k] = (unsigned long long)((long long)qmax - (long long)qmin + 1);
    }
    const double E = (double)(d + 6) * 0x1.0p-24 * A / c * (1.0 + 1e-6) + 3e-12 / c;
    P->E[t][k] = __double2float_ru(E);
  }
  __syncthreads();
  if (tid < m) {
    const int t = tid;
    unsigned long long strd = 1;
    bool of = false;
    for (int k = 0; k < kMaxDim; ++k) {
      if (k < d) {
        P->stride[t][k] = strd;
        const unsigned long long e = P->ext[t][k];
        if (__umul64hi(strd, e) != 0) of = true;
        strd *= e;
      } else {
        P->stride[t][k] = 0;
      }
    }
    bits_t[t] = of ? 65u : (strd <= 1 ? 0u : 64u - (unsigned)__clzll((long long)(strd - 1)));
  }
  __syncthreads();
  if (tid == 0) {
    unsigned int B = 0;
    for (int t = 0; t < m; ++t) B = max(B, bits_t[t]);
    const unsigned int gb = m <= 1 ? 0u : 32u - (unsigned)__clz(m - 1);
    if (B > 64 || B + gb > 64) atomicOr(&st->errors, kErrKeyOverflow);
    if ((int)(B + gb) > assumed_bits) atomicOr(&st->errors, kErrKeyBits);
    st->key_bits = B;
    st->grid_bits = gb;
    P->key_bits = (int)B;
    P->grid_bits = (int)gb;
    P->n = n;
    P->d = d;
    P->m = m;
    P->dtype = dtype;
    P->c = c;
    P->r = r;
    const double rr = __dmul_rn(r, r);
    P->rr = rr;
    P->inv_c = __double2float_rn(1.0 / c);
    // Distance filter.  With S the exact squared distance and e_f the FP32 differences,
    // |fl32-chain(e_f) - S| <= 2|eta| sqrt(S) + |eta|^2 + d 2^-24 (sqrt(S) + |eta|)^2 where
    // eta_l bounds |e_f,l - e_l|: 2^-24 (|p_a,l| + |p_b,l|) from rounding FP64 input to FP32
    // plus 2^-24 |e_l| from the FP32 subtraction.  Evaluated at S <= 2 rr; the FP64
    // reference chain adds (d + 3) 2^-53 S.  The 3e-12 rr term sends every pair within
    // 1e-12 r of r to FP64, where the near-r diagnostic is counted.
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
    P->filter_on = on ? 1 : 0;
    P->s_lo = on ? __double2float_rd(rr - Es) : 0.0f;
    P->s_hi = on ? __double2float_ru(rr + Es) : 0.0f;
  }
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

template <typename K, int DPAD>
__global__ void __launch_bounds__(128) k_keys(const float* __restrict__ pf,
                                              const void* __restrict__ pts, int dtype,
                                              const double* __restrict__ T64,
                                              const Plan* __restrict__ P, Status* st,
                                              K* __restrict__ key_mat, K* __restrict__ comp,
                                              uint32_t* __restrict__ vals, int n, int d, int m,
                                              double c) {
  extern __shared__ __align__(16) unsigned char smem[];
  // layout: qlo, ext, stride (m*d 8-byte each), R (m*d*DPAD floats), s, E (m*d floats)
  long long* sqlo = reinterpret_cast<long long*>(smem);
  unsigned long long* sext = reinterpret_cast<unsigned long long*>(sqlo + m * d);
  unsigned long long* sstr = sext + m * d;
  float* sR = reinterpret_cast<float*>(sstr + m * d);
  float* ss = sR + m * d * DPAD;
  float* sE = ss + m * d;
  for (int x = threadIdx.x; x < m * d; x += blockDim.x) {
    const int t = x / d, k = x % d;
    sqlo[x] = P->qlo[t][k];
    sext[x] = P->ext[t][k];
    sstr[x] = P->stride[t][k];
    ss[x] = P->sf[t][k];
    sE[x] = P->E[t][k];
  }
  for (int x = threadIdx.x; x < m * d * DPAD; x += blockDim.x) {
    const int t = x / (d * DPAD), rem = x % (d * DPAD), k = rem / DPAD, l = rem % DPAD;
    sR[x] = P->Rf[t][k * kMaxDim + l];
  }
  __syncthreads();
  const int B = P->key_bits;
  const float inv_c = P->inv_c;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned int near_cnt = 0, rechecks = 0;
  bool range_err = false;
  if (i < n) {
    float p[DPAD];
    const float4* src = reinterpret_cast<const float4*>(pf + i * DPAD);
#pragma unroll
    for (int v = 0; v < DPAD / 4; ++v) {
      const float4 q = src[v];
      p[4 * v] = q.x;
      p[4 * v + 1] = q.y;
      p[4 * v + 2] = q.z;
      p[4 * v + 3] = q.w;
    }
    const int stride = d * d + d;
    for (int t = 0; t < m; ++t) {
      K key = 0;
      bool near = false;
      for (int k = 0; k < d; ++k) {
        const float* Rk = sR + (t * d + k) * DPAD;
        float y = ss[t * d + k];
#pragma unroll
        for (int l = 0; l < DPAD; ++l) y = fmaf(Rk[l], p[l], y);
        const float u = y * inv_c;
        const float E = sE[t * d + k];
        const float flo = floorf(__fsub_rd(u, E)), fhi = floorf(__fadd_ru(u, E));
        long long q;
        if (flo == fhi) {
          q = (long long)flo;
        } else {
          q = exact_cell(pts, dtype, i, d, T64 + (size_t)t * stride, k, c, &near);
          ++rechecks;
        }
        long long off = q - sqlo[t * d + k];
        if ((unsigned long long)off >= sext[t * d + k]) {
          range_err = true;
          off = 0;
        }
        key += (K)off * (K)sstr[t * d + k];
      }
      key_mat[(size_t)i * m + t] = key;
      comp[(size_t)t * n + i] = (m > 1 ? ((K)t << B) : (K)0) | key;
      vals[(size_t)t * n + i] = (uint32_t)i;
      near_cnt += near ? 1u : 0u;
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
}

template <int DPAD>
void prep_impl(const BuildArgs& a, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (a.n + threads - 1) / threads;
  if (blocks > 4LL * a.num_sms) blocks = 4LL * a.num_sms;
  if (blocks < 1) blocks = 1;
  k_prep<DPAD><<<(unsigned)blocks, threads, 0, s>>>(a.pts, a.dtype, a.n, a.d, a.pf, a.st);
}

template <typename K, int DPAD>
void keys_impl(const BuildArgs& a, cudaStream_t s) {
  const int threads = 128;
  const size_t smem = (size_t)a.m * a.d * (3 * 8 + (DPAD + 2) * 4);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_keys<K, DPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const unsigned blocks = (unsigned)((a.n + threads - 1) / threads);
  k_keys<K, DPAD><<<blocks, threads, smem, s>>>(a.pf, a.pts, a.dtype, a.T64, a.plan, a.st,
                                                (K*)a.key_mat, (K*)a.keys[0], a.vals[0], a.n,
                                                a.d, a.m, a.c);
}

}  // namespace

void launch_prep(const BuildArgs& a, cudaStream_t s) {
  switch (a.dpad) {
    case 4: prep_impl<4>(a, s); break;
    case 8: prep_impl<8>(a, s); break;
    default: prep_impl<16>(a, s); break;
  }
}

void launch_plan(const BuildArgs& a, int assumed_bits, cudaStream_t s) {
  int threads = a.m * kMaxDim;
  if (threads < 64) threads = 64;
  if (threads > 1024) threads = 1024;
  k_plan<<<1, threads, 0, s>>>(a.plan, a.st, a.T64, a.n, a.d, a.m, a.dtype, a.r, a.c,
                               assumed_bits);
}

void launch_keys(const BuildArgs& a, cudaStream_t s) {
  if (a.key64) {
    switch (a.dpad) {
      case 4: keys_impl<unsigned long long, 4>(a, s); break;
      case 8: keys_impl<unsigned long long, 8>(a, s); break;
      default: keys_impl<unsigned long long, 16>(a, s); break;
    }
  } else {
    switch (a.dpad) {
      case 4: keys_impl<uint32_t, 4>(a, s); break;
      case 8: keys_impl<uint32_t, 8>(a, s); break;
      default: keys_impl<uint32_t, 16>(a, s); break;
    }
  }
}

}  // namespace rtg
