// Shared pieces of the tcgen05 kernels (tensor-core brute force and dense-cell tiles) and of
// the kernels that stage gathers asynchronously: the K-major no-swizzle operand layout of a
// 128-row half-precision tile with K = 32 (16 hi + 16 lo), its shared-memory descriptor,
// cp.async copies, bounded mbarrier waits, the TMEM read of 32 columns, and the error bound
// of a tile d^2 against the exact d^2 of the rounded, centred coordinates.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rtg {

// Byte offset of element (row m, k) in a tile: core matrices of 8 rows x 16 bytes, 128 bytes
// apart along K and 512 bytes apart along M.
__host__ __device__ __forceinline__ int tile_off(int m, int k) {
  return (m / 8) * 512 + (k / 8) * 128 + (m % 8) * 16 + (k % 8) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Asynchronous global -> shared copies (cp.async): a thread issues all of its copies and waits
// once, so that its gathers are in flight together.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ uint64_t make_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;  // next core matrix along K
  d |= (uint64_t)((512u >> 4) & 0x3FFF) << 32;  // next 8 rows
  d |= (uint64_t)1 << 46;                       // descriptor version; no swizzle
  return d;
}

// Bounded wait for the completion of phase `parity` of the mbarrier at shared address bar;
// false when the limit ran out first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned int limit) {
  for (unsigned int it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// 32 columns of the warp's 32 TMEM lanes into r, without waiting (tc_ld_wait() before use).
__device__ __forceinline__ void tc_ld32_async(uint32_t addr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
}
__device__ __forceinline__ void tc_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }

__device__ __forceinline__ void tc_ld32(uint32_t addr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}


// Bound on |tile d^2 - d^2| for coordinates centred to within M of the centre (every
// coordinate), d of them, with u16 the unit roundoff of the half type:
//   centring to FP32              8 sqrt(d) 2^-24 M (2 sqrt(d) M)
//   hi/lo split + dropped lo.lo   2 d M^2 (2 u16^2 + 2^-22) + 2 d 2^-24 M   (x2 for -2x.y)
//   FP32 accumulation of 48 terms 2 * 48 * 2^-24 * 2 d M^2, times 4 for an unknown order
//   norms (two sums of d squares) 2 d 2^-24 d M^2
//   epilogue (two roundings)      3 2^-24 (4 d M^2)
__host__ __device__ inline double tc_error_bound(double M, int d, bool bf16) {
  const double u16 = bf16 ? 0x1.0p-8 : 0x1.0p-11;
  const double u32 = 0x1.0p-24;
  const double dd = (double)d, M2 = M * M;
  return 8.0 * sqrt(dd) * u32 * M * 2.0 * sqrt(dd) * M +
         2.0 * (2.0 * dd * M2 * (2.0 * u16 * u16 + 0x1.0p-22) + 2.0 * dd * 0x1.0p-25 * M) +
         4.0 * 2.0 * 48.0 * u32 * 2.0 * dd * M2 + 2.0 * dd * u32 * dd * M2 +
         3.0 * u32 * 4.0 * dd * M2;
}

// The bound when the norms ride in the MMA (A = [-2x, |x|^2 hi, lo, 1, 1], B = [x, 1, 1,
// |y|^2 hi, lo], so that the accumulator holds d^2 itself): the centring and the split of the
// coordinates as above; each norm's FP32 sum (d 2^-24 d M^2) and its split into hi + lo
// (u16^2 d M^2, plus 2^-25 for a subnormal half); the FP32 accumulation of 52 terms whose
// magnitudes sum to at most 10 d M^2, times 4 for an unknown order; no epilogue arithmetic.
__host__ __device__ inline double tc_error_bound_folded(double M, int d, bool bf16) {
  const double u16 = bf16 ? 0x1.0p-8 : 0x1.0p-11;
  const double u32 = 0x1.0p-24;
  const double dd = (double)d, M2 = M * M;
  return 8.0 * sqrt(dd) * u32 * M * 2.0 * sqrt(dd) * M +
         2.0 * (2.0 * dd * M2 * (2.0 * u16 * u16 + 0x1.0p-22) + 2.0 * dd * 0x1.0p-25 * M) +
         2.0 * (dd * u32 * dd * M2 + u16 * u16 * dd * M2 + 0x1.0p-25) +
         4.0 * 52.0 * u32 * 10.0 * dd * M2;
}

}  // namespace rtg
