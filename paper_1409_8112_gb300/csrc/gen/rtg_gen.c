/* Seeded synthetic inputs; see rtg_gen.h for the generator references. */
#include "rtg_gen.h"

#include <math.h>
#include <stddef.h>

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

void rtg_gen_rng_init(rtg_gen_rng* g, uint64_t seed, uint64_t tag) {
  /* The tag is folded into the SplitMix64 state so that each (seed, tag) pair starts an
   * unrelated stream; the four outputs then seed xoshiro256** (never all zero). */
  uint64_t x = seed ^ (0xd1b54a32d192ed03ULL * (tag + 1));
  for (int i = 0; i < 4; ++i) g->s[i] = splitmix64_next(&x);
}

uint64_t rtg_gen_next(rtg_gen_rng* g) {
  uint64_t* s = g->s;
  const uint64_t out = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

double rtg_gen_uniform(rtg_gen_rng* g) {
  return (double)(rtg_gen_next(g) >> 11) * 0x1.0p-53;
}

float rtg_gen_uniform_f32(rtg_gen_rng* g) {
  return (float)(rtg_gen_next(g) >> 40) * 0x1.0p-24f;
}

void rtg_gen_normal2(rtg_gen_rng* g, double* z0, double* z1) {
  const double two_pi = 6.283185307179586476925286766559;
  double u1 = 1.0 - rtg_gen_uniform(g); /* (0,1] so the log is finite */
  double u2 = rtg_gen_uniform(g);
  double rad = sqrt(-2.0 * log(u1));
  *z0 = rad * cos(two_pi * u2);
  *z1 = rad * sin(two_pi * u2);
}

/* Householder QR of the d x d matrix a (row-major, overwritten by R in its upper part);
 * q receives the orthogonal factor.  Then columns of q are multiplied by sign(R_kk)
 * (sign(0) = +1) so that R has a non-negative diagonal, which makes q Haar-distributed
 * when a is standard Gaussian. */
static void haar_from_gaussian(int d, double* a, double* q) {
  double v[16];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) q[i * d + j] = (i == j) ? 1.0 : 0.0;
  for (int k = 0; k + 1 < d; ++k) {
    double norm2 = 0.0;
    for (int i = k; i < d; ++i) norm2 += a[i * d + k] * a[i * d + k];
    double norm = sqrt(norm2);
    if (norm == 0.0) continue;
    double alpha = (a[k * d + k] >= 0.0) ? -norm : norm;
    double vn2 = 0.0;
    for (int i = k; i < d; ++i) {
      v[i - k] = a[i * d + k] - (i == k ? alpha : 0.0);
      vn2 += v[i - k] * v[i - k];
    }
    if (vn2 == 0.0) continue;
    /* a <- H a on rows k.., columns k.. */
    for (int j = k; j < d; ++j) {
      double dot = 0.0;
      for (int i = k; i < d; ++i) dot += v[i - k] * a[i * d + j];
      double f = 2.0 * dot / vn2;
      for (int i = k; i < d; ++i) a[i * d + j] -= f * v[i - k];
    }
    /* q <- q H on columns k.. */
    for (int i = 0; i < d; ++i) {
      double dot = 0.0;
      for (int l = k; l < d; ++l) dot += q[i * d + l] * v[l - k];
      double f = 2.0 * dot / vn2;
      for (int l = k; l < d; ++l) q[i * d + l] -= f * v[l - k];
    }
  }
  for (int k = 0; k < d; ++k) {
    if (a[k * d + k] < 0.0)
      for (int i = 0; i < d; ++i) q[i * d + k] = -q[i * d + k];
  }
}

int rtg_gen_transforms(uint64_t seed, int d, int m, double cell_side, uint32_t flags,
                       double* out) {
  if (d < 1 || d > 16 || m < 1 || !(cell_side > 0.0) || out == NULL) return -1;
  rtg_gen_rng g;
  rtg_gen_rng_init(&g, seed, RTG_GEN_TAG_TRANSFORMS);
  const int stride = d * d + d;
  double a[256];
  for (int t = 0; t < m; ++t) {
    double* R = out + (size_t)t * stride;
    double* s = R + d * d;
    if (flags & RTG_GEN_SHIFT_ONLY) {
      for (int i = 0; i < d * d; ++i) R[i] = (i % (d + 1) == 0) ? 1.0 : 0.0;
    } else {
      for (int i = 0; i < d * d; i += 2) {
        double z0, z1;
        rtg_gen_normal2(&g, &z0, &z1);
        a[i] = z0;
        if (i + 1 < d * d) a[i + 1] = z1;
      }
      haar_from_gaussian(d, a, R);
    }
    for (int k = 0; k < d; ++k) s[k] = cell_side * rtg_gen_uniform(&g);
  }
  return 0;
}

int rtg_gen_points_uniform(uint64_t seed, int64_t n, int d, int dtype, void* out) {
  if (n < 0 || d < 1 || out == NULL || (dtype != 0 && dtype != 1)) return -1;
  rtg_gen_rng g;
  rtg_gen_rng_init(&g, seed, RTG_GEN_TAG_POINTS);
  const int64_t total = n * (int64_t)d;
  if (dtype == 0) {
    double* p = (double*)out;
    for (int64_t i = 0; i < total; ++i) p[i] = rtg_gen_uniform(&g);
  } else {
    float* p = (float*)out;
    for (int64_t i = 0; i < total; ++i) p[i] = rtg_gen_uniform_f32(&g);
  }
  return 0;
}

int rtg_gen_points_mixture(uint64_t seed, int64_t n, int d, int k, double sigma, double lo,
                           double hi, int dtype, void* out) {
  if (n < 0 || d < 1 || d > 64 || k < 1 || k > 1024 || out == NULL ||
      (dtype != 0 && dtype != 1))
    return -1;
  rtg_gen_rng gm, gp;
  rtg_gen_rng_init(&gm, seed, RTG_GEN_TAG_MIXTURE);
  rtg_gen_rng_init(&gp, seed, RTG_GEN_TAG_POINTS);
  double means[1024 * 4];
  if ((int64_t)k * d > (int64_t)(sizeof means / sizeof means[0])) return -1;
  for (int i = 0; i < k * d; ++i) means[i] = lo + (hi - lo) * rtg_gen_uniform(&gm);
  double spare = 0.0;
  int have_spare = 0;
  for (int64_t i = 0; i < n; ++i) {
    int comp = (int)(rtg_gen_next(&gp) % (uint64_t)k);
    for (int l = 0; l < d; ++l) {
      double z;
      if (have_spare) {
        z = spare;
        have_spare = 0;
      } else {
        rtg_gen_normal2(&gp, &z, &spare);
        have_spare = 1;
      }
      double x = means[comp * d + l] + sigma * z;
      if (x < 0.0) x = 0.0;
      if (x > 1.0) x = 1.0;
      if (dtype == 0)
        ((double*)out)[i * d + l] = x;
      else
        ((float*)out)[i * d + l] = (float)x;
    }
  }
  return 0;
}

double rtg_gen_radius_for_degree(int64_t n, int d, double degree) {
  const double pi = 3.14159265358979323846264338327950288;
  double zeta = pow(pi, 0.5 * d) / tgamma(0.5 * d + 1.0);
  return pow(degree / ((double)n * zeta), 1.0 / d);
}
