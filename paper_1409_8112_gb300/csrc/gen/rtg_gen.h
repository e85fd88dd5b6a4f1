/* Seeded synthetic inputs for randomly transformed grids (RTG).
 *
 * This module only draws random numbers and lays them out: point sets, the m random
 * rotations + shifts of Sec. III (Alg. 1 (grid set-up) and the rotated variant), the radius
 * for a target expected degree, and request traces.  It holds none of the method's
 * arithmetic (no cell keys, no distances, no dedupe), so both the CPU oracle's tests
 * and the GPU library may draw their inputs from it.
 *
 * Generators (published definitions, written out here):
 *   SplitMix64   - Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 *                  OOPSLA 2014 (used only to seed xoshiro256**).
 *   xoshiro256** - Blackman, Vigna, "Scrambled linear pseudorandom number generators",
 *                  ACM TOMS 2021.
 *   Box-Muller   - Box, Muller, Ann. Math. Statist. 1958 (both outputs used).
 *   Haar O(d)    - QR of a d x d standard Gaussian matrix with the diagonal of R made
 *                  positive (Mezzadri, Notices AMS 2007); QR by Householder reflections.
 */
#ifndef RTG_GEN_H
#define RTG_GEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Flags for transform generation (same bit values as the library's RTG_FLAG_*). */
#define RTG_GEN_SHIFT_ONLY 1u /* R = identity: the shift-only grids of Alg. 1 */

/* Stream tags: one independent xoshiro256** stream per (seed, tag). */
#define RTG_GEN_TAG_POINTS 1u
#define RTG_GEN_TAG_TRANSFORMS 2u
#define RTG_GEN_TAG_MIXTURE 3u
#define RTG_GEN_TAG_TRACE 4u

typedef struct { uint64_t s[4]; } rtg_gen_rng;

void rtg_gen_rng_init(rtg_gen_rng* g, uint64_t seed, uint64_t tag);
uint64_t rtg_gen_next(rtg_gen_rng* g);
double rtg_gen_uniform(rtg_gen_rng* g);      /* [0,1), 53-bit grid */
float rtg_gen_uniform_f32(rtg_gen_rng* g);   /* [0,1), 24-bit grid */
void rtg_gen_normal2(rtg_gen_rng* g, double* z0, double* z1);

/* m transforms, each R (d*d, row-major) followed by the shift s (d), s_k = c * U[0,1).
 * out must hold m*(d*d+d) doubles.  Returns 0, or -1 on invalid arguments. */
int rtg_gen_transforms(uint64_t seed, int d, int m, double cell_side, uint32_t flags,
                       double* out);

/* n points i.i.d. uniform in [0,1)^d, row-major.  dtype 0: double, 1: float. */
int rtg_gen_points_uniform(uint64_t seed, int64_t n, int d, int dtype, void* out);

/* n points from a mixture of k isotropic Gaussians (means uniform in [lo,hi]^d,
 * standard deviation sigma), each coordinate clipped to [0,1].  dtype as above. */
int rtg_gen_points_mixture(uint64_t seed, int64_t n, int d, int k, double sigma, double lo,
                           double hi, int dtype, void* out);

/* Radius whose expected ball population under a uniform density on the unit cube is
 * `degree` points: r = (degree / (n * zeta_d))^(1/d), zeta_d = pi^(d/2) / Gamma(d/2+1). */
double rtg_gen_radius_for_degree(int64_t n, int d, double degree);

#ifdef __cplusplus
}
#endif
#endif
