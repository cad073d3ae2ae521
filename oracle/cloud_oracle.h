/*
 * cloud_oracle.h -- plain FP64 CPU oracle for the volumetric-cloud raymarch
 * and temporal anti-aliasing resolve of "Optimisations for Real-Time
 * Volumetric Cloudscapes" (Toft, Bowles, Zimmermann, arXiv 1609.05344).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library; it
 * is slow on purpose, evaluates every formula directly in double precision,
 * and shares no code, header, table or constant with the CUDA path.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent the oracle takes a fixed reading; those readings are marked
 * [reading] and are the same ones the CUDA library documents.
 *
 * Parity pins (what ties this oracle to something other than itself) live in
 * tests/test_oracle_*.py: homogeneous-slab closed form, telescoping identity,
 * Henyey-Greenstein normalisation and mean cosine by quadrature, step-count
 * convergence, lattice exactness and periodicity of the noise, closed-form
 * camera motion, and the TAA identities.
 */
#ifndef CLOUD_ORACLE_H
#define CLOUD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Density modes of a volume. */
#define ORC_DENSITY_NOISE    0 /* fBm noise field (normal operation)            */
#define ORC_DENSITY_CONSTANT 1 /* rho = constant everywhere (closed-form pins)  */

/* Jitter of the start offset (Sec. 3.2; Sec. 4 compares the two). */
#define ORC_JITTER_PER_PIXEL 0 /* a random offset per pixel and frame             */
#define ORC_JITTER_PER_FRAME 1 /* one offset per frame, shared by every ray       */

/* Per-step integration rules, Sec. 3.1. */
#define ORC_INTEGRATE_ANALYTIC 0 /* S = T0 L int_0^D e^{-rho alpha x} dx       */
#define ORC_INTEGRATE_BASIC    1 /* S = T L, transmittance updated first        */

typedef struct {
    uint32_t seed;
    int base_n;            /* base lattice edge, power of two >= 16             */
    int detail_n;          /* detail lattice edge, power of two >= 16, or 0     */
    int weather_n;         /* weather map edge, power of two >= 16, or 0        */
    double detail_weight;  /* weight of the subtracted detail noise            */
    double base_period;    /* metres covered by one base tile                  */
    double detail_period;  /* metres covered by one detail tile                */
    double weather_period; /* metres covered by one weather tile               */
    double coverage;       /* coverage threshold c of the remap                */
    double slab_lo;        /* cloud layer bottom altitude (m)                  */
    double slab_hi;        /* cloud layer top altitude (m)                     */
    int density_mode;      /* ORC_DENSITY_*                                    */
    double constant_density;
} orc_volume_desc;

typedef struct {
    orc_volume_desc d;
    double *base;    /* base_n^3, x fastest, fBm value in [0,1)             */
    double *detail;  /* detail_n^3 or NULL                                   */
    double *weather; /* weather_n^2 or NULL                                  */
} orc_volume;

/* Pinhole camera.  forward/right/up orthonormal, z is up; pixel row y = 0 is
 * the top row of the image. */
typedef struct {
    double pos[3];
    double forward[3];
    double right[3];
    double up[3];
    double tan_half_fovy;
} orc_camera;

typedef struct {
    double sun_dir[3];      /* direction towards the sun (normalised here)     */
    double sun_radiance[3]; /* colour x intensity of the light source          */
    double ambient[3];      /* constant ambient radiance                       */
    double hg_g;            /* Henyey-Greenstein asymmetry                     */
    double absorption;      /* alpha, per metre at density 1                   */
    double light_step;      /* light-march step length (m)                     */
    double tau_max;         /* early-out optical depth; <= 0 disables early out*/
    double t_max;           /* far clip of a view ray (m)                       */
    int jitter_mode;        /* ORC_JITTER_PER_PIXEL or ORC_JITTER_PER_FRAME      */
} orc_params;

/* Counter-based hash (PCG output permutation over one LCG step; Jarzynski and
 * Olano, JCGT 2020): the generator behind the Sec. 3.2 start offsets and the
 * noise lattice. */
uint32_t orc_pcg(uint32_t v);
uint32_t orc_hash4(uint32_t a, uint32_t b, uint32_t c, uint32_t d);
double orc_unit(uint32_t h); /* (h >> 8) * 2^-24, in [0,1) */
void orc_hash4_batch(const uint32_t *keys /* n x 4 */, long n, uint32_t *out);

/* Noise volumes: the density field Sec. 1 samples at every step ([reading]:
 * value-noise fBm tiles, coverage remap, weather map, height profile). */
int orc_volume_build(const orc_volume_desc *desc, orc_volume *vol);
void orc_volume_free(orc_volume *vol);
double orc_fbm3(uint32_t seed, uint32_t salt, int n, int kx, int ky, int kz);
double orc_fbm2(uint32_t seed, uint32_t salt, int n, int kx, int ky);
double orc_height_gradient(const orc_volume_desc *d, double z);
double orc_density(const orc_volume *vol, const double p[3]);

/* Scattering: the Henyey-Greenstein phase function Sec. 1 names. */
double orc_hg(double mu, double g);

/* Geometry: one pinhole ray per pixel and the cloud layer it crosses
 * (Sec. 1); the per-pixel / per-frame start offset (Sec. 3.2, Sec. 4). */
void orc_pixel_ray(const orc_camera *cam, int width, int height, int x, int y, double d[3]);
int orc_slab_clip(const orc_volume_desc *d, const orc_params *prm, const double o[3],
                  const double dir[3], double *t0, double *t1);
double orc_jitter(uint32_t seed, int x, int y, int frame);

/* Raymarch of one pixel (Sec. 1 march and light march, Sec. 3.1 per-step
 * integral, Sec. 3.2 start offset); out = premultiplied RGBA; *lookups counts
 * density evaluations.  jitter_frame < 0 puts every sample at the middle of
 * its step. */
void orc_render_pixel(const orc_volume *vol, const orc_camera *cam, const orc_params *prm,
                      int width, int height, int x, int y, int steps, int light_steps,
                      int jitter_frame, int integration, double out[4], long long *lookups);

/* Whole image (row-major, 4 doubles per pixel) on nthreads host threads. */
long long orc_render(const orc_volume *vol, const orc_camera *cam, const orc_params *prm,
                     int width, int height, int steps, int light_steps, int jitter_frame,
                     int integration, int nthreads, double *out);

/* A list of pixels (xs[i], ys[i]); out is n x 4. */
long long orc_render_pixels(const orc_volume *vol, const orc_camera *cam,
                            const orc_params *prm, int width, int height, int steps,
                            int light_steps, int jitter_frame, int integration,
                            const int *xs, const int *ys, int n, int nthreads, double *out);

/* Screen-space motion of each pixel from the previous camera to the current
 * one, in pixels (the reprojection the TAA of Sec. 3.2 needs): m = current
 * pixel centre - its reprojection in prev. */
void orc_motion_pixel(const orc_volume_desc *d, const orc_params *prm, const orc_camera *prev,
                      const orc_camera *cur, int width, int height, int x, int y, double m[2]);
void orc_motion(const orc_volume_desc *d, const orc_params *prm, const orc_camera *prev,
                const orc_camera *cur, int width, int height, double *motion);

/* TAA resolve of one pixel (Sec. 3.2).  history may be NULL (first frame). */
void orc_taa_pixel(const double *history, const double *current, const double *motion,
                   int width, int height, int x, int y, double blend, int clamp, double out[4]);
void orc_taa(const double *history, const double *current, const double *motion, int width,
             int height, double blend, int clamp, double *out);

/* Composite (Sec. 3.2: the resolved low-resolution buffer goes into the
 * scene; [reading] bilinear resample and premultiplied "over").  cloud: sw x sh premultiplied RGBA; bg and out:
 * dw x dh RGBA.  out = C + (1 - C.a) bg with C the bilinear sample of cloud at
 * ((x + 1/2) sw/dw - 1/2, (y + 1/2) sh/dh - 1/2), clamp to edge. */
void orc_composite(const double *cloud, int sw, int sh, const double *bg, int dw, int dh,
                   double *out);

#ifdef __cplusplus
}
#endif
#endif
