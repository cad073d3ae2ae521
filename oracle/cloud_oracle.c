/*
 * cloud_oracle.c -- plain FP64 CPU oracle (test infrastructure only; see
 * cloud_oracle.h).  Every quantity is computed directly from its definition
 * in double precision, with no blocking, fusion, caching or early skipping
 * beyond what the method itself states.
 *
 * Paper passages followed (Toft, Bowles, Zimmermann, arXiv 1609.05344):
 *   Sec. 1   one ray per pixel marched through the volume, density taken at
 *            each step, colour and alpha accumulated, march ended once alpha
 *            is one or the ray has left the volume; running transmittance by Beer-Lambert; a second march
 *            towards the sun per step; light colour x intensity x
 *            Henyey-Greenstein phase, plus an ambient term.
 *   Sec. 3.1 basic rule S = T L versus the analytic rule
 *            S = T0 L int_0^D e^{-rho alpha x} dx = T0 L (1 - e^{-rho alpha D}) / (rho alpha),
 *            density constant over a step (the printed last line has x where
 *            the evaluated bound D belongs; D is used here).
 *   Sec. 3.2 random per-pixel offset of the raymarch start, changed every
 *            frame; TAA (reprojected history, neighbourhood clamp, blend) on
 *            the cloud buffer.
 * Everything the paper does not fix is a [reading] listed in the design notes
 * of this repository; each is marked below.
 */
#include "cloud_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Counter-based hash.  [reading] The paper only asks for a random per-pixel
 * offset (Sec. 3.2).  The generator is the single-state PCG hash of Jarzynski
 * and Olano, "Hash Functions for GPU Rendering" (JCGT 9(3), 2020): one step of
 * the 32-bit PCG linear congruential generator (multiplier 747796405,
 * increment 2891336453, O'Neill 2014) followed by the RXS-M-XS output
 * permutation (multiplier 277803737). */
uint32_t orc_pcg(uint32_t v) {
    uint32_t state = v * 747796405u + 2891336453u;
    uint32_t rot = (state >> 28) + 4u;
    uint32_t word = ((state >> rot) ^ state) * 277803737u;
    return (word >> 22) ^ word;
}

/* Four-word key, nested: h(a,b,c,d) = pcg(a ^ pcg(b ^ pcg(c ^ pcg(d)))). */
uint32_t orc_hash4(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    uint32_t h = orc_pcg(d);
    h = orc_pcg(c ^ h);
    h = orc_pcg(b ^ h);
    h = orc_pcg(a ^ h);
    return h;
}

/* Top 24 bits as a uniform number in [0,1); exact in FP32 and FP64. */
double orc_unit(uint32_t h) { return (double)(h >> 8) * (1.0 / 16777216.0); }

void orc_hash4_batch(const uint32_t *keys, long n, uint32_t *out) {
    for (long i = 0; i < n; ++i)
        out[i] = orc_hash4(keys[4 * i], keys[4 * i + 1], keys[4 * i + 2], keys[4 * i + 3]);
}

/* ------------------------------------------------------------------------ */
/* Value-noise fBm volumes.  [reading] Sec. 1 samples a cloud density at
 * every step without defining the field.  The field is four octaves of
 * value noise: hashed uniform lattice values, plain trilinear interpolation,
 * octave o has M_o = (N/16) 2^o cells per tile and amplitude 2^-o, and the
 * sum is divided by the total amplitude.  Voxel k stores the noise at lattice
 * coordinate k M_o / N; lattice indices wrap modulo M_o so the tile repeats. */
#define ORC_OCTAVES 4
#define ORC_SALT_BASE 0xB45Eu
#define ORC_SALT_DETAIL 0xDE7Au
#define ORC_SALT_WEATHER 0x3EA7u
#define ORC_OCTAVE_KEY 0x9E37u
#define ORC_JITTER_KEY 0x4A17u

static int wrap_index(long long i, int m) {
    long long r = i % m;
    return (int)(r < 0 ? r + m : r);
}

static double lattice3(uint32_t key, int m, long long ix, long long iy, long long iz) {
    return orc_unit(orc_hash4((uint32_t)wrap_index(ix, m), (uint32_t)wrap_index(iy, m),
                              (uint32_t)wrap_index(iz, m), key));
}

static double lattice2(uint32_t key, int m, long long ix, long long iy) {
    return orc_unit(orc_hash4((uint32_t)wrap_index(ix, m), (uint32_t)wrap_index(iy, m), 0u, key));
}

double orc_fbm3(uint32_t seed, uint32_t salt, int n, int kx, int ky, int kz) {
    double sum = 0.0, amp_sum = 0.0, amp = 1.0;
    for (int o = 0; o < ORC_OCTAVES; ++o) {
        int m = (n / 16) << o;
        uint32_t key = seed ^ ((uint32_t)o * ORC_OCTAVE_KEY) ^ salt;
        double cx = (double)kx * m / n, cy = (double)ky * m / n, cz = (double)kz * m / n;
        double fx0 = floor(cx), fy0 = floor(cy), fz0 = floor(cz);
        long long ix = (long long)fx0, iy = (long long)fy0, iz = (long long)fz0;
        double fx = cx - fx0, fy = cy - fy0, fz = cz - fz0;
        double v = 0.0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
                    v += w * lattice3(key, m, ix + dx, iy + dy, iz + dz);
                }
        sum += amp * v;
        amp_sum += amp;
        amp *= 0.5;
    }
    return sum / amp_sum;
}

double orc_fbm2(uint32_t seed, uint32_t salt, int n, int kx, int ky) {
    double sum = 0.0, amp_sum = 0.0, amp = 1.0;
    for (int o = 0; o < ORC_OCTAVES; ++o) {
        int m = (n / 16) << o;
        uint32_t key = seed ^ ((uint32_t)o * ORC_OCTAVE_KEY) ^ salt;
        double cx = (double)kx * m / n, cy = (double)ky * m / n;
        double fx0 = floor(cx), fy0 = floor(cy);
        long long ix = (long long)fx0, iy = (long long)fy0;
        double fx = cx - fx0, fy = cy - fy0;
        double v = 0.0;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
                v += w * lattice2(key, m, ix + dx, iy + dy);
            }
        sum += amp * v;
        amp_sum += amp;
        amp *= 0.5;
    }
    return sum / amp_sum;
}

static int is_pow2_at_least16(int n) { return n >= 16 && (n & (n - 1)) == 0; }

int orc_volume_build(const orc_volume_desc *desc, orc_volume *vol) {
    memset(vol, 0, sizeof(*vol));
    vol->d = *desc;
    if (desc->density_mode == ORC_DENSITY_CONSTANT) return 0;
    if (!is_pow2_at_least16(desc->base_n)) return -1;
    if (desc->detail_n && !is_pow2_at_least16(desc->detail_n)) return -1;
    if (desc->weather_n && !is_pow2_at_least16(desc->weather_n)) return -1;
    int n = desc->base_n;
    vol->base = (double *)malloc(sizeof(double) * (size_t)n * n * n);
    if (!vol->base) return -2;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x)
                vol->base[((size_t)z * n + y) * n + x] = orc_fbm3(desc->seed, ORC_SALT_BASE, n, x, y, z);
    if (desc->detail_n) {
        int m = desc->detail_n;
        vol->detail = (double *)malloc(sizeof(double) * (size_t)m * m * m);
        if (!vol->detail) return -2;
        for (int z = 0; z < m; ++z)
            for (int y = 0; y < m; ++y)
                for (int x = 0; x < m; ++x)
                    vol->detail[((size_t)z * m + y) * m + x] =
                        orc_fbm3(desc->seed, ORC_SALT_DETAIL, m, x, y, z);
    }
    if (desc->weather_n) {
        int m = desc->weather_n;
        vol->weather = (double *)malloc(sizeof(double) * (size_t)m * m);
        if (!vol->weather) return -2;
        for (int y = 0; y < m; ++y)
            for (int x = 0; x < m; ++x)
                vol->weather[(size_t)y * m + x] = orc_fbm2(desc->seed, ORC_SALT_WEATHER, m, x, y);
    }
    return 0;
}

void orc_volume_free(orc_volume *vol) {
    free(vol->base);
    free(vol->detail);
    free(vol->weather);
    vol->base = vol->detail = vol->weather = NULL;
}

/* Trilinear, wrapped sampling of an n^3 tile spanning `period` metres; texel
 * k sits at (k + 1/2) period / n. */
static double sample3(const double *v, int n, double period, const double p[3]) {
    long long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double s = p[a] / period * n - 0.5;
        double fl = floor(s);
        i0[a] = (long long)fl;
        f[a] = s - fl;
    }
    double r = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
                int x = wrap_index(i0[0] + dx, n), y = wrap_index(i0[1] + dy, n),
                    z = wrap_index(i0[2] + dz, n);
                r += w * v[((size_t)z * n + y) * n + x];
            }
    return r;
}

static double sample2(const double *v, int n, double period, double px, double py) {
    double sx = px / period * n - 0.5, sy = py / period * n - 0.5;
    double flx = floor(sx), fly = floor(sy);
    long long ix = (long long)flx, iy = (long long)fly;
    double fx = sx - flx, fy = sy - fly;
    double r = 0.0;
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy);
            r += w * v[(size_t)wrap_index(iy + dy, n) * n + wrap_index(ix + dx, n)];
        }
    return r;
}

/* [reading] Vertical profile over the cloud layer: h = (z - lo)/(hi - lo),
 * g(h) = clamp(h/0.1, 0, 1) * clamp((1-h)/0.4, 0, 1); zero outside the layer. */
double orc_height_gradient(const orc_volume_desc *d, double z) {
    double h = (z - d->slab_lo) / (d->slab_hi - d->slab_lo);
    double a = h / 0.1, b = (1.0 - h) / 0.4;
    a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
    b = b < 0.0 ? 0.0 : (b > 1.0 ? 1.0 : b);
    return a * b;
}

/* Density at a point (Sec. 1: sampled at every step).  [reading]
 * rho = g(z) * W(x,y) * max(0, (B - w_d Dt - c) / (1 - c)), with B the base
 * noise, Dt the detail noise (absent: 0), W the weather map (absent: 1) and c
 * the coverage threshold.  The constant mode returns rho0 everywhere. */
double orc_density(const orc_volume *vol, const double p[3]) {
    const orc_volume_desc *d = &vol->d;
    if (d->density_mode == ORC_DENSITY_CONSTANT) return d->constant_density;
    double g = orc_height_gradient(d, p[2]);
    double b = sample3(vol->base, d->base_n, d->base_period, p);
    double dt = vol->detail ? sample3(vol->detail, d->detail_n, d->detail_period, p) : 0.0;
    double w = vol->weather ? sample2(vol->weather, d->weather_n, d->weather_period, p[0], p[1]) : 1.0;
    double r = (b - d->detail_weight * dt - d->coverage) / (1.0 - d->coverage);
    if (r < 0.0) r = 0.0;
    return g * w * r;
}

/* ------------------------------------------------------------------------ */
/* Henyey-Greenstein phase function (Sec. 1 names it; the formula is the
 * standard one): p(mu) = (1 - g^2) / (4 pi (1 + g^2 - 2 g mu)^{3/2}), mu the
 * cosine between the view direction and the direction towards the sun. */
double orc_hg(double mu, double g) {
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * M_PI * den * sqrt(den));
}

/* ------------------------------------------------------------------------ */
/* Pinhole rays, one per pixel (Sec. 1).  [reading]
 * d = normalize(F + a R + b U), a = (2(x+1/2)/W - 1) (W/H) tan(fovy/2),
 * b = (1 - 2(y+1/2)/H) tan(fovy/2). */
void orc_pixel_ray(const orc_camera *cam, int width, int height, int x, int y, double d[3]) {
    double aspect = (double)width / (double)height;
    double a = (2.0 * (x + 0.5) / width - 1.0) * aspect * cam->tan_half_fovy;
    double b = (1.0 - 2.0 * (y + 0.5) / height) * cam->tan_half_fovy;
    double v[3], n2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        v[k] = cam->forward[k] + a * cam->right[k] + b * cam->up[k];
        n2 += v[k] * v[k];
    }
    double n = sqrt(n2);
    for (int k = 0; k < 3; ++k) d[k] = v[k] / n;
}

/* [reading] The cloud volume is the horizontal layer slab_lo <= z <= slab_hi,
 * cut at distance t_max.  Returns 1 and [t0, t1] when the ray crosses it. */
int orc_slab_clip(const orc_volume_desc *d, const orc_params *prm, const double o[3],
                  const double dir[3], double *t0, double *t1) {
    double a, b;
    if (fabs(dir[2]) < 1e-8) {
        if (o[2] < d->slab_lo || o[2] > d->slab_hi) return 0;
        a = 0.0;
        b = prm->t_max;
    } else {
        double tl = (d->slab_lo - o[2]) / dir[2];
        double th = (d->slab_hi - o[2]) / dir[2];
        double lo = tl < th ? tl : th, hi = tl < th ? th : tl;
        a = lo > 0.0 ? lo : 0.0;
        b = hi < prm->t_max ? hi : prm->t_max;
    }
    *t0 = a;
    *t1 = b;
    return b > a;
}

/* Per-pixel, per-frame start offset in [0,1) of a step (Sec. 3.2). */
double orc_jitter(uint32_t seed, int x, int y, int frame) {
    return orc_unit(orc_hash4((uint32_t)x, (uint32_t)y, (uint32_t)frame, seed ^ ORC_JITTER_KEY));
}

static void unit_sun(const orc_params *prm, double s[3]) {
    double n = sqrt(prm->sun_dir[0] * prm->sun_dir[0] + prm->sun_dir[1] * prm->sun_dir[1] +
                    prm->sun_dir[2] * prm->sun_dir[2]);
    for (int k = 0; k < 3; ++k) s[k] = prm->sun_dir[k] / n;
}

/* ------------------------------------------------------------------------ */
/* Raymarch of one pixel (Sec. 1 and Sec. 3.1).
 *   D = (t1 - t0)/N; sample i at t0 + (i + u) D, u the jitter (1/2 without;
 *   in per-frame mode the offset of pixel (0, 0) for every pixel).
 *   Light march (Sec. 1): Ls samples at p + (j + 1/2) dl s,
 *     tau_sun = alpha sum_j rho_j dl, only where rho_i > 0 (the step adds
 *     nothing otherwise).
 *   Lighting (Sec. 1): L_in = E_sun e^{-tau_sun} p_HG(d.s) + A.
 *   [reading] L of Sec. 3.1 is the in-scattered radiance per metre,
 *     L = sigma L_in with sigma = alpha rho (single-scattering albedo 1), so
 *     the analytic step (Sec. 3.1, bound D) is
 *       C += e^{-tau} L_in (1 - e^{-sigma D}),  tau += sigma D
 *     and in the basic step the transmittance is first advanced over the
 *     step and the advanced value then weights the step's light:
 *       tau += sigma D,  C += e^{-tau} sigma L_in D.
 *   Transmittance is e^{-tau} with tau the optical-depth sum (Beer-Lambert).
 *   [reading] Early out (Sec. 1: the march ends once alpha is one): stop after the
 *     step at which tau >= tau_max.  Alpha is reported as 1 - e^{-tau}. */
void orc_render_pixel(const orc_volume *vol, const orc_camera *cam, const orc_params *prm,
                      int width, int height, int x, int y, int steps, int light_steps,
                      int jitter_frame, int integration, double out[4], long long *lookups) {
    double d[3], s[3], t0, t1;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    orc_pixel_ray(cam, width, height, x, y, d);
    if (!orc_slab_clip(&vol->d, prm, cam->pos, d, &t0, &t1)) return;
    unit_sun(prm, s);
    double D = (t1 - t0) / steps;
    double u = 0.5;
    if (jitter_frame >= 0)  /* Sec. 4: per-frame mode applies one offset to every ray */
        u = prm->jitter_mode == ORC_JITTER_PER_FRAME ? orc_jitter(vol->d.seed, 0, 0, jitter_frame)
                                                     : orc_jitter(vol->d.seed, x, y, jitter_frame);
    double phase = orc_hg(d[0] * s[0] + d[1] * s[1] + d[2] * s[2], prm->hg_g);
    double tau = 0.0, c[3] = {0.0, 0.0, 0.0};
    long long n_look = 0;
    for (int i = 0; i < steps; ++i) {
        double t = t0 + (i + u) * D;
        double p[3] = {cam->pos[0] + t * d[0], cam->pos[1] + t * d[1], cam->pos[2] + t * d[2]};
        double rho = orc_density(vol, p);
        ++n_look;
        if (rho > 0.0) {
            double tau_sun = 0.0;
            for (int j = 0; j < light_steps; ++j) {
                double l = (j + 0.5) * prm->light_step;
                double q[3] = {p[0] + l * s[0], p[1] + l * s[1], p[2] + l * s[2]};
                tau_sun += prm->absorption * orc_density(vol, q) * prm->light_step;
                ++n_look;
            }
            double sigma = prm->absorption * rho;
            double sun_t = exp(-tau_sun);
            for (int k = 0; k < 3; ++k) {
                double l_in = prm->sun_radiance[k] * sun_t * phase + prm->ambient[k];
                if (integration == ORC_INTEGRATE_ANALYTIC)
                    c[k] += exp(-tau) * l_in * (-expm1(-sigma * D));
                else
                    c[k] += exp(-(tau + sigma * D)) * sigma * l_in * D;
            }
            tau += sigma * D;
        }
        if (prm->tau_max > 0.0 && tau >= prm->tau_max) break;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = -expm1(-tau);
    if (lookups) *lookups += n_look;
}

typedef struct {
    const orc_volume *vol;
    const orc_camera *cam;
    const orc_params *prm;
    int width, height, steps, light_steps, jitter_frame, integration;
    const int *xs, *ys; /* NULL: whole image */
    long n;
    int tid, nthreads;
    double *out;
    long long lookups;
} render_job;

static void *render_worker(void *arg) {
    render_job *j = (render_job *)arg;
    for (long i = j->tid; i < j->n; i += j->nthreads) {
        int x = j->xs ? j->xs[i] : (int)(i % j->width);
        int y = j->ys ? j->ys[i] : (int)(i / j->width);
        orc_render_pixel(j->vol, j->cam, j->prm, j->width, j->height, x, y, j->steps,
                         j->light_steps, j->jitter_frame, j->integration, j->out + 4 * i,
                         &j->lookups);
    }
    return NULL;
}

static long long run_render(render_job proto, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    render_job jobs[256];
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = proto;
        jobs[t].tid = t;
        jobs[t].nthreads = nthreads;
        jobs[t].lookups = 0;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    render_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    long long total = 0;
    for (int t = 0; t < nthreads; ++t) total += jobs[t].lookups;
    return total;
}

long long orc_render(const orc_volume *vol, const orc_camera *cam, const orc_params *prm,
                     int width, int height, int steps, int light_steps, int jitter_frame,
                     int integration, int nthreads, double *out) {
    render_job j = {vol, cam, prm, width, height, steps, light_steps, jitter_frame, integration,
                    NULL, NULL, (long)width * height, 0, 1, out, 0};
    return run_render(j, nthreads);
}

long long orc_render_pixels(const orc_volume *vol, const orc_camera *cam,
                            const orc_params *prm, int width, int height, int steps,
                            int light_steps, int jitter_frame, int integration,
                            const int *xs, const int *ys, int n, int nthreads, double *out) {
    render_job j = {vol, cam, prm, width, height, steps, light_steps, jitter_frame, integration,
                    xs, ys, n, 0, 1, out, 0};
    return run_render(j, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Motion vectors for the reprojection of Sec. 3.2 (Playdead-style TAA reads
 * the history at the pixel's previous screen position).  [reading] The
 * reprojected point is the ray's entry into the cloud layer, o + t0 d, when
 * the ray enters it ahead of the camera (t0 > 0); otherwise the point at
 * t_max.  Motion = current pixel centre - that point's pixel position in the
 * previous camera.  A point behind the previous camera gets 1e9 pixels,
 * which the resolve treats as off screen. */
void orc_motion_pixel(const orc_volume_desc *d, const orc_params *prm, const orc_camera *prev,
                      const orc_camera *cur, int width, int height, int x, int y, double m[2]) {
    double dir[3], t0, t1, t;
    orc_pixel_ray(cur, width, height, x, y, dir);
    if (orc_slab_clip(d, prm, cur->pos, dir, &t0, &t1) && t0 > 0.0)
        t = t0;
    else
        t = prm->t_max;
    double q[3];
    for (int k = 0; k < 3; ++k) q[k] = cur->pos[k] + t * dir[k] - prev->pos[k];
    double cx = q[0] * prev->right[0] + q[1] * prev->right[1] + q[2] * prev->right[2];
    double cy = q[0] * prev->up[0] + q[1] * prev->up[1] + q[2] * prev->up[2];
    double cz = q[0] * prev->forward[0] + q[1] * prev->forward[1] + q[2] * prev->forward[2];
    if (cz <= 0.0) {
        m[0] = m[1] = 1e9;
        return;
    }
    double aspect = (double)width / (double)height;
    double px = (cx / cz / (aspect * prev->tan_half_fovy) + 1.0) * 0.5 * width;
    double py = (1.0 - cy / cz / prev->tan_half_fovy) * 0.5 * height;
    m[0] = (x + 0.5) - px;
    m[1] = (y + 0.5) - py;
}

void orc_motion(const orc_volume_desc *d, const orc_params *prm, const orc_camera *prev,
                const orc_camera *cur, int width, int height, double *motion) {
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x)
            orc_motion_pixel(d, prm, prev, cur, width, height, x, y,
                             motion + 2 * ((size_t)y * width + x));
}

/* ------------------------------------------------------------------------ */
/* TAA resolve (Sec. 3.2, Playdead's temporal reprojection).  [reading]
 *   q = (x + 1/2, y + 1/2) - m; off screen (q outside [0,W] x [0,H]) or no
 *   history: out = c.  Otherwise h = bilinear history at q (texel centres at
 *   +1/2, clamp to edge), [mn, mx] = per-channel min/max of the 3x3
 *   neighbourhood of the current frame (clamp to edge),
 *   out = hc + blend (c - hc), hc = clamp(h, mn, mx) (h when clamp == 0). */
static int clampi(long long v, int lo, int hi) { return (int)(v < lo ? lo : (v > hi ? hi : v)); }

void orc_taa_pixel(const double *history, const double *current, const double *motion,
                   int width, int height, int x, int y, double blend, int clamp, double out[4]) {
    const double *c = current + 4 * ((size_t)y * width + x);
    if (!history) {
        for (int k = 0; k < 4; ++k) out[k] = c[k];
        return;
    }
    double mx = motion[2 * ((size_t)y * width + x)], my = motion[2 * ((size_t)y * width + x) + 1];
    double qx = x + 0.5 - mx, qy = y + 0.5 - my;
    if (qx < 0.0 || qx > width || qy < 0.0 || qy > height) {
        for (int k = 0; k < 4; ++k) out[k] = c[k];
        return;
    }
    double sx = qx - 0.5, sy = qy - 0.5;
    double flx = floor(sx), fly = floor(sy);
    double fx = sx - flx, fy = sy - fly;
    int xa = clampi((long long)flx, 0, width - 1), xb = clampi((long long)flx + 1, 0, width - 1);
    int ya = clampi((long long)fly, 0, height - 1), yb = clampi((long long)fly + 1, 0, height - 1);
    for (int k = 0; k < 4; ++k) {
        double h00 = history[4 * ((size_t)ya * width + xa) + k];
        double h01 = history[4 * ((size_t)ya * width + xb) + k];
        double h10 = history[4 * ((size_t)yb * width + xa) + k];
        double h11 = history[4 * ((size_t)yb * width + xb) + k];
        double h = (1.0 - fy) * ((1.0 - fx) * h00 + fx * h01) + fy * ((1.0 - fx) * h10 + fx * h11);
        double mn = c[k], mxv = c[k];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int nx = clampi((long long)x + dx, 0, width - 1);
                int ny = clampi((long long)y + dy, 0, height - 1);
                double v = current[4 * ((size_t)ny * width + nx) + k];
                if (v < mn) mn = v;
                if (v > mxv) mxv = v;
            }
        double hc = h;
        if (clamp) hc = h < mn ? mn : (h > mxv ? mxv : h);
        out[k] = hc + blend * (c[k] - hc);
    }
}

void orc_taa(const double *history, const double *current, const double *motion, int width,
             int height, double blend, int clamp, double *out) {
    for (int y = 0; y < height; ++y)
        for (int x = 0; x < width; ++x)
            orc_taa_pixel(history, current, motion, width, height, x, y, blend, clamp,
                          out + 4 * ((size_t)y * width + x));
}

/* ------------------------------------------------------------------------ */
/* Composite of the cloud buffer into the scene (Sec. 3.2).  [reading] The
 * buffer is resampled to the display resolution bilinearly (texel centres at
 * +1/2, clamp to edge) and, being premultiplied, laid over the background:
 * out = C + (1 - alpha_C) bg, per channel including alpha. */
void orc_composite(const double *cloud, int sw, int sh, const double *bg, int dw, int dh,
                   double *out) {
    for (int y = 0; y < dh; ++y)
        for (int x = 0; x < dw; ++x) {
            double u = (x + 0.5) * sw / dw - 0.5, v = (y + 0.5) * sh / dh - 0.5;
            double fu = floor(u), fv = floor(v);
            double fx = u - fu, fy = v - fv;
            int xa = clampi((long long)fu, 0, sw - 1), xb = clampi((long long)fu + 1, 0, sw - 1);
            int ya = clampi((long long)fv, 0, sh - 1), yb = clampi((long long)fv + 1, 0, sh - 1);
            double c[4];
            for (int k = 0; k < 4; ++k) {
                double c00 = cloud[4 * ((size_t)ya * sw + xa) + k];
                double c01 = cloud[4 * ((size_t)ya * sw + xb) + k];
                double c10 = cloud[4 * ((size_t)yb * sw + xa) + k];
                double c11 = cloud[4 * ((size_t)yb * sw + xb) + k];
                c[k] = (1.0 - fy) * ((1.0 - fx) * c00 + fx * c01) + fy * ((1.0 - fx) * c10 + fx * c11);
            }
            for (int k = 0; k < 4; ++k) {
                size_t i = 4 * ((size_t)y * dw + x) + k;
                out[i] = c[k] + (1.0 - c[3]) * bg[i];
            }
        }
}
