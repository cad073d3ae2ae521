// render.cu -- single-view raymarch launch (cloud_render) and the host-side
// construction of the launch constants (Sec. 1, Sec. 3.1, Sec. 3.2).
//
// One thread per pixel; a 128-thread CTA covers one pixel tile (shape chosen
// by the autotuner, 16x8 by default) so the rays of a warp stay adjacent and
// touch the same region of the L2-resident noise tiles.  The device code is
// in march.cuh, the kernels in march_kernels.cuh (instantiated by
// march{8,16}_{view,batch}.cu).
#include <atomic>
#include <cmath>
#include <mutex>

#include "march.cuh"

namespace cloudvol {

// Empty-space skipping through the volume's occupancy grid (on unless a test
// turns it off to compare against the full evaluation).
static std::atomic<bool> g_use_occupancy{true};

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

int build_scene(const cloud_volume *vol, const cloud_params *prm, int light_steps, int integration,
                SceneParams *p) {
    if (light_steps < 0 || light_steps > CLOUD_MAX_LIGHT_STEPS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: light_steps outside [0, 32]");
    if (integration != CLOUD_INTEGRATE_ANALYTIC && integration != CLOUD_INTEGRATE_BASIC)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: bad integration mode");
    if (prm->jitter_mode != CLOUD_JITTER_PER_PIXEL && prm->jitter_mode != CLOUD_JITTER_PER_FRAME)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: bad jitter mode");
    if (!(prm->t_max_m > 0.0 && prm->t_max_m <= 1e6) || !(prm->light_step_m >= 0.0) ||
        !(prm->absorption_per_m >= 0.0) || !(prm->hg_g > -1.0 && prm->hg_g < 1.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: bad lighting constants");
    const double sn = std::sqrt(dot3(prm->sun_dir, prm->sun_dir));
    if (!(sn > 0.0) || !(prm->sun_dir[2] > 0.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: sun direction must have z > 0");
    const cloud_volume_desc &d = vol->desc;
    const double thick = d.slab_hi_m - d.slab_lo_m;
    const double s[3] = {prm->sun_dir[0] / sn, prm->sun_dir[1] / sn, prm->sun_dir[2] / sn};
    if (thick + light_steps * prm->light_step_m * s[2] > 32000.0)
        return set_error(CLOUD_ERR_UNSUPPORTED,
                         "cloud_render: light march reaches > 32 km above the layer bottom");
    *p = SceneParams{};
    const bool noise = d.density_mode == CLOUD_DENSITY_NOISE;
    const int L[kLatticeAxes] = {vol->log2_base,    vol->log2_base,    vol->log2_base,
                                 vol->log2_detail,  vol->log2_detail,  vol->log2_detail,
                                 vol->log2_weather, vol->log2_weather};
    const double P[kLatticeAxes] = {d.base_period_m,    d.base_period_m,    d.base_period_m,
                                    d.detail_period_m,  d.detail_period_m,  d.detail_period_m,
                                    d.weather_period_m, d.weather_period_m};
    for (int a = 0; a < kLatticeAxes; ++a) {
        const int comp = a < 6 ? a % 3 : a - 6;
        if (!noise || L[a] == 0) continue;  // absent tile: axis unused
        const double kfix = 4294967296.0 / P[a];  // 2^32 fixed-point units per tile
        split_df(kfix, &p->kfix_h[a], &p->kfix_l[a]);
        p->half_unit[a] = 1u << (31 - L[a]);
        for (int j = 0; j < light_steps; ++j) {
            const double off = (j + 0.5) * prm->light_step_m * s[comp] * kfix;
            p->loff[j][a] = (uint32_t)(unsigned long long)std::llrint(off);
        }
    }
    for (int j = 0; j < light_steps; ++j)
        p->lh[j] = (int32_t)std::llrint((j + 0.5) * prm->light_step_m * s[2] * 65536.0);
    p->h_top = (int32_t)std::llrint(thick * 65536.0);
    p->h_lo_scale = (float)(10.0 / (thick * 65536.0));
    p->h_hi_scale = (float)(2.5 / (thick * 65536.0));
    for (int k = 0; k < 3; ++k) {
        p->sun[k] = (float)s[k];
        p->sun_rad[k] = (float)prm->sun_radiance[k];
        p->ambient[k] = (float)prm->ambient[k];
    }
    p->hg_g = (float)prm->hg_g;
    p->hg_norm = (float)((1.0 - prm->hg_g * prm->hg_g) / (4.0 * M_PI));
    p->absorption = (float)prm->absorption_per_m;
    p->light_step = (float)prm->light_step_m;
    p->tau_max = prm->tau_max > 0.0 ? (float)prm->tau_max : INFINITY;
    const double wd = vol->log2_detail ? d.detail_weight : 0.0;
    p->detail_w = (float)wd;
    const double bias = texel_bias_of(d.precision);
    p->k0 = (float)(0.5 - d.coverage - 0.5 * wd - bias + wd * bias);
    p->w_off = (float)(0.5 - bias);
    p->inv_1mc = (float)(1.0 / (1.0 - d.coverage));
    p->rho0 = (float)d.constant_density;
    p->occ = noise && g_use_occupancy.load() ? vol->occ : nullptr;
    p->log2_occ = vol->log2_occ;
    p->check = check_word();
    p->log2_base = vol->log2_base;
    p->log2_detail = vol->log2_detail;
    p->log2_weather = vol->log2_weather;
    p->light_steps = light_steps;
    p->integration = integration;
    p->constant_mode = noise ? 0 : 1;
    p->detail_shift = -1;
    if (vol->log2_detail) {
        const double ratio = d.base_period_m / d.detail_period_m;
        for (int k = 0; k <= 16; ++k)
            if (ratio == std::ldexp(1.0, k)) p->detail_shift = k;
    }
    p->jitter_key = d.seed ^ kJitterKey;
    return CLOUD_OK;
}

int build_view(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *cam, int width,
               int height, int steps, int jitter_frame, float *out, int shape, ViewParams *v) {
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: width/height outside [1, 16384]");
    if (steps < 1 || steps > CLOUD_MAX_STEPS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: steps outside [1, 4096]");
    if (!(cam->tan_half_fovy > 0.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: tan_half_fovy must be > 0");
    if (!out || !aligned(out, 16))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: out_rgba null or not 16-byte aligned");
    const cloud_volume_desc &d = vol->desc;
    *v = ViewParams{};
    const double aspect = (double)width / (double)height, tf = cam->tan_half_fovy;
    const double a0 = (1.0 / width - 1.0) * aspect * tf, ax = 2.0 * aspect * tf / width;
    const double b0 = (1.0 - 1.0 / height) * tf, by = -2.0 * tf / height;
    for (int k = 0; k < 3; ++k) {
        split_df(cam->forward[k] + a0 * cam->right[k] + b0 * cam->up[k], &v->v00h[k], &v->v00l[k]);
        split_df10(ax * cam->right[k], &v->vxh[k], &v->vxl[k]);
        split_df10(by * cam->up[k], &v->vyh[k], &v->vyl[k]);
        split_df(cam->pos[k], &v->oh[k], &v->ol[k]);
    }
    split_df(d.slab_lo_m - cam->pos[2], &v->zlo_h, &v->zlo_l);
    split_df(d.slab_hi_m - cam->pos[2], &v->zhi_h, &v->zhi_l);
    split_df(prm->t_max_m, &v->tmax_h, &v->tmax_l);
    split_df(1.0 / steps, &v->invn_h, &v->invn_l);
    v->cam_in_layer = cam->pos[2] >= d.slab_lo_m && cam->pos[2] <= d.slab_hi_m;
    // a ray from below reaches the layer within t_max only if d_z >= (lo - o_z)/t_max
    v->miss_below = -INFINITY;
    v->miss_above = INFINITY;
    if (cam->pos[2] < d.slab_lo_m)
        v->miss_below = (float)((d.slab_lo_m - cam->pos[2]) / prm->t_max_m * (1.0 - 1e-4) - 1e-6);
    if (cam->pos[2] > d.slab_hi_m)
        v->miss_above = (float)(-(cam->pos[2] - d.slab_hi_m) / prm->t_max_m * (1.0 - 1e-4) + 1e-6);
    v->width = width;
    v->height = height;
    v->steps = steps;
    v->jitter_frame = jitter_frame < 0 ? -1 : jitter_frame;
    v->u_frame = -1.0f;
    if (jitter_frame >= 0 && prm->jitter_mode == CLOUD_JITTER_PER_FRAME)  // offset of pixel (0, 0)
        v->u_frame = (float)(pcg_hash4(0u, 0u, (uint32_t)jitter_frame, d.seed ^ kJitterKey) >> 8) *
                     (1.0f / 16777216.0f);
    int tw, th;
    tile_dims(shape, &tw, &th);
    v->tiles_x = (width + tw - 1) / tw;
    v->tile_count = v->tiles_x * ((height + th - 1) / th);
    v->out = (float4 *)out;
    return CLOUD_OK;
}

// ---------------------------------------------------------------------------
// Launch-configuration selection: the autotuner records the fastest (tile
// shape, view steps per warp iteration) per (storage precision, light-step
// specialisation); launches use it when present.
namespace {
std::mutex g_tune_mu;
int g_best_config[4][2] = {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}};
}  // namespace

// Untuned default: shape 3 (8x16-pixel CTA of 4x8-pixel warps), 8 view steps
// per warp iteration, the fastest for 8- and 16-step renders of every storage
// precision measured.
constexpr int kDefaultConfig = 3;

int tuned_config(int precision, int light_steps) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int c = g_best_config[precision & 3][light_steps == 6 ? 1 : 0];
    return c < 0 ? kDefaultConfig : c;
}
void set_tuned_config(int precision, int light_steps, int config) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_best_config[precision & 3][light_steps == 6 ? 1 : 0] = config;
}

bool fixed_sizes(const SceneParams &p, const cloud_volume *vol) {
    return p.light_steps == 6 && !p.constant_mode && vol->detail && vol->weather &&
           p.log2_base == kStdLog2Base && p.log2_detail == kStdLog2Detail &&
           p.log2_weather == kStdLog2Weather && p.detail_shift >= 0;
}

int launch_march(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                 unsigned long long *counter, int config, cudaStream_t s) {
    if (config_chunk(config) == 16)
        launch_march_ch<16>(p, v, vol, counter, config_shape(config), s);
    else
        launch_march_ch<8>(p, v, vol, counter, config_shape(config), s);
    return check_launch("march_kernel");
}

int launch_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                  int width, int height, int steps, int light_steps, int jitter_frame,
                  int integration, float *out, unsigned long long *counter, cudaStream_t s) {
    if (!vol || !cam || !prm || !out)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: null pointer");
    if (counter && !aligned(counter, 8))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: counter not 8-byte aligned");
    SceneParams p;
    ViewParams v;
    const int config = tuned_config(vol->desc.precision, light_steps);
    if (int rc = build_scene(vol, prm, light_steps, integration, &p)) return rc;
    if (int rc = build_view(vol, prm, cam, width, height, steps, jitter_frame, out,
                            config_shape(config), &v))
        return rc;
    return launch_march(p, v, vol, counter, config, s);
}

}  // namespace cloudvol

using namespace cloudvol;

extern "C" int cloud_render(const cloud_volume *vol, const cloud_camera *cam,
                            const cloud_params *prm, int width, int height, int steps,
                            int light_steps, int jitter_frame, int integration, float *out_rgba,
                            void *stream) {
    clear_error();
    return launch_render(vol, cam, prm, width, height, steps, light_steps, jitter_frame,
                         integration, out_rgba, nullptr, (cudaStream_t)stream);
}

extern "C" int cloud_render_count(const cloud_volume *vol, const cloud_camera *cam,
                                  const cloud_params *prm, int width, int height, int steps,
                                  int light_steps, int jitter_frame, int integration,
                                  float *out_rgba, unsigned long long *lookups, void *stream) {
    clear_error();
    if (!lookups) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render_count: null counter");
    return launch_render(vol, cam, prm, width, height, steps, light_steps, jitter_frame,
                         integration, out_rgba, lookups, (cudaStream_t)stream);
}

extern "C" int cloud_autotune_render(const cloud_volume *vol, const cloud_camera *cam,
                                     const cloud_params *prm, int width, int height, int steps,
                                     int light_steps, int jitter_frame, int integration,
                                     float *out_rgba, int repeats, float *times_ms, int *best,
                                     void *stream) {
    clear_error();
    if (!vol || !cam || !prm || !out_rgba || repeats < 1)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_autotune_render: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    SceneParams p;
    if (int rc = build_scene(vol, prm, light_steps, integration, &p)) return rc;
    cudaEvent_t e0, e1;
    if (int rc = check_cuda(cudaEventCreate(&e0), "cudaEventCreate")) return rc;
    if (int rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate")) {
        cudaEventDestroy(e0);
        return rc;
    }
    int best_config = 0, rc = CLOUD_OK;
    float best_ms = INFINITY;
    for (int config = 0; config < kConfigs && !rc; ++config) {
        ViewParams v;
        rc = build_view(vol, prm, cam, width, height, steps, jitter_frame, out_rgba,
                        config_shape(config), &v);
        if (rc) break;
        rc = launch_march(p, v, vol, nullptr, config, s);  // warm-up
        if (!rc) rc = check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
        for (int r = 0; r < repeats && !rc; ++r) rc = launch_march(p, v, vol, nullptr, config, s);
        if (!rc) rc = check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
        if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
        float ms = 0.0f;
        if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
        ms /= repeats;
        if (times_ms) times_ms[config] = ms;
        if (!rc && ms < best_ms) {
            best_ms = ms;
            best_config = config;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    set_tuned_config(vol->desc.precision, light_steps, best_config);
    if (best) *best = best_config;
    return CLOUD_OK;
}

extern "C" int cloud_get_launch_config(int precision, int light_steps, int *config) {
    clear_error();
    if (!config || precision < CLOUD_PRECISION_FP32 || precision > CLOUD_PRECISION_UNORM16)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_get_launch_config: bad arguments");
    *config = tuned_config(precision, light_steps);
    return CLOUD_OK;
}

extern "C" int cloud_set_launch_config(int precision, int light_steps, int config) {
    clear_error();
    if (precision < CLOUD_PRECISION_FP32 || precision > CLOUD_PRECISION_UNORM16 || config < 0 ||
        config >= kConfigs)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_set_launch_config: bad arguments");
    set_tuned_config(precision, light_steps, config);
    return CLOUD_OK;
}

extern "C" int cloud_debug_set_occupancy(int enabled) {
    clear_error();
    g_use_occupancy.store(enabled != 0);
    return CLOUD_OK;
}
