// render.cu -- the per-pixel cloud raymarch (Sec. 1, Sec. 3.1, Sec. 3.2).
//
// One thread per pixel; a 128-thread CTA covers a 16x8 pixel tile and each
// warp an 8x4 sub-tile, so the rays of a warp stay adjacent and touch the
// same region of the (L2-resident) noise tiles.
//
// Precision design.  Grazing rays are tens of kilometres long and, with 8
// view steps, a step is kilometres long; the estimator then multiplies any
// density error by alpha*D*L_in (hundreds), so sample positions must be far
// more accurate than FP32 world coordinates allow.  Per ray, the start and
// the step of every lattice axis (base xyz, detail xyz, weather xy) and of the
// height above the layer bottom are computed in FP64 and stored as 32-bit
// fixed-point values.  A lattice axis keeps log2(N) integer bits and
// 32-log2(N) fraction bits, so unsigned overflow is exactly the periodic wrap
// of the tile; a view step adds the ray's increment and a light sample adds a
// per-launch constant offset -- integer adds, no rounding.  The texel index is
// the top log2(N) bits, the interpolation weight the next 23 bits.  Radiance
// and the optical-depth sum are FP32.
#include <cmath>

#include "common.cuh"

namespace cloudvol {

enum Axis { kBX = 0, kBY, kBZ, kDX, kDY, kDZ, kWX, kWY, kLatticeAxes };

struct MarchParams {
    // Camera rays, unnormalised: v(x, y) = v00 + x vx + y vy, as double-float
    // pairs; vx/vy are split so that x * hi is exact (see split_df10).
    float v00h[3], v00l[3], vxh[3], vxl[3], vyh[3], vyl[3];
    float oh[3], ol[3];          // camera position
    float zlo_h, zlo_l;          // slab_lo - o_z
    float zhi_h, zhi_l;          // slab_hi - o_z
    float tmax_h, tmax_l;        // far clip distance
    float invn_h, invn_l;        // 1 / steps
    // Fixed-point lattice coordinates: unit 2^32 per tile period, so
    // coordinate = p * kfix - half_unit (mod 2^32), kfix = 2^32 / period.
    float kfix_h[kLatticeAxes], kfix_l[kLatticeAxes];
    uint32_t half_unit[kLatticeAxes];  // half a texel: 2^(31 - log2 N)
    uint32_t loff[CLOUD_MAX_LIGHT_STEPS][kLatticeAxes];  // light-sample offsets
    int32_t lh[CLOUD_MAX_LIGHT_STEPS];                   // light-sample height offsets
    int32_t h_top;                                       // layer thickness in 2^-16 m
    float h_lo_scale, h_hi_scale;  // 10/thickness, 2.5/thickness, per 2^-16 m
    float sun[3], sun_rad[3], ambient[3];
    float hg_g, hg_norm, absorption, light_step, tau_max;  // hg_norm = (1 - g^2)/(4 pi)
    float k0, b_cut, inv_1mc, detail_w, rho0;
    int log2_base, log2_detail, log2_weather;
    int width, height, steps, light_steps, jitter_frame, integration, constant_mode;
    int cam_in_layer;
    // rays with d_z below miss_below (camera under the layer) or above
    // miss_above (camera over it) cannot reach the layer within t_max
    float miss_below, miss_above;
    // detail coordinates = (base + half_base) << detail_shift - half_detail when
    // the base tile period is 2^detail_shift detail periods (-1: convert separately)
    int detail_shift;
    uint32_t jitter_key;
};

__device__ __forceinline__ float frac23(uint32_t f) {
    return __uint_as_float((f >> 9) | 0x3F800000u) - 1.0f;
}

// Corner-packed sampling at fixed-point coordinates: the record index is the
// top L bits of each coordinate, the interpolation weights the next 23 bits.
__device__ __forceinline__ uint32_t rec3(int L, uint32_t cx, uint32_t cy, uint32_t cz) {
    const int sh = 32 - L;
    return ((cz >> sh) << (2 * L)) | ((cy >> sh) << L) | (cx >> sh);
}
__device__ __forceinline__ uint32_t rec2(int L, uint32_t cx, uint32_t cy) {
    const int sh = 32 - L;
    return ((cy >> sh) << L) | (cx >> sh);
}
// Interpolation on packed FP32x2 (Blackwell FFMA2/FADD2): x first on the
// (z0, z1) pairs of both y rows, then y on the pair, then z.  Each lane of a
// packed op rounds exactly like the scalar op.
__device__ __forceinline__ float trilerp(const float c[8], int L, uint32_t cx, uint32_t cy,
                                         uint32_t cz) {
    const float fx = frac23(cx << L), fy = frac23(cy << L), fz = frac23(cz << L);
    const float2 a0 = make_float2(c[0], c[1]), a1 = make_float2(c[2], c[3]);  // dx = 0
    const float2 b0 = make_float2(c[4], c[5]), b1 = make_float2(c[6], c[7]);  // dx = 1
    const float2 fx2 = make_float2(fx, fx), fy2 = make_float2(fy, fy);
    const float2 x0 = __ffma2_rn(fx2, __fadd2_rn(b0, make_float2(-a0.x, -a0.y)), a0);  // dy = 0
    const float2 x1 = __ffma2_rn(fx2, __fadd2_rn(b1, make_float2(-a1.x, -a1.y)), a1);  // dy = 1
    const float2 yz = __ffma2_rn(fy2, __fadd2_rn(x1, make_float2(-x0.x, -x0.y)), x0);  // (z0, z1)
    return fmaf(fz, yz.y - yz.x, yz.x);
}
__device__ __forceinline__ float bilerp(const float c[4], int L, uint32_t cx, uint32_t cy) {
    const float fx = frac23(cx << L), fy = frac23(cy << L);
    const float2 a = make_float2(c[0], c[1]), b = make_float2(c[2], c[3]);  // (y0, y1) at dx
    const float2 xy = __ffma2_rn(make_float2(fx, fx), __fadd2_rn(b, make_float2(-a.x, -a.y)), a);
    return fmaf(fy, xy.y - xy.x, xy.x);
}

// Density at a sample (Sec. 1 "the density is sampled"):
//   rho = g(h) W max(0, (B - w_d Dt - c)/(1 - c)),
// tiles stored centred (value - 1/2), so (B - w_d Dt - c) = Bc - w_d Dtc + k0.
// Samples outside the layer (g = 0) return without touching memory; otherwise
// the three record loads are issued together so that one memory round trip
// serves the lookup.
template <typename T>
__device__ __forceinline__ float density(const MarchParams &p, const T *__restrict__ base,
                                         const T *__restrict__ detail,
                                         const T *__restrict__ weather, const uint32_t c[8],
                                         int32_t hq) {
    if (p.constant_mode) return p.rho0;
    const float ga = fminf(fmaxf((float)hq * p.h_lo_scale, 0.0f), 1.0f);
    const float gb = fminf(fmaxf((float)(p.h_top - hq) * p.h_hi_scale, 0.0f), 1.0f);
    const float g = ga * gb;
    if (g <= 0.0f) return 0.0f;
    float cb[8], cd[8], cw[4];
    load_rec8(base, rec3(p.log2_base, c[kBX], c[kBY], c[kBZ]), cb);
    if (detail) load_rec8(detail, rec3(p.log2_detail, c[kDX], c[kDY], c[kDZ]), cd);
    if (weather) load_rec4(weather, rec2(p.log2_weather, c[kWX], c[kWY]), cw);
    const float b = trilerp(cb, p.log2_base, c[kBX], c[kBY], c[kBZ]) - raw_bias<T>();
    float r = b + p.k0;
    if (detail) {
        const float dt = trilerp(cd, p.log2_detail, c[kDX], c[kDY], c[kDZ]) - raw_bias<T>();
        r = fmaf(-p.detail_w, dt, r);
    }
    r = fmaxf(r * p.inv_1mc, 0.0f);
    const float w = weather ? bilerp(cw, p.log2_weather, c[kWX], c[kWY]) - raw_bias<T>() + kCentre : 1.0f;
    return g * w * r;
}

__device__ __forceinline__ df df_addf(df a, float b) {
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}

// CTAs per SM the march is compiled for (register budget 65536 / (128 x this)).
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS
#define CLOUDVOL_MARCH_MIN_BLOCKS 6
#endif

constexpr int kAxes = kLatticeAxes + 1;  // lattice axes + height above the layer bottom
constexpr int kChunk = 8;                // view steps per warp-cooperative chunk
constexpr unsigned kFull = 0xFFFFFFFFu;

// Per-warp shared scratch of the march: each lane's start coordinates and
// per-step increments, the chunk's view densities, light-march sums and the
// list of (step, lane) pairs that need a light march.
struct WarpScratch {
    uint32_t c0[kAxes][32];
    uint32_t e[kAxes][32];
    float rho[kChunk][32];
    float lsum[kChunk][32];
    uint16_t pairs[kChunk * 32];
};

// sigma D of one step, rounded the same way wherever it is recomputed
__device__ __forceinline__ float step_depth(float absorption, float rho, float D) {
    return __fmul_rn(__fmul_rn(absorption, rho), D);
}

// The march of one 16x8 tile (4 warps, one pixel per lane).  View steps are
// processed in chunks of kChunk:
//   A  each lane evaluates its view densities and its early out (the optical
//      depth does not depend on the lighting);
//   B  the warp shares out every (step, lane) light march with density > 0
//      over all 32 lanes, so lanes whose own rays are empty, finished or
//      outside the layer do useful work;
//   C  each lane integrates its steps in order with the light sums from B.
// The arithmetic of every sample is the same as a per-lane march.
template <typename T, int LS>
__global__ void __launch_bounds__(128, CLOUDVOL_MARCH_MIN_BLOCKS) march_kernel(const __grid_constant__ MarchParams p,
                                                       const T *__restrict__ base,
                                                       const T *__restrict__ detail,
                                                       const T *__restrict__ weather,
                                                       float4 *__restrict__ out,
                                                       unsigned long long *__restrict__ counter) {
    __shared__ WarpScratch scratch[4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpScratch &ws = scratch[warp];
    const int x = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int y = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    const bool in_image = x < p.width && y < p.height;
    bool inside = in_image;
    const int nlight = LS >= 0 ? LS : p.light_steps;
    unsigned long long n_look = 0;
    uint32_t c[kLatticeAxes] = {}, e[kLatticeAxes] = {};
    int32_t hq = 0, eh = 0;
    float Df = 0.0f, phase = 0.0f;
    bool alive = false;
    const float xf = (float)x, yf = (float)y;
    if (inside) {
        // quick FP32 test for rays that cannot reach the layer (a 1e-4 margin
        // keeps every undecided ray on the exact path below)
        const float qx = fmaf(yf, p.vyh[0], fmaf(xf, p.vxh[0], p.v00h[0]));
        const float qy = fmaf(yf, p.vyh[1], fmaf(xf, p.vxh[1], p.v00h[1]));
        const float qz = fmaf(yf, p.vyh[2], fmaf(xf, p.vxh[2], p.v00h[2]));
        const float dz = qz * rsqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
        if (dz < p.miss_below || dz > p.miss_above) inside = false;
    }
    if (inside) {
        // --- a1: pixel ray and layer clip (double-float) ---------------------
        // p(lambda) = o + lambda v with v unnormalised; t = lambda |v|.
        df v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            df a = {p.v00h[k], p.v00l[k] + fmaf(xf, p.vxl[k], yf * p.vyl[k])};
            a = df_addf(a, xf * p.vxh[k]);  // exact products
            v[k] = df_addf(a, yf * p.vyh[k]);
        }
        const df n2 = df_add(df_add(df_mul(v[0], v[0]), df_mul(v[1], v[1])), df_mul(v[2], v[2]));
        const df rn = df_rsqrt(n2);  // 1 / |v|
        const df lam_max = df_mul({p.tmax_h, p.tmax_l}, rn);
        df lam0 = {0.0f, 0.0f}, lam1 = lam_max;
        if (fabsf(v[2].hi) * rn.hi < 1e-8f) {
            alive = p.cam_in_layer != 0;
        } else {
            const df inv = df_recip(v[2]);
            const df ll = df_mul({p.zlo_h, p.zlo_l}, inv), lh = df_mul({p.zhi_h, p.zhi_l}, inv);
            lam0 = df_max(df_min(ll, lh), lam0);
            lam1 = df_min(df_max(ll, lh), lam_max);
            alive = df_gt(lam1, lam0);
        }
        if (alive) {
            // --- a2: jittered start offset (Sec. 3.2) ---------------------------
            const df D = df_mul(df_add(lam1, df_neg(lam0)), {p.invn_h, p.invn_l});
            float u = 0.5f;
            if (p.jitter_frame >= 0)
                u = (float)(pcg_hash4((uint32_t)x, (uint32_t)y, (uint32_t)p.jitter_frame,
                                      p.jitter_key) >> 8) * (1.0f / 16777216.0f);
            const df lam_s = df_add(lam0, df_mulf(D, u));
            df pos[3], dpos[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pos[k] = df_add({p.oh[k], p.ol[k]}, df_mul(lam_s, v[k]));
                dpos[k] = df_mul(D, v[k]);
            }
#pragma unroll
            for (int a = 0; a < kLatticeAxes; ++a) {
                const int comp = a < 6 ? a % 3 : a - 6;
                if (a >= kDX && a <= kDZ && p.detail_shift >= 0) {
                    // same origin, period 2^-shift of the base tile: exact shift
                    const int b = a - kDX;
                    c[a] = ((c[b] + p.half_unit[b]) << p.detail_shift) - p.half_unit[a];
                    e[a] = e[b] << p.detail_shift;
                    continue;
                }
                const df k = {p.kfix_h[a], p.kfix_l[a]};
                c[a] = df_to_u32(df_mul(pos[comp], k)) - p.half_unit[a];
                e[a] = df_to_u32(df_mul(dpos[comp], k));
            }
            // height above the layer bottom: (o_z - slab_lo) + lambda v_z, in 2^-16 m
            const df hrel = df_add(df_mul(lam_s, v[2]), df_neg({p.zlo_h, p.zlo_l}));
            hq = (int32_t)df_to_u32({hrel.hi * 65536.0f, hrel.lo * 65536.0f});
            eh = (int32_t)df_to_u32({dpos[2].hi * 65536.0f, dpos[2].lo * 65536.0f});
            const float vlen = n2.hi * rn.hi;
            Df = D.hi * vlen;
            // --- a5: phase function, hoisted per ray ----------------------------
            const float mu = (v[0].hi * p.sun[0] + v[1].hi * p.sun[1] + v[2].hi * p.sun[2]) * rn.hi;
            // p_HG(mu) = (1 - g^2) / (4 pi) * (1 + g^2 - 2 g mu)^(-3/2)
            const float r = rsqrtf(fmaf(-2.0f * p.hg_g, mu, fmaf(p.hg_g, p.hg_g, 1.0f)));
            phase = p.hg_norm * r * r * r;
        }
    }
#pragma unroll
    for (int a = 0; a < kLatticeAxes; ++a) {
        ws.c0[a][lane] = c[a];
        ws.e[a][lane] = e[a];
    }
    ws.c0[kLatticeAxes][lane] = (uint32_t)hq;
    ws.e[kLatticeAxes][lane] = (uint32_t)eh;
    const unsigned lt_mask = (1u << lane) - 1u;
    float tau = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    for (int i0 = 0; i0 < p.steps && __any_sync(kFull, alive); i0 += kChunk) {
        // --- A: view densities and early out --------------------------------
        uint32_t act = 0;
        int nA = 0;
        if (alive) {
            float tau_a = tau;
#pragma unroll 1
            for (int k = 0; k < kChunk; ++k) {
                if (i0 + k >= p.steps) break;
                // --- a3: density lookup ---------------------------------------
                const float rho = density(p, base, detail, weather, c, hq);
                ws.rho[k][lane] = rho;
                nA = k + 1;
                if (rho > 0.0f) {
                    act |= 1u << k;
                    tau_a = __fadd_rn(tau_a, step_depth(p.absorption, rho, Df));
                }
#pragma unroll
                for (int a = 0; a < kLatticeAxes; ++a) c[a] += e[a];
                hq += eh;
                // --- a7: early out once alpha is ~1 (Sec. 1) --------------------
                if (tau_a >= p.tau_max) {
                    alive = false;
                    break;
                }
            }
            n_look += nA + nlight * __popc(act);
        }
        if (!__any_sync(kFull, act != 0u)) {
            // no step of this chunk has density anywhere in the warp
            continue;
        }
        // --- B: light marches shared out over the warp (a4, Sec. 1) ----------
        unsigned offs[kChunk + 1];
        offs[0] = 0;
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            const unsigned m = __ballot_sync(kFull, (act >> k) & 1u);
            if ((act >> k) & 1u) ws.pairs[offs[k] + __popc(m & lt_mask)] = (uint16_t)((k << 5) | lane);
            offs[k + 1] = offs[k] + __popc(m);
        }
        __syncwarp();
        for (unsigned q = lane; q < offs[kChunk]; q += 32) {
            const unsigned pr = ws.pairs[q], k = pr >> 5, ow = pr & 31u;
            const uint32_t i = (uint32_t)(i0 + (int)k);
            uint32_t cs[kLatticeAxes];
#pragma unroll
            for (int a = 0; a < kLatticeAxes; ++a) cs[a] = ws.c0[a][ow] + i * ws.e[a][ow];
            const int32_t hs = (int32_t)(ws.c0[kLatticeAxes][ow] + i * ws.e[kLatticeAxes][ow]);
            float rho_sum = 0.0f;
#pragma unroll
            for (int j = 0; j < (LS >= 0 ? LS : CLOUD_MAX_LIGHT_STEPS); ++j) {
                if (LS < 0 && j >= nlight) break;
                uint32_t cj[kLatticeAxes];
#pragma unroll
                for (int a = 0; a < kLatticeAxes; ++a) cj[a] = cs[a] + p.loff[j][a];
                rho_sum += density(p, base, detail, weather, cj, hs + p.lh[j]);
            }
            ws.lsum[k][ow] = rho_sum;
        }
        __syncwarp();
        // --- C: in-scattered light and the per-step integral, in step order ---
        for (int k = 0; k < nA; ++k) {
            if (!((act >> k) & 1u)) continue;
            const float rho = ws.rho[k][lane];
            // --- a5: in-scattered light ---------------------------------------
            const float sun_t = expf(-p.absorption * p.light_step * ws.lsum[k][lane]) * phase;
            const float lr = fmaf(p.sun_rad[0], sun_t, p.ambient[0]);
            const float lg = fmaf(p.sun_rad[1], sun_t, p.ambient[1]);
            const float lb = fmaf(p.sun_rad[2], sun_t, p.ambient[2]);
            // --- a6: per-step integral (Sec. 3.1) ------------------------------
            const float sd = step_depth(p.absorption, rho, Df);
            float wgt;
            if (p.integration == CLOUD_INTEGRATE_ANALYTIC) {
                wgt = expf(-tau) * -expm1f(-sd);
                tau = __fadd_rn(tau, sd);
            } else {
                tau = __fadd_rn(tau, sd);
                wgt = expf(-tau) * sd;
            }
            cr = fmaf(wgt, lr, cr);
            cg = fmaf(wgt, lg, cg);
            cb = fmaf(wgt, lb, cb);
        }
        __syncwarp();
    }
    // --- a8: premultiplied RGBA, one 16-byte store ------------------------------
    if (in_image) out[(size_t)y * p.width + x] = make_float4(cr, cg, cb, -expm1f(-tau));
    if (counter) {
        unsigned long long v = n_look;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(kFull, v, s);
        if (lane == 0 && v) atomicAdd(counter, v);
    }
}

double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

int build_params(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                 int width, int height, int steps, int light_steps, int jitter_frame,
                 int integration, MarchParams *p) {
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: width/height outside [1, 16384]");
    if (steps < 1 || steps > CLOUD_MAX_STEPS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: steps outside [1, 4096]");
    if (light_steps < 0 || light_steps > CLOUD_MAX_LIGHT_STEPS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: light_steps outside [0, 32]");
    if (integration != CLOUD_INTEGRATE_ANALYTIC && integration != CLOUD_INTEGRATE_BASIC)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: bad integration mode");
    if (!(cam->tan_half_fovy > 0.0) || !(prm->t_max_m > 0.0 && prm->t_max_m <= 1e6) ||
        !(prm->light_step_m >= 0.0) ||
        !(prm->absorption_per_m >= 0.0) || !(prm->hg_g > -1.0 && prm->hg_g < 1.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: bad camera or lighting constants");
    const double sn = std::sqrt(dot3(prm->sun_dir, prm->sun_dir));
    if (!(sn > 0.0) || !(prm->sun_dir[2] > 0.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: sun direction must have z > 0");
    const cloud_volume_desc &d = vol->desc;
    const double thick = d.slab_hi_m - d.slab_lo_m;
    const double s[3] = {prm->sun_dir[0] / sn, prm->sun_dir[1] / sn, prm->sun_dir[2] / sn};
    if (thick + light_steps * prm->light_step_m * s[2] > 32000.0)
        return set_error(CLOUD_ERR_UNSUPPORTED, "cloud_render: light march reaches > 32 km above the layer bottom");

    *p = MarchParams{};
    const double aspect = (double)width / (double)height, tf = cam->tan_half_fovy;
    const double a0 = (1.0 / width - 1.0) * aspect * tf, ax = 2.0 * aspect * tf / width;
    const double b0 = (1.0 - 1.0 / height) * tf, by = -2.0 * tf / height;
    for (int k = 0; k < 3; ++k) {
        split_df(cam->forward[k] + a0 * cam->right[k] + b0 * cam->up[k], &p->v00h[k], &p->v00l[k]);
        split_df10(ax * cam->right[k], &p->vxh[k], &p->vxl[k]);
        split_df10(by * cam->up[k], &p->vyh[k], &p->vyl[k]);
        split_df(cam->pos[k], &p->oh[k], &p->ol[k]);
    }
    split_df(d.slab_lo_m - cam->pos[2], &p->zlo_h, &p->zlo_l);
    split_df(d.slab_hi_m - cam->pos[2], &p->zhi_h, &p->zhi_l);
    split_df(prm->t_max_m, &p->tmax_h, &p->tmax_l);
    split_df(1.0 / steps, &p->invn_h, &p->invn_l);
    p->cam_in_layer = cam->pos[2] >= d.slab_lo_m && cam->pos[2] <= d.slab_hi_m;
    // a ray from below reaches the layer within t_max only if d_z >= (lo - o_z)/t_max
    p->miss_below = -INFINITY;
    p->miss_above = INFINITY;
    if (cam->pos[2] < d.slab_lo_m)
        p->miss_below = (float)((d.slab_lo_m - cam->pos[2]) / prm->t_max_m * (1.0 - 1e-4) - 1e-6);
    if (cam->pos[2] > d.slab_hi_m)
        p->miss_above = (float)(-(cam->pos[2] - d.slab_hi_m) / prm->t_max_m * (1.0 - 1e-4) + 1e-6);
    p->detail_shift = -1;
    if (vol->log2_detail) {
        const double ratio = d.base_period_m / d.detail_period_m;
        for (int k = 0; k <= 16; ++k)
            if (ratio == std::ldexp(1.0, k)) p->detail_shift = k;
    }
    const bool noise = d.density_mode == CLOUD_DENSITY_NOISE;
    const int L[kLatticeAxes] = {vol->log2_base,   vol->log2_base,   vol->log2_base,
                                 vol->log2_detail, vol->log2_detail, vol->log2_detail,
                                 vol->log2_weather, vol->log2_weather};
    const double P[kLatticeAxes] = {d.base_period_m,   d.base_period_m,   d.base_period_m,
                                    d.detail_period_m, d.detail_period_m, d.detail_period_m,
                                    d.weather_period_m, d.weather_period_m};
    for (int a = 0; a < kLatticeAxes; ++a) {
        const int comp = a < 6 ? a % 3 : a - 6;
        if (!noise || L[a] == 0) continue;  // absent tile: axis unused
        const double kfix = 4294967296.0 / P[a];  // 2^32 fixed-point units per tile
        split_df(kfix, &p->kfix_h[a], &p->kfix_l[a]);
        p->half_unit[a] = 1u << (31 - L[a]);
        for (int j = 0; j < light_steps; ++j) {
            const double v = (j + 0.5) * prm->light_step_m * s[comp] * kfix;
            p->loff[j][a] = (uint32_t)(unsigned long long)std::llrint(v);
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
    p->k0 = (float)(0.5 - d.coverage - 0.5 * wd);
    p->b_cut = (float)(0.5 - d.coverage);
    p->inv_1mc = (float)(1.0 / (1.0 - d.coverage));
    p->rho0 = (float)d.constant_density;
    p->log2_base = vol->log2_base;
    p->log2_detail = vol->log2_detail;
    p->log2_weather = vol->log2_weather;
    p->width = width;
    p->height = height;
    p->steps = steps;
    p->light_steps = light_steps;
    p->jitter_frame = jitter_frame < 0 ? -1 : jitter_frame;
    p->integration = integration;
    p->constant_mode = noise ? 0 : 1;
    p->jitter_key = d.seed ^ kJitterKey;
    return CLOUD_OK;
}

// The common light-march length (6, Sec. 1) is compiled with its offsets as
// constants; any other length uses the generic loop.
template <typename T>
int launch_typed(const MarchParams &p, const cloud_volume *vol, float *out,
                 unsigned long long *counter, dim3 grid, cudaStream_t s) {
    const T *b = (const T *)vol->base, *d = (const T *)vol->detail, *w = (const T *)vol->weather;
    if (p.light_steps == 6)
        march_kernel<T, 6><<<grid, 128, 0, s>>>(p, b, d, w, (float4 *)out, counter);
    else
        march_kernel<T, -1><<<grid, 128, 0, s>>>(p, b, d, w, (float4 *)out, counter);
    return check_launch("march_kernel");
}

int launch_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                  int width, int height, int steps, int light_steps, int jitter_frame,
                  int integration, float *out, unsigned long long *counter, cudaStream_t s) {
    if (!vol || !cam || !prm || !out)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: null pointer");
    if (!aligned(out, 16)) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: out_rgba not 16-byte aligned");
    if (counter && !aligned(counter, 8))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_render: counter not 8-byte aligned");
    MarchParams p;
    if (int rc = build_params(vol, cam, prm, width, height, steps, light_steps, jitter_frame,
                              integration, &p))
        return rc;
    const dim3 grid((width + 15) / 16, (height + 7) / 8);
    switch (vol->desc.precision) {
        case CLOUD_PRECISION_FP32:
            return launch_typed<float>(p, vol, out, counter, grid, s);
        case CLOUD_PRECISION_FP16:
            return launch_typed<__half>(p, vol, out, counter, grid, s);
        case CLOUD_PRECISION_BF16:
            return launch_typed<__nv_bfloat16>(p, vol, out, counter, grid, s);
        default:
            return launch_typed<uint16_t>(p, vol, out, counter, grid, s);
    }
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
