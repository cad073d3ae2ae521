// taa.cu -- reprojection motion and the temporal anti-aliasing resolve
// (Sec. 3.2: jittered frames are accumulated by Playdead-style TAA).
//
// Both kernels are memory-bound streaming passes: one thread per pixel,
// 32x8 CTAs, 16-byte RGBA loads/stores (8-byte for FP16 history).  The 3x3
// neighbourhood reads of the current frame and the 2x2 history footprint are
// served by L1; each pixel's own current value, motion and output are the
// compulsory traffic.
#include "common.cuh"

namespace cloudvol {

struct MotionParams {
    double v00[3], vx[3], vy[3], o[3];  // current camera rays, as in the raymarch
    double op[3], rp[3], up[3], fp[3];  // previous camera
    double slab_lo, slab_hi, t_max;
    double inv_atp, inv_tp;             // 1/(aspect tan) and 1/tan of the previous camera
    int width, height;
};

// Motion of one pixel (FP64: the reprojection depth reaches 40 km and the
// result is a difference of nearly equal pixel positions).
__global__ void __launch_bounds__(256) motion_kernel(const __grid_constant__ MotionParams p,
                                                     float2 *__restrict__ motion) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= p.width || y >= p.height) return;
    double v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = fma((double)y, p.vy[k], fma((double)x, p.vx[k], p.v00[k]));
    const double rn = rsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double d[3] = {v[0] * rn, v[1] * rn, v[2] * rn};
    double t = p.t_max;
    if (fabs(d[2]) >= 1e-8) {
        const double inv = 1.0 / d[2];
        const double tl = (p.slab_lo - p.o[2]) * inv, th = (p.slab_hi - p.o[2]) * inv;
        const double t0 = fmax(fmin(tl, th), 0.0), t1 = fmin(fmax(tl, th), p.t_max);
        if (t1 > t0 && t0 > 0.0) t = t0;
    }
    double q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = fma(t, d[k], p.o[k] - p.op[k]);
    const double cx = q[0] * p.rp[0] + q[1] * p.rp[1] + q[2] * p.rp[2];
    const double cy = q[0] * p.up[0] + q[1] * p.up[1] + q[2] * p.up[2];
    const double cz = q[0] * p.fp[0] + q[1] * p.fp[1] + q[2] * p.fp[2];
    float2 m;
    if (cz <= 0.0) {
        m = make_float2(1e9f, 1e9f);
    } else {
        const double icz = 1.0 / cz;
        const double px = (cx * icz * p.inv_atp + 1.0) * 0.5 * p.width;
        const double py = (1.0 - cy * icz * p.inv_tp) * 0.5 * p.height;
        m = make_float2((float)((x + 0.5) - px), (float)((y + 0.5) - py));
    }
    motion[(size_t)y * p.width + x] = m;
}

__device__ __forceinline__ float4 load_hist(const float4 *h, size_t i) { return __ldg(h + i); }
__device__ __forceinline__ float4 load_hist(const uint2 *h, size_t i) {
    const uint2 r = __ldg(h + i);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_hist(float4 *h, size_t i, float4 v) { h[i] = v; }
__device__ __forceinline__ void store_hist(uint2 *h, size_t i, float4 v) {
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 r;
    r.x = *reinterpret_cast<const uint32_t *>(&a);
    r.y = *reinterpret_cast<const uint32_t *>(&b);
    h[i] = r;
}

__device__ __forceinline__ float4 fmin4(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}
__device__ __forceinline__ float4 fmax4(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}
__device__ __forceinline__ float bil(float fx, float fy, float h00, float h01, float h10, float h11) {
    return (1.0f - fy) * ((1.0f - fx) * h00 + fx * h01) + fy * ((1.0f - fx) * h10 + fx * h11);
}

// TAA resolve (Sec. 3.2): reprojected, bilinearly filtered history clamped
// to the current frame's 3x3 range, blended with the current frame.
template <typename H>
__global__ void __launch_bounds__(256) taa_kernel(const H *__restrict__ hist,
                                                  const float4 *__restrict__ cur,
                                                  const float2 *__restrict__ mot,
                                                  H *__restrict__ out, int W, int Hh, float blend) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= Hh) return;
    const size_t i = (size_t)y * W + x;
    const float4 c = __ldg(cur + i);
    float4 res = c;
    if (hist) {
        const float2 m = __ldg(mot + i);
        const float xc = (float)x + 0.5f, yc = (float)y + 0.5f;
        // q = centre - m outside [0,W] x [0,H]: exact comparisons in FP32
        const bool off = (m.x > xc) || (m.x < xc - (float)W) || (m.y > yc) || (m.y < yc - (float)Hh);
        if (!off) {
            // sample position (x - m.x, y - m.y) in texel-centre coordinates,
            // split into integer and fraction without rounding
            const float nx = -m.x, ny = -m.y;
            const float flx = floorf(nx), fly = floorf(ny);
            const float fx = nx - flx, fy = ny - fly;
            const int ix = x + (int)flx, iy = y + (int)fly;
            const int xa = min(max(ix, 0), W - 1), xb = min(max(ix + 1, 0), W - 1);
            const int ya = min(max(iy, 0), Hh - 1), yb = min(max(iy + 1, 0), Hh - 1);
            const float4 h00 = load_hist(hist, (size_t)ya * W + xa);
            const float4 h01 = load_hist(hist, (size_t)ya * W + xb);
            const float4 h10 = load_hist(hist, (size_t)yb * W + xa);
            const float4 h11 = load_hist(hist, (size_t)yb * W + xb);
            float4 h = make_float4(bil(fx, fy, h00.x, h01.x, h10.x, h11.x),
                                   bil(fx, fy, h00.y, h01.y, h10.y, h11.y),
                                   bil(fx, fy, h00.z, h01.z, h10.z, h11.z),
                                   bil(fx, fy, h00.w, h01.w, h10.w, h11.w));
            float4 mn = c, mx = c;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny2 = min(max(y + dy, 0), Hh - 1);
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    const int nx2 = min(max(x + dx, 0), W - 1);
                    const float4 v = __ldg(cur + (size_t)ny2 * W + nx2);
                    mn = fmin4(mn, v);
                    mx = fmax4(mx, v);
                }
            }
            h = fmin4(fmax4(h, mn), mx);
            res = make_float4(fmaf(blend, c.x - h.x, h.x), fmaf(blend, c.y - h.y, h.y),
                              fmaf(blend, c.z - h.z, h.z), fmaf(blend, c.w - h.w, h.w));
        }
    }
    store_hist(out, i, res);
}

int build_motion_params(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                        const cloud_camera *cur, int width, int height, MotionParams *p) {
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: width/height outside [1, 16384]");
    if (!(cur->tan_half_fovy > 0.0) || !(prev->tan_half_fovy > 0.0) || !(prm->t_max_m > 0.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: bad camera or t_max");
    const double aspect = (double)width / (double)height, tf = cur->tan_half_fovy;
    const double a0 = (1.0 / width - 1.0) * aspect * tf, ax = 2.0 * aspect * tf / width;
    const double b0 = (1.0 - 1.0 / height) * tf, by = -2.0 * tf / height;
    for (int k = 0; k < 3; ++k) {
        p->v00[k] = cur->forward[k] + a0 * cur->right[k] + b0 * cur->up[k];
        p->vx[k] = ax * cur->right[k];
        p->vy[k] = by * cur->up[k];
        p->o[k] = cur->pos[k];
        p->op[k] = prev->pos[k];
        p->rp[k] = prev->right[k];
        p->up[k] = prev->up[k];
        p->fp[k] = prev->forward[k];
    }
    p->slab_lo = vol->desc.slab_lo_m;
    p->slab_hi = vol->desc.slab_hi_m;
    p->t_max = prm->t_max_m;
    p->inv_atp = 1.0 / (aspect * prev->tan_half_fovy);
    p->inv_tp = 1.0 / prev->tan_half_fovy;
    p->width = width;
    p->height = height;
    return CLOUD_OK;
}

int launch_motion(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                  const cloud_camera *cur, int width, int height, float *motion, cudaStream_t s) {
    if (!vol || !prm || !prev || !cur || !motion)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: null pointer");
    if (!aligned(motion, 8)) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: motion not 8-byte aligned");
    MotionParams p;
    if (int rc = build_motion_params(vol, prm, prev, cur, width, height, &p)) return rc;
    const dim3 grid((width + 31) / 32, (height + 7) / 8), block(32, 8);
    motion_kernel<<<grid, block, 0, s>>>(p, (float2 *)motion);
    return check_launch("motion_kernel");
}

int launch_taa(const void *history, const float *current, const float *motion, void *history_out,
               int width, int height, int fmt, float blend, cudaStream_t s) {
    if (!current || !motion || !history_out)
        return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: null pointer");
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: width/height outside [1, 16384]");
    if (fmt != CLOUD_HISTORY_FP32 && fmt != CLOUD_HISTORY_FP16)
        return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: bad history format");
    if (!(blend >= 0.0f && blend <= 1.0f))
        return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: blend outside [0, 1]");
    const size_t px = (size_t)width * height, eb = fmt == CLOUD_HISTORY_FP32 ? 16 : 8;
    if (!aligned(current, 16) || !aligned(motion, 8) || !aligned(history_out, eb) ||
        (history && !aligned(history, eb)))
        return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: misaligned buffer");
    if (history) {
        const char *a = (const char *)history, *b = (const char *)history_out;
        if (a < b + px * eb && b < a + px * eb)
            return set_error(CLOUD_ERR_INVALID_ARG, "taa_resolve: history and history_out overlap");
    }
    const dim3 grid((width + 31) / 32, (height + 7) / 8), block(32, 8);
    if (fmt == CLOUD_HISTORY_FP32)
        taa_kernel<float4><<<grid, block, 0, s>>>((const float4 *)history, (const float4 *)current,
                                                  (const float2 *)motion, (float4 *)history_out,
                                                  width, height, blend);
    else
        taa_kernel<uint2><<<grid, block, 0, s>>>((const uint2 *)history, (const float4 *)current,
                                                 (const float2 *)motion, (uint2 *)history_out,
                                                 width, height, blend);
    return check_launch("taa_kernel");
}

}  // namespace cloudvol

using namespace cloudvol;

extern "C" int cloud_motion(const cloud_volume *vol, const cloud_params *prm,
                            const cloud_camera *prev, const cloud_camera *cur, int width,
                            int height, float *motion, void *stream) {
    clear_error();
    return launch_motion(vol, prm, prev, cur, width, height, motion, (cudaStream_t)stream);
}

extern "C" int taa_resolve(const void *history, const float *current, const float *motion,
                           void *history_out, int width, int height, int history_fmt, float blend,
                           void *stream) {
    clear_error();
    return launch_taa(history, current, motion, history_out, width, height, history_fmt, blend,
                      (cudaStream_t)stream);
}
