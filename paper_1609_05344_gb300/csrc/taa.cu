// taa.cu -- reprojection motion and the temporal anti-aliasing resolve
// (Sec. 3.2: jittered frames are accumulated by Playdead-style TAA).
//
// Both kernels are memory-bound streaming passes: one thread per pixel,
// 32x8 CTAs, 16-byte RGBA loads/stores (8-byte for FP16 history).  The 3x3
// neighbourhood reads of the current frame and the 2x2 history footprint are
// served by L1; each pixel's own current value, motion and output are the
// compulsory traffic.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace cloudvol {

struct MotionParams {
    // current camera, camera-space ray slopes: a = a0 + x ax, b = b0 + y by;
    // the ray is (a, b, 1) in (right, up, forward) coordinates
    float a0, ax, b0, by;
    float rz, uz, fz;      // world z of the current right, up, forward
    float zlo, zhi, tmax;  // slab_lo - o_z, slab_hi - o_z, far clip
    // previous camera: q = dlt + lambda (I + G) (a, b, 1), G = R' R^T - I,
    // dlt = R' (o - o'); projections compared as differences of slopes
    float G[3][3], dlt[3];
    float kx, ky, kx1, ky1;  // aT'/aT, T'/T, and the same minus 1
    float sx, sy;            // W / (2 aT'), H / (2 T')
    int width, height, cam_in_layer;
    // double-float restatement of the world-space ray for near-tie layer-entry
    // decisions: v(x, y) = v00 + x vx + y vy (vx, vy split so that x * hi is
    // exact), slab_lo - o_z, slab_hi - o_z and the far clip
    float v00h[3], v00l[3], vxh[3], vxl[3], vyh[3], vyl[3];
    float zlo_h, zlo_l, zhi_h, zhi_l, tmax_h, tmax_l;
    unsigned *check;  // status word of the checked build, else nullptr
};

// Reprojection depth parameter lambda (t / |v|) of the layer entry point, or
// of the far clip when the ray does not enter the layer ahead of the camera,
// in double-float FP32 (about 48 bits, the layer clip of the raymarch): for the
// rays whose entry FP32 cannot decide.
__device__ __noinline__ float entry_lambda_exact(const MotionParams &p, int x, int y) {
    const float xf = (float)x, yf = (float)y;
    df r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        df a = {p.v00h[k], p.v00l[k] + fmaf(xf, p.vxl[k], yf * p.vyl[k])};
        a = df_addf(a, xf * p.vxh[k]);  // exact products
        r[k] = df_addf(a, yf * p.vyh[k]);
    }
    const df n2 = df_add(df_add(df_mul(r[0], r[0]), df_mul(r[1], r[1])), df_mul(r[2], r[2]));
    const df rn = df_rsqrt(n2);  // 1 / |v|
    const df lam_max = df_mul({p.tmax_h, p.tmax_l}, rn);
    if (fabsf(r[2].hi) * rn.hi < 1e-8f) return lam_max.hi;  // horizontal ray
    const df inv = df_recip(r[2]);
    const df ll = df_mul({p.zlo_h, p.zlo_l}, inv), lh = df_mul({p.zhi_h, p.zhi_l}, inv);
    const df zero = {0.0f, 0.0f};
    const df l0 = df_max(df_min(ll, lh), zero), l1 = df_min(df_max(ll, lh), lam_max);
    return (df_gt(l1, l0) && df_gt(l0, zero)) ? l0.hi : lam_max.hi;
}

// Motion of one pixel.  The motion is a small difference of nearly equal
// pixel positions; it is computed directly as a difference of camera-space
// slopes (no large terms cancel), so FP32 keeps it to ~1e-6 pixel.  Split in
// three parts so that a thread can share the column terms between pixels and
// interleave the arithmetic of several pixels: the column terms, the depth
// parameter of the layer entry (FP32, with a flag for the near ties that the
// double-float restatement decides), and the projection into the previous
// camera.
struct MotionCol {
    float a, n2x, vzx, gx0, gx1, gx2, akx, nx0;
};
__device__ __forceinline__ MotionCol motion_col(const MotionParams &p, int x) {
    MotionCol c;
    c.a = fmaf((float)x, p.ax, p.a0);
    c.n2x = fmaf(c.a, c.a, 1.0f);
    c.vzx = fmaf(c.a, p.rz, p.fz);
    c.gx0 = fmaf(p.G[0][0], c.a, p.G[0][2]);
    c.gx1 = fmaf(p.G[1][0], c.a, p.G[1][2]);
    c.gx2 = fmaf(p.G[2][0], c.a, p.G[2][2]);
    c.akx = c.a * p.kx;
    c.nx0 = fmaf(c.akx, p.dlt[2], -p.dlt[0]);
    return c;
}
// Depth parameter lambda (t / |v|) of the layer entry, or of the far clip;
// *exact is set when FP32 cannot call the entry (the caller then takes
// entry_lambda_exact).  b is the row slope.
__device__ __forceinline__ float motion_lambda(const MotionParams &p, const MotionCol &c, float b,
                                               bool *exact) {
    const float n2 = fmaf(b, b, c.n2x);
    const float vz = fmaf(b, p.uz, c.vzx);
    // divisions by hardware reciprocals (relative error ~1e-7, far below the
    // 1e-5 margin of the near-tie test and the motion's own accuracy)
    const float lmax = p.tmax * rsqrtf(n2);
    float lam = lmax;
    *exact = false;
    if (vz * vz >= 1e-16f * n2) {  // |d_z| >= 1e-8
        const float ivz = __fdividef(1.0f, vz);
        const float ll = p.zlo * ivz, lh = p.zhi * ivz;
        const float l0 = fmaxf(fminf(ll, lh), 0.0f), l1 = fminf(fmaxf(ll, lh), lmax);
        if (fabsf(l1 - l0) <= 1e-5f * fmaxf(l1, l0))
            *exact = true;  // too close to call in FP32
        else if (l1 > l0 && l0 > 0.0f)
            lam = l0;
    }
    return lam;
}
__device__ __forceinline__ float2 motion_project(const MotionParams &p, const MotionCol &c, float b,
                                                 float lam) {
    const float g0 = fmaf(p.G[0][1], b, c.gx0);
    const float g1 = fmaf(p.G[1][1], b, c.gx1);
    const float g2 = fmaf(p.G[2][1], b, c.gx2);
    const float qz = fmaf(lam, 1.0f + g2, p.dlt[2]);
    if (qz <= 0.0f) return make_float2(1e9f, 1e9f);
    // a kx qz - qx and qy - b ky qz, expanded so the O(lambda) terms cancel exactly
    const float bky = b * p.ky;
    const float nx = c.nx0 + lam * fmaf(c.a, p.kx1, fmaf(c.akx, g2, -g0));
    const float ny = fmaf(-bky, p.dlt[2], p.dlt[1]) + lam * fmaf(-b, p.ky1, fmaf(-bky, g2, g1));
    const float iq = __fdividef(1.0f, qz);
    return make_float2(p.sx * nx * iq, p.sy * ny * iq);
}
__device__ __forceinline__ float2 motion_at(const MotionParams &p, int x, int y) {
    const MotionCol c = motion_col(p, x);
    const float b = fmaf((float)y, p.by, p.b0);
    bool ex;
    float lam = motion_lambda(p, c, b, &ex);
    if (ex) lam = entry_lambda_exact(p, x, y);
    return motion_project(p, c, b, lam);
}

__global__ void __launch_bounds__(256) motion_kernel(const __grid_constant__ MotionParams p,
                                                     float2 *__restrict__ motion) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= p.width || y >= p.height) return;
    motion[(size_t)y * p.width + x] = motion_at(p, x, y);
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
// Three-input minimum / maximum (sm_100+ PTX min/max with three sources),
// per channel; exact, like every min/max.
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float4 min3_4(float4 a, float4 b, float4 c) {
    return make_float4(min3f(a.x, b.x, c.x), min3f(a.y, b.y, c.y), min3f(a.z, b.z, c.z), min3f(a.w, b.w, c.w));
}
__device__ __forceinline__ float4 max3_4(float4 a, float4 b, float4 c) {
    return make_float4(max3f(a.x, b.x, c.x), max3f(a.y, b.y, c.y), max3f(a.z, b.z, c.z), max3f(a.w, b.w, c.w));
}
// a + t (b - a) on packed FP32x2 lanes (each lane rounds like the scalar form)
__device__ __forceinline__ float2 lerp2(float2 a, float2 b, float t) {
    return __ffma2_rn(make_float2(t, t), __fadd2_rn(b, make_float2(-a.x, -a.y)), a);
}
// Bilinear filter of four RGBA texels: x on both rows, then y.
__device__ __forceinline__ float4 bil4(float fx, float fy, float4 h00, float4 h01, float4 h10, float4 h11) {
    const float2 xy = lerp2(lerp2(make_float2(h00.x, h00.y), make_float2(h01.x, h01.y), fx),
                            lerp2(make_float2(h10.x, h10.y), make_float2(h11.x, h11.y), fx), fy);
    const float2 zw = lerp2(lerp2(make_float2(h00.z, h00.w), make_float2(h01.z, h01.w), fx),
                            lerp2(make_float2(h10.z, h10.w), make_float2(h11.z, h11.w), fx), fy);
    return make_float4(xy.x, xy.y, zw.x, zw.y);
}
// TAA blend h + b (c - h) of the clamped history towards the current value
__device__ __forceinline__ float4 blend4(float4 h, float4 c, float b) {
    const float2 xy = lerp2(make_float2(h.x, h.y), make_float2(c.x, c.y), b);
    const float2 zw = lerp2(make_float2(h.z, h.w), make_float2(c.z, c.w), b);
    return make_float4(xy.x, xy.y, zw.x, zw.y);
}

// TAA resolve (Sec. 3.2): reprojected, bilinearly filtered history clamped
// to the current frame's 3x3 range, blended with the current frame.
template <typename H>
__global__ void __launch_bounds__(256) taa_kernel(const H *__restrict__ hist,
                                                  const float4 *__restrict__ cur,
                                                  const float2 *__restrict__ mot,
                                                  H *__restrict__ out, int W, int Hh, float blend,
                                                  unsigned *check) {
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
            if (!in_range(check, xa >= 0 && xb < W && ya >= 0 && yb < Hh, kChkHistory)) return;
            const float4 h00 = load_hist(hist, (size_t)ya * W + xa);
            const float4 h01 = load_hist(hist, (size_t)ya * W + xb);
            const float4 h10 = load_hist(hist, (size_t)yb * W + xa);
            const float4 h11 = load_hist(hist, (size_t)yb * W + xb);
            float4 h = bil4(fx, fy, h00, h01, h10, h11);
            float4 mn = c, mx = c;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny2 = min(max(y + dy, 0), Hh - 1);
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (dx == 0 && dy == 0) continue;
                    const int nx2 = min(max(x + dx, 0), W - 1);
                    if (!in_range(check, nx2 >= 0 && nx2 < W && ny2 >= 0 && ny2 < Hh, kChkHistory)) continue;
                    const float4 v = __ldg(cur + (size_t)ny2 * W + nx2);
                    mn = fmin4(mn, v);
                    mx = fmax4(mx, v);
                }
            }
            res = blend4(fmin4(fmax4(h, mn), mx), c, blend);
        }
    }
    store_hist(out, i, res);
}

// Reprojection and TAA resolve fused (Sec. 3.2): each pixel's motion is
// computed in registers (the motion kernel's arithmetic, bitwise) instead
// of being written and read back; the current frame's 3x3 neighbourhoods come
// from a shared-memory tile with a clamped one-pixel halo, brought in by one
// TMA bulk tensor copy while the motion is computed; each thread resolves
// ResolvePix<H> vertically adjacent pixels, whose 3x3 windows share rows, and
// filters their history footprints before it waits for the tile.
#ifndef CLOUDVOL_TAA_PIX_F32
#define CLOUDVOL_TAA_PIX_F32 4  // pixels per thread, FP32 history (79 registers)
#endif
#ifndef CLOUDVOL_TAA_PIX_F16
#define CLOUDVOL_TAA_PIX_F16 2  // pixels per thread, FP16 history
#endif
template <typename H>
struct ResolvePix {
    static constexpr int value = CLOUDVOL_TAA_PIX_F32;
    static constexpr int rows = 8 * value;  // pixel rows of a tile
};
template <>
struct ResolvePix<uint2> {
    static constexpr int value = CLOUDVOL_TAA_PIX_F16;
    static constexpr int rows = 8 * value;
};
constexpr int kTW = 32;  // pixel tile of a 32x8-thread CTA: 32 x ResolvePix<H>::rows
#ifndef CLOUDVOL_TAA_MIN_BLOCKS
#define CLOUDVOL_TAA_MIN_BLOCKS 3  // CTAs per SM the fused kernel is compiled for
#endif

// Waits that gave up (a bulk copy that did not complete in time): counted on
// the device, read by cloud_device_wait_timeouts; a launch may also be given a
// counter of its own (`status`, device or mapped host memory) that its caller
// reads.  Every wait below is bounded.  The first wait polls `first_polls`
// times (kWaitPolls by default; cloud_debug_set_wait_polls changes it for
// tests); after a give-up one thread waits once more, at most kDrainPolls
// polls with a short sleep between them (about 0.1 s), for the copy already
// issued, so that it lands before the block exits.
__device__ unsigned int g_wait_timeouts = 0;
constexpr int kWaitPolls = 1 << 16;
constexpr int kDrainPolls = 1 << 20;
std::atomic<int> g_first_polls{kWaitPolls};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
// Bounded wait for phase `parity` of an mbarrier: at most `polls` polls
// (with a sleep of `sleep_ns` between them); false when it gave up.
__device__ __forceinline__ bool mbar_wait(const uint64_t *bar, unsigned parity, int polls,
                                          unsigned sleep_ns = 0) {
    const unsigned a = smem_addr(bar);
    for (int it = 0; it < polls; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return false;
}

// One 32x16-pixel tile (bx, by) of the fused resolve: the body of both the
// single-view kernel and the multi-view kernel.  tile_map points to the
// current frame's tensor map (kernel parameter or global memory), tile and bar
// are the block's shared memory.
template <typename H>
__device__ __forceinline__ void resolve_tile(const CUtensorMap *tile_map, const MotionParams &mp,
                                             const H *__restrict__ hist, H *__restrict__ out,
                                             float blend, int bx, int by,
                                             float4 (&tile)[ResolvePix<H>::rows + 2][kTW + 2],
                                             uint64_t &bar, int first_polls, unsigned int *status) {
    constexpr int kPix = ResolvePix<H>::value, kTH = ResolvePix<H>::rows;
    const int W = mp.width, Hh = mp.height;
    const int x0 = bx * kTW, y0 = by * kTH;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = x0 + tx;
    const int tid = ty * 32 + tx;
    // 1. current-frame tile with a one-pixel halo (34 x kTH + 2 texels), one TMA
    //    bulk copy issued by one thread, landing while the motion is computed.
    //    The box starts at texel (x0 - 1, y0 - 1): its x offset in bytes is
    //    16 (x0 - 1), a multiple of 16; texels outside the frame arrive as
    //    zeros and are replaced by their clamped neighbours below.
    //    Thread 0 initialises the barrier and issues the copy; the other
    //    threads only touch the barrier after the __syncthreads below, so the
    //    motion arithmetic starts at once.
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        constexpr unsigned kTileBytes = (kTH + 2) * (kTW + 2) * 16;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     ::"r"(smem_addr(&bar)), "r"(kTileBytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];\n"
            ::"r"(smem_addr(&tile[0][0])), "l"(tile_map), "r"(4 * (x0 - 1)), "r"(y0 - 1),
              "r"(smem_addr(&bar))
            : "memory");
    }
    // 2. motion (registers only) and the history footprint of the thread's
    //    pixels (rows kPix ty .. kPix ty + kPix - 1 of the tile): column terms
    //    once, the pixels' arithmetic interleaved, the rare near-tie calls after
    bool use[kPix];
    float fxs[kPix], fys[kPix];
    float4 h00[kPix], h01[kPix], h10[kPix], h11[kPix];
#pragma unroll
    for (int r = 0; r < kPix; ++r) use[r] = false;
    if (hist && x < W) {
        const MotionCol col = motion_col(mp, x);
        float bs[kPix], lam[kPix];
        bool ex[kPix];
#pragma unroll
        for (int r = 0; r < kPix; ++r) {
            bs[r] = fmaf((float)(y0 + kPix * ty + r), mp.by, mp.b0);
            lam[r] = motion_lambda(mp, col, bs[r], &ex[r]);
        }
#pragma unroll
        for (int r = 0; r < kPix; ++r)
            if (ex[r]) lam[r] = entry_lambda_exact(mp, x, y0 + kPix * ty + r);
#pragma unroll
        for (int r = 0; r < kPix; ++r) {
            const int y = y0 + kPix * ty + r;
            if (y >= Hh) continue;
            const float2 m = motion_project(mp, col, bs[r], lam[r]);
            const float xc = (float)x + 0.5f, yc = (float)y + 0.5f;
            if ((m.x > xc) || (m.x < xc - (float)W) || (m.y > yc) || (m.y < yc - (float)Hh)) continue;
            const float nx = -m.x, ny = -m.y;
            const float flx = floorf(nx), fly = floorf(ny);
            fxs[r] = nx - flx;
            fys[r] = ny - fly;
            const int ix = x + (int)flx, iy = y + (int)fly;
            const int xa = min(max(ix, 0), W - 1), xb = min(max(ix + 1, 0), W - 1);
            const int ya = min(max(iy, 0), Hh - 1), yb = min(max(iy + 1, 0), Hh - 1);
            if (!in_range(mp.check, xa >= 0 && xb < W && ya >= 0 && yb < Hh, kChkHistory)) continue;
            const H *ra = hist + (size_t)ya * W, *rb = hist + (size_t)yb * W;
            h00[r] = load_hist(ra, xa);
            h01[r] = load_hist(ra, xb);
            h10[r] = load_hist(rb, xa);
            h11[r] = load_hist(rb, xb);
            use[r] = true;
        }
    }
    float4 hf[kPix];  // filtered history, before the wait for the tile
#pragma unroll
    for (int r = 0; r < kPix; ++r)
        if (use[r]) hf[r] = bil4(fxs[r], fys[r], h00[r], h01[r], h10[r], h11[r]);
    __syncthreads();  // the barrier's initialisation is visible to every thread
    const bool landed = mbar_wait(&bar, 0, first_polls);
    if (!__syncthreads_and(landed)) {
        // the copy did not complete within the bounded wait: count it (globally
        // and in the launch's own counter), leave the outputs of this tile
        // unwritten, and give the copy already issued one more bounded wait
        // (about 0.1 s) before the block exits; if that wait also gives up the
        // copy may still be pending, which counts a second time
        if (tid == 0) {
            atomicAdd(&g_wait_timeouts, 1u);
            if (status) atomicAdd_system(status, 1u);
            if (!mbar_wait(&bar, 0, kDrainPolls, 100)) {
                atomicAdd(&g_wait_timeouts, 1u);
                if (status) atomicAdd_system(status, 1u);
            }
        }
        return;
    }
    // texels outside the frame: clamp to the edge (border tiles only); every
    // source is an in-frame texel of the tile and every target an outside one
    const int r_lo = max(0, 1 - y0), r_hi = min(kTH + 1, Hh - y0);
    const int c_lo = max(0, 1 - x0), c_hi = min(kTW + 1, W - x0);
    if (r_lo > 0 || c_lo > 0 || r_hi < kTH + 1 || c_hi < kTW + 1) {
        for (int i = tid; i < (kTH + 2) * (kTW + 2); i += 256) {
            const int r = i / (kTW + 2), c = i - r * (kTW + 2);
            const int rr = min(max(r, r_lo), r_hi), cc = min(max(c, c_lo), c_hi);
            if (!in_range(mp.check, rr >= 0 && rr < kTH + 2 && cc >= 0 && cc < kTW + 2, kChkTile)) continue;
            if (rr != r || cc != c) tile[r][c] = tile[rr][cc];
        }
        __syncthreads();
    }
    if (x >= W) return;
    if (!in_range(mp.check, tx + 2 < kTW + 2 && kPix * ty + kPix + 1 < kTH + 2, kChkTile)) return;
    // 3. 3x3 ranges from the kPix + 2 tile rows the thread's windows cover
    //    (three-input min/max): each row's three texels reduced once, each
    //    pixel combines three row results as soon as its last row is in;
    //    clamp the filtered history, blend
    float4 rmn[kPix + 2], rmx[kPix + 2], cen[kPix + 2];
#pragma unroll
    for (int j = 0; j < kPix + 2; ++j) {
        const float4 a = tile[kPix * ty + j][tx], b = tile[kPix * ty + j][tx + 1],
                     d = tile[kPix * ty + j][tx + 2];
        rmn[j] = min3_4(a, b, d);
        rmx[j] = max3_4(a, b, d);
        cen[j] = b;
        if (j < 2) continue;
        const int r = j - 2;  // the pixel whose window ends at row j
        const int y = y0 + kPix * ty + r;
        if (y >= Hh) continue;
        const float4 c = cen[r + 1];
        float4 res = c;
        if (use[r]) {
            const float4 mn = min3_4(rmn[r], rmn[r + 1], rmn[r + 2]);
            const float4 mx = max3_4(rmx[r], rmx[r + 1], rmx[r + 2]);
            res = blend4(fmin4(fmax4(hf[r], mn), mx), c, blend);
        }
        if (in_range(mp.check, y >= 0 && x >= 0, kChkPixel)) store_hist(out, (size_t)y * W + x, res);
    }
}

template <typename H>
__global__ void __launch_bounds__(256, CLOUDVOL_TAA_MIN_BLOCKS)
    taa_reproject_kernel(const __grid_constant__ CUtensorMap tile_map,
                         const __grid_constant__ MotionParams mp, const H *__restrict__ hist,
                         H *__restrict__ out, float blend, int first_polls, unsigned int *status) {
    __shared__ __align__(128) float4 tile[ResolvePix<H>::rows + 2][kTW + 2];
    __shared__ __align__(8) uint64_t bar;
    resolve_tile<H>(&tile_map, mp, hist, out, blend, blockIdx.x, blockIdx.y, tile, bar, first_polls,
                    status);
}

// Many views' resolves in one launch (the render server's batches): block b
// is tile b of the concatenated views' tile lists; its view is found by
// binary search over the views' first tiles and its motion constants staged
// in shared memory.  Each tile is computed exactly as by taa_reproject_kernel.
struct alignas(128) ResolveView {  // the tensor map's own alignment
    CUtensorMap map;  // the view's current frame
    MotionParams mp;
    const void *hist;
    void *out;
    float blend;
    int tiles_x, tile_begin;
};

template <typename H>
__global__ void __launch_bounds__(256, CLOUDVOL_TAA_MIN_BLOCKS)
    taa_reproject_batch_kernel(const ResolveView *__restrict__ views, int n_views, int first_polls,
                               unsigned int *status) {
    __shared__ __align__(128) float4 tile[ResolvePix<H>::rows + 2][kTW + 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ MotionParams smp;
    __shared__ int s_view;
    const int t = blockIdx.x, tid = threadIdx.y * 32 + threadIdx.x;
    if (tid == 0) {
        int lo = 0, hi = n_views - 1;  // last view with tile_begin <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (views[mid].tile_begin <= t) lo = mid;
            else hi = mid - 1;
        }
        s_view = lo;
    }
    __syncthreads();
    const ResolveView &rv = views[s_view];
    const int *src = reinterpret_cast<const int *>(&rv.mp);
    int *dst = reinterpret_cast<int *>(&smp);
    for (int i = tid; i < (int)(sizeof(MotionParams) / 4); i += 256) dst[i] = src[i];
    __syncthreads();
    const int local = t - rv.tile_begin;
    if (!in_range(smp.check, s_view >= 0 && s_view < n_views && local >= 0, kChkView)) return;
    resolve_tile<H>(&rv.map, smp, (const H *)rv.hist, (H *)rv.out, rv.blend, local % rv.tiles_x,
                    local / rv.tiles_x, tile, bar, first_polls, status);
}

int build_motion_params(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                        const cloud_camera *cur, int width, int height, MotionParams *p) {
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: width/height outside [1, 16384]");
    if (!(cur->tan_half_fovy > 0.0) || !(prev->tan_half_fovy > 0.0) || !(prm->t_max_m > 0.0))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_motion: bad camera or t_max");
    *p = MotionParams{};
    const double aspect = (double)width / (double)height;
    const double aT = aspect * cur->tan_half_fovy, aTp = aspect * prev->tan_half_fovy;
    const double T = cur->tan_half_fovy, Tp = prev->tan_half_fovy;
    p->a0 = (float)((1.0 / width - 1.0) * aT);
    p->ax = (float)(2.0 * aT / width);
    p->b0 = (float)((1.0 - 1.0 / height) * T);
    p->by = (float)(-2.0 * T / height);
    p->rz = (float)cur->right[2];
    p->uz = (float)cur->up[2];
    p->fz = (float)cur->forward[2];
    p->zlo = (float)(vol->desc.slab_lo_m - cur->pos[2]);
    p->zhi = (float)(vol->desc.slab_hi_m - cur->pos[2]);
    p->tmax = (float)prm->t_max_m;
    // rows of R (current) and R' (previous): right, up, forward
    const double *R[3] = {cur->right, cur->up, cur->forward};
    const double *Rp[3] = {prev->right, prev->up, prev->forward};
    for (int i = 0; i < 3; ++i) {
        double dl = 0.0;
        for (int k = 0; k < 3; ++k) dl += Rp[i][k] * (cur->pos[k] - prev->pos[k]);
        p->dlt[i] = (float)dl;
        for (int j = 0; j < 3; ++j) {
            double mij = 0.0;  // (R' R^T)_ij = Rp_i . R_j
            for (int k = 0; k < 3; ++k) mij += Rp[i][k] * R[j][k];
            p->G[i][j] = (float)(mij - (i == j ? 1.0 : 0.0));
        }
    }
    p->kx = (float)(aTp / aT);
    p->ky = (float)(Tp / T);
    p->kx1 = (float)((aTp - aT) / aT);
    p->ky1 = (float)((Tp - T) / T);
    p->sx = (float)(width / (2.0 * aTp));
    p->sy = (float)(height / (2.0 * Tp));
    p->width = width;
    p->height = height;
    p->cam_in_layer = cur->pos[2] >= vol->desc.slab_lo_m && cur->pos[2] <= vol->desc.slab_hi_m;
    const double a0 = (1.0 / width - 1.0) * aT, ax = 2.0 * aT / width;
    const double b0 = (1.0 - 1.0 / height) * T, by = -2.0 * T / height;
    for (int k = 0; k < 3; ++k) {
        split_df(cur->forward[k] + a0 * cur->right[k] + b0 * cur->up[k], &p->v00h[k], &p->v00l[k]);
        split_df10(ax * cur->right[k], &p->vxh[k], &p->vxl[k]);
        split_df10(by * cur->up[k], &p->vyh[k], &p->vyl[k]);
    }
    split_df(vol->desc.slab_lo_m - cur->pos[2], &p->zlo_h, &p->zlo_l);
    split_df(vol->desc.slab_hi_m - cur->pos[2], &p->zhi_h, &p->zhi_l);
    split_df(prm->t_max_m, &p->tmax_h, &p->tmax_l);
    p->check = check_word();
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
                                                  width, height, blend, check_word());
    else
        taa_kernel<uint2><<<grid, block, 0, s>>>((const uint2 *)history, (const float4 *)current,
                                                 (const float2 *)motion, (uint2 *)history_out,
                                                 width, height, blend, check_word());
    return check_launch("taa_kernel");
}

// Tensor map of the current frame for the resolve's tile copy: the frame as
// a 2-D FP32 array of 4 W x H elements (row stride 16 W bytes), box 4 (kTW + 2)
// x (rows + 2) elements, zero fill outside.  The encoder is the driver's,
// fetched through the runtime once.
static int current_tile_map(const float *current, int width, int height, int rows, CUtensorMap *map) {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return set_error(CLOUD_ERR_CUDA, "cloud_taa_reproject: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {4ull * (cuuint64_t)width, (cuuint64_t)height};
    const cuuint64_t strides[1] = {16ull * (cuuint64_t)width};
    const cuuint32_t box[2] = {4u * (kTW + 2), (cuuint32_t)(rows + 2)};
    const cuuint32_t elem[2] = {1u, 1u};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(current), dims,
                              strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(CLOUD_ERR_CUDA, "cloud_taa_reproject: tensor map rejected");
    return CLOUD_OK;
}

int launch_taa_reproject(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                         const cloud_camera *cur, const void *history, const float *current,
                         void *history_out, int width, int height, int fmt, float blend,
                         unsigned int *status, cudaStream_t s) {
    if (!vol || !prm || !cur || !current || !history_out || (history && !prev))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_taa_reproject: null pointer");
    if (fmt != CLOUD_HISTORY_FP32 && fmt != CLOUD_HISTORY_FP16)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_taa_reproject: bad history format");
    if (!(blend >= 0.0f && blend <= 1.0f))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_taa_reproject: blend outside [0, 1]");
    MotionParams p;
    if (int rc = build_motion_params(vol, prm, history ? prev : cur, cur, width, height, &p)) return rc;
    const size_t px = (size_t)width * height, eb = fmt == CLOUD_HISTORY_FP32 ? 16 : 8;
    if (!aligned(current, 16) || !aligned(history_out, eb) || (history && !aligned(history, eb)))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_taa_reproject: misaligned buffer");
    if (history) {
        const char *a = (const char *)history, *b = (const char *)history_out;
        if (a < b + px * eb && b < a + px * eb)
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_taa_reproject: history and history_out overlap");
    }
    const int rows = fmt == CLOUD_HISTORY_FP32 ? ResolvePix<float4>::rows : ResolvePix<uint2>::rows;
    CUtensorMap map;
    if (int rc = current_tile_map(current, width, height, rows, &map)) return rc;
    const dim3 grid((width + kTW - 1) / kTW, (height + rows - 1) / rows), block(32, 8);
    const int polls = g_first_polls.load();
    if (fmt == CLOUD_HISTORY_FP32)
        taa_reproject_kernel<float4><<<grid, block, 0, s>>>(map, p, (const float4 *)history,
                                                            (float4 *)history_out, blend, polls,
                                                            status);
    else
        taa_reproject_kernel<uint2><<<grid, block, 0, s>>>(map, p, (const uint2 *)history,
                                                           (uint2 *)history_out, blend, polls,
                                                           status);
    return check_launch("taa_reproject_kernel");
}

int launch_taa_reproject_batch(const cloud_volume *vol, const cloud_params *prm,
                               const ResolveRequest *reqs, int n, int fmt, float blend,
                               void *h_table_v, void *d_table_v, unsigned int *status,
                               cudaStream_t s) {
    if (!vol || !prm || !reqs || n < 1 || !h_table_v || !d_table_v)
        return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: bad arguments");
    if (fmt != CLOUD_HISTORY_FP32 && fmt != CLOUD_HISTORY_FP16)
        return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: bad history format");
    if (!(blend >= 0.0f && blend <= 1.0f))
        return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: blend outside [0, 1]");
    ResolveView *h_table = static_cast<ResolveView *>(h_table_v);
    int next = 0;
    const size_t eb = fmt == CLOUD_HISTORY_FP32 ? 16 : 8;
    const int rows = fmt == CLOUD_HISTORY_FP32 ? ResolvePix<float4>::rows : ResolvePix<uint2>::rows;
    for (int i = 0; i < n; ++i) {
        const ResolveRequest &r = reqs[i];
        if (!r.cur || !r.current || !r.out || (r.history && !r.prev))
            return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: null pointer");
        ResolveView &v = h_table[i];
        if (int rc = build_motion_params(vol, prm, r.history ? r.prev : r.cur, r.cur, r.width,
                                         r.height, &v.mp))
            return rc;
        const size_t px = (size_t)r.width * r.height;
        if (!aligned(r.current, 16) || !aligned(r.out, eb) || (r.history && !aligned(r.history, eb)))
            return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: misaligned buffer");
        if (r.history) {
            const char *a = (const char *)r.history, *b = (const char *)r.out;
            if (a < b + px * eb && b < a + px * eb)
                return set_error(CLOUD_ERR_INVALID_ARG, "resolve batch: history and output overlap");
        }
        if (int rc = current_tile_map(r.current, r.width, r.height, rows, &v.map)) return rc;
        v.hist = r.history;
        v.out = r.out;
        v.blend = blend;
        v.tiles_x = (r.width + kTW - 1) / kTW;
        v.tile_begin = next;
        next += v.tiles_x * ((r.height + rows - 1) / rows);
    }
    if (int rc = check_cuda(cudaMemcpyAsync(d_table_v, h_table, sizeof(ResolveView) * n,
                                            cudaMemcpyHostToDevice, s),
                            "resolve batch: upload table"))
        return rc;
    const ResolveView *d_table = static_cast<const ResolveView *>(d_table_v);
    const int polls = g_first_polls.load();
    if (fmt == CLOUD_HISTORY_FP32)
        taa_reproject_batch_kernel<float4><<<next, dim3(32, 8), 0, s>>>(d_table, n, polls, status);
    else
        taa_reproject_batch_kernel<uint2><<<next, dim3(32, 8), 0, s>>>(d_table, n, polls, status);
    return check_launch("taa_reproject_batch_kernel");
}

size_t resolve_view_bytes() { return sizeof(ResolveView); }

// Composite (Sec. 3.2): the low-resolution cloud buffer, resampled
// bilinearly to the display size, laid over the background (premultiplied
// "over").  Streaming: the background is read and the result written once
// (32 B per pixel); the small cloud buffer is served by L1/L2.
// Source texel coordinate of output pixel x: u = (2x + 1) sw / (2 dw) - 1/2,
// split into floor(u) and frac(u) with integer arithmetic so that the texel
// choice is exact and frac is one correctly rounded division.
__device__ __forceinline__ void src_coord(int x, int sw, int dw, int &i0, float &f) {
    const int num = (2 * x + 1) * sw - dw, den = 2 * dw;  // < 2^31 for sizes <= 16384
    const int q = num >= 0 ? num / den : -1;              // num >= -dw > -den
    f = (float)(num - q * den) / (float)den;
    i0 = q;
}

template <typename H>
__global__ void __launch_bounds__(256) composite_kernel(const H *__restrict__ cloud, int sw, int sh,
                                                        const float4 *__restrict__ bg, float4 *out,
                                                        int dw, int dh, unsigned *check) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= dw || y >= dh) return;
    int u0, v0;
    float fx, fy;
    src_coord(x, sw, dw, u0, fx);
    src_coord(y, sh, dh, v0, fy);
    const int xa = max(u0, 0), xb = min(u0 + 1, sw - 1);
    const int ya = max(v0, 0), yb = min(v0 + 1, sh - 1);
    if (!in_range(check, xa < sw && xb >= 0 && ya < sh && yb >= 0, kChkHistory)) return;
    const float4 c00 = load_hist(cloud, (size_t)ya * sw + xa), c01 = load_hist(cloud, (size_t)ya * sw + xb);
    const float4 c10 = load_hist(cloud, (size_t)yb * sw + xa), c11 = load_hist(cloud, (size_t)yb * sw + xb);
    const float4 c = bil4(fx, fy, c00, c01, c10, c11);
    const size_t i = (size_t)y * dw + x;
    const float4 b = __ldg(bg + i);
    const float t = 1.0f - c.w;
    out[i] = make_float4(fmaf(t, b.x, c.x), fmaf(t, b.y, c.y), fmaf(t, b.z, c.z), fmaf(t, b.w, c.w));
}

int launch_composite(const void *cloud, int fmt, int sw, int sh, const float *bg, float *out, int dw,
                     int dh, cudaStream_t s) {
    if (!cloud || !bg || !out) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_composite: null pointer");
    if (sw < 1 || sh < 1 || dw < 1 || dh < 1 || sw > CLOUD_MAX_DIM || sh > CLOUD_MAX_DIM ||
        dw > CLOUD_MAX_DIM || dh > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_composite: sizes outside [1, 16384]");
    if (fmt != CLOUD_HISTORY_FP32 && fmt != CLOUD_HISTORY_FP16)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_composite: bad cloud format");
    if (!aligned(cloud, fmt == CLOUD_HISTORY_FP32 ? 16 : 8) || !aligned(bg, 16) || !aligned(out, 16))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_composite: misaligned buffer");
    const dim3 grid((dw + 31) / 32, (dh + 7) / 8), block(32, 8);
    if (fmt == CLOUD_HISTORY_FP32)
        composite_kernel<float4><<<grid, block, 0, s>>>((const float4 *)cloud, sw, sh, (const float4 *)bg,
                                                        (float4 *)out, dw, dh, check_word());
    else
        composite_kernel<uint2><<<grid, block, 0, s>>>((const uint2 *)cloud, sw, sh, (const float4 *)bg,
                                                       (float4 *)out, dw, dh, check_word());
    return check_launch("composite_kernel");
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

extern "C" int cloud_taa_reproject(const cloud_volume *vol, const cloud_params *prm,
                                   const cloud_camera *prev, const cloud_camera *cur,
                                   const void *history, const float *current, void *history_out,
                                   int width, int height, int history_fmt, float blend,
                                   void *stream) {
    clear_error();
    return launch_taa_reproject(vol, prm, prev, cur, history, current, history_out, width, height,
                                history_fmt, blend, nullptr, (cudaStream_t)stream);
}

extern "C" int cloud_composite(const void *cloud, int cloud_fmt, int cloud_width, int cloud_height,
                               const float *background, float *out, int width, int height,
                               void *stream) {
    clear_error();
    return launch_composite(cloud, cloud_fmt, cloud_width, cloud_height, background, out, width,
                            height, (cudaStream_t)stream);
}

extern "C" int cloud_device_wait_timeouts(unsigned int *count, int reset) {
    clear_error();
    if (!count) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_device_wait_timeouts: null pointer");
    if (int rc = check_cuda(cudaMemcpyFromSymbol(count, g_wait_timeouts, sizeof(unsigned int)),
                            "cloud_device_wait_timeouts"))
        return rc;
    if (reset) {
        const unsigned int zero = 0;
        return check_cuda(cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(unsigned int)),
                          "cloud_device_wait_timeouts");
    }
    return CLOUD_OK;
}

extern "C" int cloud_debug_set_wait_polls(int first_polls) {
    clear_error();
    if (first_polls > (1 << 30))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_debug_set_wait_polls: more than 2^30 polls");
    g_first_polls.store(first_polls < 0 ? kWaitPolls : first_polls);
    return CLOUD_OK;
}
