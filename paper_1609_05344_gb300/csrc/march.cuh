// march.cuh -- device side of the per-pixel cloud raymarch (Sec. 1, Sec. 3.1,
// Sec. 3.2), shared by the single-view kernel (render.cu) and the persistent
// multi-view kernel (batch.cu).
//
// Precision design.  Grazing rays are tens of kilometres long and, with 8
// view steps, a step is kilometres long; the estimator then multiplies any
// density error by alpha*D*L_in (hundreds), so sample positions must be far
// more accurate than FP32 world coordinates allow.  Per ray, the start and
// the step of every lattice axis (base xyz, detail xyz, weather xy) and of the
// height above the layer bottom are computed in double-float FP32 and stored
// as 32-bit fixed-point values: 2^32 units per tile period, so unsigned
// overflow is exactly the periodic wrap of the tile.  A view step adds the
// ray's increment and a light sample adds a per-launch constant offset --
// integer adds, no rounding.  The texel index is the top log2(N) bits, the
// interpolation weight the next 23 bits.  Radiance and the optical-depth sum
// are FP32.
#pragma once

#include "common.cuh"

// CTAs per SM the march is compiled for (register budget 65536 / (128 x this)),
// for FP32 records and for 16-bit records (which need fewer registers).
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_F32
#define CLOUDVOL_MARCH_MIN_BLOCKS_F32 5
#endif
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_16
#define CLOUDVOL_MARCH_MIN_BLOCKS_16 6
#endif

namespace cloudvol {

// Records at the standard tile sizes, 8 view steps per warp iteration: 8 CTAs
// (64 registers, no spills; FP32 148.8 us at fast-1080p against 154.5 us with
// 7 and 154.2 us with 9; FP16 152.4 us against 153.0 us with 7).  With 16 steps
// per iteration the per-warp scratch is 1.7x larger and 8 CTAs would leave the
// L1 28 KB: 7 CTAs for FP32 records and 6 for 16-bit ones (the 64-view batch,
// BF16: 18.7 ms against 19.5 ms with 8).
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX
#define CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX 8
#endif
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_16_FX
#define CLOUDVOL_MARCH_MIN_BLOCKS_16_FX 8
#endif
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX16
#define CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX16 7
#endif
#ifndef CLOUDVOL_MARCH_MIN_BLOCKS_16_FX16
#define CLOUDVOL_MARCH_MIN_BLOCKS_16_FX16 6
#endif
template <typename T, bool FX, int CH>
struct MarchBlocks {
    static constexpr bool f32 = sizeof(T) == 4;
    static constexpr int value =
        !FX ? (f32 ? CLOUDVOL_MARCH_MIN_BLOCKS_F32 : CLOUDVOL_MARCH_MIN_BLOCKS_16)
        : CH <= 8 ? (f32 ? CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX : CLOUDVOL_MARCH_MIN_BLOCKS_16_FX)
                  : (f32 ? CLOUDVOL_MARCH_MIN_BLOCKS_F32_FX16 : CLOUDVOL_MARCH_MIN_BLOCKS_16_FX16);
};

// The standard tile sizes (128^3 base, 32^3 detail, 512^2 weather records) as
// compile-time constants: with FX the record-index and weight shifts of every
// lookup are immediates instead of per-launch values.
constexpr int kStdLog2Base = 7, kStdLog2Detail = 5, kStdLog2Weather = 9;

// Light samples of a march evaluated per iteration of the light loop (the
// density code is inlined that many times).
#ifndef CLOUDVOL_LIGHT_UNROLL_F32
#define CLOUDVOL_LIGHT_UNROLL_F32 6
#endif
#ifndef CLOUDVOL_LIGHT_UNROLL_16
#define CLOUDVOL_LIGHT_UNROLL_16 2
#endif
// View lookups a lane evaluates per round of the shared-out view phase (their
// record loads can overlap; more of them cost registers): one for FP32
// records; for 16-bit records one with 8 view steps per iteration (the
// registers buy an eighth CTA per SM instead) and two with 16.
#ifndef CLOUDVOL_VIEW_BATCH_F32
#define CLOUDVOL_VIEW_BATCH_F32 1
#endif
#ifndef CLOUDVOL_VIEW_BATCH_16
#define CLOUDVOL_VIEW_BATCH_16 1
#endif
#ifndef CLOUDVOL_VIEW_BATCH_16_CH16
#define CLOUDVOL_VIEW_BATCH_16_CH16 2
#endif
template <typename T, int CH>
struct ViewBatch {
    static constexpr int value = sizeof(T) == 4 ? CLOUDVOL_VIEW_BATCH_F32
                                 : CH <= 8      ? CLOUDVOL_VIEW_BATCH_16
                                                : CLOUDVOL_VIEW_BATCH_16_CH16;
};
template <typename T>
struct LightUnroll { static constexpr int value = CLOUDVOL_LIGHT_UNROLL_16; };
template <>
struct LightUnroll<float> { static constexpr int value = CLOUDVOL_LIGHT_UNROLL_F32; };

enum Axis { kBX = 0, kBY, kBZ, kDX, kDY, kDZ, kWX, kWY, kLatticeAxes };

// Constants shared by every view of a launch: volume, lighting, light march.
struct SceneParams {
    // Fixed-point lattice coordinates: coordinate = p * kfix - half_unit
    // (mod 2^32), kfix = 2^32 / tile period.
    float kfix_h[kLatticeAxes], kfix_l[kLatticeAxes];
    uint32_t half_unit[kLatticeAxes];                    // half a texel: 2^(31 - log2 N)
    uint32_t loff[CLOUD_MAX_LIGHT_STEPS][kLatticeAxes];  // light-sample offsets
    int32_t lh[CLOUD_MAX_LIGHT_STEPS];                   // light-sample height offsets
    int32_t h_top;                                       // layer thickness in 2^-16 m
    float h_lo_scale, h_hi_scale;  // 10/thickness, 2.5/thickness, per 2^-16 m
    float sun[3], sun_rad[3], ambient[3];
    float hg_g, hg_norm, absorption, light_step, tau_max;  // hg_norm = (1 - g^2)/(4 pi)
    // k0 = 1/2 - c - w_d/2 minus the record decode bias b folded in:
    // k0 - b + w_d b; w_off = 1/2 - b (weather values are stored centred)
    float k0, inv_1mc, detail_w, rho0, w_off;
    // occupancy grid of the volume (bit set: density may be > 0 somewhere in
    // the macro-cell of 2^kOccShift records per axis), or nullptr; log2 of its
    // cells per axis
    const uint32_t *occ;
    int log2_occ;
    unsigned *check;  // status word of the checked build, else nullptr
    int log2_base, log2_detail, log2_weather;
    int light_steps, integration, constant_mode;
    // detail coordinates = (base + half_base) << detail_shift - half_detail when
    // the base tile period is 2^detail_shift detail periods (-1: convert separately)
    int detail_shift;
    uint32_t jitter_key;
};

// One camera view: rays, layer clip, step count, jitter frame, output.
struct ViewParams {
    // Camera rays, unnormalised: v(x, y) = v00 + x vx + y vy, as double-float
    // pairs; vx/vy are split so that x * hi is exact (see split_df10).
    float v00h[3], v00l[3], vxh[3], vxl[3], vyh[3], vyl[3];
    float oh[3], ol[3];    // camera position
    float zlo_h, zlo_l;    // slab_lo - o_z
    float zhi_h, zhi_l;    // slab_hi - o_z
    float tmax_h, tmax_l;  // far clip distance
    float invn_h, invn_l;  // 1 / steps
    // rays with d_z below miss_below (camera under the layer) or above
    // miss_above (camera over it) cannot reach the layer within t_max
    float miss_below, miss_above;
    int cam_in_layer, width, height, steps, jitter_frame;
    float u_frame;   // >= 0: the start offset of every ray (per-frame jitter); < 0: per pixel
    int tiles_x;     // tiles per image row
    int tile_begin;  // first work-queue index of this view (multi-view launches)
    int tile_count;
    float4 *out;     // device RGBA, width * height
};

// CTA pixel-tile shapes (4 warps of 32 lanes); the autotuner picks one.
//   shape 0: warp 8x4,  CTA 2x2 warps -> 16x8 pixels
//   shape 1: warp 8x4,  CTA 4x1 warps -> 32x4 pixels
//   shape 2: warp 16x2, CTA 2x2 warps -> 32x4 pixels
//   shape 3: warp 4x8,  CTA 2x2 warps -> 8x16 pixels
constexpr int kShapes = 4;
template <int S>
struct TileShape;
template <>
struct TileShape<0> { static constexpr int WX = 8, WY = 4, CX = 2, CY = 2; };
template <>
struct TileShape<1> { static constexpr int WX = 8, WY = 4, CX = 4, CY = 1; };
template <>
struct TileShape<2> { static constexpr int WX = 16, WY = 2, CX = 2, CY = 2; };
template <>
struct TileShape<3> { static constexpr int WX = 4, WY = 8, CX = 2, CY = 2; };
inline void tile_dims(int shape, int *tw, int *th) {
    static const int w[kShapes] = {16, 32, 32, 8}, h[kShapes] = {8, 4, 4, 16};
    *tw = w[shape];
    *th = h[shape];
}

constexpr int kAxes = kLatticeAxes + 1;  // lattice axes + height above the layer bottom
// Launch configurations the autotuner chooses from: a pixel-tile shape and the
// number of view steps a warp evaluates per iteration of its march (the chunk
// of phase A/B/C below).  config = shape + kShapes * chunk index.
constexpr int CHSizes[2] = {8, 16};
constexpr int kConfigs = kShapes * 2;
inline int config_shape(int config) { return config % kShapes; }
inline int config_chunk(int config) { return CHSizes[(config / kShapes) & 1]; }
constexpr unsigned kFull = 0xFFFFFFFFu;

// Axes whose start and increment a warp stages for step_coords: all of them,
// or (FX: the base tile period is 2^detail_shift detail periods) the base,
// weather and height axes only, the detail coordinates following from the
// base ones by an exact shift.
template <bool FX>
struct StagedAxes { static constexpr int value = kAxes; };
template <>
struct StagedAxes<true> { static constexpr int value = 6; };  // BX BY BZ WX WY, height

// Per-warp shared scratch of the march: each lane's start coordinates and
// per-step increments, the chunk's view densities, light-march sums and the
// list of (step, lane) pairs that need a light march (CH view steps a chunk).
template <int CH, bool FX>
struct WarpScratch {
    uint32_t c0[StagedAxes<FX>::value][32];
    uint32_t e[StagedAxes<FX>::value][32];
    float rho[CH][32];
    float lsum[CH][32];
    uint16_t pairs[CH * 32];
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
// (z0, z1) pairs of both y rows (the x differences come with the record),
// then y on the pair, then z.  Each lane of a packed op rounds exactly like
// the scalar op.
__device__ __forceinline__ float trilerp(const float c[8], int L, uint32_t cx, uint32_t cy,
                                         uint32_t cz) {
    const float fx = frac23(cx << L), fy = frac23(cy << L), fz = frac23(cz << L);
    const float2 a0 = make_float2(c[0], c[1]), a1 = make_float2(c[2], c[3]);  // dx = 0
    const float2 d0 = make_float2(c[4], c[5]), d1 = make_float2(c[6], c[7]);  // dx = 1 minus dx = 0
    const float2 fx2 = make_float2(fx, fx), fy2 = make_float2(fy, fy);
    const float2 x0 = __ffma2_rn(fx2, d0, a0);  // dy = 0
    const float2 x1 = __ffma2_rn(fx2, d1, a1);  // dy = 1
    const float2 yz = __ffma2_rn(fy2, __fadd2_rn(x1, make_float2(-x0.x, -x0.y)), x0);  // (z0, z1)
    return fmaf(fz, yz.y - yz.x, yz.x);
}
__device__ __forceinline__ float bilerp(const float c[4], int L, uint32_t cx, uint32_t cy) {
    const float fx = frac23(cx << L), fy = frac23(cy << L);
    const float2 a = make_float2(c[0], c[1]), d = make_float2(c[2], c[3]);  // (y0, y1): dx = 0, difference
    const float2 xy = __ffma2_rn(make_float2(fx, fx), d, a);
    return fmaf(fy, xy.y - xy.x, xy.x);
}

// Height profile g(h) of the layer at a fixed-point height (2^-16 m above the
// layer bottom): clamp(h / 0.1, 0, 1) clamp((1 - h) / 0.4, 0, 1), h in layer
// thicknesses.
__device__ __forceinline__ float height_profile(const SceneParams &p, int32_t hq) {
    const float ga = fminf(fmaxf((float)hq * p.h_lo_scale, 0.0f), 1.0f);
    const float gb = fminf(fmaxf((float)(p.h_top - hq) * p.h_hi_scale, 0.0f), 1.0f);
    return ga * gb;
}

// Occupancy bit of the macro-cell holding a sample's base record: clear where
// the volume's bound proves B - w_d Dt - c < 0, i.e. zero density.
template <bool FX>
__device__ __forceinline__ bool occupied(const SceneParams &p, uint32_t bx, uint32_t by, uint32_t bz) {
    // macro-cell = record index >> kOccShift on each axis; bits x fastest
    const int lo = FX ? kStdLog2Base - kOccShift : p.log2_occ, sh = 32 - lo;
    const uint32_t cell = ((bz >> sh) << (2 * lo)) | ((by >> sh) << lo) | (bx >> sh);
    if (!in_range(p.check, cell < (1u << (3 * lo)), kChkOccupancy)) return true;
    return (__ldg(p.occ + (cell >> 5)) >> (cell & 31u)) & 1u;
}

// Density at a sample (Sec. 1):
//   rho = g(h) W max(0, (B - w_d Dt - c)/(1 - c)),
// tiles stored centred (value - 1/2), so (B - w_d Dt - c) = Bc - w_d Dtc + k0;
// the records' decode bias is folded into k0 and w_off.
// Samples outside the layer (g = 0) return without touching memory; the
// three record loads are issued together so that one memory round trip serves
// the lookup.
template <bool FX, typename T>
__device__ __forceinline__ float density(const SceneParams &p, const T *__restrict__ base,
                                         const T *__restrict__ detail,
                                         const T *__restrict__ weather, const uint32_t c[8],
                                         int32_t hq) {
    const int lb = FX ? kStdLog2Base : p.log2_base, ld = FX ? kStdLog2Detail : p.log2_detail,
              lw = FX ? kStdLog2Weather : p.log2_weather;
    if (!FX && p.constant_mode) return p.rho0;
    const float g = height_profile(p, hq);
    if (g <= 0.0f) return 0.0f;
    float cb[8], cd[8], cw[4];
    const uint32_t rb = rec3(lb, c[kBX], c[kBY], c[kBZ]), rd = rec3(ld, c[kDX], c[kDY], c[kDZ]),
                   rw = rec2(lw, c[kWX], c[kWY]);
    if (!in_range(p.check,
                  rb < (1u << (3 * lb)) && (!(FX || detail) || rd < (1u << (3 * ld))) &&
                      (!(FX || weather) || rw < (1u << (2 * lw))),
                  kChkRecord))
        return 0.0f;
    const float ob = load_rec8(base, rb, cb);
    float od = 0.0f, ow = 0.0f;
    if (FX || detail) od = load_rec8(detail, rd, cd);
    if (FX || weather) ow = load_rec4(weather, rw, cw);
    const float b = trilerp(cb, lb, c[kBX], c[kBY], c[kBZ]) + ob;
    float r = b + p.k0;
    if (FX || detail) {
        const float dt = trilerp(cd, ld, c[kDX], c[kDY], c[kDZ]) + od;
        r = fmaf(-p.detail_w, dt, r);
    }
    r = fmaxf(r * p.inv_1mc, 0.0f);
    const float w = (FX || weather) ? bilerp(cw, lw, c[kWX], c[kWY]) + ow + p.w_off : 1.0f;
    return g * w * r;
}

// Staging of one lane's start coordinates and increments (lattice axes, then
// the height) into the warp's scratch.
template <int CH, bool FX>
__device__ __forceinline__ void stage_coords(WarpScratch<CH, FX> &ws, unsigned lane,
                                             const uint32_t c[kLatticeAxes],
                                             const uint32_t e[kLatticeAxes], int32_t hq, int32_t eh) {
    constexpr int kS = StagedAxes<FX>::value;
#pragma unroll
    for (int a = 0, s = 0; a < kLatticeAxes; ++a) {
        if (FX && a >= kDX && a <= kDZ) continue;
        ws.c0[s][lane] = c[a];
        ws.e[s][lane] = e[a];
        ++s;
    }
    ws.c0[kS - 1][lane] = (uint32_t)hq;
    ws.e[kS - 1][lane] = (uint32_t)eh;
}

// Coordinates of view step i of ray `ow` of the warp from its staged start and
// increment (integer arithmetic: the same values as adding the increment step
// by step; for FX the detail coordinates are the base ones shifted exactly,
// as the ray setup derives them).  Returns the height.
template <int CH, bool FX>
__device__ __forceinline__ int32_t step_coords(const SceneParams &p, const WarpScratch<CH, FX> &ws,
                                               unsigned ow, uint32_t i, uint32_t cs[kLatticeAxes]) {
    constexpr int kS = StagedAxes<FX>::value;
#pragma unroll
    for (int a = 0, s = 0; a < kLatticeAxes; ++a) {
        if (FX && a >= kDX && a <= kDZ) {
            const int b = a - kDX;
            cs[a] = ((cs[b] + p.half_unit[b]) << p.detail_shift) - p.half_unit[a];
            continue;
        }
        cs[a] = ws.c0[s][ow] + i * ws.e[s][ow];
        ++s;
    }
    return (int32_t)(ws.c0[kS - 1][ow] + i * ws.e[kS - 1][ow]);
}

// sigma D of one step, rounded the same way wherever it is recomputed
__device__ __forceinline__ float step_depth(float absorption, float rho, float D) {
    return __fmul_rn(__fmul_rn(absorption, rho), D);
}

// The march of one CTA pixel tile (4 warps, one pixel per lane).  View steps
// are processed in chunks of CH:
//   A  view densities and the early out (the optical depth does not depend on
//      the lighting): each lane marks which of its steps need a lookup (inside
//      the layer, occupied macro-cell), the warp shares those lookups out over
//      all 32 lanes, ViewBatch per lane at a time, and each lane then walks its
//      own steps in order for the optical depth and the early out;
//   B  the warp shares out every (step, lane) light march with density > 0
//      over all 32 lanes, so lanes whose own rays are empty, finished or
//      outside the layer do useful work;
//   C  each lane integrates its steps in order with the light sums from B.
// The arithmetic of every sample is the same as a per-lane march (a skipped
// lookup is one whose density is exactly 0).  Returns the number of density
// lookups this lane's ray performed in the method's sense (Sec. 1: one per
// view step walked, plus the light steps of each step with density).
template <typename T, int LS, int SHAPE, bool FX, int CH>
__device__ __forceinline__ unsigned long long march_tile(
    const SceneParams &p, const ViewParams &v, int tile_x, int tile_y, WarpScratch<CH, FX> &ws,
    const T *__restrict__ base, const T *__restrict__ detail, const T *__restrict__ weather) {
    using S = TileShape<SHAPE>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = tile_x * (S::WX * S::CX) + (warp % S::CX) * S::WX + (lane % S::WX);
    const int y = tile_y * (S::WY * S::CY) + (warp / S::CX) * S::WY + (lane / S::WX);
    const bool in_image = x < v.width && y < v.height;
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
        const float qx = fmaf(yf, v.vyh[0], fmaf(xf, v.vxh[0], v.v00h[0]));
        const float qy = fmaf(yf, v.vyh[1], fmaf(xf, v.vxh[1], v.v00h[1]));
        const float qz = fmaf(yf, v.vyh[2], fmaf(xf, v.vxh[2], v.v00h[2]));
        const float dz = qz * rsqrtf(fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
        if (dz < v.miss_below || dz > v.miss_above) inside = false;
    }
    if (inside) {
        // --- a1: pixel ray and layer clip (double-float) ---------------------
        // p(lambda) = o + lambda v with v unnormalised; t = lambda |v|.
        df r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            df a = {v.v00h[k], v.v00l[k] + fmaf(xf, v.vxl[k], yf * v.vyl[k])};
            a = df_addf(a, xf * v.vxh[k]);  // exact products
            r[k] = df_addf(a, yf * v.vyh[k]);
        }
        // |v| in FP32 for the step length and the phase angle; the far clip
        // lambda_max = t_max / |v| in double-float only where it can decide the
        // layer exit (an FP32 test with a 1e-5 margin, far above its error)
        const float n2f = fmaf(r[0].hi, r[0].hi, fmaf(r[1].hi, r[1].hi, r[2].hi * r[2].hi));
        const float rnf = rsqrtf(n2f);  // 1 / |v|
        const auto lam_max = [&]() {
            const df n2 = df_add(df_add(df_mul(r[0], r[0]), df_mul(r[1], r[1])), df_mul(r[2], r[2]));
            return df_mul({v.tmax_h, v.tmax_l}, df_rsqrt(n2));
        };
        df lam0 = {0.0f, 0.0f}, lam1;
        if (fabsf(r[2].hi) * rnf < 1e-8f) {
            alive = v.cam_in_layer != 0;
            lam1 = lam_max();
        } else {
            const df inv = df_recip(r[2]);
            const df ll = df_mul({v.zlo_h, v.zlo_l}, inv), lh = df_mul({v.zhi_h, v.zhi_l}, inv);
            lam0 = df_max(df_min(ll, lh), lam0);
            lam1 = df_max(ll, lh);
            if (!(lam1.hi < v.tmax_h * rnf * (1.0f - 1e-5f))) lam1 = df_min(lam1, lam_max());
            alive = df_gt(lam1, lam0);
        }
        if (alive) {
            // --- a2: jittered start offset (Sec. 3.2) ---------------------------
            const df D = df_mul(df_add(lam1, df_neg(lam0)), {v.invn_h, v.invn_l});
            float u = 0.5f;
            if (v.u_frame >= 0.0f)
                u = v.u_frame;
            else if (v.jitter_frame >= 0)
                u = (float)(pcg_hash4((uint32_t)x, (uint32_t)y, (uint32_t)v.jitter_frame,
                                      p.jitter_key) >> 8) * (1.0f / 16777216.0f);
            const df lam_s = df_add(lam0, df_mulf(D, u));
            df pos[3], dpos[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                pos[k] = df_add({v.oh[k], v.ol[k]}, df_mul(lam_s, r[k]));
                dpos[k] = df_mul(D, r[k]);
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
            const df hrel = df_add(df_mul(lam_s, r[2]), df_neg({v.zlo_h, v.zlo_l}));
            hq = (int32_t)df_to_u32({hrel.hi * 65536.0f, hrel.lo * 65536.0f});
            eh = (int32_t)df_to_u32({dpos[2].hi * 65536.0f, dpos[2].lo * 65536.0f});
            const float vlen = n2f * rnf;
            Df = D.hi * vlen;
            // --- a5: phase function, hoisted per ray ----------------------------
            // p_HG(mu) = (1 - g^2) / (4 pi) * (1 + g^2 - 2 g mu)^(-3/2)
            const float mu = (r[0].hi * p.sun[0] + r[1].hi * p.sun[1] + r[2].hi * p.sun[2]) * rnf;
            const float q = rsqrtf(fmaf(-2.0f * p.hg_g, mu, fmaf(p.hg_g, p.hg_g, 1.0f)));
            phase = p.hg_norm * q * q * q;
        }
    }
    stage_coords(ws, lane, c, e, hq, eh);
    const unsigned lt_mask = (1u << lane) - 1u;
    float tau = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
    for (int i0 = 0; i0 < v.steps && __any_sync(kFull, alive); i0 += CH) {
        // --- A1: which of this lane's CH steps need a density lookup: inside the
        //     layer and in an occupied macro-cell of the occupancy grid (the grid
        //     words of all CH steps are loaded together) -------------------------
        uint32_t need = 0;
        if (alive) {
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                if (i0 + k >= v.steps) break;
                bool nd = true;
                if (FX || !p.constant_mode) {
                    // g(h) > 0 exactly when 0 < h < layer thickness: both clamp
                    // factors are then at least ~1e-8, their product far above
                    // the FP32 underflow, and otherwise one of them is 0
                    const int32_t hk = hq + k * eh;
                    nd = hk > 0 && hk < p.h_top;
                    if (nd && p.occ)
                        nd = occupied<FX>(p, c[kBX] + k * e[kBX], c[kBY] + k * e[kBY],
                                          c[kBZ] + k * e[kBZ]);
                }
                if (nd) need |= 1u << k;
            }
        }
        // --- A2: those (step, lane) lookups shared out over the warp, one or two
        //     per lane at a time (ViewBatch) so that their loads overlap (a3) ---
        unsigned nq = 0;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const unsigned m = __ballot_sync(kFull, (need >> k) & 1u);
            const unsigned slot = nq + __popc(m & lt_mask);
            if (((need >> k) & 1u) && in_range(p.check, slot < CH * 32u, kChkWork))
                ws.pairs[slot] = (uint16_t)((k << 5) | lane);
            nq += __popc(m);
        }
        __syncwarp();
        constexpr int kViewBatch = ViewBatch<T, CH>::value;
        for (unsigned q = lane; q < nq; q += 32 * kViewBatch) {
            // a lane without a further lookup repeats its first (same value, same entry)
            unsigned pr[kViewBatch];
            float rho[kViewBatch];
#pragma unroll
            for (int b = 0; b < kViewBatch; ++b) pr[b] = ws.pairs[q + 32 * b < nq ? q + 32 * b : q];
            bool ok = in_range(p.check, q < CH * 32u, kChkWork);
#pragma unroll
            for (int b = 0; b < kViewBatch; ++b) ok = ok && in_range(p.check, (pr[b] >> 5) < (unsigned)CH, kChkWork);
            if (!ok) continue;
#pragma unroll
            for (int b = 0; b < kViewBatch; ++b) {
                uint32_t cs[kLatticeAxes];
                const int32_t hs = step_coords(p, ws, pr[b] & 31u, (uint32_t)i0 + (pr[b] >> 5), cs);
                rho[b] = density<FX>(p, base, detail, weather, cs, hs);
            }
#pragma unroll
            for (int b = 0; b < kViewBatch; ++b) ws.rho[pr[b] >> 5][pr[b] & 31u] = rho[b];
        }
        __syncwarp();
        // --- A3: each lane walks its steps in order: optical depth and the early
        //     out (a7, Sec. 1: stop once alpha is ~1) ---------------------------
        uint32_t act = 0;
        int nA = 0;
        if (alive) {
            float tau_a = tau;
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                if (i0 + k >= v.steps) break;
                const float rho = ((need >> k) & 1u) ? ws.rho[k][lane] : 0.0f;
                nA = k + 1;
                if (rho > 0.0f) {
                    act |= 1u << k;
                    tau_a = __fadd_rn(tau_a, step_depth(p.absorption, rho, Df));
                }
                if (tau_a >= p.tau_max) {
                    alive = false;
                    break;
                }
            }
            n_look += nA + nlight * __popc(act);
        }
#pragma unroll
        for (int a = kBX; a <= kBZ; ++a) c[a] += CH * e[a];
        hq += CH * eh;
        if (!__any_sync(kFull, act != 0u)) continue;  // no density in this chunk, warp-wide
        // --- B: light marches shared out over the warp (a4, Sec. 1) ----------
        unsigned offs[CH + 1];
        offs[0] = 0;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            const unsigned m = __ballot_sync(kFull, (act >> k) & 1u);
            const unsigned slot = offs[k] + __popc(m & lt_mask);
            if (((act >> k) & 1u) && in_range(p.check, slot < CH * 32u, kChkWork))
                ws.pairs[slot] = (uint16_t)((k << 5) | lane);
            offs[k + 1] = offs[k] + __popc(m);
        }
        __syncwarp();
        const unsigned npairs = offs[CH];
        for (unsigned q = lane; q < npairs; q += 32) {
            const unsigned pr = ws.pairs[q], k = pr >> 5, ow = pr & 31u;
            if (!in_range(p.check, q < CH * 32u && k < (unsigned)CH, kChkWork)) continue;
            uint32_t cs[kLatticeAxes];
            const int32_t hs = step_coords(p, ws, ow, (uint32_t)(i0 + (int)k), cs);
            float rho_sum = 0.0f;
            if (LS >= 0) {
                constexpr int kU = LightUnroll<T>::value;
#pragma unroll kU
                for (int j = 0; j < (LS >= 0 ? LS : 0); ++j) {
                    uint32_t cj[kLatticeAxes];
#pragma unroll
                    for (int a = 0; a < kLatticeAxes; ++a) cj[a] = cs[a] + p.loff[j][a];
                    rho_sum += density<FX>(p, base, detail, weather, cj, hs + p.lh[j]);
                }
            } else {
#pragma unroll 2
                for (int j = 0; j < nlight; ++j) {
                    uint32_t cj[kLatticeAxes];
#pragma unroll
                    for (int a = 0; a < kLatticeAxes; ++a) cj[a] = cs[a] + p.loff[j][a];
                    rho_sum += density<FX>(p, base, detail, weather, cj, hs + p.lh[j]);
                }
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
    if (in_image && in_range(p.check, x >= 0 && y >= 0, kChkPixel))
        v.out[(size_t)y * v.width + x] = make_float4(cr, cg, cb, -expm1f(-tau));
    return n_look;
}

// Warp-aggregated add of the lookup count (counting launches only).
__device__ __forceinline__ void count_lookups(unsigned long long *counter, unsigned long long n) {
    if (!counter) return;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) n += __shfl_down_sync(kFull, n, s);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(counter, n);
}

// Host side (render.cu).
int build_scene(const cloud_volume *vol, const cloud_params *prm, int light_steps, int integration,
                SceneParams *p);
int build_view(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *cam, int width,
               int height, int steps, int jitter_frame, float *out, int shape, ViewParams *v);
// The autotuned launch configuration for (storage precision, light steps).
int tuned_config(int precision, int light_steps);
// Raymarch of one view with the given configuration (render.cu); the
// per-chunk-size kernels and their dispatch are instantiated in
// march{8,16}_{view,batch}.cu.
int launch_march(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                 unsigned long long *counter, int config, cudaStream_t s);
template <int CH>
void launch_march_ch(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                     unsigned long long *counter, int shape, cudaStream_t s);
template <int CH>
const void *batch_kernel_ch(int precision, int light_steps, bool fx, int shape);
// True when a launch can use the FX march: the standard tile sizes, all three
// tiles present, noise density, six light steps and a base tile period of 2^k
// detail periods (the detail coordinates then follow from the base ones).
bool fixed_sizes(const SceneParams &p, const cloud_volume *vol);

}  // namespace cloudvol
