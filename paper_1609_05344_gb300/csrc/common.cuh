// common.cuh -- internal definitions shared by the CUDA translation units of
// libcloudvol.so (not part of the public ABI; see include/cloudvol.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>

#include "../../include/cloudvol.h"

namespace cloudvol {

// ---------------------------------------------------------------------------
// Error reporting: every entry point returns a status and records a one-line
// message for cloud_last_error_message() on the calling thread.
int set_error(int status, const std::string &msg);
int check_cuda(cudaError_t e, const char *what);
int check_launch(const char *what);
void clear_error();

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---------------------------------------------------------------------------
// Checked build (CLOUDVOL_CHECKED=1, a separate library used by tests in place
// of a memory checker): kernels verify the ranges their index arithmetic is
// meant to stay in (tile records, occupancy words, work lists, pixels, history
// texels, shared tiles, views), skip an access that fails and record the site
// in a device status word read by cloud_debug_check_status.  In normal builds
// the checks compile away.
#ifndef CLOUDVOL_CHECKED
#define CLOUDVOL_CHECKED 0
#endif
enum CheckSite : unsigned {
    kChkRecord = 1u,      // a tile record index
    kChkOccupancy = 2u,   // an occupancy-grid word
    kChkWork = 4u,        // a (step, lane) work-list entry
    kChkPixel = 8u,       // an output pixel
    kChkHistory = 16u,    // a history or source texel
    kChkTile = 32u,       // a shared-memory tile texel
    kChkView = 64u,       // a view or tile of a multi-view launch
};
__device__ __forceinline__ bool in_range(unsigned *word, bool ok, unsigned site) {
#if CLOUDVOL_CHECKED
    if (!ok && word) atomicOr(word, site);
    return ok;
#else
    (void)word;
    (void)ok;
    (void)site;
    return true;
#endif
}
// Host: the current device's status word in checked builds, else nullptr.
unsigned *check_word();

// ---------------------------------------------------------------------------
// Counter-based hash: single-state PCG hash (Jarzynski & Olano, JCGT 2020):
// one 32-bit PCG LCG step (multiplier 747796405, increment 2891336453) and
// the RXS-M-XS output permutation (multiplier 277803737).  Four-word keys
// nest: h(a,b,c,d) = pcg(a ^ pcg(b ^ pcg(c ^ pcg(d)))).
__host__ __device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    uint32_t s = v * 747796405u + 2891336453u;
    uint32_t w = ((s >> ((s >> 28u) + 4u)) ^ s) * 277803737u;
    return (w >> 22u) ^ w;
}

__host__ __device__ __forceinline__ uint32_t pcg_hash4(uint32_t a, uint32_t b, uint32_t c,
                                                       uint32_t d) {
    return pcg_hash(a ^ pcg_hash(b ^ pcg_hash(c ^ pcg_hash(d))));
}

// Key words mixed into the hash for each use.
constexpr uint32_t kJitterKey = 0x4A17u;
constexpr uint32_t kOctaveKey = 0x9E37u;
constexpr uint32_t kSaltBase = 0xB45Eu;
constexpr uint32_t kSaltDetail = 0xDE7Au;
constexpr uint32_t kSaltWeather = 0x3EA7u;
constexpr int kOctaves = 4;

// Noise tiles are stored centred: texel = fBm - 1/2, which halves the
// magnitude (and so the rounding error) of reduced-precision storage.
constexpr float kCentre = 0.5f;

// ---------------------------------------------------------------------------
// Volume handle (cloud_volume in the ABI).
}  // namespace cloudvol

struct cloud_volume {
    cloud_volume_desc desc;
    int log2_base, log2_detail, log2_weather;  // 0 when the tile is absent
    void *base;      // device, base_n^3 corner-packed records of the storage precision
    void *detail;    // device or nullptr (detail_n^3 records)
    void *weather;   // device or nullptr (weather_n^2 records)
    // occupancy grid: one bit per cell of 2^kOccShift base records per axis (x fastest),
    // clear where the density is provably 0 throughout (see build_occupancy)
    uint32_t *occ;   // device or nullptr (constant density)
    int log2_occ;    // macro-cells per axis = 2^log2_occ = base_n / 2^kOccShift
    int device;
};

namespace cloudvol {

inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

inline size_t precision_bytes(int p) { return p == CLOUD_PRECISION_FP32 ? 4 : 2; }

// Occupancy grid cell: 2^kOccShift base records per axis.
#ifndef CLOUDVOL_OCC_SHIFT
#define CLOUDVOL_OCC_SHIFT -1
#endif
constexpr int kOccShift = CLOUDVOL_OCC_SHIFT;

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2, about
// 48 significant bits from FP32 operations only (error-free transformations
// of Knuth/Dekker: two-sum, fast-two-sum, FMA-based two-product).  Used where
// a per-ray quantity needs more than FP32 precision; GB300's FP64 rate is far
// below its FP32 rate.
struct df {
    float hi, lo;
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df df_addf(df a, float b) {
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return fast_two_sum(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = a.hi * b;
    const float e = fmaf(a.hi, b, -p);
    return fast_two_sum(p, fmaf(a.lo, b, e));
}
// 1/b: one Newton step on the hardware reciprocal estimate (PTX rcp.approx,
// relative error about 2^-23; the step squares it, like df_rsqrt's).
__device__ __forceinline__ df df_recip(df b) {
    float q;
    asm("rcp.approx.f32 %0, %1;" : "=f"(q) : "f"(b.hi));
    const df p = df_mulf(b, q);                 // b q = 1 - r
    const float r = (1.0f - p.hi) - p.lo;
    return fast_two_sum(q, q * r);
}
// 1/sqrt(a): one Newton step on the FP32 estimate.
__device__ __forceinline__ df df_rsqrt(df a) {
    const float r = rsqrtf(a.hi);
    const df t = df_mulf(df_mulf(a, r), r);     // a r^2 = 1 - e
    const float e = (1.0f - t.hi) - t.lo;
    return fast_two_sum(r, 0.5f * r * e);
}
__device__ __forceinline__ bool df_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ df df_max(df a, df b) { return df_gt(a, b) ? a : b; }
__device__ __forceinline__ df df_min(df a, df b) { return df_gt(a, b) ? b : a; }
// round(a) modulo 2^32 (fixed-point wrap) of a double-float with |a| < 2^55:
// k = round(a.hi / 2^32) and r = a.hi - k 2^32 are exact (|r| <= 2^31, a
// multiple of ulp(a.hi)); the integer part of r and the rounded remainder
// (r - round(r)) + a.lo are converted with 32-bit conversions only.
__device__ __forceinline__ uint32_t df_to_u32(df a) {
    const float k = rintf(a.hi * 2.3283064365386963e-10f);
    const float r = fmaf(-k, 4294967296.0f, a.hi);
    const float rr = rintf(r);
    return (uint32_t)__float2int_rn(rr) + (uint32_t)__float2int_rn((r - rr) + a.lo);
}

// Host: split an FP64 value into a double-float pair.
inline void split_df(double v, float *hi, float *lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
}
// Host: split so that x * hi is exact in FP32 for integer |x| < 2^14 (hi keeps
// 10 significant bits) and lo carries the rest.
inline void split_df10(double v, float *hi, float *lo) {
    if (v == 0.0) {
        *hi = *lo = 0.0f;
        return;
    }
    int e;
    std::frexp(v, &e);
    const double q = std::ldexp(1.0, e - 10);
    *hi = (float)(std::nearbyint(v / q) * q);
    *lo = (float)(v - (double)*hi);
}

// ---------------------------------------------------------------------------
// Corner-packed tiles.  Record k of an N^3 tile holds the 8 texels of the
// trilinear footprint whose lowest corner is texel k, with the periodic wrap
// already applied, in the order r = 4 dx + 2 dy + dz (dz fastest), so that
// (r, r+1) are the two z-neighbours a packed FP32x2 lerp works on; record k
// of an N^2 tile holds the 4 texels of the bilinear footprint, r = 2 dx + dy.
// One lookup is one contiguous record load (16 B for 16-bit texels, 32 B for
// FP32) instead of 8 (or 4) scattered texel loads.  Texels are stored centred
// (fBm - 1/2).
//
// Record formats, by storage precision:
//   FP32     the texels, except that the dx = 1 half holds its differences
//            from the dx = 0 half (rounded at packing exactly as the x lerp
//            would round them);
//   UNORM16  each texel as 16-bit fixed point q = round((t + 1/2) 2^16);
//   FP16 / BF16  corner 0 as 16-bit fixed point (as UNORM16), the other dx = 0
//            corners as IEEE half (bfloat16) differences from that decoded
//            corner 0, and the dx = 1 corners as differences from the decoded
//            dx = 0 corner next to them.  Neighbouring texels differ little, so
//            the 11-bit (8-bit) significand rounds a small difference instead
//            of the texel itself.
// A loader returns the corners with the dx = 1 half as differences from the
// dx = 0 half (the operand the x lerp needs) and returns an offset: the lerp
// of the returned corners plus the offset, minus texel_bias<T>(), is the
// centred texel value at a point.  FP32 records: offset 0, bias 0.  UNORM16:
// corners decoded to 1 + q 2^-16 by bit operations, offset 0, bias 3/2.
// FP16 / BF16: corners relative to corner 0 (so corner 0 is 0), offset the
// decoded corner 0 as 1 + q 2^-16, bias 3/2.  The bias is folded into the
// density's constants (SceneParams::k0, w_off).
template <typename T>
__host__ __device__ constexpr float texel_bias() { return 1.5f; }
template <>
__host__ __device__ constexpr float texel_bias<float>() { return 0.0f; }
inline float texel_bias_of(int precision) { return precision == CLOUD_PRECISION_FP32 ? 0.0f : 1.5f; }

// An FP32 record is one 32-byte sector, fetched by a single 256-bit load
// (sm_100+ ld.global .v8): one L1 wavefront instead of two.
__device__ __forceinline__ float load_rec8(const float *tile, uint32_t rec, float c[8]) {
    const float *p = tile + 8 * (size_t)rec;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]), "=f"(c[4]), "=f"(c[5]), "=f"(c[6]),
          "=f"(c[7])
        : "l"(p));
    return 0.0f;
}
__device__ __forceinline__ float load_rec4(const float *tile, uint32_t rec, float c[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(tile) + rec);
    c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
    return 0.0f;
}

// 16-bit fields of a 32-bit word: 1 + q 2^-16 for fixed point (exact, bit
// operations only); half and bfloat16 converted exactly.
__device__ __forceinline__ float unorm_lo(uint32_t w) {
    return __uint_as_float(0x3F800000u | ((w << 7) & 0x007FFF80u));
}
__device__ __forceinline__ float unorm_hi(uint32_t w) {
    return __uint_as_float(0x3F800000u | ((w >> 9) & 0x007FFF80u));
}
__device__ __forceinline__ float f16_hi(uint32_t w, const __half *) {
    return __half2float(__ushort_as_half((unsigned short)(w >> 16)));
}
__device__ __forceinline__ float f16_hi(uint32_t w, const __nv_bfloat16 *) {
    return __uint_as_float(w & 0xFFFF0000u);
}
__device__ __forceinline__ void unpack16(uint32_t w, const __half *, float &lo, float &hi) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
    lo = f.x;
    hi = f.y;
}
__device__ __forceinline__ void unpack16(uint32_t w, const __nv_bfloat16 *, float &lo, float &hi) {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xFFFF0000u);
}

__device__ __forceinline__ float load_rec8(const uint16_t *tile, uint32_t rec, float c[8]) {
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(tile) + rec);
    c[0] = unorm_lo(r.x); c[1] = unorm_hi(r.x);
    c[2] = unorm_lo(r.y); c[3] = unorm_hi(r.y);
    const float2 d0 = __fadd2_rn(make_float2(unorm_lo(r.z), unorm_hi(r.z)), make_float2(-c[0], -c[1]));
    const float2 d1 = __fadd2_rn(make_float2(unorm_lo(r.w), unorm_hi(r.w)), make_float2(-c[2], -c[3]));
    c[4] = d0.x; c[5] = d0.y; c[6] = d1.x; c[7] = d1.y;
    return 0.0f;
}
__device__ __forceinline__ float load_rec4(const uint16_t *tile, uint32_t rec, float c[4]) {
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(tile) + rec);
    c[0] = unorm_lo(r.x); c[1] = unorm_hi(r.x);
    const float2 d = __fadd2_rn(make_float2(unorm_lo(r.y), unorm_hi(r.y)), make_float2(-c[0], -c[1]));
    c[2] = d.x; c[3] = d.y;
    return 0.0f;
}

// Difference records (FP16 / BF16 volumes): relative corners (0, d1, d2, d3)
// of the dx = 0 face and the x differences of the dx = 1 face, as stored.
template <typename T>
__device__ __forceinline__ float load_rec8(const T *tile, uint32_t rec, float c[8]) {
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(tile) + rec);
    c[0] = 0.0f;
    c[1] = f16_hi(r.x, tile);
    unpack16(r.y, tile, c[2], c[3]);
    unpack16(r.z, tile, c[4], c[5]);
    unpack16(r.w, tile, c[6], c[7]);
    return unorm_lo(r.x);
}
template <typename T>
__device__ __forceinline__ float load_rec4(const T *tile, uint32_t rec, float c[4]) {
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(tile) + rec);
    c[0] = 0.0f;
    c[1] = f16_hi(r.x, tile);
    unpack16(r.y, tile, c[2], c[3]);
    return unorm_lo(r.x);
}

// Host side of the multi-view resolve (taa.cu), used by the render server:
// one request per view (prev == NULL and history == NULL for a first frame).
struct ResolveRequest {
    const cloud_camera *prev, *cur;
    const void *history;
    const float *current;
    void *out;
    int width, height;
};
// Builds the per-view table in h_table (pinned host, resolve_view_bytes() per
// view), uploads it to d_table on s and launches one kernel over all views.
// status (device or mapped host memory, may be NULL) counts the launch's
// bounded waits that gave up.
int launch_taa_reproject_batch(const cloud_volume *vol, const cloud_params *prm,
                               const ResolveRequest *reqs, int n, int fmt, float blend,
                               void *h_table, void *d_table, unsigned int *status, cudaStream_t s);
size_t resolve_view_bytes();

// Texel k of a packed tile (corner 0 of record k, `stride` values per
// record), decoded to the centred value.
__device__ __forceinline__ float load_corner0(const float *p, uint32_t rec, int stride) {
    return __ldg(p + (size_t)stride * rec);
}
template <typename T>
__device__ __forceinline__ float load_corner0(const T *p, uint32_t rec, int stride) {
    const uint16_t q = __ldg(reinterpret_cast<const uint16_t *>(p) + (size_t)stride * rec);
    return __uint_as_float(0x3F800000u | ((uint32_t)q << 7)) - 1.5f;
}

}  // namespace cloudvol
