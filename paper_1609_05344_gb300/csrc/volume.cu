// volume.cu -- cloud density volumes: creation, fBm generation, export, and
// the device hash test hook.
//
// Sec. 1 samples a cloud density at every step and does not define the
// field.  The field here is value-noise fBm: 4 octaves,
// octave o with (N/16) 2^o lattice cells per tile and amplitude 2^-o, summed
// and divided by the total amplitude; lattice values are hash(ix, iy, iz,
// seed ^ o*0x9E37 ^ salt) >> 8 scaled to [0,1); plain trilinear
// interpolation; voxel k holds the noise at lattice coordinate k M_o / N.
// The generation arithmetic runs in FP64 on the device so every stored texel
// is the correctly rounded fBm value (minus the 1/2 centring offset).
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"

namespace cloudvol {

namespace {
thread_local std::string g_last_error;
}

int set_error(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}
void clear_error() { g_last_error.clear(); }

int check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CLOUD_OK;
    if (e == cudaErrorMemoryAllocation)
        return set_error(CLOUD_ERR_OUT_OF_MEMORY, std::string(what) + ": " + cudaGetErrorString(e));
    return set_error(CLOUD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int check_launch(const char *what) { return check_cuda(cudaGetLastError(), what); }

unsigned *check_word() {
#if CLOUDVOL_CHECKED
    static std::mutex mu;
    static unsigned *words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!words[dev] && cudaMalloc(&words[dev], sizeof(unsigned)) == cudaSuccess)
        cudaMemset(words[dev], 0, sizeof(unsigned));
    return words[dev];
#else
    return nullptr;
#endif
}

__device__ __forceinline__ double unit_value(uint32_t h) {
    return (double)(h >> 8) * (1.0 / 16777216.0);
}

// 16-bit fixed point of a centred texel t: q = round((t + 1/2) 2^16), clamped.
__device__ __forceinline__ uint16_t encode_unorm16(double t) {
    const double q = rint((t + (double)kCentre) * 65536.0);
    return (uint16_t)(q < 0.0 ? 0.0 : (q > 65535.0 ? 65535.0 : q));
}
__device__ __forceinline__ double decode_unorm16(uint16_t q) { return q * (1.0 / 65536.0) - (double)kCentre; }
__device__ __forceinline__ uint16_t encode16(double v, const __half *) {
    return __half_as_ushort(__double2half(v));
}
__device__ __forceinline__ uint16_t encode16(double v, const __nv_bfloat16 *) {
    return __bfloat16_as_ushort(__double2bfloat16(v));
}

__global__ void fbm3_kernel(double *__restrict__ out, int log2n, uint32_t seed, uint32_t salt) {
    const uint32_t n = 1u << log2n;
    const uint64_t total = (uint64_t)n * n * n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k[3] = {(uint32_t)(i & (n - 1)), (uint32_t)((i >> log2n) & (n - 1)),
                               (uint32_t)(i >> (2 * log2n))};
        double sum = 0.0, amp_sum = 0.0, amp = 1.0;
        for (int o = 0; o < kOctaves; ++o) {
            const uint32_t m = (n >> 4) << o;  // cells per tile
            const uint32_t key = seed ^ ((uint32_t)o * kOctaveKey) ^ salt;
            uint32_t c0[3], c1[3];
            double f[3];
            for (int a = 0; a < 3; ++a) {
                const uint32_t km = k[a] * m;  // lattice coordinate k m / n, exactly
                c0[a] = km >> log2n;
                c1[a] = (c0[a] + 1u) % m;
                f[a] = (double)(km & (n - 1)) / (double)n;
            }
            double v = 0.0;
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                                         (dz ? f[2] : 1.0 - f[2]);
                        v += w * unit_value(pcg_hash4(dx ? c1[0] : c0[0], dy ? c1[1] : c0[1],
                                                      dz ? c1[2] : c0[2], key));
                    }
            sum += amp * v;
            amp_sum += amp;
            amp *= 0.5;
        }
        out[i] = sum / amp_sum - (double)kCentre;
    }
}

__global__ void fbm2_kernel(double *__restrict__ out, int log2n, uint32_t seed, uint32_t salt) {
    const uint32_t n = 1u << log2n;
    const uint64_t total = (uint64_t)n * n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k[2] = {(uint32_t)(i & (n - 1)), (uint32_t)(i >> log2n)};
        double sum = 0.0, amp_sum = 0.0, amp = 1.0;
        for (int o = 0; o < kOctaves; ++o) {
            const uint32_t m = (n >> 4) << o;
            const uint32_t key = seed ^ ((uint32_t)o * kOctaveKey) ^ salt;
            uint32_t c0[2], c1[2];
            double f[2];
            for (int a = 0; a < 2; ++a) {
                const uint32_t km = k[a] * m;
                c0[a] = km >> log2n;
                c1[a] = (c0[a] + 1u) % m;
                f[a] = (double)(km & (n - 1)) / (double)n;
            }
            double v = 0.0;
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]);
                    v += w * unit_value(pcg_hash4(dx ? c1[0] : c0[0], dy ? c1[1] : c0[1], 0u, key));
                }
            sum += amp * v;
            amp_sum += amp;
            amp *= 0.5;
        }
        out[i] = sum / amp_sum - (double)kCentre;
    }
}

// Corner-packing of a generated tile (centred FP64 texels) into the records
// of the storage precision (formats in common.cuh).
template <int R>
__device__ __forceinline__ void store_record(float *dst, const double (&t)[R]) {
    float f[R];
#pragma unroll
    for (int r = 0; r < R; ++r) f[r] = (float)t[r];
#pragma unroll
    for (int r = 0; r < R / 2; ++r) dst[r] = f[r];
#pragma unroll
    for (int r = R / 2; r < R; ++r) dst[r] = __fsub_rn(f[r], f[r - R / 2]);  // as the x lerp rounds it
}
template <int R>
__device__ __forceinline__ void store_record(uint16_t *dst, const double (&t)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r] = encode_unorm16(t[r]);
}
__device__ __forceinline__ double decode16(uint16_t u, const __half *) {
    return (double)__half2float(__ushort_as_half(u));
}
__device__ __forceinline__ double decode16(uint16_t u, const __nv_bfloat16 *) {
    return (double)__bfloat162float(__ushort_as_bfloat16(u));
}
// FP16 / BF16: corner 0 as 16-bit fixed point, the other dx = 0 corners as
// differences from its decoded value, the dx = 1 corners as differences from
// the decoded dx = 0 corner beside them; each rounded once from FP64, against
// the values the loader will reconstruct
template <typename T, int R>
__device__ __forceinline__ void store_record(T *dst, const double (&t)[R]) {
    uint16_t *u = reinterpret_cast<uint16_t *>(dst);
    const uint16_t q0 = encode_unorm16(t[0]);
    const double c0 = decode_unorm16(q0);
    double dec[R / 2];
    u[0] = q0;
    dec[0] = c0;
#pragma unroll
    for (int r = 1; r < R / 2; ++r) {
        u[r] = encode16(t[r] - c0, dst);
        dec[r] = c0 + decode16(u[r], dst);
    }
#pragma unroll
    for (int r = R / 2; r < R; ++r) u[r] = encode16(t[r] - dec[r - R / 2], dst);
}

template <typename T>
__global__ void pack3_kernel(const double *__restrict__ plain, T *__restrict__ packed, int log2n) {
    const uint32_t mask = (1u << log2n) - 1u;
    const uint64_t total = 1ull << (3 * log2n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)i & mask, y = (uint32_t)(i >> log2n) & mask,
                       z = (uint32_t)(i >> (2 * log2n));
        double t[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {  // r = 4 dx + 2 dy + dz
            const uint32_t xx = (x + (r >> 2)) & mask, yy = (y + ((r >> 1) & 1)) & mask,
                           zz = (z + (r & 1)) & mask;
            t[r] = plain[((uint64_t)zz << (2 * log2n)) | (yy << log2n) | xx];
        }
        store_record(packed + 8 * i, t);
    }
}

template <typename T>
__global__ void pack2_kernel(const double *__restrict__ plain, T *__restrict__ packed, int log2n) {
    const uint32_t mask = (1u << log2n) - 1u;
    const uint64_t total = 1ull << (2 * log2n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)i & mask, y = (uint32_t)(i >> log2n);
        double t[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {  // r = 2 dx + dy
            const uint32_t xx = (x + (r >> 1)) & mask, yy = (y + (r & 1)) & mask;
            t[r] = plain[(yy << log2n) | xx];
        }
        store_record(packed + 4 * i, t);
    }
}

// Texel k of a packed tile is corner 0 of record k.
template <typename T>
__global__ void decode_kernel(const T *__restrict__ packed, int stride, float *__restrict__ out,
                              uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = load_corner0(packed, (uint32_t)i, stride) + kCentre;
}

// Smallest and largest centred value any trilinear lookup of record `rec` can
// interpolate: the extremes of its corners as the march decodes them (for
// FP32 records the dx = 1 corners are the dx = 0 corners plus the stored
// differences).  Rounding of the lerps is covered by the caller's margin.
template <typename T>
__device__ __forceinline__ void record_corners(const T *tile, uint32_t rec, float v[8]) {
    float c[8];
    const float off = load_rec8(tile, rec, c) - texel_bias<T>();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[r] = c[r] + off;
        v[r + 4] = (c[r] + c[r + 4]) + off;
    }
}
template <typename T>
__device__ __forceinline__ void record_range(const T *tile, uint32_t rec, float &lo, float &hi) {
    float v[8];
    record_corners(tile, rec, v);
    lo = hi = v[0];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
        lo = fminf(lo, v[r]);
        hi = fmaxf(hi, v[r]);
    }
}
// Trilinear value of a record's corners (r = 4 dx + 2 dy + dz) at fractions f.
__device__ __forceinline__ float trilinear_at(const float v[8], float fx, float fy, float fz) {
    float yz[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) yz[r] = fmaf(fx, v[r + 4] - v[r], v[r]);  // (dy, dz) pairs
    const float z0 = fmaf(fy, yz[2] - yz[0], yz[0]), z1 = fmaf(fy, yz[3] - yz[1], yz[1]);
    return fmaf(fz, z1 - z0, z0);
}

// Occupancy grid.  Macro-cell (X, Y, Z) covers the base records mX..mX+m-1 on
// each axis (m = 2^kOccShift), i.e. every sample whose base record lies there.  Its bit is
// clear when, for every such sample,
//   B - w_d Dt - c <= max B - w_d min Dt - c < 0      (w_d >= 0; max Dt if < 0)
// with max B over the corners of those base records and the Dt extreme over
// the corners of every detail record such a sample can use: the density
// max(0, .) is then exactly 0 there.  The detail records of a macro-cell are
// found from the periods when the base period is 2^k detail periods (the
// detail coordinate is then a fixed function of the base coordinate);
// otherwise the extreme over the whole detail tile is used.  The margin
// 1e-5 covers FP32 rounding of the lerps and of the remap.
template <typename T>
__global__ void occupancy_kernel(const T *__restrict__ base, int log2b, const T *__restrict__ detail,
                                 int log2d, float ratio, float dt_all_lo, float dt_all_hi,
                                 float k0, float wd, uint32_t *__restrict__ occ) {
    const int lo2 = log2b - kOccShift;
    const uint32_t M = 1u << lo2, nd = 1u << log2d;
    const uint32_t total = M * M * M;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < (total + 31) / 32;
         w += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t b = 0; b < 32 && 32 * w + b < total; ++b) {
            const uint32_t cell = 32 * w + b;
            const uint32_t X = cell & (M - 1), Y = (cell >> lo2) & (M - 1), Z = cell >> (2 * lo2);
            constexpr uint32_t m = 1u << (kOccShift > 0 ? kOccShift : 0);  // base records per cell and axis
            float bmax = -INFINITY;
            for (uint32_t dz = 0; dz < m; ++dz)
                for (uint32_t dy = 0; dy < m; ++dy)
                    for (uint32_t dx = 0; dx < m; ++dx) {
                        float l, h;
                        record_range(base, (((m * Z + dz) << (2 * log2b)) | ((m * Y + dy) << log2b) |
                                            (m * X + dx)), l, h);
                        bmax = fmaxf(bmax, h);
                    }
            float dlo = dt_all_lo, dhi = dt_all_hi;
            if (detail && ratio > 0.0f) {
                // detail record range along each axis: samples with base texel-centre
                // coordinate s in [m K, m K + m) have detail coordinate (s + 1/2) ratio - 1/2
                const uint32_t K[3] = {X, Y, Z};
                int r0[3], r1[3];
                for (int a = 0; a < 3; ++a) {
                    r0[a] = (int)floorf(((float)(m * K[a]) + 0.5f) * ratio - 0.5f);
                    r1[a] = (int)floorf(((float)(m * K[a] + m) + 0.5f) * ratio - 0.5f);
                }
                dlo = INFINITY;
                dhi = -INFINITY;
                for (int z = r0[2]; z <= r1[2]; ++z)
                    for (int y = r0[1]; y <= r1[1]; ++y)
                        for (int x = r0[0]; x <= r1[0]; ++x) {
                            float l, h;
                            const uint32_t rec = (((uint32_t)z & (nd - 1)) << (2 * log2d)) |
                                                 (((uint32_t)y & (nd - 1)) << log2d) |
                                                 ((uint32_t)x & (nd - 1));
                            record_range(detail, rec, l, h);
                            dlo = fminf(dlo, l);
                            dhi = fmaxf(dhi, h);
                        }
            }
            const float bound = bmax + k0 - wd * (wd >= 0.0f ? dlo : dhi);
            if (bound > -1e-5f) bits |= 1u << b;
        }
        occ[w] = bits;
    }
}

// Occupancy grid of half-texel cells (kOccShift = -1): cell (X, Y, Z) covers
// base texel-centre coordinates [X/2, X/2 + 1/2) (and likewise on y, z), inside
// base record (X/2, Y/2, Z/2).  Trilinear interpolation restricted to a box is
// trilinear in the box's corners, so max B over the cell is the largest of
// B at its 8 corners (evaluated from the record); Dt over the cell's detail
// coordinates (the same box mapped by the fixed base-to-detail shift) is
// extreme at the box corners or at the detail lattice planes inside it, so its
// minimum is taken over those points.  The bit is clear when
// max B - w_d min Dt - c < -1e-5 (room for FP32 rounding).
template <typename T>
__global__ void occupancy_half_kernel(const T *__restrict__ base, int log2b,
                                      const T *__restrict__ detail, int log2d, float ratio,
                                      float dt_all_lo, float dt_all_hi, float k0, float wd,
                                      uint32_t *__restrict__ occ) {
    const int lc = log2b + 1;
    const uint32_t C = 1u << lc, nd = 1u << log2d;
    const uint32_t total = C * C * C;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < (total + 31) / 32;
         w += gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (uint32_t b = 0; b < 32 && 32 * w + b < total; ++b) {
            const uint32_t cell = 32 * w + b;
            const uint32_t K[3] = {cell & (C - 1), (cell >> lc) & (C - 1), cell >> (2 * lc)};
            float v[8];
            record_corners(base, ((K[2] >> 1) << (2 * log2b)) | ((K[1] >> 1) << log2b) | (K[0] >> 1), v);
            float bmax = -INFINITY;
            for (int r = 0; r < 8; ++r)
                bmax = fmaxf(bmax, trilinear_at(v, 0.5f * ((K[0] & 1) + (r >> 2)),
                                                0.5f * ((K[1] & 1) + ((r >> 1) & 1)),
                                                0.5f * ((K[2] & 1) + (r & 1))));
            float dlo = dt_all_lo, dhi = dt_all_hi;
            if (detail && ratio > 0.0f) {
                // per axis: the cell's detail coordinates [lo, hi) and the points
                // where Dt can be extreme (lo, the lattice integers inside, hi);
                // ratio is a power of two and K < 2^16, so these are exact in FP32
                float pts[3][6];
                int np[3];
                bool ok = true;
                for (int a = 0; a < 3; ++a) {
                    const float lo = (0.5f * (float)K[a] + 0.5f) * ratio - 0.5f;
                    const float hi = (0.5f * (float)K[a] + 1.0f) * ratio - 0.5f;
                    int n = 0;
                    pts[a][n++] = lo;
                    for (float q = floorf(lo) + 1.0f; q < hi && n < 5; q += 1.0f) pts[a][n++] = q;
                    if (floorf(lo) + 1.0f + (float)(n - 1) < hi) ok = false;  // more planes than kept
                    pts[a][n++] = hi;
                    np[a] = n;
                }
                if (ok) {
                    dlo = INFINITY;
                    dhi = -INFINITY;
                    for (int iz = 0; iz < np[2]; ++iz)
                        for (int iy = 0; iy < np[1]; ++iy)
                            for (int ix = 0; ix < np[0]; ++ix) {
                                const float sp[3] = {pts[0][ix], pts[1][iy], pts[2][iz]};
                                uint32_t ri[3];
                                float f[3];
                                for (int a = 0; a < 3; ++a) {
                                    const float fl = floorf(sp[a]);
                                    ri[a] = (uint32_t)((int)fl & (int)(nd - 1));
                                    f[a] = sp[a] - fl;
                                }
                                float dv[8];
                                record_corners(detail, (ri[2] << (2 * log2d)) | (ri[1] << log2d) | ri[0], dv);
                                const float val = trilinear_at(dv, f[0], f[1], f[2]);
                                dlo = fminf(dlo, val);
                                dhi = fmaxf(dhi, val);
                            }
                }
            }
            const float bound = bmax + k0 - wd * (wd >= 0.0f ? dlo : dhi);
            if (bound > -1e-5f) bits |= 1u << b;
        }
        occ[w] = bits;
    }
}

// Extremes of the corners of every record of a tile (for occupancy bounds
// that cannot localise the detail tile); one block of 1024 threads.
template <typename T>
__global__ void __launch_bounds__(1024) tile_range_kernel(const T *__restrict__ tile, uint32_t n,
                                                          float *__restrict__ out) {
    __shared__ float slo[32], shi[32];
    float lo = INFINITY, hi = -INFINITY;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        float l, h;
        record_range(tile, i, l, h);
        lo = fminf(lo, l);
        hi = fmaxf(hi, h);
    }
    for (int s = 16; s > 0; s >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, s));
        hi = fmaxf(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, s));
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fminf(lo, slo[w]);
            hi = fmaxf(hi, shi[w]);
        }
        out[0] = lo;
        out[1] = hi;
    }
}

__global__ void hash4_kernel(const uint4 *__restrict__ keys, uint32_t *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 k = keys[i];
        out[i] = pcg_hash4(k.x, k.y, k.z, k.w);
    }
}

unsigned grid_for(uint64_t n, unsigned block) {
    uint64_t g = (n + block - 1) / block;
    const uint64_t cap = 152ull * 16ull;  // grid-stride beyond 16 waves of CTAs per SM
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// Builds the occupancy grid of a volume from its packed records.
template <typename T>
int build_occupancy(cloud_volume *v, cudaStream_t s) {
    const cloud_volume_desc &d = v->desc;
    v->log2_occ = v->log2_base - kOccShift;
    const uint64_t cells = 1ull << (3 * v->log2_occ), words = (cells + 31) / 32;
    if (int rc = check_cuda(cudaMalloc(&v->occ, words * sizeof(uint32_t)), "cudaMalloc occupancy"))
        return rc;
    const double wd = v->detail ? d.detail_weight : 0.0;
    const float k0 = (float)(0.5 - d.coverage - 0.5 * wd);
    // detail texels per base texel when the detail coordinate is a function of
    // the base coordinate (base period an integer number of detail periods)
    double ratio = -1.0;
    float range[2] = {0.0f, 0.0f};
    if (v->detail) {
        const double per = d.base_period_m / d.detail_period_m;
        const bool exact_shift = per >= 1.0 && per <= 65536.0 &&
                                 std::ldexp(1.0, (int)std::lround(std::log2(per))) == per;
        if (exact_shift)
            ratio = per * std::ldexp(1.0, v->log2_detail - v->log2_base);
        float *d_range = nullptr;
        if (int rc = check_cuda(cudaMalloc(&d_range, 2 * sizeof(float)), "cudaMalloc range")) return rc;
        tile_range_kernel<T><<<1, 1024, 0, s>>>((const T *)v->detail, 1u << (3 * v->log2_detail), d_range);
        int rc = check_launch("tile_range_kernel");
        if (!rc) rc = check_cuda(cudaMemcpyAsync(range, d_range, sizeof(range), cudaMemcpyDeviceToHost, s),
                                 "copy detail range");
        if (!rc) rc = check_cuda(cudaStreamSynchronize(s), "detail range");
        cudaFree(d_range);
        if (rc) return rc;
    }
    if (kOccShift < 0)
        occupancy_half_kernel<T><<<grid_for(words, 128), 128, 0, s>>>(
            (const T *)v->base, v->log2_base, (const T *)v->detail, v->log2_detail, (float)ratio, range[0],
            range[1], k0, (float)wd, v->occ);
    else
        occupancy_kernel<T><<<grid_for(words, 128), 128, 0, s>>>(
            (const T *)v->base, v->log2_base, (const T *)v->detail, v->log2_detail, (float)ratio, range[0],
            range[1], k0, (float)wd, v->occ);
    return check_launch("occupancy_kernel");
}

// Generates each tile in FP64 into a plain scratch array, corner-packs it into
// the records of the storage precision, then builds the occupancy grid.
template <typename T>
int generate(cloud_volume *v, cudaStream_t s) {
    const cloud_volume_desc &d = v->desc;
    const uint64_t nb = 1ull << (3 * v->log2_base);
    const uint64_t nd = v->detail ? 1ull << (3 * v->log2_detail) : 0;
    const uint64_t nw = v->weather ? 1ull << (2 * v->log2_weather) : 0;
    const uint64_t most = nb > nd ? (nb > nw ? nb : nw) : (nd > nw ? nd : nw);
    double *tmp = nullptr;
    int rc = check_cuda(cudaMalloc(&tmp, most * sizeof(double)), "cudaMalloc generation scratch");
    if (rc) return rc;
    fbm3_kernel<<<grid_for(nb, 256), 256, 0, s>>>(tmp, v->log2_base, d.seed, kSaltBase);
    pack3_kernel<T><<<grid_for(nb, 256), 256, 0, s>>>(tmp, (T *)v->base, v->log2_base);
    rc = check_launch("generate base");
    if (!rc && v->detail) {
        fbm3_kernel<<<grid_for(nd, 256), 256, 0, s>>>(tmp, v->log2_detail, d.seed, kSaltDetail);
        pack3_kernel<T><<<grid_for(nd, 256), 256, 0, s>>>(tmp, (T *)v->detail, v->log2_detail);
        rc = check_launch("generate detail");
    }
    if (!rc && v->weather) {
        fbm2_kernel<<<grid_for(nw, 256), 256, 0, s>>>(tmp, v->log2_weather, d.seed, kSaltWeather);
        pack2_kernel<T><<<grid_for(nw, 256), 256, 0, s>>>(tmp, (T *)v->weather, v->log2_weather);
        rc = check_launch("generate weather");
    }
    if (!rc) rc = build_occupancy<T>(v, s);
    const int rs = check_cuda(cudaStreamSynchronize(s), "generation");
    cudaFree(tmp);
    return rc ? rc : rs;
}

template <typename T>
int decode_all(const cloud_volume *v, float *base, float *detail, float *weather, cudaStream_t s) {
    if (base && v->base) {
        const uint64_t n = 1ull << (3 * v->log2_base);
        decode_kernel<T><<<grid_for(n, 256), 256, 0, s>>>((const T *)v->base, 8, base, n);
        if (int rc = check_launch("decode base")) return rc;
    }
    if (detail && v->detail) {
        const uint64_t n = 1ull << (3 * v->log2_detail);
        decode_kernel<T><<<grid_for(n, 256), 256, 0, s>>>((const T *)v->detail, 8, detail, n);
        if (int rc = check_launch("decode detail")) return rc;
    }
    if (weather && v->weather) {
        const uint64_t n = 1ull << (2 * v->log2_weather);
        decode_kernel<T><<<grid_for(n, 256), 256, 0, s>>>((const T *)v->weather, 4, weather, n);
        if (int rc = check_launch("decode weather")) return rc;
    }
    return CLOUD_OK;
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

void free_volume(cloud_volume *v) {
    if (!v) return;
    if (v->base) cudaFree(v->base);
    if (v->detail) cudaFree(v->detail);
    if (v->weather) cudaFree(v->weather);
    if (v->occ) cudaFree(v->occ);
    delete v;
}

}  // namespace cloudvol

using namespace cloudvol;

extern "C" const char *cloud_status_string(int status) {
    switch (status) {
        case CLOUD_OK: return "ok";
        case CLOUD_ERR_INVALID_ARG: return "invalid argument";
        case CLOUD_ERR_OUT_OF_MEMORY: return "out of memory";
        case CLOUD_ERR_CUDA: return "CUDA error";
        case CLOUD_ERR_TIMEOUT: return "timeout";
        case CLOUD_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char *cloud_last_error_message(void) { return g_last_error.c_str(); }

extern "C" int cloud_volume_create(const cloud_volume_desc *desc, void *stream, cloud_volume **out) {
    clear_error();
    if (!desc || !out) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: null pointer");
    const cloud_volume_desc &d = *desc;
    if (d.precision < CLOUD_PRECISION_FP32 || d.precision > CLOUD_PRECISION_UNORM16)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: bad precision");
    if (d.density_mode != CLOUD_DENSITY_NOISE && d.density_mode != CLOUD_DENSITY_CONSTANT)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: bad density_mode");
    if (!(d.slab_hi_m > d.slab_lo_m))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: slab_hi_m <= slab_lo_m");
    if (d.slab_hi_m - d.slab_lo_m > 30000.0)
        return set_error(CLOUD_ERR_UNSUPPORTED, "cloud_volume_create: layer thicker than 30 km");
    if (d.density_mode == CLOUD_DENSITY_NOISE) {
        if (!pow2_in(d.base_n, 16, 1024))
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: base_n must be 2^k in [16,1024]");
        if (d.detail_n && !pow2_in(d.detail_n, 16, 1024))
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: detail_n must be 0 or 2^k in [16,1024]");
        if (d.weather_n && !pow2_in(d.weather_n, 16, 4096))
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: weather_n must be 0 or 2^k in [16,4096]");
        if (!(d.base_period_m >= 1.0) || (d.detail_n && !(d.detail_period_m >= 1.0)) ||
            (d.weather_n && !(d.weather_period_m >= 1.0)))
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: periods must be >= 1 m");
        if (!(d.coverage >= 0.0 && d.coverage < 1.0))
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: coverage outside [0,1)");
    } else if (!(d.constant_density >= 0.0)) {
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_create: constant_density < 0");
    }
    cloud_volume *v = new (std::nothrow) cloud_volume();
    if (!v) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_volume_create: host allocation");
    v->desc = d;
    cudaGetDevice(&v->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (d.density_mode == CLOUD_DENSITY_NOISE) {
        const size_t eb = precision_bytes(d.precision);
        v->log2_base = ilog2(d.base_n);
        v->log2_detail = d.detail_n ? ilog2(d.detail_n) : 0;
        v->log2_weather = d.weather_n ? ilog2(d.weather_n) : 0;
        // corner-packed records: 8 texels per 3-D record, 4 per 2-D record
        int rc = check_cuda(cudaMalloc(&v->base, (8 * eb) << (3 * v->log2_base)), "cudaMalloc base");
        if (!rc && d.detail_n)
            rc = check_cuda(cudaMalloc(&v->detail, (8 * eb) << (3 * v->log2_detail)), "cudaMalloc detail");
        if (!rc && d.weather_n)
            rc = check_cuda(cudaMalloc(&v->weather, (4 * eb) << (2 * v->log2_weather)), "cudaMalloc weather");
        if (!rc) {
            if (d.precision == CLOUD_PRECISION_FP32) rc = generate<float>(v, s);
            else if (d.precision == CLOUD_PRECISION_FP16) rc = generate<__half>(v, s);
            else if (d.precision == CLOUD_PRECISION_BF16) rc = generate<__nv_bfloat16>(v, s);
            else rc = generate<uint16_t>(v, s);
        }
        if (rc) {
            cudaStreamSynchronize(s);
            free_volume(v);
            return rc;
        }
    }
    *out = v;
    return CLOUD_OK;
}

extern "C" int cloud_volume_destroy(cloud_volume *vol) {
    clear_error();
    if (!vol) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_destroy: null volume");
    free_volume(vol);
    return CLOUD_OK;
}

extern "C" int cloud_volume_export(const cloud_volume *vol, float *base, float *detail,
                                   float *weather, void *stream) {
    clear_error();
    if (!vol) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_export: null volume");
    cudaStream_t s = (cudaStream_t)stream;
    switch (vol->desc.precision) {
        case CLOUD_PRECISION_FP32: return decode_all<float>(vol, base, detail, weather, s);
        case CLOUD_PRECISION_FP16: return decode_all<__half>(vol, base, detail, weather, s);
        case CLOUD_PRECISION_BF16: return decode_all<__nv_bfloat16>(vol, base, detail, weather, s);
        default: return decode_all<uint16_t>(vol, base, detail, weather, s);
    }
}

extern "C" int cloud_hash4_batch(const uint32_t *keys, int64_t n, uint32_t *out, void *stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!keys || !out)))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_hash4_batch: bad arguments");
    if (!aligned(keys, 16)) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_hash4_batch: keys not 16-byte aligned");
    if (n == 0) return CLOUD_OK;
    hash4_kernel<<<grid_for((uint64_t)n, 256), 256, 0, (cudaStream_t)stream>>>(
        (const uint4 *)keys, out, n);
    return check_launch("hash4_kernel");
}

extern "C" int cloud_volume_occupancy(const cloud_volume *vol, uint32_t *out, int64_t words,
                                      int *log2_cells, void *stream) {
    clear_error();
    if (!vol || !log2_cells) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_occupancy: null pointer");
    if (!vol->occ) {
        *log2_cells = -1;
        return CLOUD_OK;
    }
    *log2_cells = vol->log2_occ;
    const int64_t need = (int64_t)(((1ull << (3 * vol->log2_occ)) + 31) / 32);
    if (!out) return CLOUD_OK;
    if (words != need)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_volume_occupancy: words must be ceil(cells / 32)");
    return check_cuda(cudaMemcpyAsync(out, vol->occ, need * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream),
                      "cloud_volume_occupancy");
}

extern "C" int cloud_debug_check_status(unsigned int *bits, int reset) {
    clear_error();
    if (!bits) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_debug_check_status: null pointer");
    *bits = 0;
#if CLOUDVOL_CHECKED
    unsigned *w = check_word();
    if (!w) return set_error(CLOUD_ERR_CUDA, "cloud_debug_check_status: no status word");
    if (int rc = check_cuda(cudaMemcpy(bits, w, sizeof(unsigned), cudaMemcpyDeviceToHost),
                            "cloud_debug_check_status"))
        return rc;
    if (reset) return check_cuda(cudaMemset(w, 0, sizeof(unsigned)), "cloud_debug_check_status");
    return CLOUD_OK;
#else
    (void)reset;
    return set_error(CLOUD_ERR_UNSUPPORTED, "cloud_debug_check_status: not a checked build");
#endif
}
