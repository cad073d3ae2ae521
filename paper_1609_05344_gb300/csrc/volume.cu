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

__device__ __forceinline__ double unit_value(uint32_t h) {
    return (double)(h >> 8) * (1.0 / 16777216.0);
}

template <typename T>
__device__ __forceinline__ T encode(double v);
template <>
__device__ __forceinline__ float encode<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half encode<__half>(double v) { return __double2half(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 encode<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

template <>
__device__ __forceinline__ uint16_t encode<uint16_t>(double v) {
    const double q = rint((v + (double)kCentre) * 65536.0);
    return (uint16_t)(q < 0.0 ? 0.0 : (q > 65535.0 ? 65535.0 : q));
}

template <typename T>
__global__ void fbm3_kernel(T *__restrict__ out, int log2n, uint32_t seed, uint32_t salt) {
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
        out[i] = encode<T>(sum / amp_sum - (double)kCentre);
    }
}

template <typename T>
__global__ void fbm2_kernel(T *__restrict__ out, int log2n, uint32_t seed, uint32_t salt) {
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
        out[i] = encode<T>(sum / amp_sum - (double)kCentre);
    }
}

// Corner-packing of a generated tile (see common.cuh).
// Record layout (see common.cuh): the dx = 0 half of a record holds texels,
// the dx = 1 half holds them as differences from the dx = 0 half for FP32
// tiles (rounded exactly as the lerp would round them) and as texels for
// 16-bit tiles (whose loaders form the differences after decoding).
template <typename T, int R>
__device__ __forceinline__ void store_record(T *dst, const T (&t)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r] = t[r];
}
template <int R>
__device__ __forceinline__ void store_record(float *dst, const float (&t)[R]) {
#pragma unroll
    for (int r = 0; r < R / 2; ++r) dst[r] = t[r];
#pragma unroll
    for (int r = R / 2; r < R; ++r) dst[r] = __fsub_rn(t[r], t[r - R / 2]);
}

template <typename T>
__global__ void pack3_kernel(const T *__restrict__ plain, T *__restrict__ packed, int log2n) {
    const uint32_t mask = (1u << log2n) - 1u;
    const uint64_t total = 1ull << (3 * log2n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)i & mask, y = (uint32_t)(i >> log2n) & mask,
                       z = (uint32_t)(i >> (2 * log2n));
        T t[8];
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
__global__ void pack2_kernel(const T *__restrict__ plain, T *__restrict__ packed, int log2n) {
    const uint32_t mask = (1u << log2n) - 1u;
    const uint64_t total = 1ull << (2 * log2n);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)i & mask, y = (uint32_t)(i >> log2n);
        T t[4];
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
        out[i] = load_texel(packed, (uint32_t)(stride * i)) + kCentre;
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

// Generates each tile into a plain scratch array, then corner-packs it.
template <typename T>
int generate(cloud_volume *v, cudaStream_t s) {
    const cloud_volume_desc &d = v->desc;
    const uint64_t nb = 1ull << (3 * v->log2_base);
    const uint64_t nd = v->detail ? 1ull << (3 * v->log2_detail) : 0;
    const uint64_t nw = v->weather ? 1ull << (2 * v->log2_weather) : 0;
    const uint64_t most = nb > nd ? (nb > nw ? nb : nw) : (nd > nw ? nd : nw);
    T *tmp = nullptr;
    int rc = check_cuda(cudaMalloc(&tmp, most * sizeof(T)), "cudaMalloc generation scratch");
    if (rc) return rc;
    fbm3_kernel<T><<<grid_for(nb, 256), 256, 0, s>>>(tmp, v->log2_base, d.seed, kSaltBase);
    pack3_kernel<T><<<grid_for(nb, 256), 256, 0, s>>>(tmp, (T *)v->base, v->log2_base);
    rc = check_launch("generate base");
    if (!rc && v->detail) {
        fbm3_kernel<T><<<grid_for(nd, 256), 256, 0, s>>>(tmp, v->log2_detail, d.seed, kSaltDetail);
        pack3_kernel<T><<<grid_for(nd, 256), 256, 0, s>>>(tmp, (T *)v->detail, v->log2_detail);
        rc = check_launch("generate detail");
    }
    if (!rc && v->weather) {
        fbm2_kernel<T><<<grid_for(nw, 256), 256, 0, s>>>(tmp, v->log2_weather, d.seed, kSaltWeather);
        pack2_kernel<T><<<grid_for(nw, 256), 256, 0, s>>>(tmp, (T *)v->weather, v->log2_weather);
        rc = check_launch("generate weather");
    }
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
