// common.cuh -- internal definitions shared by the CUDA translation units of
// libcloudvol.so (not part of the public ABI; see include/cloudvol.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

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
    void *base;      // device, base_n^3 texels of the storage precision
    void *detail;    // device or nullptr
    void *weather;   // device or nullptr
    int device;
};

namespace cloudvol {

inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

inline size_t precision_bytes(int p) { return p == CLOUD_PRECISION_FP32 ? 4 : 2; }

// Texel loads through the read-only path, decoded to float.
__device__ __forceinline__ float load_texel(const float *p, uint32_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_texel(const __half *p, uint32_t i) {
    return __half2float(__ldg(p + i));
}
__device__ __forceinline__ float load_texel(const __nv_bfloat16 *p, uint32_t i) {
    return __bfloat162float(__ldg(p + i));
}

}  // namespace cloudvol
