// march_kernels.cuh -- the raymarch kernels (one view; many views from a work
// queue) and their dispatch over storage type, light-step specialisation, tile
// sizes and tile shape, for one chunk size CH.  Included only by
// march{8,16}_{view,batch}.cu, which instantiate the single-view and the
// multi-view kernels for CH = 8 and CH = 16 (four units compiled in parallel).
#pragma once

#include "march.cuh"

namespace cloudvol {

template <typename T, int LS, int SHAPE, bool FX, int CH>
__global__ void __launch_bounds__(128, MarchBlocks<T, FX, CH>::value)
    march_kernel(const __grid_constant__ SceneParams p, const __grid_constant__ ViewParams v,
                 const T *__restrict__ base, const T *__restrict__ detail,
                 const T *__restrict__ weather, unsigned long long *__restrict__ counter) {
    __shared__ WarpScratch<CH, FX> scratch[4];
    const unsigned long long n = march_tile<T, LS, SHAPE, FX, CH>(
        p, v, blockIdx.x, blockIdx.y, scratch[threadIdx.x >> 5], base, detail, weather);
    count_lookups(counter, n);
}

// Persistent multi-view march: one CTA per resident slot takes (view, tile)
// items from a device counter until the queue is empty; the view of an item
// is found by binary search over the views' first tile indices and staged in
// shared memory.
template <typename T, int LS, int SHAPE, bool FX, int CH>
__global__ void __launch_bounds__(128, MarchBlocks<T, FX, CH>::value)
    march_batch_kernel(const __grid_constant__ SceneParams p, const ViewParams *__restrict__ views,
                       int n_views, int total_tiles, unsigned int *__restrict__ work,
                       const T *__restrict__ base, const T *__restrict__ detail,
                       const T *__restrict__ weather, unsigned long long *__restrict__ counter) {
    __shared__ WarpScratch<CH, FX> scratch[4];
    __shared__ ViewParams sv;
    __shared__ int s_tile, s_view;
    unsigned long long n_look = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = (int)atomicAdd(work, 1u);
            s_tile = t;
            if (t < total_tiles) {
                int lo = 0, hi = n_views - 1;  // last view with tile_begin <= t
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (views[mid].tile_begin <= t) lo = mid;
                    else hi = mid - 1;
                }
                s_view = lo;
            }
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= total_tiles) break;
        const int *src = reinterpret_cast<const int *>(views + s_view);
        int *dst = reinterpret_cast<int *>(&sv);
        for (int i = threadIdx.x; i < (int)(sizeof(ViewParams) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        const int local = t - sv.tile_begin;
        if (in_range(p.check, s_view >= 0 && s_view < n_views && local >= 0 && local < sv.tile_count,
                     kChkView))
            n_look += march_tile<T, LS, SHAPE, FX, CH>(p, sv, local % sv.tiles_x, local / sv.tiles_x,
                                                       scratch[threadIdx.x >> 5], base, detail, weather);
        __syncthreads();  // s_tile / sv are rewritten by the next iteration
    }
    count_lookups(counter, n_look);
}

template <typename T, int SHAPE, int CH>
void launch_shape(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                  unsigned long long *counter, cudaStream_t s) {
    int tw, th;
    tile_dims(SHAPE, &tw, &th);
    const dim3 grid(v.tiles_x, (v.height + th - 1) / th);
    const T *b = (const T *)vol->base, *d = (const T *)vol->detail, *w = (const T *)vol->weather;
    if (fixed_sizes(p, vol))
        march_kernel<T, 6, SHAPE, true, CH><<<grid, 128, 0, s>>>(p, v, b, d, w, counter);
    else if (p.light_steps == 6)
        march_kernel<T, 6, SHAPE, false, CH><<<grid, 128, 0, s>>>(p, v, b, d, w, counter);
    else
        march_kernel<T, -1, SHAPE, false, CH><<<grid, 128, 0, s>>>(p, v, b, d, w, counter);
}

template <typename T, int CH>
void launch_typed(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                  unsigned long long *counter, int shape, cudaStream_t s) {
    switch (shape) {
        case 1: launch_shape<T, 1, CH>(p, v, vol, counter, s); break;
        case 2: launch_shape<T, 2, CH>(p, v, vol, counter, s); break;
        case 3: launch_shape<T, 3, CH>(p, v, vol, counter, s); break;
        default: launch_shape<T, 0, CH>(p, v, vol, counter, s);
    }
}

template <int CH>
void launch_march_ch(const SceneParams &p, const ViewParams &v, const cloud_volume *vol,
                     unsigned long long *counter, int shape, cudaStream_t s) {
    switch (vol->desc.precision) {
        case CLOUD_PRECISION_FP32: launch_typed<float, CH>(p, v, vol, counter, shape, s); break;
        case CLOUD_PRECISION_FP16: launch_typed<__half, CH>(p, v, vol, counter, shape, s); break;
        case CLOUD_PRECISION_BF16: launch_typed<__nv_bfloat16, CH>(p, v, vol, counter, shape, s); break;
        default: launch_typed<uint16_t, CH>(p, v, vol, counter, shape, s);
    }
}

template <typename T, int SHAPE, int CH>
const void *batch_kernel_ptr(int light_steps, bool fx) {
    if (fx) return (const void *)march_batch_kernel<T, 6, SHAPE, true, CH>;
    return light_steps == 6 ? (const void *)march_batch_kernel<T, 6, SHAPE, false, CH>
                            : (const void *)march_batch_kernel<T, -1, SHAPE, false, CH>;
}
template <typename T, int CH>
const void *batch_kernel_typed(int light_steps, bool fx, int shape) {
    switch (shape) {
        case 1: return batch_kernel_ptr<T, 1, CH>(light_steps, fx);
        case 2: return batch_kernel_ptr<T, 2, CH>(light_steps, fx);
        case 3: return batch_kernel_ptr<T, 3, CH>(light_steps, fx);
        default: return batch_kernel_ptr<T, 0, CH>(light_steps, fx);
    }
}
template <int CH>
const void *batch_kernel_ch(int precision, int light_steps, bool fx, int shape) {
    switch (precision) {
        case CLOUD_PRECISION_FP32: return batch_kernel_typed<float, CH>(light_steps, fx, shape);
        case CLOUD_PRECISION_FP16: return batch_kernel_typed<__half, CH>(light_steps, fx, shape);
        case CLOUD_PRECISION_BF16: return batch_kernel_typed<__nv_bfloat16, CH>(light_steps, fx, shape);
        default: return batch_kernel_typed<uint16_t, CH>(light_steps, fx, shape);
    }
}

}  // namespace cloudvol
