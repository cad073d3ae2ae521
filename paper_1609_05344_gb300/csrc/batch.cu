// batch.cu -- many views of uneven size and step count in one persistent
// launch (the raymarch of Sec. 1 / Sec. 3.1 / Sec. 3.2 per view).
//
// The work queue is the concatenation of every view's pixel tiles, ordered by
// decreasing per-tile cost (step count) so that the long tiles start first
// and the tail is made of short ones.  One CTA per resident slot loops: take
// the next tile index from a device counter, find its view (binary search over
// the views' first tile indices), stage the view constants in shared memory,
// march the tile.  The launch (counter reset + kernel) is captured once into a
// CUDA graph and replayed; per-frame camera changes only rewrite the device
// view table.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "march.cuh"

namespace cloudvol {

static const void *batch_kernel(int precision, int light_steps, bool fx, int config) {
    return config_chunk(config) == 16
               ? batch_kernel_ch<16>(precision, light_steps, fx, config_shape(config))
               : batch_kernel_ch<8>(precision, light_steps, fx, config_shape(config));
}

// Enqueue counter reset + persistent kernel for the given table on stream s.
int launch_batch(const cloud_volume *vol, const SceneParams &scene, const ViewParams *d_views,
                 int n_views, int total_tiles, int config, unsigned int *d_work,
                 unsigned long long *counter, cudaStream_t s) {
    if (total_tiles == 0) return CLOUD_OK;
    const void *fn = batch_kernel(vol->desc.precision, scene.light_steps, fixed_sizes(scene, vol), config);
    int dev = 0, sms = 0, per_sm = 0;
    if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
    if (int rc = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                            "cudaDeviceGetAttribute"))
        return rc;
    if (int rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 128, 0),
                            "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
        return rc;
    const int grid = std::max(1, std::min(total_tiles, sms * std::max(per_sm, 1)));
    if (int rc = check_cuda(cudaMemsetAsync(d_work, 0, sizeof(unsigned int), s), "reset work counter"))
        return rc;
    SceneParams scene_arg = scene;
    const void *b = vol->base, *d = vol->detail, *w = vol->weather;
    void *args[] = {(void *)&scene_arg, (void *)&d_views, (void *)&n_views, (void *)&total_tiles,
                    (void *)&d_work, (void *)&b, (void *)&d, (void *)&w, (void *)&counter};
    return check_cuda(cudaLaunchKernel(fn, dim3(grid), dim3(128), args, 0, s), "march_batch_kernel");
}

}  // namespace cloudvol

using namespace cloudvol;

struct cloud_batch {
    const cloud_volume *vol;
    cloud_params prm;
    SceneParams scene;
    int n_views, total_tiles, config;  // config: tile shape + view steps per iteration
    std::vector<cloud_view> views;  // caller order
    std::vector<int> order;         // queue order (decreasing steps)
    std::vector<ViewParams> table;  // queue order
    ViewParams *d_views;
    unsigned int *d_work;
    cudaGraphExec_t exec;
    cudaStream_t capture_stream;
};

namespace {

void drop_graph(cloud_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

void free_batch(cloud_batch *b) {
    if (!b) return;
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->d_views) cudaFree(b->d_views);
    if (b->d_work) cudaFree(b->d_work);
    delete b;
}

// (Re)build the view table in queue order for the batch's tile shape (from its
// launch configuration) and upload it on stream s.
int build_table(cloud_batch *b, cudaStream_t s) {
    b->table.resize(b->n_views);
    int next = 0;
    for (int q = 0; q < b->n_views; ++q) {
        const cloud_view &cv = b->views[b->order[q]];
        ViewParams &v = b->table[q];
        if (int rc = build_view(b->vol, &b->prm, &cv.camera, cv.width, cv.height, cv.steps,
                                cv.jitter_frame, cv.out_rgba, config_shape(b->config), &v))
            return rc;
        v.tile_begin = next;
        next += v.tile_count;
    }
    b->total_tiles = next;
    return check_cuda(cudaMemcpyAsync(b->d_views, b->table.data(), sizeof(ViewParams) * b->n_views,
                                      cudaMemcpyHostToDevice, s),
                      "upload view table");
}

}  // namespace

extern "C" int cloud_batch_create(const cloud_volume *vol, const cloud_params *prm, int light_steps,
                                  int integration, const cloud_view *views, int n_views,
                                  cloud_batch **out) {
    clear_error();
    if (!vol || !prm || !views || !out || n_views < 1 || n_views > CLOUD_MAX_VIEWS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_create: bad arguments");
    cloud_batch *b = new (std::nothrow) cloud_batch();
    if (!b) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_batch_create: host allocation");
    b->vol = vol;
    b->prm = *prm;
    b->n_views = n_views;
    b->config = tuned_config(vol->desc.precision, light_steps);
    b->views.assign(views, views + n_views);
    b->order.resize(n_views);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
        return b->views[a].steps > b->views[c].steps;  // longest tiles first
    });
    int rc = build_scene(vol, prm, light_steps, integration, &b->scene);
    if (!rc) rc = check_cuda(cudaMalloc(&b->d_views, sizeof(ViewParams) * n_views), "cudaMalloc views");
    if (!rc) rc = check_cuda(cudaMalloc(&b->d_work, sizeof(unsigned int)), "cudaMalloc work counter");
    if (!rc) rc = check_cuda(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking),
                             "cudaStreamCreate");
    if (!rc) rc = build_table(b, b->capture_stream);
    if (!rc) rc = check_cuda(cudaStreamSynchronize(b->capture_stream), "cudaStreamSynchronize");
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return CLOUD_OK;
}

extern "C" int cloud_batch_destroy(cloud_batch *b) {
    clear_error();
    if (!b) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_destroy: null batch");
    cudaStreamSynchronize(b->capture_stream);
    free_batch(b);
    return CLOUD_OK;
}

extern "C" int cloud_batch_set_views(cloud_batch *b, const cloud_view *views, int n_views,
                                     void *stream) {
    clear_error();
    if (!b || !views || n_views != b->n_views)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_set_views: bad arguments");
    for (int i = 0; i < n_views; ++i)
        if (views[i].width != b->views[i].width || views[i].height != b->views[i].height ||
            views[i].steps != b->views[i].steps)
            return set_error(CLOUD_ERR_INVALID_ARG,
                             "cloud_batch_set_views: sizes and step counts must not change");
    b->views.assign(views, views + n_views);
    return build_table(b, (cudaStream_t)stream);
}

extern "C" int cloud_batch_render(cloud_batch *b, void *stream) {
    clear_error();
    if (!b) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_render: null batch");
    return launch_batch(b->vol, b->scene, b->d_views, b->n_views, b->total_tiles, b->config,
                        b->d_work, nullptr, (cudaStream_t)stream);
}

extern "C" int cloud_batch_render_graph(cloud_batch *b, void *stream) {
    clear_error();
    if (!b) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_render_graph: null batch");
    if (!b->exec) {
        cudaStream_t cs = b->capture_stream;
        int rc = check_cuda(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal),
                            "cudaStreamBeginCapture");
        if (rc) return rc;
        const int lrc = launch_batch(b->vol, b->scene, b->d_views, b->n_views, b->total_tiles,
                                     b->config, b->d_work, nullptr, cs);
        cudaGraph_t g = nullptr;
        rc = check_cuda(cudaStreamEndCapture(cs, &g), "cudaStreamEndCapture");
        if (lrc || rc) {
            if (g) cudaGraphDestroy(g);
            return lrc ? lrc : rc;
        }
        rc = check_cuda(cudaGraphInstantiate(&b->exec, g, 0), "cudaGraphInstantiate");
        cudaGraphDestroy(g);
        if (rc) {
            b->exec = nullptr;
            return rc;
        }
    }
    return check_cuda(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "cudaGraphLaunch");
}

extern "C" int cloud_batch_render_per_view(cloud_batch *b, void *stream) {
    clear_error();
    if (!b) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_render_per_view: null batch");
    for (int q = 0; q < b->n_views; ++q)
        if (int rc = launch_march(b->scene, b->table[q], b->vol, nullptr, b->config,
                                  (cudaStream_t)stream))
            return rc;
    return CLOUD_OK;
}

extern "C" int cloud_batch_autotune(cloud_batch *b, int repeats, float *times_ms, int *best,
                                    void *stream) {
    clear_error();
    if (!b || repeats < 1) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_autotune: bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (int rc = check_cuda(cudaEventCreate(&e0), "cudaEventCreate")) return rc;
    if (int rc = check_cuda(cudaEventCreate(&e1), "cudaEventCreate")) {
        cudaEventDestroy(e0);
        return rc;
    }
    drop_graph(b);
    int rc = CLOUD_OK, best_config = 0;
    float best_ms = INFINITY;
    for (int config = 0; config < kConfigs && !rc; ++config) {
        b->config = config;
        rc = build_table(b, s);
        if (!rc) rc = cloud_batch_render(b, s);  // warm-up
        if (!rc) rc = check_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
        for (int r = 0; r < repeats && !rc; ++r) rc = cloud_batch_render(b, s);
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
    b->config = best_config;
    if (int r2 = build_table(b, s)) return r2;
    if (best) *best = best_config;
    return CLOUD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the multi-view launch.  Its scratch (the work
// counter and the view table) lives in one file-scope device array sized for
// CLOUD_STATIC_MAX_VIEWS views, which every GPU that loads the library keeps
// until the process exits.  Host code cannot pass the array's name to a
// kernel (on the host it only stands in for the symbol), so the device address
// is looked up once per device with that device current and cached.
namespace {
constexpr size_t kStaticTableOffset = 256;  // the counter sits in the first 256 bytes
constexpr size_t kStaticBytes = kStaticTableOffset + sizeof(ViewParams) * CLOUD_STATIC_MAX_VIEWS;
// the documented size of the array (include/cloudvol.h); fails to compile if ViewParams changes
static_assert(kStaticBytes == 47360, "static scratch size changed: update its documentation");
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

static int static_scratch_address(void **out) {
    int dev = 0;
    if (int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(CLOUD_ERR_UNSUPPORTED, "cloud_batch_render_static: device index >= 64");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        if (int rc = check_cuda(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress"))
            return rc;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return CLOUD_OK;
}

extern "C" int cloud_batch_render_static(const cloud_volume *vol, const cloud_params *prm,
                                         int light_steps, int integration, const cloud_view *views,
                                         int n_views, void *stream) {
    clear_error();
    if (!vol || !prm || !views || n_views < 1)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_batch_render_static: bad arguments");
    if (n_views > CLOUD_STATIC_MAX_VIEWS)
        return set_error(CLOUD_ERR_INVALID_ARG,
                         "cloud_batch_render_static: more views than the static scratch holds (256)");
    SceneParams scene;
    if (int rc = build_scene(vol, prm, light_steps, integration, &scene)) return rc;
    // host staging of the table: per-thread static storage, no per-call allocation
    thread_local ViewParams table[CLOUD_STATIC_MAX_VIEWS];
    int order[CLOUD_STATIC_MAX_VIEWS];
    for (int i = 0; i < n_views; ++i) order[i] = i;
    for (int i = 1; i < n_views; ++i)  // stable insertion sort, longest step counts first
        for (int j = i; j > 0 && views[order[j]].steps > views[order[j - 1]].steps; --j)
            std::swap(order[j], order[j - 1]);
    const int config = tuned_config(vol->desc.precision, light_steps);
    int next = 0;
    for (int q = 0; q < n_views; ++q) {
        const cloud_view &cv = views[order[q]];
        if (int rc = build_view(vol, prm, &cv.camera, cv.width, cv.height, cv.steps, cv.jitter_frame,
                                cv.out_rgba, config_shape(config), &table[q]))
            return rc;
        table[q].tile_begin = next;
        next += table[q].tile_count;
    }
    void *base = nullptr;
    if (int rc = static_scratch_address(&base)) return rc;
    unsigned int *work = static_cast<unsigned int *>(base);
    ViewParams *d_views = reinterpret_cast<ViewParams *>(static_cast<char *>(base) + kStaticTableOffset);
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = check_cuda(cudaMemcpyAsync(d_views, table, sizeof(ViewParams) * n_views,
                                            cudaMemcpyHostToDevice, s),
                            "cloud_batch_render_static: upload view table"))
        return rc;
    return launch_batch(vol, scene, d_views, n_views, next, config, work, nullptr, s);
}
