// session.cu -- one camera's stream of TAA frames (Sec. 3.2: a jittered,
// reduced-step render every frame, resolved against the reprojected history).
//
// The session owns its device buffers and the frame index that selects the
// per-frame jitter; a frame is render -> (motion + TAA resolve, fused) -> swap.
#include <cstring>
#include <new>

#include "common.cuh"

namespace cloudvol {
int launch_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                  int width, int height, int steps, int light_steps, int jitter_frame,
                  int integration, float *out, unsigned long long *counter, cudaStream_t s);
int launch_taa_reproject(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                         const cloud_camera *cur, const void *history, const float *current,
                         void *history_out, int width, int height, int fmt, float blend,
                         cudaStream_t s);
}  // namespace cloudvol

struct cloud_session {
    const cloud_volume *vol;
    int width, height, fmt;
    float *current;  // device RGBA float, the raw jittered render
    void *hist[2];   // device history ping-pong
    int latest;      // index of the latest resolved frame in hist
    bool has_history;
    int frame;
    cloud_camera prev_cam;
};

using namespace cloudvol;

namespace {
void free_session(cloud_session *s) {
    if (!s) return;
    if (s->current) cudaFree(s->current);
    if (s->hist[0]) cudaFree(s->hist[0]);
    if (s->hist[1]) cudaFree(s->hist[1]);
    delete s;
}
}  // namespace

extern "C" int cloud_session_create(const cloud_volume *vol, int width, int height, int history_fmt,
                                    cloud_session **out) {
    clear_error();
    if (!vol || !out) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_create: null pointer");
    if (width < 1 || height < 1 || width > CLOUD_MAX_DIM || height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_create: width/height outside [1, 16384]");
    if (history_fmt != CLOUD_HISTORY_FP32 && history_fmt != CLOUD_HISTORY_FP16)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_create: bad history format");
    cloud_session *s = new (std::nothrow) cloud_session();
    if (!s) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_session_create: host allocation");
    s->vol = vol;
    s->width = width;
    s->height = height;
    s->fmt = history_fmt;
    const size_t px = (size_t)width * height;
    const size_t hb = px * (history_fmt == CLOUD_HISTORY_FP32 ? 16 : 8);
    int rc = check_cuda(cudaMalloc(&s->current, px * 16), "cudaMalloc current");
    if (!rc) rc = check_cuda(cudaMalloc(&s->hist[0], hb), "cudaMalloc history");
    if (!rc) rc = check_cuda(cudaMalloc(&s->hist[1], hb), "cudaMalloc history");
    if (rc) {
        free_session(s);
        return rc;
    }
    *out = s;
    return CLOUD_OK;
}

extern "C" int cloud_session_destroy(cloud_session *s) {
    clear_error();
    if (!s) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_destroy: null session");
    free_session(s);
    return CLOUD_OK;
}

extern "C" int cloud_session_reset(cloud_session *s) {
    clear_error();
    if (!s) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_reset: null session");
    s->has_history = false;
    return CLOUD_OK;
}

extern "C" int cloud_session_frame(cloud_session *s, const cloud_camera *cam,
                                   const cloud_params *prm, int steps, int light_steps,
                                   int integration, float blend, void *host_out,
                                   const void **dev_out, void *stream) {
    clear_error();
    if (!s || !cam || !prm) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_frame: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_render(s->vol, cam, prm, s->width, s->height, steps, light_steps, s->frame,
                           integration, s->current, nullptr, st);
    if (rc) return rc;
    const int next = 1 - s->latest;
    // reprojection motion and TAA resolve fused (the motion is never stored)
    rc = launch_taa_reproject(s->vol, prm, s->has_history ? &s->prev_cam : nullptr, cam,
                              s->has_history ? s->hist[s->latest] : nullptr, s->current,
                              s->hist[next], s->width, s->height, s->fmt, blend, st);
    if (rc) return rc;
    s->latest = next;
    s->has_history = true;
    s->prev_cam = *cam;
    s->frame += 1;
    if (dev_out) *dev_out = s->hist[s->latest];
    if (host_out) {
        const size_t bytes = (size_t)s->width * s->height * (s->fmt == CLOUD_HISTORY_FP32 ? 16 : 8);
        rc = check_cuda(cudaMemcpyAsync(host_out, s->hist[s->latest], bytes, cudaMemcpyDeviceToHost, st),
                        "cudaMemcpyAsync resolved frame");
        if (rc) return rc;
        rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    }
    return rc;
}
