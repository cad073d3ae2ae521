// session.cu -- one camera's stream of TAA frames (Sec. 3.2: a jittered,
// reduced-step render every frame, resolved against the reprojected history).
//
// The session owns its device buffers and the frame index that selects the
// per-frame jitter; a frame is render -> (motion + TAA resolve, fused) -> swap.
#include <chrono>
#include <cstring>
#include <string>
#include <new>
#include <thread>

#include "common.cuh"

namespace cloudvol {
int launch_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                  int width, int height, int steps, int light_steps, int jitter_frame,
                  int integration, float *out, unsigned long long *counter, cudaStream_t s);
int launch_taa_reproject(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                         const cloud_camera *cur, const void *history, const float *current,
                         void *history_out, int width, int height, int fmt, float blend,
                         unsigned int *status, cudaStream_t s);
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
    // asynchronous read-back: D2H copies of resolved frames run on their own
    // stream; copied[i] marks the end of the last copy out of hist[i], so the
    // resolve that next overwrites hist[i] waits for it
    cudaStream_t copy_stream;
    cudaEvent_t resolved[2], copied[2];
    bool copy_pending[2];
    int copy_frame[2];  // frame index whose copy was last issued from hist[i]
    // bounded waits of this session's resolves that gave up: a counter in
    // mapped pinned host memory the resolve kernel increments (never reset, so
    // no reset can race with a kernel in flight); wait_seen is the value last
    // accounted for.  A give-up leaves a tile of the history unwritten, so the
    // session reports CLOUD_ERR_TIMEOUT until cloud_session_reset.
    unsigned int *h_wait, *d_wait;
    unsigned int wait_seen;
    bool wait_failed;
};

using namespace cloudvol;

namespace {
void free_session(cloud_session *s) {
    if (!s) return;
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    for (int i = 0; i < 2; ++i) {
        if (s->resolved[i]) cudaEventDestroy(s->resolved[i]);
        if (s->copied[i]) cudaEventDestroy(s->copied[i]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->current) cudaFree(s->current);
    if (s->hist[0]) cudaFree(s->hist[0]);
    if (s->hist[1]) cudaFree(s->hist[1]);
    if (s->h_wait) cudaFreeHost(s->h_wait);
    delete s;
}

// CLOUD_ERR_TIMEOUT once a resolve of this session has given up a bounded
// wait (seen through the mapped counter), until cloud_session_reset.
int check_waits(cloud_session *s, const char *where) {
    const unsigned int v = *reinterpret_cast<volatile unsigned int *>(s->h_wait);
    if (v != s->wait_seen) {
        s->wait_seen = v;
        s->wait_failed = true;
    }
    if (s->wait_failed)
        return set_error(CLOUD_ERR_TIMEOUT, std::string(where) +
                                                ": a bounded wait of the TAA resolve gave up, the "
                                                "history misses a tile until cloud_session_reset");
    return CLOUD_OK;
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
    if (!rc) rc = check_cuda(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking),
                             "cudaStreamCreate");
    if (!rc) rc = check_cuda(cudaHostAlloc((void **)&s->h_wait, sizeof(unsigned int), cudaHostAllocMapped),
                             "cudaHostAlloc wait counter");
    if (!rc) {
        *s->h_wait = 0;
        rc = check_cuda(cudaHostGetDevicePointer((void **)&s->d_wait, s->h_wait, 0),
                        "cudaHostGetDevicePointer wait counter");
    }
    for (int i = 0; i < 2 && !rc; ++i) {
        rc = check_cuda(cudaEventCreateWithFlags(&s->resolved[i], cudaEventDisableTiming), "cudaEventCreate");
        if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming), "cudaEventCreate");
        s->copy_frame[i] = -1;
    }
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
    s->wait_seen = *reinterpret_cast<volatile unsigned int *>(s->h_wait);
    s->wait_failed = false;
    return CLOUD_OK;
}

namespace {
// Render + fused resolve of one frame on `st`; returns the history index written.
int session_render(cloud_session *s, const cloud_camera *cam, const cloud_params *prm, int steps,
                   int light_steps, int integration, float blend, cudaStream_t st, int *written) {
    int rc = launch_render(s->vol, cam, prm, s->width, s->height, steps, light_steps, s->frame,
                           integration, s->current, nullptr, st);
    if (rc) return rc;
    const int next = 1 - s->latest;
    // a read-back of hist[next] still in flight must finish before it is overwritten
    if (s->copy_pending[next]) {
        rc = check_cuda(cudaStreamWaitEvent(st, s->copied[next], 0), "cudaStreamWaitEvent");
        if (rc) return rc;
        s->copy_pending[next] = false;
    }
    // reprojection motion and TAA resolve fused (the motion is never stored)
    rc = launch_taa_reproject(s->vol, prm, s->has_history ? &s->prev_cam : nullptr, cam,
                              s->has_history ? s->hist[s->latest] : nullptr, s->current,
                              s->hist[next], s->width, s->height, s->fmt, blend, s->d_wait, st);
    if (rc) return rc;
    s->latest = next;
    s->has_history = true;
    s->prev_cam = *cam;
    s->frame += 1;
    *written = next;
    return CLOUD_OK;
}

size_t frame_bytes(const cloud_session *s) {
    return (size_t)s->width * s->height * (s->fmt == CLOUD_HISTORY_FP32 ? 16 : 8);
}
}  // namespace

extern "C" int cloud_session_frame(cloud_session *s, const cloud_camera *cam,
                                   const cloud_params *prm, int steps, int light_steps,
                                   int integration, float blend, void *host_out,
                                   const void **dev_out, void *stream) {
    clear_error();
    if (!s || !cam || !prm) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_frame: null pointer");
    if (int rc = check_waits(s, "cloud_session_frame")) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int written = 0;
    int rc = session_render(s, cam, prm, steps, light_steps, integration, blend, st, &written);
    if (rc) return rc;
    if (dev_out) *dev_out = s->hist[written];
    if (host_out) {
        rc = check_cuda(cudaMemcpyAsync(host_out, s->hist[written], frame_bytes(s),
                                        cudaMemcpyDeviceToHost, st),
                        "cudaMemcpyAsync resolved frame");
        if (rc) return rc;
        rc = check_cuda(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        if (!rc) rc = check_waits(s, "cloud_session_frame");
    }
    return rc;
}

extern "C" int cloud_session_frame_async(cloud_session *s, const cloud_camera *cam,
                                         const cloud_params *prm, int steps, int light_steps,
                                         int integration, float blend, void *host_out,
                                         int *frame_index, void *stream) {
    clear_error();
    if (!s || !cam || !prm || !host_out)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_frame_async: null pointer");
    if (int rc = check_waits(s, "cloud_session_frame_async")) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int index = s->frame;
    int written = 0;
    int rc = session_render(s, cam, prm, steps, light_steps, integration, blend, st, &written);
    if (rc) return rc;
    // the read-back runs on the copy stream, overlapping the next frame's render
    rc = check_cuda(cudaEventRecord(s->resolved[written], st), "cudaEventRecord");
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(s->copy_stream, s->resolved[written], 0),
                             "cudaStreamWaitEvent");
    if (!rc) rc = check_cuda(cudaMemcpyAsync(host_out, s->hist[written], frame_bytes(s),
                                             cudaMemcpyDeviceToHost, s->copy_stream),
                             "cudaMemcpyAsync resolved frame");
    if (!rc) rc = check_cuda(cudaEventRecord(s->copied[written], s->copy_stream), "cudaEventRecord");
    if (rc) return rc;
    s->copy_pending[written] = true;
    s->copy_frame[written] = index;
    if (frame_index) *frame_index = index;
    return CLOUD_OK;
}

extern "C" int cloud_session_wait_frame(cloud_session *s, int frame_index, int timeout_ms) {
    clear_error();
    if (!s) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_wait_frame: null session");
    // copies complete in issue order on the copy stream, so the earliest tracked
    // copy at or after frame_index finishing implies that frame's copy finished
    int slot = -1;
    for (int i = 0; i < 2; ++i)
        if (s->copy_frame[i] >= frame_index &&
            (slot < 0 || s->copy_frame[i] < s->copy_frame[slot]))
            slot = i;
    if (frame_index < 0 || slot < 0)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_wait_frame: no such frame");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {  // bounded host-side polling of the copy's completion event
        const cudaError_t q = cudaEventQuery(s->copied[slot]);
        if (q == cudaSuccess) return check_waits(s, "cloud_session_wait_frame");
        if (q != cudaErrorNotReady) return check_cuda(q, "cudaEventQuery");
        if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
            return set_error(CLOUD_ERR_TIMEOUT, "cloud_session_wait_frame: read-back not finished");
        std::this_thread::yield();
    }
}

// ---------------------------------------------------------------------------
// Snapshot / restore: the state a session needs to continue -- its latest
// resolved frame (the history the next resolve reprojects), whether it has
// one, its frame index (the next jitter frame) and the previous camera -- as
// one block of host memory: a header followed by the history pixels.
namespace {
constexpr uint32_t kSnapMagic = 0x43564C53u;  // "SLVC"
constexpr uint32_t kSnapVersion = 1;
struct SnapHeader {
    uint32_t magic, version;
    int32_t width, height, fmt, has_history, frame, reserved;
    cloud_camera prev_cam;
};
}  // namespace

extern "C" int cloud_session_snapshot_bytes(const cloud_session *s, size_t *bytes) {
    clear_error();
    if (!s || !bytes) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_snapshot_bytes: null pointer");
    *bytes = sizeof(SnapHeader) + frame_bytes(s);
    return CLOUD_OK;
}

extern "C" int cloud_session_snapshot(cloud_session *s, void *dst, size_t bytes, void *stream) {
    clear_error();
    if (!s || !dst) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_snapshot: null pointer");
    if (bytes != sizeof(SnapHeader) + frame_bytes(s))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_snapshot: wrong size (see cloud_session_snapshot_bytes)");
    if (int rc = check_waits(s, "cloud_session_snapshot")) return rc;
    SnapHeader h{};
    h.magic = kSnapMagic;
    h.version = kSnapVersion;
    h.width = s->width;
    h.height = s->height;
    h.fmt = s->fmt;
    h.has_history = s->has_history ? 1 : 0;
    h.frame = s->frame;
    h.prev_cam = s->prev_cam;
    std::memcpy(dst, &h, sizeof(h));
    char *pix = static_cast<char *>(dst) + sizeof(h);
    cudaStream_t st = (cudaStream_t)stream;
    if (s->has_history) {
        if (int rc = check_cuda(cudaMemcpyAsync(pix, s->hist[s->latest], frame_bytes(s),
                                                cudaMemcpyDeviceToHost, st),
                                "cloud_session_snapshot: copy history"))
            return rc;
        if (int rc = check_cuda(cudaStreamSynchronize(st), "cloud_session_snapshot")) return rc;
    } else {
        std::memset(pix, 0, frame_bytes(s));
    }
    return CLOUD_OK;
}

extern "C" int cloud_session_restore(cloud_session *s, const void *src, size_t bytes, void *stream) {
    clear_error();
    if (!s || !src) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_restore: null pointer");
    if (bytes != sizeof(SnapHeader) + frame_bytes(s))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_restore: wrong size for this session");
    SnapHeader h;
    std::memcpy(&h, src, sizeof(h));
    if (h.magic != kSnapMagic || h.version != kSnapVersion)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_restore: not a session snapshot");
    if (h.width != s->width || h.height != s->height || h.fmt != s->fmt)
        return set_error(CLOUD_ERR_INVALID_ARG,
                         "cloud_session_restore: snapshot of a session of another size or history format");
    if (h.frame < 0) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_session_restore: bad frame index");
    // read-backs still in flight from the history buffers finish first
    if (int rc = check_cuda(cudaStreamSynchronize(s->copy_stream), "cloud_session_restore")) return rc;
    s->copy_pending[0] = s->copy_pending[1] = false;
    cudaStream_t st = (cudaStream_t)stream;
    if (h.has_history) {
        if (int rc = check_cuda(cudaMemcpyAsync(s->hist[0], static_cast<const char *>(src) + sizeof(h),
                                                frame_bytes(s), cudaMemcpyHostToDevice, st),
                                "cloud_session_restore: copy history"))
            return rc;
        if (int rc = check_cuda(cudaStreamSynchronize(st), "cloud_session_restore")) return rc;
    }
    s->latest = 0;
    s->has_history = h.has_history != 0;
    s->frame = h.frame;
    s->prev_cam = h.prev_cam;
    s->wait_seen = *reinterpret_cast<volatile unsigned int *>(s->h_wait);
    s->wait_failed = false;
    return CLOUD_OK;
}
