/*
 * cloudvol.h -- C ABI of libcloudvol.so, a GB300 (sm_103a) implementation of
 * the volumetric-cloud raymarch and temporal anti-aliasing resolve of Toft,
 * Bowles and Zimmermann, "Optimisations for Real-Time Volumetric
 * Cloudscapes" (arXiv 1609.05344).
 *
 * Conventions shared by every call:
 *  - Every call returns an int status: CLOUD_OK (0) or a negative CLOUD_ERR_*
 *    code.  No call aborts, traps or exits; cloud_last_error_message() gives
 *    a one-line description of the last failure on the calling thread.
 *  - "device" pointers are CUDA global-memory addresses on the current
 *    device; "host" pointers are ordinary CPU memory.  Buffers passed in are
 *    owned by the caller unless a call says otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that take a stream only enqueue work on it and return
 *    without waiting, unless stated otherwise.
 *  - Images are row-major, row y = 0 at the top, pixel (x, y) at index
 *    y * width + x.  RGBA images are 4 floats per pixel, premultiplied by
 *    alpha.  Motion fields are 2 floats per pixel, in pixels.
 *  - Cameras are pinholes in a right-handed world with z up, metres.
 */
#ifndef CLOUDVOL_H
#define CLOUDVOL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CLOUD_OK 0
#define CLOUD_ERR_INVALID_ARG (-1)   /* a size, pointer, alignment or enum is invalid */
#define CLOUD_ERR_OUT_OF_MEMORY (-2) /* a device or host allocation failed           */
#define CLOUD_ERR_CUDA (-3)          /* the CUDA runtime reported an error           */
#define CLOUD_ERR_TIMEOUT (-4)       /* a bounded device wait gave up                */
#define CLOUD_ERR_UNSUPPORTED (-5)   /* valid request this build does not provide    */

/* ---- enumerations ------------------------------------------------------ */
/* Storage of the noise tiles.  Tiles are kept as corner-packed records (the 8
 * texels of a trilinear footprint, 4 of a bilinear one); the 16-bit formats
 * halve the record bytes of FP32. */
#define CLOUD_PRECISION_FP32 0    /* texels as float                                */
#define CLOUD_PRECISION_FP16 1    /* corner 0 as 16-bit fixed point, the other
                                     corners as IEEE half differences from it      */
#define CLOUD_PRECISION_BF16 2    /* corner 0 as 16-bit fixed point, the other
                                     corners as bfloat16 differences from it       */
#define CLOUD_PRECISION_UNORM16 3 /* texels as 16-bit fixed point v * 65536         */

#define CLOUD_DENSITY_NOISE 0    /* fBm base - detail, coverage remap, weather    */
#define CLOUD_DENSITY_CONSTANT 1 /* constant density everywhere (closed forms)   */

#define CLOUD_INTEGRATE_ANALYTIC 0 /* Sec. 3.1 analytic step integral            */
#define CLOUD_INTEGRATE_BASIC 1    /* Sec. 3.1 basic S = T L                     */

#define CLOUD_JITTER_PER_PIXEL 0 /* Sec. 3.2: random offset per pixel and frame   */
#define CLOUD_JITTER_PER_FRAME 1 /* Sec. 4: one offset per frame for every ray    */

#define CLOUD_HISTORY_FP32 0 /* TAA history: 4 x float per pixel (16 B)          */
#define CLOUD_HISTORY_FP16 1 /* TAA history: 4 x IEEE half per pixel (8 B)       */

#define CLOUD_MAX_LIGHT_STEPS 32
#define CLOUD_MAX_STEPS 4096
#define CLOUD_MAX_DIM 16384
#define CLOUD_MAX_VIEWS 4096
#define CLOUD_STATIC_MAX_VIEWS 256

/* ---- descriptors ------------------------------------------------------- */

/* Cloud density volume.  The paper samples "the density" of a cloud volume
 * at every step (Sec. 1) without defining it; the field is value-noise fBm:
 *   rho(p) = g(z) * W(x, y) * max(0, (B(p) - detail_weight * Dt(p) - coverage)
 *                                      / (1 - coverage))
 * B: base_n^3 fBm tile spanning base_period_m; Dt: detail_n^3 tile (0 = none,
 * then Dt = 0); W: weather_n^2 map (0 = none, then W = 1); g: piecewise-linear
 * height profile over [slab_lo_m, slab_hi_m] (0 outside).  Lattice edges are
 * powers of two in [16, 1024] (weather up to 4096).  Noise lattice values come
 * from the counter-based hash keyed by `seed`. */
typedef struct {
    uint32_t seed;
    int32_t base_n;
    int32_t detail_n;
    int32_t weather_n;
    double detail_weight;
    double base_period_m;
    double detail_period_m;
    double weather_period_m;
    double coverage;         /* in [0, 1)                                      */
    double slab_lo_m;
    double slab_hi_m;        /* > slab_lo_m                                    */
    int32_t density_mode;    /* CLOUD_DENSITY_*                                */
    double constant_density; /* rho for CLOUD_DENSITY_CONSTANT                 */
    int32_t precision;       /* CLOUD_PRECISION_*                              */
} cloud_volume_desc;

/* Pinhole camera: forward/right/up orthonormal; vertical field of view
 * 2 atan(tan_half_fovy); the horizontal one follows from width/height. */
typedef struct {
    double pos[3];
    double forward[3];
    double right[3];
    double up[3];
    double tan_half_fovy;
} cloud_camera;

/* Lighting and march constants (Sec. 1): sun direction (towards the sun,
 * any length, z > 0), sun colour x intensity, ambient radiance, the
 * Henyey-Greenstein asymmetry g in (-1, 1), absorption alpha per metre at
 * density 1, light-march step length, early-out optical depth (<= 0 turns the
 * early out off), far clip of a view ray, and the jitter mode
 * (CLOUD_JITTER_PER_PIXEL; CLOUD_JITTER_PER_FRAME shares one offset, that of
 * pixel (0, 0), between all rays of a frame). */
typedef struct {
    double sun_dir[3];
    double sun_radiance[3];
    double ambient[3];
    double hg_g;
    double absorption_per_m;
    double light_step_m;
    double tau_max;
    double t_max_m;
    int32_t jitter_mode;
} cloud_params;

/* One view of a multi-view launch: camera, image size, view steps, jitter
 * frame (< 0: no jitter) and its output (device, width*height*4 floats,
 * 16-byte aligned, caller-owned). */
typedef struct {
    cloud_camera camera;
    int32_t width;
    int32_t height;
    int32_t steps;
    int32_t jitter_frame;
    float *out_rgba;
} cloud_view;

typedef struct cloud_volume cloud_volume;   /* opaque, immutable once created */
typedef struct cloud_session cloud_session; /* opaque, one TAA stream of frames */
typedef struct cloud_batch cloud_batch;     /* opaque, a set of views rendered together */
typedef struct cloud_server cloud_server;   /* opaque, continuous-batching render server */

/* Render server configuration. */
typedef struct {
    int32_t max_batch_views; /* requests per batch, 1..CLOUD_MAX_VIEWS (1 = a launch per frame) */
    int32_t slots;           /* batches in flight at once (one stream each), 1..8 */
    int32_t max_sessions;    /* session table size, 1..65536 */
    int32_t history_fmt;     /* CLOUD_HISTORY_* */
    float blend;             /* TAA blend, [0, 1] */
    uint64_t reserve_bytes;  /* device memory left free when admitting a session */
    uint64_t budget_bytes;   /* 0: none; else the most all sessions may hold */
} cloud_server_config;

/* Per-request timing returned by cloud_server_wait. */
typedef struct {
    int32_t session;
    int32_t steps;
    int32_t batch_size; /* requests in the batch that carried it */
    double queue_ms;    /* submit -> batch launch */
    double latency_ms;  /* submit -> device work complete */
} cloud_request_info;

typedef struct {
    uint64_t completed;
    uint64_t batches;
    uint64_t batched_views;
    uint64_t queued;
    int32_t open_sessions;
    uint64_t session_bytes;
} cloud_server_counters;

/* ---- status ------------------------------------------------------------ */

/* Name of a status code (library plumbing; no counterpart in the paper). */
const char *cloud_status_string(int status);
/* Last failure on the calling thread ("" if none). */
const char *cloud_last_error_message(void);

/* ---- volumes ----------------------------------------------------------- */

/* Creates the density volume described by *desc on the current device and
 * generates its noise tiles on `stream` (the density field Sec. 1
 * samples; parameters as in cloud_volume_desc).  The library allocates and owns the device
 * memory; the handle may be shared read-only by any number of streams once
 * `stream` has passed the generation work.  *out is set only on success. */
int cloud_volume_create(const cloud_volume_desc *desc, void *stream, cloud_volume **out);

/* Frees a volume.  The caller guarantees that no enqueued work still uses it.
 * (Volume lifetime; the tiles are those of cloud_volume_create, Sec. 1.)
 */
int cloud_volume_destroy(cloud_volume *vol);

/* Copies the noise tiles into caller-owned device buffers as float values
 * in [0, 1) (decoding reduced-precision storage): base base_n^3, detail
 * detail_n^3, weather weather_n^2, x fastest.  Any pointer may be NULL to
 * skip that tile.  For tests and tools.
 * (The density tiles of Sec. 1, decoded for checks.)
 */
int cloud_volume_export(const cloud_volume *vol, float *base, float *detail, float *weather,
                        void *stream);

/* Copies the volume's occupancy grid into `out` (device, `words` uint32,
 * caller-owned): one bit per cell of half a base-tile texel on each axis
 * (8 per trilinear record), 2^(3 * *log2_cells) cells with x fastest, bit i
 * of word i / 32 for cell i.
 * A clear bit means the density is provably zero for every sample in the cell
 * (max B - detail_weight min Dt - coverage < 0, with the exact extremes of the
 * interpolated tiles over the cell); the raymarch then skips that lookup's memory reads,
 * which changes no result.  With out == NULL only *log2_cells is set (-1 for
 * a constant-density volume, which has no grid).  words must be
 * ceil(2^(3 * *log2_cells) / 32).  For tests and tools.
 * (Empty-space skipping for the density samples of Sec. 1.) */
int cloud_volume_occupancy(const cloud_volume *vol, uint32_t *out, int64_t words, int *log2_cells,
                           void *stream);

/* ---- render (Sec. 1, Sec. 3.1, Sec. 3.2) -------------------------------- */

/* Raymarches every pixel of a width x height image into out_rgba (device,
 * width*height*4 floats, 16-byte aligned, caller-owned):
 *   steps view samples per ray over the ray's span [t0, t1] inside the
 *   cloud layer (D = (t1 - t0)/steps, sample i at t0 + (i + u) D);
 *   u = 1/2, or for jitter_frame >= 0 a per-pixel per-frame value from the
 *   hash of (x, y, jitter_frame, seed) (Sec. 3.2);
 *   light_steps samples towards the sun per view sample with density > 0,
 *   giving L_in = E_sun e^{-tau_sun} p_HG(d.s) + ambient (Sec. 1);
 *   integration CLOUD_INTEGRATE_ANALYTIC adds e^{-tau} L_in (1 - e^{-sigma D})
 *   per step, CLOUD_INTEGRATE_BASIC the step-dependent S = T L form
 *   (Sec. 3.1), sigma = absorption * rho, tau the optical-depth sum;
 *   the ray stops after the step at which tau >= tau_max (Sec. 1);
 *   out = (C.rgb, 1 - e^{-tau}).  Rays that miss the layer write 0.
 * Limits: 1 <= steps <= CLOUD_MAX_STEPS, 0 <= light_steps <=
 * CLOUD_MAX_LIGHT_STEPS, 1 <= width, height <= CLOUD_MAX_DIM. */
int cloud_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                 int width, int height, int steps, int light_steps, int jitter_frame,
                 int integration, float *out_rgba, void *stream);

/* As cloud_render, and also adds the number of density evaluations the
 * launch performed to *lookups (device, one uint64, caller-owned; the caller
 * zeroes it).  Measures the effective work of a frame.
 * (The lookups are the density samples of Sec. 1: one per view step
 * plus one per light step of each step with density.)
 */
int cloud_render_count(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                       int width, int height, int steps, int light_steps, int jitter_frame,
                       int integration, float *out_rgba, unsigned long long *lookups,
                       void *stream);

/* Launch configurations of the raymarch that the autotuners choose from:
 * config = shape + 4 * k, with shape the pixel tile of a 128-thread CTA (0:
 * 16x8, 1: 32x4 of 8x4-pixel warps, 2: 32x4 of 16x2-pixel warps, 3: 8x16) and
 * k selecting the view steps a warp evaluates per iteration of its march
 * (0: 8, 1: 16).  Every configuration gives bitwise the same pixels.  Until a
 * configuration is tuned or set, launches use 3 (8x16, 8 steps). */
#define CLOUD_TUNE_CONFIGS 8

/* Times every launch configuration of the raymarch on this workload (repeats
 * launches each, writing out_rgba), remembers the fastest for the volume's
 * storage precision and light-step count (later cloud_render, new batches and
 * new servers use it), and returns it in *best (and the per-configuration mean
 * times in times_ms[CLOUD_TUNE_CONFIGS] if not NULL).  Waits for the stream. */
int cloud_autotune_render(const cloud_volume *vol, const cloud_camera *cam, const cloud_params *prm,
                          int width, int height, int steps, int light_steps, int jitter_frame,
                          int integration, float *out_rgba, int repeats, float *times_ms,
                          int *best, void *stream);

/* Reads / sets the launch configuration that cloud_render, new batches and
 * new servers use for volumes of `precision` rendered with `light_steps`
 * light steps (e.g. to restore a configuration an earlier autotune found).
 * config outside [0, CLOUD_TUNE_CONFIGS) or a bad precision is
 * CLOUD_ERR_INVALID_ARG.  Process-wide; host only.
 * Scheduling only; no counterpart in the paper (the pixel results do not
 * depend on it).
 */
int cloud_get_launch_config(int precision, int light_steps, int *config);
int cloud_set_launch_config(int precision, int light_steps, int config);

/* ---- multi-view batches (each view as cloud_render) --------------------- */

/* A batch renders n_views (1..CLOUD_MAX_VIEWS) views of one volume with the
 * same lighting, light steps and integration rule in ONE persistent launch:
 * the views' pixel tiles form a work queue (longest step counts first) that
 * resident CTAs drain through a device counter.  The library allocates and
 * owns the view table and the counter.  Each view's output equals a
 * cloud_render of that view.
 * (Each view is the raymarch of Sec. 1 / Sec. 3.1 / Sec. 3.2 exactly as
 * cloud_render; batching itself has no counterpart in the paper.)
 */
int cloud_batch_create(const cloud_volume *vol, const cloud_params *prm, int light_steps,
                       int integration, const cloud_view *views, int n_views, cloud_batch **out);
int cloud_batch_destroy(cloud_batch *b);
/* New cameras, jitter frames or outputs (sizes and step counts unchanged);
 * the device view table is rewritten on `stream`. */
int cloud_batch_set_views(cloud_batch *b, const cloud_view *views, int n_views, void *stream);
/* Counter reset + persistent kernel on `stream`. */
int cloud_batch_render(cloud_batch *b, void *stream);
/* The same two operations captured once into a CUDA graph, replayed on
 * `stream` (the graph reads the current view table from device memory). */
int cloud_batch_render_graph(cloud_batch *b, void *stream);
/* One cloud_render launch per view (the unbatched comparison). */
int cloud_batch_render_per_view(cloud_batch *b, void *stream);
/* Times each launch configuration (CLOUD_TUNE_CONFIGS of them; times_ms
 * holds that many if not NULL) for this batch and keeps the fastest (waits). */
int cloud_batch_autotune(cloud_batch *b, int repeats, float *times_ms, int *best, void *stream);

/* Renders n_views views exactly as cloud_batch_create + cloud_batch_render
 * would, but allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library call.  The paper has no counterpart to this entry point; it is for
 * callers that cannot allocate device memory at render time, such as a
 * real-time render thread or an engine with a fixed device-memory budget,
 * where cudaMalloc/cudaFree may block, synchronize the device or fail.
 * The caller still owns every view's out_rgba.  The scratch (work counter and
 * view table) is one library-wide static device array sized for
 * CLOUD_STATIC_MAX_VIEWS (256) views, 47360 bytes, which every GPU that loads
 * the library holds until the process exits; n_views above 256 returns
 * CLOUD_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address (a runtime query), so make it before any stream capture.
 * Every call reuses the same array and resets the counter itself; calls whose
 * work overlaps on the GPU (e.g. on two streams) race on it, so issue them on
 * one stream or otherwise order them. */
int cloud_batch_render_static(const cloud_volume *vol, const cloud_params *prm, int light_steps,
                              int integration, const cloud_view *views, int n_views, void *stream);

/* ---- motion and TAA (Sec. 3.2) ----------------------------------------- */

/* Screen-space motion (device, width*height*2 floats, 8-byte aligned) of
 * each pixel of camera `cur` relative to camera `prev`: the pixel's ray
 * entry point into the cloud layer (or the point at t_max for rays that do
 * not enter it ahead of the camera) is projected into `prev`;
 * motion = pixel centre - that projection.  Points behind `prev` get 1e9.
 * (The per-pixel reprojection the TAA of Sec. 3.2 needs.)
 */
int cloud_motion(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                 const cloud_camera *cur, int width, int height, float *motion, void *stream);

/* Temporal anti-aliasing resolve (Sec. 3.2, Playdead-style):
 *   q = pixel centre - motion; if history == NULL or q is outside
 *   [0, width] x [0, height]: out = current; otherwise
 *   h = bilinear sample of history at q (clamp to edge),
 *   hc = clamp(h, min, max of the 3x3 neighbourhood of current),
 *   out = hc + blend (current - hc).
 * history / history_out: device, width*height*4 values of history_fmt,
 * 16-byte (FP32) or 8-byte (FP16) aligned; they must not overlap.
 * current: device RGBA float (16-byte aligned); motion: device float2. */
int taa_resolve(const void *history, const float *current, const float *motion,
                void *history_out, int width, int height, int history_fmt, float blend,
                void *stream);

/* cloud_motion followed by taa_resolve, fused into one kernel: the motion of
 * each pixel (camera `prev` -> `cur`, exactly as cloud_motion computes it) is
 * used in registers and never stored.  history == NULL is a first frame (prev
 * may then be NULL).  Buffers as in taa_resolve; `current` is read through a
 * TMA tensor map built for this call (width*height contiguous float4), so it
 * must stay valid until the launch completes.  Results are bitwise those of
 * cloud_motion + taa_resolve.
 * (Sec. 3.2: reprojection and the TAA resolve.)
 */
int cloud_taa_reproject(const cloud_volume *vol, const cloud_params *prm, const cloud_camera *prev,
                        const cloud_camera *cur, const void *history, const float *current,
                        void *history_out, int width, int height, int history_fmt, float blend,
                        void *stream);

/* Composite (Sec. 3.2: the resolved cloud buffer is composited into the
 * scene): the cloud buffer (cloud_width x cloud_height RGBA of cloud_fmt,
 * CLOUD_HISTORY_*, premultiplied; e.g. a half- or quarter-resolution session
 * output) is resampled bilinearly to width x height (texel centres, clamp to
 * edge) and laid over `background` (device RGBA float, width x height):
 * out = C + (1 - C.alpha) background.  out may equal background. */
int cloud_composite(const void *cloud, int cloud_fmt, int cloud_width, int cloud_height,
                    const float *background, float *out, int width, int height, void *stream);

/* Number of bounded device-side waits that gave up since the last reset,
 * over every launch of the library in this process.  The fused resolve
 * brings its current-frame tile into shared memory with one bulk copy and
 * waits for it a bounded number of polls; if the copy has not landed by then
 * the tile's outputs are left unwritten (no wait is unbounded) and the
 * give-up is counted here and, for session and server frames, reported by
 * those calls as CLOUD_ERR_TIMEOUT.  Zero in normal operation.  Synchronous;
 * reset != 0 clears the counter.
 * Failure reporting; no counterpart in the paper.
 */
int cloud_device_wait_timeouts(unsigned int *count, int reset);

/* ---- sessions: one camera's stream of TAA frames ------------------------- */

/* A session owns the device buffers of one view (current frame, two history
 * buffers of history_fmt) and its frame index, which is the jitter frame of
 * Sec. 3.2.  The library allocates and owns the memory. */
int cloud_session_create(const cloud_volume *vol, int width, int height, int history_fmt,
                         cloud_session **out);
int cloud_session_destroy(cloud_session *s);

/* Failure reporting shared by the session calls below: if a bounded wait in
 * one of this session's resolves gave up (cloud_device_wait_timeouts), a tile
 * of the resolved frame and so of the history was not written.  The first
 * session call that observes it (cloud_session_frame with host_out, after it
 * waits; any later frame call; cloud_session_wait_frame) returns
 * CLOUD_ERR_TIMEOUT, and every frame call does so without rendering until
 * cloud_session_reset. */

/* One frame of Sec. 3.2: render with jitter_frame = the session's frame
 * index, then the fused reprojection (motion from the previous frame's
 * camera) and TAA resolve into the other history buffer
 * (cloud_taa_reproject), advance the index.  If host_out is not NULL the resolved frame
 * (width*height*4 values of the history format) is copied to it and the
 * call waits for the stream; otherwise it returns after enqueueing.
 * *dev_out (if not NULL) receives the device address of the resolved frame,
 * valid until the next call on this session. */
int cloud_session_frame(cloud_session *s, const cloud_camera *cam, const cloud_params *prm,
                        int steps, int light_steps, int integration, float blend,
                        void *host_out, const void **dev_out, void *stream);

/* As cloud_session_frame, but the copy of the resolved frame into host_out
 * (pinned host memory recommended) runs on the session's own copy stream and
 * the call returns at once, so the read-back of frame k overlaps the render of
 * frame k+1; a later frame's resolve waits for the copy out of the history
 * buffer it overwrites.  *frame_index receives this frame's index; host_out is
 * complete after cloud_session_wait_frame(s, index). */
int cloud_session_frame_async(cloud_session *s, const cloud_camera *cam, const cloud_params *prm,
                              int steps, int light_steps, int integration, float blend,
                              void *host_out, int *frame_index, void *stream);
/* Waits at most timeout_ms (CLOUD_ERR_TIMEOUT) for the read-back of a frame
 * issued by cloud_session_frame_async. */
int cloud_session_wait_frame(cloud_session *s, int frame_index, int timeout_ms);

/* Forgets the history: the next frame is a first frame (index kept); also
 * clears a CLOUD_ERR_TIMEOUT state. */
int cloud_session_reset(cloud_session *s);

/* Checkpoint of a session: the state its next frame depends on -- the latest
 * resolved frame (the history Sec. 3.2 reprojects), whether there is one, the
 * frame index (the next jitter frame) and the previous camera -- copied to or
 * from caller-owned host memory of cloud_session_snapshot_bytes bytes (a
 * header, then width*height*4 history values).  cloud_session_snapshot
 * enqueues the copy on `stream` (after the session's frames issued on that
 * stream) and waits for it; it refuses a session in the CLOUD_ERR_TIMEOUT
 * state.  cloud_session_restore loads a snapshot into a session of the same
 * size and history format (a fresh one, or one on another device), waiting
 * for the copy and for the session's own read-backs; its next frame then
 * continues exactly as the snapshotted session's would (bitwise the same
 * pixels).  A buffer that is not a snapshot of this size and format is
 * CLOUD_ERR_INVALID_ARG.  Checkpointing has no counterpart in the paper. */
int cloud_session_snapshot_bytes(const cloud_session *s, size_t *bytes);
int cloud_session_snapshot(cloud_session *s, void *dst, size_t bytes, void *stream);
int cloud_session_restore(cloud_session *s, const void *src, size_t bytes, void *stream);

/* ---- continuous-batching render server ----------------------------------- */

/* A server renders TAA frames (as cloud_session_frame, Sec. 3.2) for many
 * sessions of one volume.  A worker thread forms batches from the request
 * queue whenever an in-flight slot is free: in arrival order, at most one
 * request per session (its next frame needs the history of the previous one)
 * and at most max_batch_views requests; a batch is one persistent raymarch
 * over its views plus each request's motion and TAA resolve on the slot's
 * stream, so with slots > 1 batches overlap on the device.  Requests that
 * arrive while batches run join the next batch.  Each session's result is
 * the same whether it is rendered alone or among others.  The library
 * allocates and owns all buffers. */
int cloud_server_create(const cloud_volume *vol, const cloud_params *prm, int light_steps,
                        const cloud_server_config *cfg, cloud_server **out);
/* Stops the worker, waits for in-flight batches, frees everything. */
int cloud_server_destroy(cloud_server *srv);
/* Admits a session of width x height if the free device memory minus its
 * buffers stays above reserve_bytes and the budget allows it
 * (CLOUD_ERR_OUT_OF_MEMORY otherwise).  Its history, raw frame, motion and
 * jitter index live on the device. */
int cloud_server_open_session(cloud_server *srv, int width, int height, int *session_id);
/* Frees a session with no queued request; waits (at most 10 s) for an
 * in-flight frame.  From the start of the call cloud_server_submit refuses
 * the session. */
int cloud_server_close_session(cloud_server *srv, int session_id);
/* Queues the next frame of a session (camera, view steps); returns at once. */
int cloud_server_submit(cloud_server *srv, int session_id, const cloud_camera *cam, int steps,
                        uint64_t *ticket);
/* Waits at most timeout_ms for a request (CLOUD_ERR_TIMEOUT otherwise), then
 * returns its timing and forgets the ticket.  A request whose batch had a
 * resolve wait give up (cloud_device_wait_timeouts) also ends with
 * CLOUD_ERR_TIMEOUT (ticket forgotten); its session's next frame is then a
 * first frame. */
int cloud_server_wait(cloud_server *srv, uint64_t ticket, int timeout_ms, cloud_request_info *info);
/* Device address of a session's latest resolved frame (history format),
 * NULL before its first frame; invalid while a frame of it is in flight. */
int cloud_server_session_output(cloud_server *srv, int session_id, const void **dev_out);
/* Copies a session's latest resolved frame (width*height*4 values of the
 * history format, `bytes` must match) to dst (host or device); waits. */
int cloud_server_copy_output(cloud_server *srv, int session_id, void *dst, size_t bytes);
/* Holds (paused != 0) or releases batch formation; queued requests wait. */
int cloud_server_pause(cloud_server *srv, int paused);
/* Counters; returns the server's sticky error status (CLOUD_OK if none). */
int cloud_server_stats(cloud_server *srv, cloud_server_counters *st);

/* ---- test hooks -------------------------------------------------------- */

/* out[i] = hash(keys[4i], keys[4i+1], keys[4i+2], keys[4i+3]) on the device
 * (the counter-based hash of the jitter and the noise lattice).  keys and
 * out are device buffers of 4n and n uint32.
 * (The counter-based hash behind the Sec. 3.2 offsets and the noise lattice.)
 */
int cloud_hash4_batch(const uint32_t *keys, int64_t n, uint32_t *out, void *stream);

/* Sets how many times the fused resolve polls for its tile copy before it
 * gives up (the first of its two bounded waits; < 0 restores the default of
 * 65536, at most 2^30), for launches issued after the call.  For tests of
 * the failure reporting: with 0 every tile gives up at once, the copy still
 * lands within the second bounded wait, and the tiles' outputs stay
 * unwritten.  Process-wide.
 * Failure reporting; no counterpart in the paper. */
int cloud_debug_set_wait_polls(int first_polls);

/* Turns the raymarch's use of the occupancy grid (cloud_volume_occupancy) off
 * (enabled == 0) or back on, for launches issued after the call, so that tests
 * can compare against the full evaluation of every lookup; the pixels are the
 * same either way.  Process-wide; on by default.
 * Scheduling only; no counterpart in the paper. */
int cloud_debug_set_occupancy(int enabled);

/* Checked builds only (the library compiled with CLOUDVOL_CHECKED=1, a test
 * build in place of a memory checker): the kernels verify that their index
 * arithmetic stays in range (tile records 1, occupancy words 2, work lists 4,
 * output pixels 8, history and source texels 16, shared-memory tiles 32,
 * views and tiles of multi-view launches 64), skip an access that fails and
 * OR its bit into a device status word.  *bits receives that word (reset != 0
 * clears it); synchronous.  A normal build sets *bits = 0 and returns
 * CLOUD_ERR_UNSUPPORTED.  No counterpart in the paper. */
int cloud_debug_check_status(unsigned int *bits, int reset);

#ifdef __cplusplus
}
#endif
#endif /* CLOUDVOL_H */
