// server.cu -- continuous-batching render server: many sessions, each a
// camera's stream of jittered frames resolved by TAA (Sec. 3.2), served from
// one volume.
//
// Requests (session, camera, step count) arrive at any time.  A worker thread
// forms a batch from the queue as soon as an in-flight slot is free: at most
// one request per session (a session's next frame needs the history its
// previous frame produces) and at most max_batch_views requests, in arrival
// order.  The batch's raymarch is one persistent launch over all its views,
// followed by one launch resolving every request (fused motion + TAA), all on
// the slot's stream; a host callback at the end of the stream work stamps the completion
// time.  With two or more slots, a batch formed while another is on the GPU
// overlaps with it.  Sessions keep their history, raw frame and jitter index
// on the device; opening one is admitted only while the free
// device memory stays above the configured reserve.  Every host wait is
// bounded and reports CLOUD_ERR_TIMEOUT; nothing waits on the device without
// a limit.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "march.cuh"

namespace cloudvol {
int launch_batch(const cloud_volume *vol, const SceneParams &scene, const ViewParams *d_views,
                 int n_views, int total_tiles, int config, unsigned int *d_work,
                 unsigned long long *counter, cudaStream_t s);
}  // namespace cloudvol

using namespace cloudvol;

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Session {
    int width = 0, height = 0;
    float *current = nullptr;  // raw jittered render
    void *hist[2] = {nullptr, nullptr};
    int latest = 0;
    bool has_history = false;
    int frame = 0;  // jitter index of the next frame
    cloud_camera prev_cam{};
    bool busy = false;  // a frame of this session is in flight
    bool open = false;
    bool closing = false;  // cloud_server_close_session is waiting for it: no new requests
    size_t bytes = 0;
};

struct Request {
    uint64_t id = 0;
    int session = 0;
    cloud_camera cam{};
    int steps = 0;
    double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
    int status = 0;   // 0 queued, 1 in flight, 2 done, <0 failed
    int batch_size = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    ViewParams *h_table = nullptr;  // pinned
    ViewParams *d_table = nullptr;
    void *h_rtable = nullptr;       // pinned: the resolve's per-view table
    void *d_rtable = nullptr;
    unsigned int *d_work = nullptr;
    // bounded waits of this slot's resolves that gave up: mapped pinned host
    // counter (never reset) and the value last accounted for
    unsigned int *h_wait = nullptr, *d_wait = nullptr;
    unsigned int wait_seen = 0;
    bool busy = false;
    std::vector<uint64_t> reqs;
    std::vector<ResolveRequest> resolves;
};

}  // namespace

struct cloud_server {
    const cloud_volume *vol = nullptr;
    cloud_params prm{};
    SceneParams scene{};
    cloud_server_config cfg{};
    int device = 0;
    int config = 0;  // launch configuration (tile shape, view steps per iteration)
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Session> sessions;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
    uint64_t next_id = 1;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false, paused = false;
    int error = CLOUD_OK;
    std::string error_msg;
    uint64_t completed = 0, batches = 0, batched_views = 0;
};

namespace {

struct Completion {
    cloud_server *srv;
    int slot;
};

void CUDART_CB on_slot_done(void *arg) {
    // runs on a CUDA callback thread: host bookkeeping only, no CUDA calls
    Completion *c = static_cast<Completion *>(arg);
    cloud_server *srv = c->srv;
    const double t = now_ms();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        Slot &sl = srv->slots[c->slot];
        // a resolve tile that gave up its bounded wait was left unwritten: the
        // batch's requests fail with CLOUD_ERR_TIMEOUT and their sessions'
        // next frames start without history
        const unsigned int waits = *reinterpret_cast<volatile unsigned int *>(sl.h_wait);
        const bool gave_up = waits != sl.wait_seen;
        sl.wait_seen = waits;
        for (uint64_t id : sl.reqs) {
            auto it = srv->requests.find(id);
            if (it == srv->requests.end()) continue;
            Request &r = *it->second;
            r.t_done = t;
            r.status = gave_up ? CLOUD_ERR_TIMEOUT : 2;
            srv->sessions[r.session].busy = false;
            if (gave_up) srv->sessions[r.session].has_history = false;
            ++srv->completed;
        }
        sl.reqs.clear();
        sl.busy = false;
    }
    srv->cv.notify_all();
    delete c;
}

// Enqueue one batch on slot `si`.  Called WITHOUT the server mutex: the
// requests are immutable once queued, and the sessions of a batch are marked
// busy, so no other thread touches their state until the slot completes.
int launch_slot(cloud_server *srv, int si, const std::vector<Request *> &batch) {
    Slot &sl = srv->slots[si];
    const int n = (int)batch.size();
    // order the queue by decreasing step count (long tiles first)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return batch[a]->steps > batch[b]->steps; });
    int next = 0;
    for (int q = 0; q < n; ++q) {
        const Request &r = *batch[order[q]];
        const Session &se = srv->sessions[r.session];
        ViewParams &v = sl.h_table[q];
        if (int rc = build_view(srv->vol, &srv->prm, &r.cam, se.width, se.height, r.steps, se.frame,
                                se.current, config_shape(srv->config), &v))
            return rc;
        v.tile_begin = next;
        next += v.tile_count;
    }
    if (int rc = check_cuda(cudaMemcpyAsync(sl.d_table, sl.h_table, sizeof(ViewParams) * n,
                                            cudaMemcpyHostToDevice, sl.stream),
                            "server: upload view table"))
        return rc;
    if (int rc = launch_batch(srv->vol, srv->scene, sl.d_table, n, next, srv->config, sl.d_work,
                              nullptr, sl.stream))
        return rc;
    // every request's reprojection motion and TAA resolve in one launch (the
    // motion is never stored)
    sl.resolves.resize(n);
    for (int i = 0; i < n; ++i) {
        const Request &r = *batch[i];
        const Session &se = srv->sessions[r.session];
        sl.resolves[i] = ResolveRequest{se.has_history ? &se.prev_cam : nullptr, &r.cam,
                                        se.has_history ? se.hist[se.latest] : nullptr, se.current,
                                        se.hist[1 - se.latest], se.width, se.height};
    }
    if (int rc = launch_taa_reproject_batch(srv->vol, &srv->prm, sl.resolves.data(), n,
                                            srv->cfg.history_fmt, srv->cfg.blend, sl.h_rtable,
                                            sl.d_rtable, sl.d_wait, sl.stream))
        return rc;
    for (const Request *rp : batch) {
        // the session stays busy until this slot completes, so its state can advance now
        const Request &r = *rp;
        Session &se = srv->sessions[r.session];
        se.latest = 1 - se.latest;
        se.has_history = true;
        se.prev_cam = r.cam;
        se.frame += 1;
    }
    Completion *c = new (std::nothrow) Completion{srv, si};
    if (!c) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "server: host allocation");
    const int rc = check_cuda(cudaLaunchHostFunc(sl.stream, on_slot_done, c), "cudaLaunchHostFunc");
    if (rc) delete c;
    return rc;
}

void worker_main(cloud_server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        srv->cv.wait_for(lk, std::chrono::milliseconds(50), [&] {
            if (srv->stop) return true;
            if (srv->paused || srv->error || srv->queue.empty()) return false;
            for (size_t i = 0; i < srv->slots.size(); ++i)
                if (!srv->slots[i].busy) return true;
            return false;
        });
        if (srv->stop) break;
        if (srv->paused || srv->error || srv->queue.empty()) continue;
        int si = -1;
        for (size_t i = 0; i < srv->slots.size(); ++i)
            if (!srv->slots[i].busy) {
                si = (int)i;
                break;
            }
        if (si < 0) continue;
        // continuous batching: take queued requests of idle sessions in arrival order
        std::vector<Request *> batch;
        std::vector<uint64_t> ids;
        for (auto it = srv->queue.begin();
             it != srv->queue.end() && (int)batch.size() < srv->cfg.max_batch_views;) {
            Request *r = srv->requests[*it].get();
            Session &se = srv->sessions[r->session];
            if (!se.open) {
                // cannot happen while close_session refuses sessions with queued
                // requests; fail the request rather than render into freed buffers
                r->status = CLOUD_ERR_INVALID_ARG;
                it = srv->queue.erase(it);
                srv->cv.notify_all();
                continue;
            }
            if (!se.busy) {
                se.busy = true;  // also excludes a second request of this session
                batch.push_back(r);
                ids.push_back(*it);
                it = srv->queue.erase(it);
            } else {
                ++it;
            }
        }
        if (batch.empty()) {
            // every queued request belongs to a session with a frame in flight
            srv->cv.wait_for(lk, std::chrono::milliseconds(1));
            continue;
        }
        const double t = now_ms();
        for (Request *r : batch) {
            r->status = 1;
            r->t_start = t;
            r->batch_size = (int)batch.size();
        }
        Slot &sl = srv->slots[si];
        sl.busy = true;
        sl.reqs = ids;
        ++srv->batches;
        srv->batched_views += batch.size();
        lk.unlock();
        const int rc = launch_slot(srv, si, batch);
        const std::string msg = rc ? cloud_last_error_message() : "";
        lk.lock();
        if (rc) {
            srv->error = rc;
            srv->error_msg = msg;
            for (Request *r : batch) r->status = rc;
            srv->cv.notify_all();
        }
    }
}

void free_session_buffers(Session &se) {
    if (se.current) cudaFree(se.current);
    if (se.hist[0]) cudaFree(se.hist[0]);
    if (se.hist[1]) cudaFree(se.hist[1]);
    se = Session{};
}

}  // namespace

extern "C" int cloud_server_create(const cloud_volume *vol, const cloud_params *prm,
                                   int light_steps, const cloud_server_config *cfg,
                                   cloud_server **out) {
    clear_error();
    if (!vol || !prm || !cfg || !out)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_create: null pointer");
    if (cfg->max_batch_views < 1 || cfg->max_batch_views > CLOUD_MAX_VIEWS || cfg->slots < 1 ||
        cfg->slots > 8 || cfg->max_sessions < 1 || cfg->max_sessions > 65536 ||
        (cfg->history_fmt != CLOUD_HISTORY_FP32 && cfg->history_fmt != CLOUD_HISTORY_FP16) ||
        !(cfg->blend >= 0.0f && cfg->blend <= 1.0f))
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_create: bad configuration");
    cloud_server *srv = new (std::nothrow) cloud_server();
    if (!srv) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_server_create: host allocation");
    srv->vol = vol;
    srv->prm = *prm;
    srv->cfg = *cfg;
    int rc = check_cuda(cudaGetDevice(&srv->device), "cudaGetDevice");
    if (!rc) rc = build_scene(vol, prm, light_steps, CLOUD_INTEGRATE_ANALYTIC, &srv->scene);
    srv->config = tuned_config(vol->desc.precision, light_steps);
    srv->sessions.resize(cfg->max_sessions);
    srv->slots.resize(cfg->slots);
    for (auto &sl : srv->slots) {
        if (rc) break;
        rc = check_cuda(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "cudaStreamCreate");
        if (!rc)
            rc = check_cuda(cudaMallocHost(&sl.h_table, sizeof(ViewParams) * cfg->max_batch_views),
                            "cudaMallocHost view table");
        if (!rc)
            rc = check_cuda(cudaMalloc(&sl.d_table, sizeof(ViewParams) * cfg->max_batch_views),
                            "cudaMalloc view table");
        if (!rc) rc = check_cuda(cudaMalloc(&sl.d_work, sizeof(unsigned int)), "cudaMalloc counter");
        if (!rc)
            rc = check_cuda(cudaMallocHost(&sl.h_rtable, resolve_view_bytes() * cfg->max_batch_views),
                            "cudaMallocHost resolve table");
        if (!rc)
            rc = check_cuda(cudaMalloc(&sl.d_rtable, resolve_view_bytes() * cfg->max_batch_views),
                            "cudaMalloc resolve table");
        if (!rc)
            rc = check_cuda(cudaHostAlloc((void **)&sl.h_wait, sizeof(unsigned int), cudaHostAllocMapped),
                            "cudaHostAlloc wait counter");
        if (!rc) {
            *sl.h_wait = 0;
            rc = check_cuda(cudaHostGetDevicePointer((void **)&sl.d_wait, sl.h_wait, 0),
                            "cudaHostGetDevicePointer wait counter");
        }
    }
    if (!rc) {
        try {
            srv->worker = std::thread(worker_main, srv);
        } catch (...) {
            rc = set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_server_create: cannot start worker");
        }
    }
    if (rc) {
        for (auto &sl : srv->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.h_table) cudaFreeHost(sl.h_table);
            if (sl.d_table) cudaFree(sl.d_table);
            if (sl.d_work) cudaFree(sl.d_work);
            if (sl.h_rtable) cudaFreeHost(sl.h_rtable);
            if (sl.d_rtable) cudaFree(sl.d_rtable);
            if (sl.h_wait) cudaFreeHost(sl.h_wait);
        }
        delete srv;
        return rc;
    }
    *out = srv;
    return CLOUD_OK;
}

extern "C" int cloud_server_destroy(cloud_server *srv) {
    clear_error();
    if (!srv) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_destroy: null server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    srv->worker.join();
    for (auto &sl : srv->slots) cudaStreamSynchronize(sl.stream);
    for (auto &sl : srv->slots) {
        cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_table);
        cudaFree(sl.d_table);
        cudaFree(sl.d_work);
        cudaFreeHost(sl.h_rtable);
        cudaFree(sl.d_rtable);
        cudaFreeHost(sl.h_wait);
    }
    for (auto &se : srv->sessions)
        if (se.open) free_session_buffers(se);
    delete srv;
    return CLOUD_OK;
}

extern "C" int cloud_server_open_session(cloud_server *srv, int width, int height, int *session_id) {
    clear_error();
    if (!srv || !session_id || width < 1 || height < 1 || width > CLOUD_MAX_DIM ||
        height > CLOUD_MAX_DIM)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_open_session: bad arguments");
    const size_t px = (size_t)width * height;
    const size_t hb = px * (srv->cfg.history_fmt == CLOUD_HISTORY_FP32 ? 16 : 8);
    const size_t bytes = px * 16 + 2 * hb;  // raw frame + two histories
    std::lock_guard<std::mutex> lk(srv->mu);
    int id = -1;
    for (size_t i = 0; i < srv->sessions.size(); ++i)
        if (!srv->sessions[i].open) {
            id = (int)i;
            break;
        }
    if (id < 0) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_server_open_session: all session slots in use");
    // admission by free device memory
    size_t free_b = 0, total_b = 0;
    if (int rc = check_cuda(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo")) return rc;
    size_t used = 0;
    for (auto &se : srv->sessions) used += se.open ? se.bytes : 0;
    if (free_b < bytes + srv->cfg.reserve_bytes ||
        (srv->cfg.budget_bytes && used + bytes > srv->cfg.budget_bytes))
        return set_error(CLOUD_ERR_OUT_OF_MEMORY,
                         "cloud_server_open_session: not admitted, device memory budget exhausted");
    Session &se = srv->sessions[id];
    se = Session{};
    se.width = width;
    se.height = height;
    se.bytes = bytes;
    int rc = check_cuda(cudaMalloc(&se.current, px * 16), "cudaMalloc current");
    if (!rc) rc = check_cuda(cudaMalloc(&se.hist[0], hb), "cudaMalloc history");
    if (!rc) rc = check_cuda(cudaMalloc(&se.hist[1], hb), "cudaMalloc history");
    if (rc) {
        free_session_buffers(se);
        return rc;
    }
    se.open = true;
    *session_id = id;
    return CLOUD_OK;
}

extern "C" int cloud_server_close_session(cloud_server *srv, int session_id) {
    clear_error();
    if (!srv) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_close_session: null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    if (session_id < 0 || session_id >= (int)srv->sessions.size() || !srv->sessions[session_id].open ||
        srv->sessions[session_id].closing)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_close_session: no such session");
    for (uint64_t id : srv->queue)
        if (srv->requests[id]->session == session_id)
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_close_session: requests still queued");
    // from here on cloud_server_submit refuses this session, so the queue
    // cannot gain a request for it while the wait below releases the lock
    srv->sessions[session_id].closing = true;
    if (!srv->cv.wait_for(lk, std::chrono::seconds(10),
                          [&] { return !srv->sessions[session_id].busy || srv->error; })) {
        srv->sessions[session_id].closing = false;
        return set_error(CLOUD_ERR_TIMEOUT, "cloud_server_close_session: frame still in flight");
    }
    if (srv->sessions[session_id].busy) {
        // the server failed with a frame of this session still enqueued: let
        // the slot streams drain before the buffers they use are freed
        lk.unlock();
        for (auto &sl : srv->slots) cudaStreamSynchronize(sl.stream);
        lk.lock();
    }
    free_session_buffers(srv->sessions[session_id]);
    return CLOUD_OK;
}

extern "C" int cloud_server_submit(cloud_server *srv, int session_id, const cloud_camera *cam,
                                   int steps, uint64_t *ticket) {
    clear_error();
    if (!srv || !cam || !ticket || steps < 1 || steps > CLOUD_MAX_STEPS)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_submit: bad arguments");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return set_error(CLOUD_ERR_OUT_OF_MEMORY, "cloud_server_submit: host allocation");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->error) return set_error(srv->error, "cloud_server_submit: server failed: " + srv->error_msg);
        if (session_id < 0 || session_id >= (int)srv->sessions.size() || !srv->sessions[session_id].open ||
            srv->sessions[session_id].closing)
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_submit: no such session");
        r->id = srv->next_id++;
        r->session = session_id;
        r->cam = *cam;
        r->steps = steps;
        r->t_submit = now_ms();
        *ticket = r->id;
        srv->queue.push_back(r->id);
        srv->requests.emplace(r->id, std::move(r));
    }
    srv->cv.notify_all();
    return CLOUD_OK;
}

extern "C" int cloud_server_wait(cloud_server *srv, uint64_t ticket, int timeout_ms,
                                 cloud_request_info *info) {
    clear_error();
    if (!srv) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_wait: null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->requests.find(ticket);
    if (it == srv->requests.end()) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_wait: unknown ticket");
    Request *r = it->second.get();
    const bool ok = srv->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                     [&] { return r->status == 2 || r->status < 0; });
    if (!ok) return set_error(CLOUD_ERR_TIMEOUT, "cloud_server_wait: request not finished in time");
    if (r->status < 0) {
        const int st = r->status;
        srv->requests.erase(it);
        if (st == CLOUD_ERR_TIMEOUT)
            return set_error(st, "cloud_server_wait: a bounded wait of this frame's TAA resolve gave "
                                 "up; the frame misses a tile and the session's history was reset");
        return set_error(st, "cloud_server_wait: " + srv->error_msg);
    }
    if (info) {
        info->session = r->session;
        info->steps = r->steps;
        info->batch_size = r->batch_size;
        info->queue_ms = r->t_start - r->t_submit;
        info->latency_ms = r->t_done - r->t_submit;
    }
    srv->requests.erase(it);
    return CLOUD_OK;
}

extern "C" int cloud_server_session_output(cloud_server *srv, int session_id, const void **dev_out) {
    clear_error();
    if (!srv || !dev_out) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_session_output: bad arguments");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (session_id < 0 || session_id >= (int)srv->sessions.size() || !srv->sessions[session_id].open)
        return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_session_output: no such session");
    const Session &se = srv->sessions[session_id];
    if (se.busy) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_session_output: frame in flight");
    *dev_out = se.has_history ? se.hist[se.latest] : nullptr;
    return CLOUD_OK;
}

extern "C" int cloud_server_pause(cloud_server *srv, int paused) {
    clear_error();
    if (!srv) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_pause: null server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->paused = paused != 0;
    }
    srv->cv.notify_all();
    return CLOUD_OK;
}

extern "C" int cloud_server_stats(cloud_server *srv, cloud_server_counters *st) {
    clear_error();
    if (!srv || !st) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_stats: bad arguments");
    std::lock_guard<std::mutex> lk(srv->mu);
    st->completed = srv->completed;
    st->batches = srv->batches;
    st->batched_views = srv->batched_views;
    st->queued = srv->queue.size();
    int open = 0;
    size_t bytes = 0;
    for (auto &se : srv->sessions)
        if (se.open) {
            ++open;
            bytes += se.bytes;
        }
    st->open_sessions = open;
    st->session_bytes = bytes;
    return srv->error;
}

extern "C" int cloud_server_copy_output(cloud_server *srv, int session_id, void *dst, size_t bytes) {
    clear_error();
    if (!srv || !dst) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_copy_output: bad arguments");
    const void *src = nullptr;
    size_t need = 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (session_id < 0 || session_id >= (int)srv->sessions.size() || !srv->sessions[session_id].open)
            return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_copy_output: no such session");
        const Session &se = srv->sessions[session_id];
        if (se.busy) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_copy_output: frame in flight");
        if (!se.has_history) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_copy_output: no frame yet");
        src = se.hist[se.latest];
        need = (size_t)se.width * se.height * (srv->cfg.history_fmt == CLOUD_HISTORY_FP32 ? 16 : 8);
    }
    if (bytes != need) return set_error(CLOUD_ERR_INVALID_ARG, "cloud_server_copy_output: wrong size");
    return check_cuda(cudaMemcpy(dst, src, need, cudaMemcpyDefault), "cloud_server_copy_output");
}
