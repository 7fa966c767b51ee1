// Serving loop: scan-integration requests from many map sessions, with
// continuous batching on the GPU.
//
// Every session owns a map that stays resident in device memory; sessions are
// admitted against a device-memory budget. Requests (a host point cloud, a
// pose and optionally a new window origin) are copied into pinned slabs at
// submission, or, when the points already lie in device-mapped pinned memory,
// read in place by the batch; requests are queued per session. A worker thread forms batches from the
// requests that have arrived: at most one request per session per batch and
// at most one batch per session in flight, so each map sees its scans in
// submission order. Each batch goes to a free stream slot: host-to-device
// copies of the points, the shifts, one batched integration launch
// (tsdf_batch_integrate, a persistent cooperative kernel over all maps of the
// batch, whose last phase also writes each map's counters into mapped host
// memory; a batch of one or two requests runs as plain per-map integrations,
// which publish their counters the same way), then an event; a map without
// that mapped copy gets a device-to-host copy of its counters.
// While one slot's batch runs, requests that arrive are formed into the next
// batch on the other slot, so copies and kernels of consecutive batches
// overlap on the device. Because each map's integration is bit-identical in
// any batch composition, a session's result is the same alone and in the mix.
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <sys/prctl.h>

#include "tsdf_internal.cuh"
#include "../../include/tsdf.h"

using namespace tsdf;

namespace {

double now_us() {
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

struct Request {
    uint64_t ticket = 0;
    int32_t session = 0;
    int64_t n = 0;
    float pose[12];
    bool shift = false;
    int64_t origin[3] = {0, 0, 0};
    float4* host = nullptr;   // pinned slab
    int slab = -1;
    const float4* mapped = nullptr;   // the caller's pinned buffer, read in place (no slab copy)
    tsdf_request_result res{};
    bool done = false;
};

struct Session {
    tsdf_map* map = nullptr;
    size_t bytes = 0;
    std::deque<Request*> queue;
    bool in_flight = false;
    int outstanding = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    tsdf_batch* batch = nullptr;
    float4* dev_pts = nullptr;          // max_batch x max_points
    long long* counters = nullptr;      // pinned, max_batch x 3 (maps without mapped counters)
    cudaEvent_t done = nullptr;
    std::vector<Request*> reqs;
    std::vector<const volatile long long*> src;   // per request: where its counters are read
    bool busy = false;
    bool launching = false;             // being filled by the worker outside the lock
};

// Device-tier slots of a session's global store (rounded up to the 8 MiB
// segments the store allocates).
size_t session_store_chunks(const tsdf_params& p, int32_t store_chunks) {
    const size_t bricks = (size_t)p.dims[0] * p.dims[1] * p.dims[2] / 512;
    size_t c = store_chunks > 0 ? (size_t)store_chunks : bricks / 8;
    if (c < 1) c = 1;
    return (c + 4095) / 4096 * 4096;
}

size_t session_bytes(const tsdf_params& p, int64_t max_points, int32_t store_chunks) {
    const size_t voxels = (size_t)p.dims[0] * p.dims[1] * p.dims[2];
    const size_t bricks = voxels / 512;
    return voxels * (4 + 8) + bricks * (1 + 4) + (size_t)max_points * 32 + 8192 +
           session_store_chunks(p, store_chunks) * 2048;
}

}  // namespace

struct tsdf_server {
    tsdf_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::atomic<uint64_t> submitted{0};   // requests queued so far (an idle worker spins on it briefly)
    int worker_error = TSDF_OK;
    std::map<int32_t, Session> sessions;
    int32_t next_session = 1;
    std::unordered_map<uint64_t, Request*> requests;
    uint64_t next_ticket = 1;
    size_t used_bytes = 0;
    std::vector<Slot> slots;
    std::vector<float4*> slabs;
    std::vector<int> free_slabs;
    // totals for tsdf_server_get_stats
    int64_t completed = 0, batches = 0, batched_requests = 0;
};

namespace {

// Batches of at most this many requests run as plain per-map integrations
// (four short kernels each) instead of one cooperative batched launch, whose
// fixed cost (five phases, grid barriers) dominates when it carries only a
// scan or two: the latency of a lone request is what a lightly loaded server
// sees.
#ifndef TSDF_SERVER_PLAIN_BATCH
#define TSDF_SERVER_PLAIN_BATCH 2
#endif

void release_request(tsdf_server* s, Request* r) {
    if (r->slab >= 0) s->free_slabs.push_back(r->slab);
    delete r;
}

// Launch a batch on slot `k`. Called WITHOUT the lock: the requests and the
// slot belong to the worker until it records the launch (`maps` were taken
// under the lock; sessions in flight cannot be closed).
int launch_batch(tsdf_server* s, int k, std::vector<Request*>& reqs, const std::vector<tsdf_map*>& smaps) {
    Slot& sl = s->slots[k];
    const int count = (int)reqs.size();
    std::vector<tsdf_map*> maps(count);
    std::vector<const float*> pts(count);
    std::vector<int64_t> ns(count);
    std::vector<float> poses(12 * (size_t)count);
    cudaError_t e = cudaSuccess;
    const double t0 = now_us();
    for (int i = 0; i < count; ++i) {
        Request* r = reqs[i];
        maps[i] = smaps[i];
        float4* dst = sl.dev_pts + (size_t)i * s->cfg.max_points;
        if (r->mapped) {
            pts[i] = reinterpret_cast<const float*>(r->mapped);   // read in place over the host link
        } else {
            if (r->n > 0 && e == cudaSuccess)
                e = cudaMemcpyAsync(dst, r->host, (size_t)r->n * sizeof(float4), cudaMemcpyHostToDevice,
                                    sl.stream);
            pts[i] = reinterpret_cast<const float*>(dst);
        }
        ns[i] = r->n;
        std::memcpy(&poses[12 * (size_t)i], r->pose, sizeof(r->pose));
        if (r->shift && e == cudaSuccess) {
            int rc = tsdf_shift(maps[i], r->origin, sl.stream);
            if (rc != TSDF_OK) return rc;
        }
        r->res.t_start_us = t0;
    }
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    int rc = TSDF_OK;
    if (count <= TSDF_SERVER_PLAIN_BATCH) {
        for (int i = 0; i < count && rc == TSDF_OK; ++i)
            rc = tsdf_integrate(maps[i], pts[i], ns[i], &poses[12 * (size_t)i], sl.stream);
    } else {
        rc = tsdf_batch_integrate(sl.batch, maps.data(), pts.data(), ns.data(), poses.data(), count, sl.stream);
    }
    if (rc != TSDF_OK) return rc;
    // counters: the mapped host copy the batch writes (no copy to issue), else
    // a device-to-host copy (one call per map costs microseconds of host time)
    sl.src.resize(count);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
        sl.src[i] = map_host_counters(maps[i]);
        if (!sl.src[i]) {
            e = cudaMemcpyAsync(sl.counters + 3 * i, map_last_counters(maps[i]), 3 * sizeof(long long),
                                cudaMemcpyDeviceToHost, sl.stream);
            sl.src[i] = sl.counters + 3 * i;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) return TSDF_ERR_CUDA;
    return TSDF_OK;
}

// Poll interval of the worker while batches are in flight. The thread's
// timer slack is set to 1 us so that the short waits are not stretched to the
// default 50 us, which would add that much to every request's latency.
#ifndef TSDF_SERVER_POLL_US
#define TSDF_SERVER_POLL_US 5
#endif
// An idle worker watches for the next submission this long (yielding the
// core between checks) before it sleeps on the condition variable, whose
// wake-up would add its latency to the request.
#ifndef TSDF_SERVER_IDLE_SPIN_US
#define TSDF_SERVER_IDLE_SPIN_US 500
#endif

void worker_loop(tsdf_server* s) {
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);   // nanoseconds; failure only costs latency
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        // 1. completions
        for (Slot& sl : s->slots) {
            if (!sl.busy || sl.launching || cudaEventQuery(sl.done) != cudaSuccess) continue;
            const double t = now_us();
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                Request* r = sl.reqs[i];
                r->res.stats.valid_rays = sl.src[i][0];
                r->res.stats.hits = sl.src[i][1];
                r->res.stats.touched = sl.src[i][2];
                r->res.t_done_us = t;
                r->res.batch_size = (int32_t)sl.reqs.size();
                r->res.status = TSDF_OK;
                r->done = true;
                s->sessions[r->session].in_flight = false;
                s->completed++;
            }
            sl.reqs.clear();
            sl.busy = false;
            progress = true;
        }
        if (progress) s->cv_done.notify_all();
        // 2. a new batch on a free slot from the requests that have arrived
        for (size_t k = 0; k < s->slots.size(); ++k) {
            if (s->slots[k].busy) continue;
            std::vector<Request*> reqs;
            for (auto& kv : s->sessions) {
                Session& ss = kv.second;
                if (ss.in_flight || ss.queue.empty()) continue;
                reqs.push_back(ss.queue.front());
                if ((int)reqs.size() >= s->cfg.max_batch) break;
            }
            if (reqs.empty()) break;
            // oldest first is implicit in the per-session queues; mark, then
            // launch outside the lock so that submissions are not held up
            std::vector<tsdf_map*> maps;
            for (Request* r : reqs) {
                Session& ss = s->sessions[r->session];
                ss.queue.pop_front();
                ss.in_flight = true;
                maps.push_back(ss.map);
            }
            Slot& sl = s->slots[k];
            sl.busy = true;
            sl.launching = true;
            lk.unlock();
            int rc = launch_batch(s, (int)k, reqs, maps);
            lk.lock();
            sl.launching = false;
            if (rc == TSDF_OK) {
                sl.reqs = reqs;
                s->batches++;
                s->batched_requests += (int64_t)reqs.size();
            } else {
                sl.busy = false;
                for (Request* r : reqs) {
                    r->res.status = rc;
                    r->res.t_done_us = now_us();
                    r->done = true;
                    s->sessions[r->session].in_flight = false;
                }
                s->worker_error = rc;
                s->cv_done.notify_all();
            }
            progress = true;
        }
        bool any_busy = false;
        for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
        if (!progress) {
            if (any_busy) {
                s->cv_work.wait_for(lk, std::chrono::microseconds(TSDF_SERVER_POLL_US));
            } else {
                const uint64_t seen = s->submitted.load(std::memory_order_acquire);
                lk.unlock();
                const double t0 = now_us();
                while (s->submitted.load(std::memory_order_acquire) == seen && now_us() - t0 < TSDF_SERVER_IDLE_SPIN_US)
                    std::this_thread::yield();
                lk.lock();
                if (!s->stop && s->submitted.load(std::memory_order_acquire) == seen)
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

void destroy_server(tsdf_server* s) {
    for (Slot& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.batch) tsdf_batch_destroy(sl.batch);
        cudaFree(sl.dev_pts);
        if (sl.counters) cudaFreeHost(sl.counters);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto& kv : s->requests) delete kv.second;
    for (auto& kv : s->sessions)
        if (kv.second.map) tsdf_map_destroy(kv.second.map);
    for (float4* p : s->slabs) cudaFreeHost(p);
    delete s;
}

}  // namespace

extern "C" {

int tsdf_server_create(const tsdf_server_config* cfg, tsdf_server** out) {
    if (!cfg || !out) return TSDF_ERR_INVALID;
    *out = nullptr;
    if (cfg->max_batch < 1 || cfg->max_batch > 1024 || cfg->streams < 1 || cfg->streams > 8 || cfg->max_points < 1 ||
        cfg->max_points > TSDF_MAX_POINTS || cfg->max_outstanding < 1 || cfg->max_outstanding > 65536 ||
        cfg->hbm_budget_bytes < 0 || cfg->store_chunks < 0 || cfg->store_chunks > (1 << 30))
        return TSDF_ERR_INVALID;
    tsdf_server* s = new tsdf_server();
    s->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s->device);
    s->slots.resize((size_t)cfg->streams);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&sl.dev_pts, (size_t)cfg->max_batch * cfg->max_points * sizeof(float4));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.counters, (size_t)cfg->max_batch * 3 * sizeof(long long));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        int rc = tsdf_batch_create(cfg->max_batch, &sl.batch);
        if (rc != TSDF_OK) {
            destroy_server(s);
            return rc;
        }
        // each slot's launch uses its share of the GPU so that batches on
        // different slots can be resident together
        tsdf_batch_set_option(sl.batch, TSDF_BATCH_OPT_GRID_FRACTION, 100 / cfg->streams);
        // the sort configurations allocate each map's sort buffers: served
        // batches allocate no device memory
        tsdf_batch_set_option(sl.batch, TSDF_BATCH_OPT_TUNE_SORT, 0);
    }
    for (int i = 0; i < cfg->max_outstanding && e == cudaSuccess; ++i) {
        float4* p = nullptr;
        e = cudaMallocHost(&p, (size_t)cfg->max_points * sizeof(float4));
        if (e == cudaSuccess) {
            s->slabs.push_back(p);
            s->free_slabs.push_back(i);
        }
    }
    if (e != cudaSuccess) {
        destroy_server(s);
        return e == cudaErrorMemoryAllocation ? TSDF_ERR_OOM : TSDF_ERR_CUDA;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return TSDF_OK;
}

int tsdf_server_destroy(tsdf_server* s) {
    if (!s) return TSDF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    destroy_server(s);
    return TSDF_OK;
}

int tsdf_server_open_session(tsdf_server* s, const tsdf_params* params, int32_t* session) {
    if (!s || !params || !session) return TSDF_ERR_INVALID;
    const size_t bytes = session_bytes(*params, s->cfg.max_points, s->cfg.store_chunks);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((long long)(s->used_bytes + bytes) > s->cfg.hbm_budget_bytes) return TSDF_ERR_ADMISSION;
        s->used_bytes += bytes;   // reserve before the (slow) allocation
    }
    // the session's map lives on the server's device, whichever device is
    // current on the calling thread (restored before returning)
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(s->device) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->used_bytes -= bytes;
        return TSDF_ERR_CUDA;
    }
    tsdf_map* m = nullptr;
    int rc = tsdf_map_create(params, &m);
    // size the per-ray buffers for the largest scan now, so that no request
    // reallocates them (which would synchronise the device) while batches run
    if (rc == TSDF_OK) {
        rc = map_reserve_points(m, s->cfg.max_points);
        // the store's device tier too: served shifts allocate no device memory
        if (rc == TSDF_OK)
            rc = tsdf_map_reserve_store(m, (int64_t)session_store_chunks(*params, s->cfg.store_chunks));
        if (rc != TSDF_OK) {
            tsdf_map_destroy(m);
            m = nullptr;
        }
    }
    cudaSetDevice(prev);
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc != TSDF_OK) {
        s->used_bytes -= bytes;
        return rc;
    }
    const int32_t id = s->next_session++;
    Session& ss = s->sessions[id];
    ss.map = m;
    ss.bytes = bytes;
    *session = id;
    return TSDF_OK;
}

int tsdf_server_close_session(tsdf_server* s, int32_t session) {
    if (!s) return TSDF_ERR_INVALID;
    tsdf_map* m = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->sessions.find(session);
        if (it == s->sessions.end()) return TSDF_ERR_INVALID;
        if (it->second.outstanding > 0 || it->second.in_flight) return TSDF_ERR_BUSY;
        m = it->second.map;
        s->used_bytes -= it->second.bytes;
        s->sessions.erase(it);
    }
    return tsdf_map_destroy(m);
}

int tsdf_server_submit(tsdf_server* s, int32_t session, const float* points_host, int64_t n, const float pose[12],
                       const int64_t* new_origin, uint64_t* ticket) {
    if (!s || !pose || !ticket || n < 0 || n > s->cfg.max_points || (n > 0 && !points_host)) return TSDF_ERR_INVALID;
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(pose[i])) return TSDF_ERR_INVALID;
    if (new_origin)
        for (int a = 0; a < 3; ++a)
            if (new_origin[a] % 8 != 0) return TSDF_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->sessions.find(session);
    if (it == s->sessions.end()) return TSDF_ERR_INVALID;
    if (s->worker_error != TSDF_OK) return s->worker_error;
    if (s->free_slabs.empty()) return TSDF_ERR_BUSY;   // back-pressure: wait for results first
    Request* r = new Request();
    r->slab = s->free_slabs.back();
    s->free_slabs.pop_back();
    r->host = s->slabs[r->slab];
    r->ticket = s->next_ticket++;
    r->session = session;
    r->n = n;
    std::memcpy(r->pose, pose, sizeof(r->pose));
    if (new_origin) {
        r->shift = true;
        for (int a = 0; a < 3; ++a) r->origin[a] = new_origin[a];
    }
    r->res.ticket = r->ticket;
    r->res.session = session;
    r->res.t_submit_us = now_us();
    lk.unlock();
    if (n > 0) {
        // pinned host memory mapped into the device is read in place by the
        // batch (the caller keeps it unchanged until the request completes);
        // anything else is copied into the request's slab
        cudaPointerAttributes at{};
        if (((uintptr_t)points_host & 15u) == 0 && cudaPointerGetAttributes(&at, points_host) == cudaSuccess &&
            at.type == cudaMemoryTypeHost && at.devicePointer != nullptr && ((uintptr_t)at.devicePointer & 15u) == 0) {
            r->mapped = static_cast<const float4*>(at.devicePointer);
        } else {
            cudaGetLastError();
            std::memcpy(r->host, points_host, (size_t)n * sizeof(float4));   // slab is ours alone
        }
    }
    lk.lock();
    it = s->sessions.find(session);
    if (it == s->sessions.end()) {
        release_request(s, r);
        return TSDF_ERR_INVALID;
    }
    it->second.queue.push_back(r);
    it->second.outstanding++;
    s->requests[r->ticket] = r;
    *ticket = r->ticket;
    s->submitted.fetch_add(1, std::memory_order_release);
    lk.unlock();
    s->cv_work.notify_one();
    return TSDF_OK;
}

int tsdf_server_submit_many(tsdf_server* s, int32_t count, const int32_t* sessions, const float* const* points_host,
                            const int64_t* n, const float* poses, uint64_t* tickets, int32_t* submitted) {
    if (!s || count < 0 || !submitted || (count > 0 && (!sessions || !points_host || !n || !poses || !tickets)))
        return TSDF_ERR_INVALID;
    *submitted = 0;
    for (int32_t k = 0; k < count; ++k) {
        const int rc = tsdf_server_submit(s, sessions[k], points_host[k], n[k], poses + 12 * (size_t)k, nullptr,
                                          tickets + k);
        if (rc != TSDF_OK) return rc;
        *submitted = k + 1;
    }
    return TSDF_OK;
}

int tsdf_server_wait(tsdf_server* s, uint64_t ticket, tsdf_request_result* out, int64_t timeout_us) {
    if (!s || !out) return TSDF_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) return TSDF_ERR_INVALID;
    Request* r = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (!r->done) {
        if (timeout_us < 0) s->cv_done.wait(lk);
        else if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) return TSDF_ERR_TIMEOUT;
    }
    *out = r->res;
    auto sit = s->sessions.find(r->session);
    if (sit != s->sessions.end()) sit->second.outstanding--;
    s->requests.erase(it);
    release_request(s, r);
    return out->status;
}

int tsdf_server_wait_many(tsdf_server* s, int32_t count, const uint64_t* tickets, tsdf_request_result* out,
                          int64_t timeout_us) {
    if (!s || count < 0 || (count > 0 && (!tickets || !out))) return TSDF_ERR_INVALID;
    int first = TSDF_OK;
    for (int32_t i = 0; i < count; ++i) {
        const int rc = tsdf_server_wait(s, tickets[i], out + i, timeout_us);
        if (rc == TSDF_ERR_TIMEOUT || rc == TSDF_ERR_INVALID) {
            // not taken: mark the slot so the caller can tell it from a result
            out[i] = tsdf_request_result{};
            out[i].ticket = tickets[i];
            out[i].status = rc;
        }
        if (first == TSDF_OK) first = rc;
    }
    return first;
}

int tsdf_server_session_map(tsdf_server* s, int32_t session, tsdf_map** out) {
    if (!s || !out) return TSDF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->sessions.find(session);
    if (it == s->sessions.end()) return TSDF_ERR_INVALID;
    *out = it->second.map;
    return TSDF_OK;
}

int tsdf_server_get_stats(tsdf_server* s, tsdf_server_stats* out) {
    if (!s || !out) return TSDF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out->sessions = (int32_t)s->sessions.size();
    out->used_bytes = (int64_t)s->used_bytes;
    out->completed = s->completed;
    out->batches = s->batches;
    out->mean_batch = s->batches ? (double)s->batched_requests / (double)s->batches : 0.0;
    int64_t queued = 0;
    for (auto& kv : s->sessions) queued += (int64_t)kv.second.queue.size();
    out->queued = queued;
    return TSDF_OK;
}

}  // extern "C"
