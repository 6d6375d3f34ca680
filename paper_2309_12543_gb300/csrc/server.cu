// Serving engine: a request loop that batches incoming trajectory checks as they
// arrive (continuous batching) against the latest published obstacle cloud.
//
// The paper's controller needs distances along the executing trajectory in every
// control cycle (about 10 ms; 8 ms for the b-CAP protocol, Sec. I).  Clients submit
// trajectories from any thread; one engine thread forms batches whenever one of
// `slots` in-flight slots is free and the device-memory budget admits the batch,
// launches it with check_batch on the slot's own stream (so batches overlap on the
// device).  The kernels read the joint values from, and write the results to, the
// slot's page-locked buffers (over the CPU-GPU link, no copies); a one-thread
// finish kernel then publishes the status and a completion count in page-locked
// memory, which the engine polls while batches are in flight.  Grids, robots and
// the latest cloud stay resident on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    const sdf_robot* robot = nullptr;
    std::vector<float> q;            // W x dof
    int W = 0;
    size_t bytes = 0;                // device footprint of its buffers
    Clock::time_point submitted;
    int state = 0;                   // 0 pending, 1 in flight, 2 done
    int status = SDF_OK;
    std::vector<float> dist;
    std::vector<int32_t> link, point;
    double latency_us = 0.0;
};

struct CloudBuf {
    float* d = nullptr;              // device, max_points x 3
    float* h = nullptr;              // pinned staging
    int N = 0;
    int refs = 0;                    // in-flight batches using it
    cudaEvent_t ready = nullptr;     // its upload finished
};

struct Slot {
    sdf_server* srv = nullptr;
    sdf_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    float* h_q = nullptr;            // page-locked, max_waypoints x max_dof: read by the kernels
    float* h_out = nullptr;          // page-locked, dist | link | point, max_waypoints each:
                                     // written by the kernels
    std::vector<std::shared_ptr<Request>> reqs;
    int cloud = -1;
    size_t bytes = 0;
    std::atomic<bool> finished{false};   // set only when the launch itself failed
    unsigned seq = 0;                    // completion count the batch's finish kernel publishes
    bool busy = false;
};

}  // namespace

struct sdf_server {
    sdf_server_config cfg;
    std::vector<std::unique_ptr<Slot>> slots;
    std::vector<CloudBuf> clouds;
    cudaStream_t upload = nullptr;
    int current_cloud = -1;
    std::mutex mu;
    std::condition_variable cv;      // engine wake-up and client wake-up
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> by_ticket;
    uint64_t next_ticket = 1;
    size_t in_flight_bytes = 0;
    size_t scratch_bytes = 0;        // per batch: sorted cloud and spheres
    bool stop = false;
    std::atomic<uint64_t> submits{0};   // bumped by every submission (wakes a polling engine)
    std::thread engine;
    // statistics
    std::vector<double> latencies;
    uint64_t completed = 0, rejected = 0, batches = 0, batched_requests = 0;
    int in_flight = 0, peak_in_flight = 0;
    std::string err;
    // surrogate form (requests on the surrogate's grids), or none
    const sdf_surrogate* surrogate = nullptr;
    const sdf_grids* surrogate_grids = nullptr;
    float margin = 0.f, eps = 0.f;
};

namespace {

// Whether a slot's batch has completed: its finish kernel has published the
// expected count (the acquire load orders the reads of the results after it), or
// its launch failed.
bool slot_done(const Slot& s) {
    return s.finished.load(std::memory_order_acquire) || __atomic_load_n(s.ctx->h_done, __ATOMIC_ACQUIRE) == s.seq;
}

// The status word the finish kernel published, as a return code.
int published_status(const Slot& s) {
    const int st = __atomic_load_n(s.ctx->h_status, __ATOMIC_ACQUIRE);
    if (st & sdf::kStatusTimeout) return SDF_ERR_TIMEOUT;
    if (st & sdf::kStatusNonFinite) return SDF_ERR_NONFINITE;
    return SDF_OK;
}

size_t request_bytes(const sdf_server* S, int W, int dof) {
    (void)S;
    return (size_t)W * ((size_t)dof * sizeof(float) + sizeof(float) + 2 * sizeof(int32_t));
}

// Retire finished batches: results to their requests, memory and cloud released.
void retire(sdf_server* S, std::unique_lock<std::mutex>& lk) {
    (void)lk;
    for (auto& sp : S->slots) {
        Slot& s = *sp;
        if (!s.busy || !slot_done(s)) continue;
        const int rc = s.finished.load(std::memory_order_relaxed) ? SDF_OK : published_status(s);
        const auto now = Clock::now();
        const int maxw = S->cfg.max_waypoints;
        int off = 0;
        for (auto& r : s.reqs) {
            r->dist.assign(s.h_out + off, s.h_out + off + r->W);
            const int32_t* li = reinterpret_cast<const int32_t*>(s.h_out + maxw);
            const int32_t* pi = reinterpret_cast<const int32_t*>(s.h_out + 2 * maxw);
            r->link.assign(li + off, li + off + r->W);
            r->point.assign(pi + off, pi + off + r->W);
            if (r->status == SDF_OK) r->status = rc;
            r->latency_us = std::chrono::duration<double, std::micro>(now - r->submitted).count();
            r->state = 2;
            S->latencies.push_back(r->latency_us);
            ++S->completed;
            off += r->W;
        }
        s.reqs.clear();
        S->in_flight_bytes -= s.bytes;
        S->clouds[s.cloud].refs--;
        s.busy = false;
        s.finished.store(false, std::memory_order_relaxed);
        --S->in_flight;
    }
}

// Form and launch batches while a slot is free and requests are waiting.
void launch(sdf_server* S) {
    while (!S->pending.empty() && S->current_cloud >= 0) {
        Slot* slot = nullptr;
        for (auto& sp : S->slots)
            if (!sp->busy) { slot = sp.get(); break; }
        if (!slot) return;
        if (S->cfg.batch_window_us > 0 && (int)S->pending.size() < S->cfg.max_batch) {
            const auto waited = std::chrono::duration_cast<std::chrono::microseconds>(
                Clock::now() - S->pending.front()->submitted).count();
            if (waited < S->cfg.batch_window_us) return;   // the engine wakes every 200 us
        }
        // admission: requests in arrival order while the batch fits the slot and the
        // memory budget (in-flight batches included)
        size_t bytes = S->scratch_bytes;
        int W = 0, n = 0;
        for (auto& r : S->pending) {
            if (n == S->cfg.max_batch || W + r->W > S->cfg.max_waypoints) break;
            if (S->in_flight_bytes + bytes + r->bytes > (size_t)S->cfg.memory_budget_bytes) break;
            bytes += r->bytes;
            W += r->W;
            ++n;
        }
        if (n == 0) return;   // wait for memory to be released
        Slot& s = *slot;
        s.reqs.assign(S->pending.begin(), S->pending.begin() + n);
        S->pending.erase(S->pending.begin(), S->pending.begin() + n);
        CloudBuf& cb = S->clouds[S->current_cloud];
        s.cloud = S->current_cloud;
        cb.refs++;
        // pack joint values; the check reads them and writes its results in the
        // slot's page-locked buffers; then the finish kernel
        const int maxw = S->cfg.max_waypoints;
        std::vector<sdf_check_request> req(n);
        size_t qoff = 0;
        int woff = 0;
        for (int i = 0; i < n; ++i) {
            Request& r = *s.reqs[i];
            std::memcpy(s.h_q + qoff, r.q.data(), r.q.size() * sizeof(float));
            req[i].robot = r.robot;
            req[i].q_dev = s.h_q + qoff;
            req[i].W = r.W;
            req[i].points_dev = cb.d;
            req[i].N = cb.N;
            req[i].dist_dev = s.h_out + woff;
            req[i].argmin_link_dev = reinterpret_cast<int32_t*>(s.h_out + maxw) + woff;
            req[i].argmin_point_dev = reinterpret_cast<int32_t*>(s.h_out + 2 * maxw) + woff;
            qoff += r.q.size();
            woff += r.W;
            r.state = 1;
        }
        int rc = SDF_OK;
        if (cudaStreamWaitEvent(s.stream, cb.ready, 0) != cudaSuccess) rc = SDF_ERR_CUDA;
        if (rc == SDF_OK && S->surrogate) {
            // the surrogate form, one request after the other on the slot's stream;
            // requests on other grids take the grid path together
            std::vector<sdf_check_request> rest;
            for (auto& q : req) {
                if (rc != SDF_OK) break;
                if (q.robot->grids == S->surrogate_grids)
                    rc = check_trajectory_surrogate(s.ctx, q.robot, S->surrogate, q.q_dev, q.W, q.points_dev, q.N,
                                                    S->margin, S->eps, q.dist_dev, q.argmin_link_dev,
                                                    q.argmin_point_dev, nullptr, nullptr);
                else
                    rest.push_back(q);
            }
            if (rc == SDF_OK && !rest.empty()) rc = check_batch(s.ctx, rest.data(), (int)rest.size());
        } else if (rc == SDF_OK) {
            rc = check_batch(s.ctx, req.data(), n);
        }
        if (rc == SDF_OK) {
            s.seq = s.ctx->seq + 1u;
            if (sdf::launch_finish(s.ctx->status, s.ctx->h_status, s.ctx->d_seq, s.ctx->h_done, s.stream) ==
                cudaSuccess)
                s.ctx->seq = s.seq;
            else
                rc = SDF_ERR_CUDA;
        }
        s.bytes = bytes;
        s.busy = true;
        S->in_flight_bytes += bytes;
        S->in_flight++;
        S->peak_in_flight = std::max(S->peak_in_flight, S->in_flight);
        S->batches++;
        S->batched_requests += (uint64_t)n;
        if (rc != SDF_OK) {
            // report the failure on these requests; the slot is released at once
            for (auto& r : s.reqs) r->status = rc;
            s.finished.store(true, std::memory_order_release);
        }
    }
}

void engine_loop(sdf_server* S) {
    cudaSetDevice(S->cfg.device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        retire(S, lk);
        launch(S);
        S->cv.notify_all();   // clients waiting on results
        if (S->in_flight > 0) {
            // batches in flight: poll their completion words, without the lock, until
            // one completes, a request arrives, or 100 us pass (the batch window)
            const uint64_t sub0 = S->submits.load(std::memory_order_relaxed);
            lk.unlock();
            const auto t0 = Clock::now();
            for (unsigned i = 0;; ++i) {
                bool any = false;
                for (auto& sp : S->slots)   // only this thread changes the slots
                    if (sp->busy && slot_done(*sp)) any = true;
                if (any || S->submits.load(std::memory_order_relaxed) != sub0) break;
                if ((i & 63u) == 63u && Clock::now() - t0 > std::chrono::microseconds(100)) break;
            }
            lk.lock();
        } else {
            S->cv.wait_for(lk, std::chrono::microseconds(200));
        }
    }
}

void free_server(sdf_server* S) {
    for (auto& sp : S->slots) {
        Slot& s = *sp;
        if (s.stream) cudaStreamSynchronize(s.stream);
        sdf::hfree(s.h_q);
        sdf::hfree(s.h_out);
        if (s.ctx) sdf_ctx_destroy(s.ctx);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    for (auto& c : S->clouds) {
        sdf::dfree(c.d);
        sdf::hfree(c.h);
        if (c.ready) cudaEventDestroy(c.ready);
    }
    if (S->upload) cudaStreamDestroy(S->upload);
    delete S;
}

}  // namespace

extern "C" {

int sdf_server_create(const sdf_server_config* cfg, sdf_server** out) {
    if (!cfg || !out) return SDF_ERR_INVALID_ARG;
    *out = nullptr;
    sdf_server_config c = *cfg;
    if (c.slots < 1 || c.slots > 16 || c.max_batch < 1 || c.max_batch > SDF_MAX_BATCH || c.max_waypoints < 1 ||
        c.max_points < 0 || c.max_points > SDF_MAX_POINTS || c.max_dof < 0 || c.max_dof + 1 > SDF_MAX_LINKS ||
        c.memory_budget_bytes < 0 || c.batch_window_us < 0)
        return SDF_ERR_INVALID_ARG;
    if (cudaSetDevice(c.device) != cudaSuccess) return SDF_ERR_INVALID_ARG;
    if (c.memory_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return SDF_ERR_CUDA;
        c.memory_budget_bytes = (int64_t)(fr / 4);
    }
    sdf_server* S = new (std::nothrow) sdf_server();
    if (!S) return SDF_ERR_OOM;
    S->cfg = c;
    const size_t np = (size_t)std::max(c.max_points, 1);
    S->scratch_bytes = np * sizeof(float4) + (np / 32 + 2) * sizeof(float4) * 2 + 64;
    int rc = SDF_OK;
    if (cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking) != cudaSuccess) rc = SDF_ERR_CUDA;
    const int kClouds = c.slots + 2;   // enough that a free buffer exists while slots hold theirs
    S->clouds.resize(kClouds);
    for (auto& cb : S->clouds) {
        if (rc != SDF_OK) break;
        if (sdf::dmalloc(&cb.d, np * 3 * sizeof(float)) != cudaSuccess ||
            sdf::hmalloc(&cb.h, np * 3 * sizeof(float)) != cudaSuccess ||
            cudaEventCreateWithFlags(&cb.ready, cudaEventDisableTiming) != cudaSuccess)
            rc = SDF_ERR_OOM;
    }
    const size_t qn = (size_t)c.max_waypoints * std::max(c.max_dof, 1);
    for (int i = 0; i < c.slots && rc == SDF_OK; ++i) {
        S->slots.emplace_back(new Slot());
        Slot& s = *S->slots.back();
        s.srv = S;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess) { rc = SDF_ERR_CUDA; break; }
        rc = sdf_ctx_create(&s.ctx, c.device, s.stream);
        if (rc != SDF_OK) break;
        rc = sdf_ctx_reserve(s.ctx, c.max_points, c.max_waypoints, (int64_t)c.max_waypoints * (c.max_dof + 1),
                             c.max_batch);
        if (rc != SDF_OK) break;
        if (sdf::hmalloc(&s.h_q, qn * sizeof(float)) != cudaSuccess ||
            sdf::hmalloc(&s.h_out, 3 * (size_t)c.max_waypoints * sizeof(float)) != cudaSuccess)
            rc = SDF_ERR_OOM;
    }
    if (rc != SDF_OK) {
        free_server(S);
        return rc;
    }
    S->engine = std::thread(engine_loop, S);
    *out = S;
    return SDF_OK;
}

void sdf_server_destroy(sdf_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->engine.joinable()) S->engine.join();
    cudaSetDevice(S->cfg.device);
    free_server(S);
}

int sdf_server_set_surrogate(sdf_server* S, const sdf_surrogate* surrogate, float margin, float eps) {
    if (!S || !(margin >= 0.f) || !(eps >= 0.f)) return SDF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->surrogate = surrogate;
    S->surrogate_grids = surrogate ? sdf::surrogate_grids(surrogate) : nullptr;
    S->margin = margin;
    S->eps = eps;
    return SDF_OK;
}

int sdf_server_set_cloud(sdf_server* S, const float* points_host, int32_t N) {
    if (!S || N < 0 || N > S->cfg.max_points || (N > 0 && !points_host)) return SDF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    int pick = -1;
    for (int i = 0; i < (int)S->clouds.size(); ++i)
        if (i != S->current_cloud && S->clouds[i].refs == 0) { pick = i; break; }
    if (pick < 0) return SDF_ERR_TIMEOUT;   // every buffer is held by in-flight batches
    CloudBuf& cb = S->clouds[pick];
    // the previous upload into this buffer is complete once no batch holds it and its
    // own upload event has fired
    if (cudaEventSynchronize(cb.ready) != cudaSuccess) return SDF_ERR_CUDA;
    cudaSetDevice(S->cfg.device);
    std::memcpy(cb.h, points_host, (size_t)N * 3 * sizeof(float));
    cb.N = N;
    if (N > 0 && cudaMemcpyAsync(cb.d, cb.h, (size_t)N * 3 * sizeof(float), cudaMemcpyHostToDevice, S->upload) !=
                     cudaSuccess)
        return SDF_ERR_CUDA;
    if (cudaEventRecord(cb.ready, S->upload) != cudaSuccess) return SDF_ERR_CUDA;
    S->current_cloud = pick;
    S->cv.notify_all();
    return SDF_OK;
}

int sdf_server_submit(sdf_server* S, const sdf_robot* robot, const float* q_host, int32_t W, uint64_t* ticket) {
    if (!S || !robot || !ticket || W < 1 || (robot->dof > 0 && !q_host)) return SDF_ERR_INVALID_ARG;
    if (robot->device != S->cfg.device || robot->dof > S->cfg.max_dof || W > S->cfg.max_waypoints)
        return SDF_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->robot = robot;
    r->W = W;
    r->q.assign(q_host, q_host + (size_t)W * robot->dof);
    r->bytes = request_bytes(S, W, robot->dof);
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->bytes + S->scratch_bytes > (size_t)S->cfg.memory_budget_bytes) {
        ++S->rejected;
        return SDF_ERR_OOM;   // could never be admitted
    }
    r->ticket = S->next_ticket++;
    r->submitted = Clock::now();
    S->pending.push_back(r);
    S->submits.fetch_add(1, std::memory_order_relaxed);
    S->by_ticket[r->ticket] = r;
    *ticket = r->ticket;
    S->cv.notify_all();
    return SDF_OK;
}

int sdf_server_poll(sdf_server* S, uint64_t ticket, int64_t wait_us, float* dist, int32_t* link, int32_t* point,
                    double* latency_us) {
    if (!S) return SDF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return SDF_ERR_INVALID_ARG;
    std::shared_ptr<Request> r = it->second;
    if (r->state != 2 && wait_us != 0) {
        const auto until = Clock::now() + std::chrono::microseconds(wait_us < 0 ? 60000000 : wait_us);
        S->cv.wait_until(lk, until, [&] { return r->state == 2 || S->stop; });
    }
    if (r->state != 2) return wait_us != 0 ? SDF_ERR_TIMEOUT : SDF_PENDING;
    if (dist) std::memcpy(dist, r->dist.data(), (size_t)r->W * sizeof(float));
    if (link) std::memcpy(link, r->link.data(), (size_t)r->W * sizeof(int32_t));
    if (point) std::memcpy(point, r->point.data(), (size_t)r->W * sizeof(int32_t));
    if (latency_us) *latency_us = r->latency_us;
    S->by_ticket.erase(it);
    return r->status;
}

int sdf_server_stats(sdf_server* S, double* out, int32_t n, int32_t reset) {
    if (!S || n < 0 || (n > 0 && !out)) return SDF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->latencies;
    auto pct = [&](double p) -> double {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
        std::nth_element(v.begin(), v.begin() + k, v.end());
        return v[k];
    };
    double mean = 0.0;
    for (double x : S->latencies) mean += x;
    if (!S->latencies.empty()) mean /= (double)S->latencies.size();
    const double vals[SDF_SERVER_STAT_COUNT] = {
        pct(0.50), pct(0.99), mean, (double)S->completed, (double)S->rejected, (double)S->batches,
        S->batches ? (double)S->batched_requests / (double)S->batches : 0.0, (double)S->peak_in_flight,
        (double)S->pending.size(), v.empty() ? 0.0 : *std::max_element(S->latencies.begin(), S->latencies.end())};
    for (int i = 0; i < n && i < SDF_SERVER_STAT_COUNT; ++i) out[i] = vals[i];
    if (reset) {
        S->latencies.clear();
        S->completed = S->rejected = S->batches = S->batched_requests = 0;
        S->peak_in_flight = S->in_flight;
    }
    return SDF_OK;
}

}  // extern "C"
