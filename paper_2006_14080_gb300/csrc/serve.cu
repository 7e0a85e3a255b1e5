// Serving loop: continuous batching of reconstruction requests under a
// device-memory budget.
//
// Requests arrive from host memory (mri_server_submit copies them into
// library-owned pinned staging and returns a ticket).  A scheduler thread
// admits the oldest pending request as soon as a stream slot is free and its
// device memory fits the budget, so requests that arrive while others run
// start as slots and memory free up and their kernels overlap on the GPU.
// A cache of plan entries keeps DFT factors, coil maps and the request
// buffers resident: an entry is a plan for one shape and trajectory (its
// factors) plus fixed device buffers for k-space, coil maps and the image.
// A request whose trajectory and coil maps equal an idle entry's (compared
// byte for byte against host copies the entry keeps) uploads only its
// k-space; from the first such request on, the entry's reconstruction is a
// CUDA graph captured once and replayed (the fixed buffers keep the launch
// arguments the same).  Idle entries are evicted least-recently-used when
// the budget needs room; an idle entry of the request's shape is given the
// new trajectory in place when nothing else fits.  Entries and per-request
// buffers come from a stream-ordered pool and are freed stream-ordered, so
// no step of the loop, eviction included, synchronises the device.  Each
// request is reconstructed by exactly the kernels it would use alone (own
// plan, own workspace), so its result does not depend on what else is in
// flight, nor on whether it ran from a graph.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

uint64_t fnv1a(const void *data, size_t n, uint64_t h = 1469598103934665603ull) {
    const uint8_t *p = (const uint8_t *)data;
    for (size_t q = 0; q < n; ++q) {
        h ^= p[q];
        h *= 1099511628211ull;
    }
    return h;
}

struct PlanEntry {
    int nx, ny, nk, nc;
    uint64_t traj_hash;
    mri_plan *plan = nullptr;
    bool busy = false;
    uint64_t last_use = 0;
    size_t bytes = 0;                    // the plan's device bytes plus the three buffers below
    cudaStream_t last_stream = nullptr;  // stream of the entry's last work (stream-ordered free)
    void *d_k = nullptr, *d_maps = nullptr, *d_img = nullptr;  // fixed request buffers
    // host copies (ordinary memory) of the trajectory the plan's factors hold
    // and of the maps d_maps holds, compared byte for byte with a request's
    std::vector<uint8_t> h_traj, h_maps;
    int hits = 0;  // requests that found this entry holding their trajectory
};

struct Job {
    uint64_t ticket = 0;
    mri_server_request req{};
    uint64_t traj_hash = 0;
    size_t traj_bytes = 0, k_bytes = 0, maps_bytes = 0, img_bytes = 0;
    void *h_traj = nullptr, *h_k = nullptr, *h_maps = nullptr, *h_img = nullptr;  // pinned staging
    void *d_traj = nullptr;  // device trajectory, only while the entry's factors are (re)generated
    size_t dev_bytes = 0;    // transient device bytes of the request (its trajectory upload)
    PlanEntry *entry = nullptr;
    bool hit = false;       // the entry already holds this trajectory's factors
    bool retarget = false;  // the entry is an idle plan of the same shape given this request's trajectory
    int slot = -1;
    cudaEvent_t done_ev = nullptr;
    Clock::time_point t_submit, t_done;
    enum State { kPending, kRunning, kDone, kFailed } state = kPending;
    int status = MRI_OK;
    std::string error;
};

}  // namespace

struct mri_server {
    int device = 0, precision = MRI_BF16X3, max_inflight = 4;
    size_t budget = 0, resident = 0, peak_resident = 0;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    cudaMemPool_t pool = nullptr;  // request buffers; keeps up to the budget mapped between requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> pending;
    std::vector<Job *> running;
    std::unordered_map<uint64_t, Job *> jobs;
    std::vector<PlanEntry *> plans;
    std::multimap<size_t, void *> pinned_pool;  // free pinned staging buffers by size
    std::vector<double> latencies_ms;
    uint64_t next_ticket = 1, use_clock = 0, completed = 0, failed = 0;
    uint64_t plan_hits = 0, plan_retargets = 0, maps_reused = 0, graph_replays = 0;
    bool stop = false;
    std::thread worker;
};

namespace {

void *pinned_get(mri_server *s, size_t bytes) {
    auto it = s->pinned_pool.find(bytes);
    if (it != s->pinned_pool.end()) {
        void *p = it->second;
        s->pinned_pool.erase(it);
        return p;
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_put(mri_server *s, void *p, size_t bytes) {
    if (p) s->pinned_pool.emplace(bytes, p);
}

// The image staging buffer carries one extra 16-byte word for the status.
size_t stage_img_bytes(const Job *j) { return j->img_bytes + 16; }
int *job_status_word(Job *j) { return (int *)((char *)j->h_img + j->img_bytes); }

// Device bytes of an entry's fixed request buffers (k-space, maps, image).
size_t entry_buffer_bytes(const Job *j) { return j->k_bytes + j->maps_bytes + j->img_bytes; }

// Frees an entry (no work of it pending on `st` beyond what is already
// ordered there) and takes its bytes off the resident count.
void drop_entry(mri_server *s, PlanEntry *pe, cudaStream_t st) {
    if (pe->plan) mri::plan_destroy_async(pe->plan, st);
    void *bufs[] = {pe->d_k, pe->d_maps, pe->d_img};
    for (void *b : bufs)
        if (b) cudaFreeAsync(b, st);
    s->resident -= pe->bytes;
    s->plans.erase(std::find(s->plans.begin(), s->plans.end(), pe));
    delete pe;
}

void fail_job(mri_server *s, Job *j, int code, const std::string &msg) {
    j->state = Job::kFailed;
    j->status = code;
    j->error = msg;
    j->t_done = Clock::now();
    s->failed += 1;
}

// Starts a job on its slot (called by the worker with the lock held).
int start_job(mri_server *s, Job *j) {
    mri::NvtxRange range("mri_server_start_job");
    cudaStream_t st = s->streams[j->slot];
    const mri_server_request &r = j->req;
    PlanEntry *pe = j->entry;
    pe->last_stream = st;
    cudaError_t e = cudaSuccess;
    if (!pe->d_k) {  // a new entry: its fixed buffers
        void **bufs[] = {&pe->d_k, &pe->d_maps, &pe->d_img};
        size_t sizes[] = {j->k_bytes, j->maps_bytes, j->img_bytes};
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaMallocFromPoolAsync(bufs[q], sizes[q], s->pool, st);
    }
    if (e == cudaSuccess && !j->hit) {
        e = cudaMallocFromPoolAsync(&j->d_traj, j->traj_bytes, s->pool, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(j->d_traj, j->h_traj, j->traj_bytes, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(pe->d_k, j->h_k, j->k_bytes, cudaMemcpyHostToDevice, st);
    // coil maps: resident when they equal what the entry already holds
    const bool maps_same = pe->h_maps.size() == j->maps_bytes &&
                           std::memcmp(pe->h_maps.data(), j->h_maps, j->maps_bytes) == 0;
    if (e == cudaSuccess && !maps_same) {
        pe->h_maps.clear();  // the entry's maps are unknown until the copy is queued
        e = cudaMemcpyAsync(pe->d_maps, j->h_maps, j->maps_bytes, cudaMemcpyHostToDevice, st);
        const uint8_t *m = (const uint8_t *)j->h_maps;
        if (e == cudaSuccess) pe->h_maps.assign(m, m + j->maps_bytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MRI_ERR_CUDA;
    }
    if (maps_same) s->maps_reused += 1;
    if (!pe->plan) {
        // plan buffers come from the server's pool, so that evicting the plan
        // later frees them stream-ordered instead of synchronising the device
        int rc = mri::plan_create(&pe->plan, r.nx, r.ny, r.nk, r.nc, (const float *)j->d_traj, s->precision, st, s->pool);
        if (rc != MRI_OK) return rc;
        mri_plan_set_graphs(pe->plan, 0);
        const uint8_t *t = (const uint8_t *)j->h_traj;
        pe->h_traj.assign(t, t + j->traj_bytes);
    } else if (j->retarget) {
        // same shape, other trajectory: regenerate the factors in place (Alg. 1);
        // the plan's buffers, and so its captured graph, stay valid
        pe->traj_hash = 0;
        int rc = mri_plan_set_trajectory(pe->plan, (const float *)j->d_traj, st);
        if (rc != MRI_OK) return rc;
        pe->traj_hash = j->traj_hash;
        const uint8_t *t = (const uint8_t *)j->h_traj;
        pe->h_traj.assign(t, t + j->traj_bytes);
        s->plan_retargets += 1;
    } else {
        s->plan_hits += 1;
    }
    // from the first request that finds the entry holding its trajectory,
    // the whole reconstruction is a CUDA graph over the entry's fixed
    // buffers: captured once, then replayed (a new trajectory regenerated in
    // place keeps it valid).  Entries that never see their trajectory again
    // launch directly and pay no capture.  Requests run concurrently, so the
    // CG steps are two ordinary kernels (a cooperative grid would wait for the
    // whole GPU), with the same results as alone.
    if (j->hit) pe->hits += 1;
    mri_plan_set_graphs(pe->plan, pe->hits >= 1);
    const long long replays0 = pe->plan->graph_replays;
    int rc = mri::run_admm(pe->plan, (const mri_c64 *)pe->d_k, (const mri_c64 *)pe->d_maps, &r.params,
                           (mri_c64 *)pe->d_img, nullptr, nullptr, mri::AdmmWarm(), st, false);
    if (rc != MRI_OK) return rc;
    s->graph_replays += (uint64_t)(pe->plan->graph_replays - replays0);
    e = cudaMemcpyAsync(j->h_img, pe->d_img, j->img_bytes, cudaMemcpyDeviceToHost, st);
    // the plan's deferred status word (bounded device waits) travels with the image
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(job_status_word(j), &pe->plan->scal->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(j->done_ev, st);
    return e == cudaSuccess ? MRI_OK : MRI_ERR_CUDA;
}

void release_job_device(mri_server *s, Job *j) {
    cudaStream_t st = s->streams[j->slot];
    if (j->d_traj) cudaFreeAsync(j->d_traj, st);
    j->d_traj = nullptr;
    s->resident -= j->dev_bytes;
    j->dev_bytes = 0;
    s->slot_busy[j->slot] = false;
    if (j->entry) {
        j->entry->busy = false;
        j->entry->last_use = ++s->use_clock;
    }
}

// Evict idle cached entries, least recently used first, until `need` more bytes fit.
void make_room(mri_server *s, size_t need) {
    while (s->resident + need > s->budget) {
        PlanEntry *victim = nullptr;
        for (PlanEntry *pe : s->plans)
            if (!pe->busy && pe->plan && (!victim || pe->last_use < victim->last_use)) victim = pe;
        if (!victim) return;
        drop_entry(s, victim, victim->last_stream);  // idle: its last work has completed
    }
}

void worker_loop(mri_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        bool progressed = false;
        // completions
        for (size_t q = 0; q < s->running.size();) {
            Job *j = s->running[q];
            cudaError_t e = cudaEventQuery(j->done_ev);
            if (e == cudaErrorNotReady) {
                ++q;
                continue;
            }
            if (e == cudaSuccess) {
                const int dev_status = *job_status_word(j);
                j->t_done = Clock::now();
                if (dev_status == 0) {
                    j->state = Job::kDone;
                    s->completed += 1;
                    s->latencies_ms.push_back(
                        std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count());
                } else {
                    // clear the plan's status word before it serves again, on
                    // any stream (a failure path: waiting here is acceptable)
                    cudaMemsetAsync(&j->entry->plan->scal->status, 0, sizeof(int), s->streams[j->slot]);
                    cudaStreamSynchronize(s->streams[j->slot]);
                    fail_job(s, j, MRI_ERR_TIMEOUT,
                             "a bounded device-side wait gave up (status " + std::to_string(dev_status) + ")");
                }
            } else {
                cudaGetLastError();
                fail_job(s, j, MRI_ERR_CUDA, cudaGetErrorString(e));
            }
            release_job_device(s, j);
            s->running.erase(s->running.begin() + q);
            progressed = true;
        }
        if (progressed) s->cv_done.notify_all();
        // admission, oldest first
        while (!s->pending.empty()) {
            int slot = -1;
            for (int q = 0; q < s->max_inflight; ++q)
                if (!s->slot_busy[q]) {
                    slot = q;
                    break;
                }
            if (slot < 0) break;
            Job *j = s->pending.front();
            const mri_server_request &r = j->req;
            // entry: an idle cached entry of this shape and trajectory (the
            // trajectory compared byte for byte); else a new one if it fits;
            // else an idle entry of the same shape given this trajectory in
            // place (no allocation); else a new one after evicting
            PlanEntry *pe = nullptr, *same_shape = nullptr;
            for (PlanEntry *c : s->plans) {
                if (c->busy || c->nx != r.nx || c->ny != r.ny || c->nk != r.nk || c->nc != r.nc || !c->plan) continue;
                if (c->traj_hash == j->traj_hash && c->h_traj.size() == j->traj_bytes &&
                    std::memcmp(c->h_traj.data(), j->h_traj, j->traj_bytes) == 0) {
                    pe = c;
                    break;
                }
                if (!same_shape || c->last_use < same_shape->last_use) same_shape = c;
            }
            const size_t plan_est = pe ? 0 : mri_plan_estimate_bytes(r.nx, r.ny, r.nk, r.nc, s->precision);
            size_t entry_bytes = pe ? 0 : plan_est + entry_buffer_bytes(j);  // a new entry's resident bytes
            const size_t transient = pe ? 0 : j->traj_bytes;  // the trajectory upload for its factors
            size_t need = entry_bytes + transient;
            j->hit = pe != nullptr;
            j->retarget = false;
            if (!pe && same_shape && s->resident + need > s->budget) {
                pe = same_shape;
                j->retarget = true;
                entry_bytes = 0;
                need = transient;
            }
            if ((!pe && plan_est == 0) || need > s->budget) {
                s->pending.pop_front();
                fail_job(s, j, MRI_ERR_NOMEM,
                         plan_est == 0 && !pe ? "request shape not supported"
                                              : "request needs " + std::to_string(need) +
                                                    " bytes, more than the whole budget");
                s->cv_done.notify_all();
                continue;
            }
            if (s->resident + need > s->budget) {
                if (pe) pe->busy = true;  // keep the matching entry out of the eviction
                make_room(s, need);
                if (pe) pe->busy = false;
            }
            if (s->resident + need > s->budget) break;  // wait for completions
            s->pending.pop_front();
            if (!pe) {
                pe = new PlanEntry{r.nx, r.ny, r.nk, r.nc, j->traj_hash};
                pe->bytes = entry_bytes;
                s->plans.push_back(pe);
            }
            pe->busy = true;
            j->entry = pe;
            j->slot = slot;
            j->dev_bytes = transient;  // the entry's bytes stay resident with the cache
            s->slot_busy[slot] = true;
            s->resident += need;
            s->peak_resident = std::max(s->peak_resident, s->resident);
            j->state = Job::kRunning;
            const int rc = start_job(s, j);
            if (entry_bytes && pe->plan) {  // the plan's actual bytes instead of the estimate
                const size_t actual = mri_plan_device_bytes(pe->plan) + entry_buffer_bytes(j);
                s->resident = s->resident - pe->bytes + actual;
                pe->bytes = actual;
                s->peak_resident = std::max(s->peak_resident, s->resident);
            }
            if (rc != MRI_OK) {
                // a start that failed part-way leaves the entry's factors, maps
                // or graph in an unknown state: it leaves the cache (its frees
                // are ordered after whatever the slot's stream already holds)
                fail_job(s, j, rc, mri_last_error());
                release_job_device(s, j);
                drop_entry(s, pe, s->streams[slot]);
                j->entry = nullptr;
                s->cv_done.notify_all();
                continue;
            }
            s->running.push_back(j);
            progressed = true;
        }
        if (s->stop && s->pending.empty() && s->running.empty()) break;
        if (!progressed)
            s->cv_work.wait_for(lock, std::chrono::microseconds(s->running.empty() ? 2000 : 50));
    }
}

}  // namespace

using namespace mri;

extern "C" {

MRI_API int mri_server_create(mri_server **out, size_t hbm_budget_bytes, int max_inflight, int precision) {
    if (!out) return set_error("null output"), MRI_ERR_INVALID;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_inflight <= 0 || max_inflight > 64)
        return set_error("budget must be > 0 and max_inflight in 1..64"), MRI_ERR_INVALID;
    if (precision != MRI_FP32 && !is_tc_precision(precision)) return set_error("unknown precision"), MRI_ERR_INVALID;
    mri_server *s = new mri_server();
    s->budget = hbm_budget_bytes;
    s->max_inflight = max_inflight;
    s->precision = precision;
    cudaGetDevice(&s->device);
    s->slot_busy.assign(max_inflight, false);
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return set_error("cudaMemPoolCreate failed"), MRI_ERR_CUDA;
        }
        uint64_t keep = hbm_budget_bytes;
        cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int q = 0; q < max_inflight; ++q) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            cudaMemPoolDestroy(s->pool);
            delete s;
            return set_error("cudaStreamCreate failed"), MRI_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return MRI_OK;
}

MRI_API int mri_server_submit(mri_server *s, const mri_server_request *r, uint64_t *ticket) {
    if (!s || !r || !ticket) return set_error("null argument"), MRI_ERR_INVALID;
    if (r->nx <= 0 || r->ny <= 0 || r->nk <= 0 || r->nc <= 0 || !r->traj || !r->kspace || !r->coil_maps)
        return set_error("bad request: dimensions must be positive and host pointers non-null"), MRI_ERR_INVALID;
    Job *j = new Job();
    j->req = *r;
    j->traj_bytes = (size_t)r->nk * 2 * sizeof(float);
    j->k_bytes = (size_t)r->nc * r->nk * sizeof(mri_c64);
    j->maps_bytes = (size_t)r->nc * r->nx * r->ny * sizeof(mri_c64);
    j->img_bytes = (size_t)r->nx * r->ny * sizeof(mri_c64);
    j->traj_hash = fnv1a(r->traj, j->traj_bytes);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        j->h_traj = pinned_get(s, j->traj_bytes);
        j->h_k = pinned_get(s, j->k_bytes);
        j->h_maps = pinned_get(s, j->maps_bytes);
        j->h_img = pinned_get(s, stage_img_bytes(j));
    }
    if (!j->h_traj || !j->h_k || !j->h_maps || !j->h_img) {
        std::lock_guard<std::mutex> lock(s->mu);
        pinned_put(s, j->h_traj, j->traj_bytes);
        pinned_put(s, j->h_k, j->k_bytes);
        pinned_put(s, j->h_maps, j->maps_bytes);
        pinned_put(s, j->h_img, stage_img_bytes(j));
        delete j;
        return set_error("pinned staging allocation failed"), MRI_ERR_NOMEM;
    }
    std::memcpy(j->h_traj, r->traj, j->traj_bytes);
    std::memcpy(j->h_k, r->kspace, j->k_bytes);
    std::memcpy(j->h_maps, r->coil_maps, j->maps_bytes);
    if (cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lock(s->mu);
        pinned_put(s, j->h_traj, j->traj_bytes);
        pinned_put(s, j->h_k, j->k_bytes);
        pinned_put(s, j->h_maps, j->maps_bytes);
        pinned_put(s, j->h_img, stage_img_bytes(j));
        delete j;
        return set_error("cudaEventCreate failed"), MRI_ERR_CUDA;
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        j->ticket = s->next_ticket++;
        j->t_submit = Clock::now();
        s->jobs[j->ticket] = j;
        s->pending.push_back(j);
        *ticket = j->ticket;
    }
    s->cv_work.notify_one();
    return MRI_OK;
}

MRI_API int mri_server_poll(mri_server *s, uint64_t ticket, int *done) {
    if (!s || !done) return set_error("null argument"), MRI_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return set_error("unknown ticket"), MRI_ERR_INVALID;
    *done = it->second->state == Job::kDone || it->second->state == Job::kFailed;
    return MRI_OK;
}

MRI_API int mri_server_wait(mri_server *s, uint64_t ticket, mri_c64 *image, double *latency_ms, double timeout_s) {
    if (!s) return set_error("null server"), MRI_ERR_INVALID;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return set_error("unknown ticket"), MRI_ERR_INVALID;
    Job *j = it->second;
    auto finished = [&] { return j->state == Job::kDone || j->state == Job::kFailed; };
    if (timeout_s > 0) {
        if (!s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), finished))
            return set_error("request still running after the wait limit"), MRI_ERR_TIMEOUT;
    } else {
        s->cv_done.wait(lock, finished);
    }
    int rc = j->status;
    if (j->state == Job::kDone) {
        if (image) std::memcpy(image, j->h_img, j->img_bytes);
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
    } else {
        set_error(j->error);
    }
    pinned_put(s, j->h_traj, j->traj_bytes);
    pinned_put(s, j->h_k, j->k_bytes);
    pinned_put(s, j->h_maps, j->maps_bytes);
    pinned_put(s, j->h_img, stage_img_bytes(j));
    cudaEventDestroy(j->done_ev);
    s->jobs.erase(it);
    delete j;
    return rc;
}

MRI_API int mri_server_stats(mri_server *s, double *p50_ms, double *p99_ms, uint64_t *completed, uint64_t *failed,
                             size_t *resident_bytes, size_t *peak_resident_bytes) {
    if (!s) return set_error("null server"), MRI_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    std::vector<double> v = s->latencies_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) -> double {
        if (v.empty()) return 0.0;
        size_t idx = (size_t)std::min<double>(v.size() - 1, std::max(0.0, std::ceil(q * v.size()) - 1));
        return v[idx];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (completed) *completed = s->completed;
    if (failed) *failed = s->failed;
    if (resident_bytes) *resident_bytes = s->resident;
    if (peak_resident_bytes) *peak_resident_bytes = s->peak_resident;
    return MRI_OK;
}

MRI_API int mri_server_cache_stats(mri_server *s, uint64_t *plan_hits, uint64_t *plan_retargets,
                                   uint64_t *maps_reused, uint64_t *graph_replays) {
    if (!s) return set_error("null server"), MRI_ERR_INVALID;
    std::lock_guard<std::mutex> lock(s->mu);
    if (plan_hits) *plan_hits = s->plan_hits;
    if (plan_retargets) *plan_retargets = s->plan_retargets;
    if (maps_reused) *maps_reused = s->maps_reused;
    if (graph_replays) *graph_replays = s->graph_replays;
    return MRI_OK;
}

MRI_API int mri_server_destroy(mri_server *s) {
    if (!s) return MRI_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        // requests not yet admitted are dropped
        for (Job *j : s->pending) fail_job(s, j, MRI_ERR_INVALID, "server destroyed before the request started");
        s->pending.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : s->jobs) {
        Job *j = kv.second;
        void *hs[] = {j->h_traj, j->h_k, j->h_maps, j->h_img};
        for (void *h : hs)
            if (h) cudaFreeHost(h);
        if (j->done_ev) cudaEventDestroy(j->done_ev);
        delete j;
    }
    for (PlanEntry *pe : s->plans) {
        if (pe->plan) mri_plan_destroy(pe->plan);
        void *bufs[] = {pe->d_k, pe->d_maps, pe->d_img};
        for (void *b : bufs)
            if (b) cudaFree(b);
        delete pe;
    }
    for (auto &kv : s->pinned_pool) cudaFreeHost(kv.second);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    cudaMemPoolDestroy(s->pool);
    delete s;
    return MRI_OK;
}

}  // extern "C"
