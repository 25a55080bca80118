// server.cu -- continuous-batching request loop (lbm_server_* in include/lbm.h).
//
// A worker thread owns one batch per (lattice, storage, collision) class, each on its own stream.
// Each round it enqueues a run of K steps (lbm_batch_run) for every class with running instances,
// then -- while the GPU works -- admits waiting requests in arrival order as long as their device
// footprint fits the budget (they join the next round), waits for the round, and retires the
// instances that have run all their steps: FP64 fit of the force history, normalized damping,
// memory freed.  The batches run in their default mode, the streams mode (every instance's step
// kernel on one of 16 parallel streams; the persistent mode is lbm_server_set_batch_mode).
// Clients submit and poll from any thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lbm.h"
#include "runtime.h"

using namespace lbm;

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    long long id = 0;
    lbm_request req{};
    lbm_result res{};
    int cls = -1, slot = -1;
    size_t bytes = 0;
    std::vector<double> history;  // kept after completion until released
};

int class_key(const lbm_instance_desc& d) { return (d.lattice * 8 + d.geom.storage) * 2 + d.geom.collision; }

}  // namespace

struct lbm_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int steps_per_round = 64;
    int batch_mode = LBM_BATCH_STREAMS;  // mode of the class batches created from now on
    std::map<int, std::pair<int, int>> class_kernel;  // class -> (variant, segment) set by the client
    std::map<int, lbm_batch*> batches;
    // shared with clients
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job*> incoming;
    std::map<long long, Job*> jobs;  // every job not yet released
    long long next_id = 1;
    bool stop = false;
    int worker_error = 0;
    // worker-only
    std::deque<Job*> waiting;
    std::vector<Job*> running;
    std::thread worker;
    Clock::time_point t0;
    // statistics
    long long rounds = 0, completed = 0;
    double lattice_updates = 0.0, busy_s = 0.0;
    size_t peak_used = 0;
    int peak_running = 0;
};

namespace {

double now_s(const lbm_server* s) {
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// Admit waiting jobs in arrival order while they fit (worker thread).
void admit(lbm_server* s) {
    while (!s->waiting.empty()) {
        Job* j = s->waiting.front();
        if (s->used + j->bytes > s->budget) {
            if (s->running.empty()) {  // nothing will free memory: it can never run
                s->waiting.pop_front();
                std::lock_guard<std::mutex> lk(s->mu);
                j->res.status = LBM_ENOMEM;
                j->res.done_s = now_s(s);
                s->cv_done.notify_all();
                continue;
            }
            break;
        }
        s->waiting.pop_front();
        const int key = class_key(j->req.desc);
        lbm_batch*& b = s->batches[key];
        int rc = LBM_OK;
        if (!b) {
            rc = lbm_batch_create(j->req.desc.lattice, j->req.desc.geom.storage, j->req.desc.geom.collision, s->budget,
                                  &b);
            int mode = LBM_BATCH_STREAMS, variant = -1, segment = 0;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                mode = s->batch_mode;
                auto it = s->class_kernel.find(key);
                if (it != s->class_kernel.end()) {
                    variant = it->second.first;
                    segment = it->second.second;
                }
            }
            if (rc == LBM_OK && mode != LBM_BATCH_STREAMS) rc = lbm_batch_set_mode(b, mode);
            if (rc == LBM_OK && variant >= 0) rc = lbm_batch_set_variant(b, variant);
            if (rc == LBM_OK && segment > 0 && mode == LBM_BATCH_PERSISTENT) rc = lbm_batch_set_segment(b, segment);
            // each class batch keeps its own stream, so that the rounds of different classes
            // (D2Q9 and D2Q37, FP32 and FP16) run at the same time on the GPU
        }
        if (rc == LBM_OK) rc = lbm_batch_add(b, &j->req.desc, &j->slot);
        if (rc != LBM_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            j->res.status = rc;
            j->res.done_s = now_s(s);
            s->cv_done.notify_all();
            continue;
        }
        j->cls = key;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            j->res.status = 1;
            j->res.admit_s = now_s(s);
        }
        s->used += j->bytes;
        s->peak_used = std::max(s->peak_used, s->used);
        s->running.push_back(j);
    }
    s->peak_running = std::max(s->peak_running, (int)s->running.size());
}

// Fit, record and free every running job that has run all its steps (worker thread, after a sync).
void retire(lbm_server* s) {
    std::vector<Job*> still;
    for (Job* j : s->running) {
        lbm_batch* b = s->batches[j->cls];
        long done = 0, total = 0;
        if (lbm_batch_status(b, j->slot, &done, &total) != LBM_OK || done < total) {
            still.push_back(j);
            continue;
        }
        lbm_sim* sim = lbm_batch_instance(b, j->slot);
        j->history.assign(2 * (size_t)total, 0.0);
        size_t n = 0;
        int rc = lbm_force_history(sim, j->history.data(), (size_t)total, &n);
        double fin = 0, fq = 0, f0 = 0, gb = 0;
        if (rc == LBM_OK) rc = lbm_fit(sim, j->req.skip_periods, &fin, &fq, &f0);
        if (rc == LBM_OK && j->req.perimeter > 0 && j->req.desc.geom.u0 > 0)
            rc = lbm_gamma_bar(sim, fin, j->req.perimeter, &gb);
        lbm_info_t info;
        lbm_info(sim, &info);
        lbm_batch_remove(b, j->slot);
        s->used -= j->bytes;
        s->lattice_updates += (double)total * (double)info.n_fluid;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            j->res.f_in = fin;
            j->res.f_q = fq;
            j->res.f_0 = f0;
            j->res.gamma_bar = gb;
            j->res.steps = total;
            j->res.fluid_nodes = info.n_fluid;
            j->res.done_s = now_s(s);
            j->res.status = rc == LBM_OK ? 2 : rc;
            ++s->completed;
            s->cv_done.notify_all();
        }
    }
    s->running.swap(still);
}

void worker_main(lbm_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->running.empty() && s->waiting.empty() && s->incoming.empty() && !s->stop)
                s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            if (s->stop && s->incoming.empty() && s->waiting.empty() && s->running.empty()) break;
            if (s->stop) {  // abandon what is left
                for (Job* j : s->incoming) j->res.status = LBM_EINVAL;
                s->incoming.clear();
            }
            while (!s->incoming.empty()) {
                s->waiting.push_back(s->incoming.front());
                s->incoming.pop_front();
            }
        }
        if (s->stop) {
            if (!s->running.empty()) {
                for (auto& kv : s->batches) lbm_batch_synchronize(kv.second);
                retire(s);
            }
            std::lock_guard<std::mutex> lk(s->mu);
            for (Job* j : s->waiting) j->res.status = LBM_EINVAL;
            for (Job* j : s->running) j->res.status = LBM_EINVAL;
            s->waiting.clear();
            s->running.clear();
            s->cv_done.notify_all();
            break;
        }
        const auto tr = Clock::now();
        bool launched = false;
        for (auto& kv : s->batches) {
            lbm_batch_info_t bi;
            if (lbm_batch_info(kv.second, &bi) == LBM_OK && bi.running > 0) {
                if (lbm_batch_run(kv.second, s->steps_per_round) != LBM_OK) s->worker_error = LBM_ECUDA;
                launched = true;
            }
        }
        admit(s);  // overlaps with the runs just enqueued
        if (launched) {
            for (auto& kv : s->batches) {
                const int rc = lbm_batch_synchronize(kv.second);
                if (rc != LBM_OK) s->worker_error = rc;
            }
            s->busy_s += std::chrono::duration<double>(Clock::now() - tr).count();
            ++s->rounds;
        }
        retire(s);
    }
}

}  // namespace

extern "C" {

int lbm_server_create(size_t device_budget_bytes, int steps_per_round, lbm_server** out) {
    clear_error();
    if (!out) return set_error(LBM_EINVAL, "null output handle");
    *out = nullptr;
    if (steps_per_round < 1) return set_error(LBM_EINVAL, "steps_per_round must be >= 1");
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) return set_error(LBM_ENOMEM, "host allocation");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return set_error(LBM_ECUDA, "no CUDA device");
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return set_error(LBM_ECUDA, "cudaMemGetInfo");
    }
    const size_t margin = (size_t)2 << 30;
    s->budget = device_budget_bytes ? device_budget_bytes : (free_b > margin ? free_b - margin : free_b / 2);
    s->steps_per_round = steps_per_round;
    s->t0 = Clock::now();
    s->worker = std::thread(worker_main, s);
    *out = s;
    return LBM_OK;
}

int lbm_server_submit(lbm_server* s, const lbm_request* req, long long* id) {
    if (!s || !req || !id) return set_error(LBM_EINVAL, "null argument");
    const lbm_instance_desc& d = req->desc;
    if (d.nsteps < 1) return set_error(LBM_EINVAL, "nsteps must be >= 1");
    size_t bytes = 0;
    int rc = lbm_batch_footprint(&d, &bytes);
    if (rc) return rc;
    if (bytes > s->budget) return set_error(LBM_ENOMEM, "request needs %zu bytes, the budget is %zu", bytes, s->budget);
    if (d.geom.kind == LBM_GEOM_MASK)
        return set_error(LBM_EINVAL, "mask geometries are not served (the mask would have to outlive the call)");
    Job* j = new (std::nothrow) Job();
    if (!j) return set_error(LBM_ENOMEM, "host allocation");
    j->req = *req;
    j->bytes = bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete j;
        return set_error(LBM_EINVAL, "server is shutting down");
    }
    j->id = s->next_id++;
    j->res.id = j->id;
    j->res.status = 0;
    j->res.submit_s = now_s(s);
    s->jobs[j->id] = j;
    s->incoming.push_back(j);
    s->cv_work.notify_one();
    *id = j->id;
    return LBM_OK;
}

int lbm_server_set_batch_mode(lbm_server* s, int mode) {
    if (!s) return set_error(LBM_EINVAL, "null server");
    if (mode != LBM_BATCH_STREAMS && mode != LBM_BATCH_PERSISTENT) return set_error(LBM_EINVAL, "bad batch mode");
    std::lock_guard<std::mutex> lk(s->mu);
    s->batch_mode = mode;
    return LBM_OK;
}

int lbm_server_set_class_kernel(lbm_server* s, int lattice, int storage, int collision, int variant, int segment) {
    if (!s) return set_error(LBM_EINVAL, "null server");
    if (variant < -1 || segment < 0) return set_error(LBM_EINVAL, "bad variant or segment");
    lbm_instance_desc d{};
    d.lattice = lattice;
    d.geom.storage = storage;
    d.geom.collision = collision;
    std::lock_guard<std::mutex> lk(s->mu);
    s->class_kernel[class_key(d)] = std::make_pair(variant, segment);
    return LBM_OK;
}

int lbm_server_poll(lbm_server* s, long long id, lbm_result* out) {
    if (!s || !out) return set_error(LBM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return set_error(LBM_ERANGE, "no request %lld", id);
    *out = it->second->res;
    return out->status == 2 || out->status < 0 ? 1 : 0;
}

int lbm_server_wait(lbm_server* s, long long id, double timeout_s, lbm_result* out) {
    if (!s || !out) return set_error(LBM_EINVAL, "null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return set_error(LBM_ERANGE, "no request %lld", id);
    Job* j = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!(j->res.status == 2 || j->res.status < 0)) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout &&
            !(j->res.status == 2 || j->res.status < 0)) {
            *out = j->res;
            return 0;
        }
    }
    *out = j->res;
    return 1;
}

int lbm_server_force_history(lbm_server* s, long long id, double* out_xy, size_t cap_steps, size_t* n_steps) {
    if (!s) return set_error(LBM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return set_error(LBM_ERANGE, "no request %lld", id);
    Job* j = it->second;
    if (j->res.status != 2) return set_error(LBM_EINVAL, "request %lld has not completed", id);
    const size_t n = j->history.size() / 2;
    if (n_steps) *n_steps = n;
    const size_t m = std::min(n, cap_steps);
    if (m && !out_xy) return set_error(LBM_EINVAL, "null output buffer");
    std::copy(j->history.begin(), j->history.begin() + 2 * m, out_xy);
    return LBM_OK;
}

int lbm_server_release(lbm_server* s, long long id) {
    if (!s) return set_error(LBM_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return set_error(LBM_ERANGE, "no request %lld", id);
    if (!(it->second->res.status == 2 || it->second->res.status < 0))
        return set_error(LBM_EINVAL, "request %lld is still in flight", id);
    delete it->second;
    s->jobs.erase(it);
    return LBM_OK;
}

int lbm_server_stats(lbm_server* s, lbm_server_stats_t* o) {
    if (!s || !o) return set_error(LBM_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    o->submitted = s->next_id - 1;
    o->completed = s->completed;
    o->rounds = s->rounds;
    o->lattice_updates = s->lattice_updates;
    o->busy_s = s->busy_s;
    o->elapsed_s = now_s(s);
    o->budget_bytes = s->budget;
    o->used_bytes = s->used;
    o->peak_used_bytes = s->peak_used;
    o->peak_running = s->peak_running;
    o->worker_error = s->worker_error;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->batches) lbm_batch_destroy(kv.second);
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
}

}  // extern "C"
