// Serving: a request loop over one resident graph with continuous batching.
//
// Requests (u, eps) enter a queue.  A scheduler thread forms waves of up to
// max_batch requests and runs each wave as one batched query (the multi-RHS
// path of batch.cu) on its own CUDA stream with its own workspace.  Up to
// max_waves waves are in flight at once, admitted while their workspaces fit the
// device-memory budget; whenever a wave completes, its slot set and memory go to
// the next requests in the queue, so requests that arrive while others are on
// the GPU start as soon as a slot set frees, and the waves' kernels overlap on the
// device.  A request's result does not depend on the wave it lands in (see the
// batch path), so it is the same alone and in any mix.
//
// The scheduler never blocks on the GPU: it polls each wave's completion event.
// All waits a caller can make (esim_server_wait) are bounded by a timeout.
#include "exactsim.h"
#include "internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace esim;

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
    return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

struct Request {
    int64_t u = 0;
    double eps = 0.0;
    int32_t state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    int32_t status = 0;
    std::string error;
    std::vector<int32_t> ids;
    std::vector<double> scores;
    Clock::time_point t_submit, t_start, t_done;
};

struct Wave {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Status* status_d = nullptr;
    Status* status_h = nullptr;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int32_t* ids_h = nullptr;   // pinned, max_batch * k
    double* vals_h = nullptr;
    bool busy = false;
    std::vector<uint64_t> reqs;
};

}  // namespace

struct esim_server {
    Graph* g = nullptr;
    esim_server_config cfg{};
    double budget = 0.0;
    std::mutex mu;
    std::condition_variable cv_done;   // signalled when a request finishes
    std::condition_variable cv_work;   // signalled when work arrives or on stop
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Wave> waves;
    std::thread sched;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    // statistics
    uint64_t completed = 0, failed = 0, waves_launched = 0, batched_requests = 0;
    int32_t max_running = 0, running = 0;
    std::vector<double> latencies;
    std::string fatal;
};

namespace {

void finish_wave(esim_server* s, Wave& w) {
    // called with s->mu held
    const Status hs = *w.status_h;
    const Clock::time_point now = Clock::now();
    const int k = s->cfg.k;
    for (size_t q = 0; q < w.reqs.size(); ++q) {
        auto it = s->reqs.find(w.reqs[q]);
        if (it == s->reqs.end()) continue;
        Request& r = it->second;
        r.t_done = now;
        if (hs.err & kErrBudget) {
            r.state = 3;
            r.status = ESIM_EBUDGET;
            r.error = "pair budget exceeded";
            ++s->failed;
        } else {
            r.ids.assign(w.ids_h + q * k, w.ids_h + (q + 1) * k);
            r.scores.assign(w.vals_h + q * k, w.vals_h + (q + 1) * k);
            r.state = 2;
            r.status = ESIM_OK;
            ++s->completed;
            s->latencies.push_back(ms_since(r.t_submit, r.t_done));
        }
    }
    s->running -= (int32_t)w.reqs.size();
    w.reqs.clear();
    w.busy = false;
}

void fail_requests(esim_server* s, const std::vector<uint64_t>& ids, int status, const std::string& msg) {
    for (uint64_t id : ids) {
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) continue;
        it->second.state = 3;
        it->second.status = status;
        it->second.error = msg;
        it->second.t_done = Clock::now();
        ++s->failed;
    }
}

size_t arenas_in_use(esim_server* s, const Wave* except) {
    size_t t = 0;
    for (auto& w : s->waves)
        if (&w != except) t += w.ws_bytes;
    return t;
}

// Try to start one wave from the queue; returns true if one started.  Called with
// s->mu held; releases it around the (asynchronous) launches.
bool start_wave(esim_server* s, std::unique_lock<std::mutex>& lk) {
    if (s->pending.empty()) return false;
    Wave* w = nullptr;
    for (auto& x : s->waves)
        if (!x.busy) {
            w = &x;
            break;
        }
    if (!w) return false;
    const int maxb = s->cfg.max_batch;
    std::vector<uint64_t> take;
    std::vector<int64_t> us;
    std::vector<double> eps;
    for (uint64_t id : s->pending) {
        if ((int)take.size() == maxb) break;
        const Request& r = s->reqs[id];
        take.push_back(id);
        us.push_back(r.u);
        eps.push_back(r.eps);
    }
    BatchPlan plan;
    Graph& g = *s->g;
    if (batch_plan(g, (int32_t)take.size(), us.data(), eps.data(), s->cfg.c, s->cfg.k, &plan) != ESIM_OK) {
        for (size_t i = 0; i < take.size(); ++i) s->pending.pop_front();
        fail_requests(s, take, ESIM_EINVAL, esim_last_error());
        s->cv_done.notify_all();
        return true;
    }
    const size_t need = batch_ws_bytes(g, plan);
    if (need > w->ws_bytes) {
        // admission by device memory: the new arena must fit the budget with the others
        if ((double)(arenas_in_use(s, w) + need) > s->budget) {
            bool any_busy = false;
            for (auto& x : s->waves) any_busy |= x.busy;
            if (any_busy) return false;  // wait for a wave to free its memory
            if ((double)need > s->budget) {
                for (size_t i = 0; i < take.size(); ++i) s->pending.pop_front();
                fail_requests(s, take, ESIM_ENOMEM, "request batch does not fit the server's memory budget");
                s->cv_done.notify_all();
                return true;
            }
            // nothing is running: release idle arenas to make room
            for (auto& x : s->waves)
                if (&x != w && x.ws) {
                    cudaFree(x.ws);
                    x.ws = nullptr;
                    x.ws_bytes = 0;
                }
        }
        cudaFree(w->ws);
        w->ws = nullptr;
        w->ws_bytes = 0;
        if (cudaMalloc(&w->ws, need) != cudaSuccess) {
            cudaGetLastError();
            bool any_busy = false;
            for (auto& x : s->waves) any_busy |= x.busy;
            if (any_busy) return false;
            for (size_t i = 0; i < take.size(); ++i) s->pending.pop_front();
            fail_requests(s, take, ESIM_ENOMEM, "cudaMalloc(wave workspace)");
            s->cv_done.notify_all();
            return true;
        }
        w->ws_bytes = need;
    }
    for (size_t i = 0; i < take.size(); ++i) s->pending.pop_front();
    const Clock::time_point now = Clock::now();
    for (uint64_t id : take) {
        Request& r = s->reqs[id];
        r.state = 1;
        r.t_start = now;
    }
    w->reqs = take;
    w->busy = true;
    s->running += (int32_t)take.size();
    s->max_running = std::max(s->max_running, s->running);
    ++s->waves_launched;
    s->batched_requests += take.size();
    lk.unlock();
    Graph view = g;  // shares the graph's device arrays; own stream and status block
    view.stream = w->stream;
    view.status = w->status_d;
    view.status_host = w->status_h;
    view.timing = 0;
    int st = batch_enqueue(g, view, plan, w->ws, s->cfg.seed, s->cfg.c, nullptr, nullptr, nullptr, nullptr, w->ids_h,
                           w->vals_h, true);
    cudaError_t e = cudaSuccess;
    if (st == ESIM_OK) e = cudaEventRecord(w->done, w->stream);
    lk.lock();
    if (st != ESIM_OK || e != cudaSuccess) {
        std::string msg = st != ESIM_OK ? std::string(esim_last_error()) : std::string(cudaGetErrorString(e));
        cudaStreamSynchronize(w->stream);
        fail_requests(s, w->reqs, st != ESIM_OK ? st : ESIM_ECUDA, msg);
        s->running -= (int32_t)w->reqs.size();
        w->reqs.clear();
        w->busy = false;
        s->cv_done.notify_all();
    }
    return true;
}

void scheduler(esim_server* s) {
    cudaSetDevice(s->g->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        bool progress = false;
        for (auto& w : s->waves) {
            if (!w.busy) continue;
            const cudaError_t q = cudaEventQuery(w.done);
            if (q == cudaSuccess) {
                finish_wave(s, w);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                fail_requests(s, w.reqs, ESIM_ECUDA, cudaGetErrorString(q));
                s->running -= (int32_t)w.reqs.size();
                w.reqs.clear();
                w.busy = false;
                progress = true;
            }
        }
        if (progress) s->cv_done.notify_all();
        if (s->stop.load()) {
            bool any_busy = false;
            for (auto& w : s->waves) any_busy |= w.busy;
            if (!any_busy) break;
        } else {
            while (start_wave(s, lk)) progress = true;
        }
        if (!progress) {
            bool any_busy = false;
            for (auto& w : s->waves) any_busy |= w.busy;
            // poll in-flight waves every 50 us; sleep until work arrives otherwise
            if (any_busy) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

void release_server(esim_server* s) {
    for (auto& w : s->waves) {
        if (w.stream) cudaStreamSynchronize(w.stream);
        if (w.done) cudaEventDestroy(w.done);
        if (w.stream) cudaStreamDestroy(w.stream);
        cudaFree(w.status_d);
        cudaFree(w.ws);
        if (w.status_h) cudaFreeHost(w.status_h);
        if (w.ids_h) cudaFreeHost(w.ids_h);
        if (w.vals_h) cudaFreeHost(w.vals_h);
    }
    s->waves.clear();
}

}  // namespace

extern "C" {

esim_status esim_server_create(esim_graph* gh, const esim_server_config* cfg, esim_server** out) {
    if (!out) return (esim_status)set_error(ESIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!gh || !cfg) return (esim_status)set_error(ESIM_EINVAL, "NULL graph or config");
    if (!(cfg->c > 0.0 && cfg->c < 1.0)) return (esim_status)set_error(ESIM_EINVAL, "need 0 < c < 1");
    if (cfg->k < 1 || cfg->k > kTopkMax) return (esim_status)set_error(ESIM_EINVAL, "need 1 <= k <= 4096");
    if (cfg->max_batch < 1 || cfg->max_batch > kBatchMax)
        return (esim_status)set_error(ESIM_EINVAL, "need 1 <= max_batch <= 64");
    if (cfg->max_waves < 1 || cfg->max_waves > 8) return (esim_status)set_error(ESIM_EINVAL, "need 1 <= max_waves <= 8");
    Graph* g = graph_of(gh);
    if (cudaSetDevice(g->device) != cudaSuccess) return (esim_status)set_error(ESIM_ECUDA, "cudaSetDevice");
    esim_server* s = new (std::nothrow) esim_server();
    if (!s) return (esim_status)set_error(ESIM_ENOMEM, "host allocation");
    s->g = g;
    s->cfg = *cfg;
    if (cfg->kappa != 0.0) g->kappa = cfg->kappa;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = cfg->mem_budget_bytes > 0.0 ? cfg->mem_budget_bytes : 0.8 * (double)free_b;
    s->waves.resize((size_t)cfg->max_waves);
    for (auto& w : s->waves) {
        const size_t outs = (size_t)cfg->max_batch * (size_t)cfg->k;
        bool ok = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc((void**)&w.status_d, sizeof(Status)) == cudaSuccess &&
                  cudaMallocHost((void**)&w.status_h, sizeof(Status)) == cudaSuccess &&
                  cudaMallocHost((void**)&w.ids_h, sizeof(int32_t) * outs) == cudaSuccess &&
                  cudaMallocHost((void**)&w.vals_h, sizeof(double) * outs) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            release_server(s);
            delete s;
            return (esim_status)set_error(ESIM_ENOMEM, "server stream/buffer allocation");
        }
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    return ESIM_OK;
}

esim_status esim_server_submit(esim_server* s, int64_t u, double eps, uint64_t* id_out) {
    if (!s || !id_out) return (esim_status)set_error(ESIM_EINVAL, "NULL argument");
    if (u < 0 || u >= s->g->n) return (esim_status)set_error(ESIM_EINVAL, "source node out of range");
    if (!(eps > 0.0 && eps < 1.0)) return (esim_status)set_error(ESIM_EINVAL, "need 0 < eps < 1");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop.load()) return (esim_status)set_error(ESIM_EINVAL, "server is shutting down");
        const uint64_t id = s->next_id++;
        Request& r = s->reqs[id];
        r.u = u;
        r.eps = eps;
        r.t_submit = Clock::now();
        s->pending.push_back(id);
        *id_out = id;
    }
    s->cv_work.notify_one();
    return ESIM_OK;
}

esim_status esim_server_poll(esim_server* s, uint64_t id, int32_t* state) {
    if (!s || !state) return (esim_status)set_error(ESIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return (esim_status)set_error(ESIM_EINVAL, "unknown request id");
    *state = it->second.state;
    return ESIM_OK;
}

esim_status esim_server_wait(esim_server* s, uint64_t id, int32_t timeout_ms, int32_t* ids_out, double* scores_out,
                             double* latency_ms) {
    if (!s) return (esim_status)set_error(ESIM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return (esim_status)set_error(ESIM_EINVAL, "unknown request id");
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (it->second.state < 2) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && it->second.state < 2)
            return (esim_status)set_error(ESIM_ETIMEOUT, "request not finished within the timeout");
        it = s->reqs.find(id);
        if (it == s->reqs.end()) return (esim_status)set_error(ESIM_EINVAL, "request vanished");
    }
    Request& r = it->second;
    if (r.state == 3) {
        const std::string msg = r.error;
        const int st = r.status;
        s->reqs.erase(it);
        return (esim_status)set_error(st, msg);
    }
    if (ids_out) std::copy(r.ids.begin(), r.ids.end(), ids_out);
    if (scores_out) std::copy(r.scores.begin(), r.scores.end(), scores_out);
    if (latency_ms) *latency_ms = ms_since(r.t_submit, r.t_done);
    s->reqs.erase(it);
    return ESIM_OK;
}

esim_status esim_server_get_stats(esim_server* s, esim_server_stats* out) {
    if (!s || !out) return (esim_status)set_error(ESIM_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = esim_server_stats{};
    out->completed = s->completed;
    out->failed = s->failed;
    out->waves = s->waves_launched;
    out->mean_batch = s->waves_launched ? (double)s->batched_requests / (double)s->waves_launched : 0.0;
    out->max_running = s->max_running;
    out->queued = (int32_t)s->pending.size();
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
    }
    return ESIM_OK;
}

void esim_server_destroy(esim_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
        // queued requests are cancelled; running waves finish
        std::vector<uint64_t> q(s->pending.begin(), s->pending.end());
        s->pending.clear();
        fail_requests(s, q, ESIM_EINVAL, "server destroyed before the request ran");
    }
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    s->cv_done.notify_all();
    release_server(s);
    delete s;
}

}  // extern "C"
