/*
 * usr_server.cpp -- continuous batching of independent u-series evaluations
 * (the serving form; the paper itself evaluates one system at a time).
 *
 * Requests (one periodic system each: box, grid, cutoff, preset, charges in
 * host memory) are queued by usr_server_submit from any host thread.  A
 * worker thread admits them in arrival order onto slots; a slot is a context
 * (usr_ctx, its cell list, grids and tables resident on the device) plus its
 * own CUDA stream.  Admission needs a free slot and room in the device-memory
 * budget: a slot's context is re-targeted to the request with usr_reconfigure
 * (which reuses its buffers, allocating only when the request is larger than
 * anything the slot held before), and the bytes all slots hold may not exceed
 * the budget.  Requests that arrive while others run are admitted as soon as
 * a slot and memory free up, so evaluations of different systems overlap on
 * the device.  Each admitted request is enqueued on its slot's stream as host
 * -> device copy, the evaluation, device -> host copies, and an event;
 * completion is detected by polling the event, and the latency (submit to
 * results in host memory) is recorded.
 */
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
#include <vector>

#include "usr_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long ticket;
    usr_params params;
    std::shared_ptr<usr::Plan> plan;     // made by the worker at admission
    double need = 0.0;                   // device bytes of a fresh context for it
    int n;
    const float* xyzq;
    float* out;
    double* energy;
    Clock::time_point t_submit;
};

struct Slot {
    usr_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    double bytes = 0.0;          // device bytes the slot's context holds (it only grows)
    Request req;
};

struct Done {
    long long ticket;
    double latency_ms;
    usr_status status;
};

}  // namespace

struct usr_server {
    usr_server_params prm;
    int device = 0;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::vector<Done> done;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    std::atomic<bool> stop{false};
    long long next_ticket = 0;
    long long completed = 0;
    long long submitted = 0;
    double held_bytes = 0.0;
    usr_status first_error = USR_OK;
};

namespace {

/* Enqueue a request on a free slot (worker thread; the queue lock is not held). */
usr_status launch(usr_server* s, Slot& sl, const Request& r)
{
    usr_status st;
    if (!sl.ctx) {
        if ((st = usr_init(&r.params, &sl.ctx)) != USR_OK) return st;
    } else if ((st = usr::reconfigure_with_plan(sl.ctx, *r.plan, sl.st)) != USR_OK) {
        return st;
    }
    usr_plan_info info;
    usr_info(sl.ctx, &info);
    sl.bytes = std::max(sl.bytes, info.device_bytes);
    if (r.n > 0 && (st = usr_eval_host_async(sl.ctx, r.n, r.xyzq, r.out, r.energy, sl.st)) != USR_OK) return st;
    if (r.n == 0 && r.energy) std::memset(r.energy, 0, 4 * sizeof(double));
    if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return USR_ERR_CUDA;
    sl.req = r;
    sl.busy = true;
    return USR_OK;
}

/* Plan a queued request once (the worker keeps the plan with the request). */
void plan_request(Request& r)
{
    if (r.plan) return;
    r.plan = std::make_shared<usr::Plan>();
    r.need = usr::make_plan(&r.params, r.plan.get()) == USR_OK ? usr::plan_device_bytes(*r.plan) : -1.0;
}

/* Free the contexts of idle slots (all but `keep`): the only way held memory shrinks. */
void release_idle(usr_server* s, int keep)
{
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot& sl = s->slots[i];
        if ((int)i == keep || sl.busy || !sl.ctx) continue;
        usr_destroy(sl.ctx);
        sl.ctx = nullptr;
        sl.bytes = 0.0;
    }
}

void worker_loop(usr_server* s)
{
    cudaSetDevice(s->device);
    const double budget = s->prm.hbm_budget_bytes;
    while (true) {
        bool progressed = false;
        // completions
        for (auto& sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            usr_status st = q == cudaSuccess ? usr_last_device_status(sl.ctx) : USR_ERR_CUDA;
            if (q != cudaSuccess) cudaGetLastError();
            const double ms = std::chrono::duration<double, std::milli>(Clock::now() - sl.req.t_submit).count();
            std::lock_guard<std::mutex> lk(s->mu);
            s->done.push_back({sl.req.ticket, ms, st});
            ++s->completed;
            sl.busy = false;
            progressed = true;
            s->cv.notify_all();
        }
        // admissions, in arrival order
        while (true) {
            Request r;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->queue.empty()) break;
                if (s->stop) {                                     // shutting down: cancel what waits
                    for (const auto& q : s->queue) s->done.push_back({q.ticket, 0.0, USR_ERR_ARG});
                    s->completed += (long long)s->queue.size();
                    s->queue.clear();
                    s->cv.notify_all();
                    break;
                }
                plan_request(s->queue.front());
                r = s->queue.front();
            }
            const double need = r.need;
            // a free slot, preferring the one holding the most (its buffers are the likeliest to fit)
            int best = -1;
            for (size_t i = 0; i < s->slots.size(); ++i) {
                const Slot& sl = s->slots[i];
                if (sl.busy) continue;
                if (best < 0 || sl.bytes > s->slots[best].bytes) best = (int)i;
            }
            if (best < 0) break;                                   // no free slot
            // a slot re-targeted to the request holds at most its current bytes plus the request's
            // own need (buffers grow to the larger of the two), so admit only if that fits
            double held = 0.0;
            bool any_busy = false;
            for (const auto& sl : s->slots) {
                held += sl.bytes;
                any_busy = any_busy || sl.busy;
            }
            double best_growth = need;
            if (need >= 0.0 && need <= budget && held + best_growth > budget && !any_busy) {
                // nothing runs, so waiting frees nothing: release idle slots, then if needed the chosen one
                release_idle(s, best);
                held = s->slots[best].bytes;
                if (held + best_growth > budget) {
                    release_idle(s, -1);
                    held = 0.0;
                }
            }
            if (need < 0.0 || need > budget || held + best_growth > budget) {
                if (need >= 0.0 && need <= budget) break;          // wait for memory
                std::lock_guard<std::mutex> lk(s->mu);             // can never fit: fail it
                s->queue.pop_front();
                s->done.push_back({r.ticket, 0.0, need < 0.0 ? USR_ERR_BOX : USR_ERR_OOM});
                ++s->completed;
                s->cv.notify_all();
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(s->mu);
                s->queue.pop_front();
            }
            Slot& sl = s->slots[best];
            const usr_status st = launch(s, sl, r);
            held = 0.0;
            for (const auto& x : s->slots) held += x.bytes;
            std::lock_guard<std::mutex> lk(s->mu);
            s->held_bytes = held;
            if (st != USR_OK) {
                if (s->first_error == USR_OK) s->first_error = st;
                s->done.push_back({r.ticket, 0.0, st});
                ++s->completed;
                sl.busy = false;
                s->cv.notify_all();
            }
            progressed = true;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop && s->queue.empty()) {
            bool any = false;
            for (const auto& sl : s->slots) any = any || sl.busy;
            if (!any) break;
        }
        if (!progressed) s->cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" usr_status usr_server_create(const usr_server_params* p, usr_server** out)
{
    if (!out) return USR_ERR_ARG;
    *out = nullptr;
    usr_server* s = new (std::nothrow) usr_server();
    if (!s) return USR_ERR_OOM;
    if (p) s->prm = *p;
    else std::memset(&s->prm, 0, sizeof(s->prm));
    if (s->prm.slots <= 0) s->prm.slots = 8;
    if (s->prm.slots > 64 || s->prm.hbm_budget_bytes < 0.0) {
        delete s;
        return USR_ERR_ARG;
    }
    if (s->prm.hbm_budget_bytes == 0.0) s->prm.hbm_budget_bytes = 16.0 * (1ull << 30);
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return USR_ERR_CUDA;
    }
    s->slots.resize(s->prm.slots);
    for (auto& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            usr_server_destroy(s);
            return USR_ERR_CUDA;
        }
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return USR_OK;
}

extern "C" usr_status usr_server_submit(usr_server* s, const usr_params* p, int n, const float* xyzq, float* out,
                                        double* energy, long long* ticket)
{
    if (!s || !p || n < 0 || (n > 0 && (!xyzq || !out)) || n > p->max_atoms) return USR_ERR_ARG;
    Request r;
    r.params = *p;
    r.n = n;
    r.xyzq = xyzq;
    r.out = out;
    r.energy = energy;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return USR_ERR_ARG;
        r.ticket = s->next_ticket++;
        ++s->submitted;
        s->queue.push_back(r);
    }
    s->cv.notify_all();
    if (ticket) *ticket = r.ticket;
    return USR_OK;
}

extern "C" int usr_server_poll(usr_server* s, long long* tickets, double* latency_ms, int* status, int max)
{
    if (!s || max <= 0) return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    const int k = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < k; ++i) {
        if (tickets) tickets[i] = s->done[i].ticket;
        if (latency_ms) latency_ms[i] = s->done[i].latency_ms;
        if (status) status[i] = s->done[i].status;
    }
    s->done.erase(s->done.begin(), s->done.begin() + k);
    return k;
}

extern "C" usr_status usr_server_wait(usr_server* s, double timeout_s)
{
    if (!s) return USR_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    while (s->completed < s->submitted) {
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout && s->completed < s->submitted)
            return USR_ERR_TIMEOUT;
    }
    return s->first_error;
}

extern "C" usr_status usr_server_info(usr_server* s, double* held_bytes, long long* queued, long long* in_flight)
{
    if (!s) return USR_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (held_bytes) *held_bytes = s->held_bytes;
    if (queued) *queued = (long long)s->queue.size();
    if (in_flight) *in_flight = s->submitted - s->completed - (long long)s->queue.size();
    return USR_OK;
}

extern "C" void usr_server_destroy(usr_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ctx) usr_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete s;
}
