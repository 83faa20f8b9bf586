/*
 * usr_server.cpp -- continuous batching of independent u-series evaluations
 * (the serving form; the paper itself evaluates one system at a time).
 *
 * Requests (one periodic system each: box, grid, cutoff, preset, charges in
 * host memory) are queued by usr_server_submit from any host thread.  Every
 * slot -- a context (usr_ctx: cell list, grids and tables resident on the
 * device) with its own CUDA stream -- is served by its own host thread, which
 * takes the next request in arrival order as soon as its slot is free, makes
 * the request's FP64 plan, waits for room in the device-memory budget,
 * re-targets its context to the request with usr_reconfigure (which reuses
 * its buffers, allocating only when the request is larger than anything the
 * slot held before), enqueues host -> device copy, evaluation and device ->
 * host copies on its stream, and waits for them.  The host work of different
 * requests (planning, table uploads, launches) therefore runs in parallel on
 * the host cores, and their device work overlaps on the GPU.  The latency of a
 * request is measured from submission to results in host memory.
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
    std::shared_ptr<usr::Plan> plan;     // made by the slot's thread after it takes the request
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
    bool busy = false;           // a request is being prepared or evaluated on it
    bool admitted = false;       // its request has its memory reserved and is being evaluated
    double bytes = 0.0;          // device bytes the slot's context holds or has reserved (it only grows)
    std::thread th;
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
    bool stop = false;
    int admitted = 0;            // slots whose request passed admission and is being evaluated
    long long next_ticket = 0;
    long long completed = 0;
    long long submitted = 0;
    double held_bytes = 0.0;
    usr_status first_error = USR_OK;
};

namespace {

/* Re-target the slot's context to the request and enqueue its evaluation (no server lock held). */
usr_status launch(Slot& sl, const Request& r)
{
    usr_status st;
    if (!sl.ctx) {
        if ((st = usr_init(&r.params, &sl.ctx)) != USR_OK) return st;
    } else if ((st = usr::reconfigure_with_plan(sl.ctx, *r.plan, sl.st)) != USR_OK) {
        return st;
    }
    if (r.n > 0 && (st = usr_eval_host_async(sl.ctx, r.n, r.xyzq, r.out, r.energy, sl.st)) != USR_OK) return st;
    if (r.n == 0 && r.energy) std::memset(r.energy, 0, 4 * sizeof(double));
    if (cudaEventRecord(sl.done, sl.st) != cudaSuccess) return USR_ERR_CUDA;
    return USR_OK;
}

/* Plan a request (the slot thread's host work before admission): need = -1 for parameters the plan
   refuses, -2 when the host ran out of memory planning it. */
void plan_request(Request& r)
{
    if (r.plan) return;
    const usr_status st = usr::guard([&] {
        r.plan = std::make_shared<usr::Plan>();
        return usr::make_plan(&r.params, r.plan.get());
    });
    r.need = st == USR_OK ? usr::plan_device_bytes(*r.plan) : (st == USR_ERR_OOM ? -2.0 : -1.0);
}

double held(const usr_server* s)
{
    double h = 0.0;
    for (const auto& sl : s->slots) h += sl.bytes;
    return h;
}

/*
 * Free the contexts of slots other than `keep` that evaluate nothing (idle, or holding a request that
 * still waits for admission: such a slot touches its context only once admitted); lock held.  This is
 * the only way held memory shrinks.
 */
void release_idle(usr_server* s, int keep)
{
    for (size_t i = 0; i < s->slots.size(); ++i) {
        Slot& sl = s->slots[i];
        if ((int)i == keep || sl.admitted || !sl.ctx) continue;
        usr_destroy(sl.ctx);
        sl.ctx = nullptr;
        sl.bytes = 0.0;
    }
}

void slot_loop(usr_server* s, int idx)
{
    cudaSetDevice(s->device);
    Slot& sl = s->slots[idx];
    const double budget = s->prm.hbm_budget_bytes;
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
        if (s->stop) {                                       // shutting down: cancel what waits
            for (const auto& q : s->queue) s->done.push_back({q.ticket, 0.0, USR_ERR_ARG});
            s->completed += (long long)s->queue.size();
            s->queue.clear();
            s->cv.notify_all();
            break;
        }
        Request r = s->queue.front();                        // arrival order
        s->queue.pop_front();
        sl.busy = true;
        lk.unlock();
        plan_request(r);                                     // in parallel with the other slots
        lk.lock();
        // admission by memory: re-targeted to r, the slot holds at most max(its bytes, r's need)
        usr_status st = r.need == -2.0 ? USR_ERR_OOM
                        : (r.need < 0.0 ? USR_ERR_BOX : (r.need > budget ? USR_ERR_OOM : USR_OK));
        while (st == USR_OK) {
            const double after = held(s) - sl.bytes + std::max(sl.bytes, r.need);
            if (after <= budget) break;
            if (s->admitted == 0) {
                // nothing is evaluated, so waiting frees nothing: release the other slots' contexts,
                // then if needed this one
                release_idle(s, idx);
                if (held(s) - sl.bytes + std::max(sl.bytes, r.need) > budget && sl.ctx) {
                    usr_destroy(sl.ctx);
                    sl.ctx = nullptr;
                    sl.bytes = 0.0;
                }
                continue;
            }
            s->cv.wait(lk);                                  // until another request completes
        }
        if (st == USR_OK) {
            sl.bytes = std::max(sl.bytes, r.need);           // reserved before the lock is released
            sl.admitted = true;
            ++s->admitted;
        }
        lk.unlock();
        usr_status lst = USR_OK;
        if (st == USR_OK) {
            lst = launch(sl, r);
            st = lst;
            if (st == USR_OK) {
                st = cudaEventSynchronize(sl.done) == cudaSuccess ? usr_last_device_status(sl.ctx) : USR_ERR_CUDA;
                if (st == USR_ERR_CUDA) cudaGetLastError();
            }
        }
        const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r.t_submit).count();
        double ctx_bytes = 0.0;
        if (sl.ctx) {
            usr_plan_info info;
            if (usr_info(sl.ctx, &info) == USR_OK) ctx_bytes = info.device_bytes;
        }
        lk.lock();
        sl.bytes = sl.ctx ? std::max(sl.bytes, ctx_bytes) : 0.0;
        s->held_bytes = held(s);
        if (lst != USR_OK && s->first_error == USR_OK) s->first_error = lst;
        s->done.push_back({r.ticket, ms, st});
        ++s->completed;
        if (sl.admitted) --s->admitted;
        sl.admitted = false;
        sl.busy = false;
        s->cv.notify_all();
    }
}

}  // namespace

extern "C" usr_status usr_server_create(const usr_server_params* p, usr_server** out)
{
    if (!out) return USR_ERR_ARG;
    *out = nullptr;
    usr_server* s = nullptr;
    try {
        s = new usr_server();
    } catch (...) {
        return USR_ERR_OOM;
    }
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
    if (usr::guard([&] {
            s->slots.resize(s->prm.slots);
            return USR_OK;
        }) != USR_OK) {
        delete s;
        return USR_ERR_OOM;
    }
    for (auto& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            usr_server_destroy(s);
            return USR_ERR_CUDA;
        }
    }
    for (int i = 0; i < (int)s->slots.size(); ++i) {
        try {
            s->slots[i].th = std::thread(slot_loop, s, i);
        } catch (...) {                      // no thread could be started: stop the ones that were
            usr_server_destroy(s);
            return USR_ERR_OOM;
        }
    }
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
        const usr_status st = usr::guard([&] {
            s->queue.push_back(r);
            return USR_OK;
        });
        if (st != USR_OK) return st;
        r.ticket = s->next_ticket++;
        s->queue.back().ticket = r.ticket;
        ++s->submitted;
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
    for (auto& sl : s->slots)
        if (sl.th.joinable()) sl.th.join();
    for (auto& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ctx) usr_destroy(sl.ctx);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete s;
}
