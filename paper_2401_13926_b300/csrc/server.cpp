// Serving runtime: many resident KKT sequences ("instances") on one GPU,
// their refactor + solve steps in flight together.
//
// The method solves a sequence of same-pattern KKT systems reusing the
// analysis, the factor storage and the Krylov space (Sections 2.1, 3.1.1);
// one such sequence keeps only part of a B300 busy (its refactorization and
// triangular solves are chains of dependent rows).  This runtime keeps many
// instances resident and lets their steps overlap: every instance is a
// context with its own stream, and a pool of worker threads takes instances
// that have a queued step and are not running one, runs that step (a
// blocking kkt_step -- refactor + solve -- on the instance's stream), and re-queues
// the instance if more steps wait.  Steps of one instance run one at a time,
// in submission order; steps of different instances run concurrently.
// Admission holds the device memory of the admitted instances within a
// budget.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "kkt.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Step {
    int64_t ticket = 0;
    std::vector<double> values, b;
    double* x = nullptr;
    double tol = 0.0;
    Clock::time_point submitted;
};

struct Instance {
    int64_t id = 0;
    kkt_ctx* ctx = nullptr;
    int32_t n = 0;
    int64_t nnz = 0;
    int64_t bytes = 0;
    std::deque<Step> pending;
    bool running = false;    // a worker holds this instance
    bool queued = false;     // in the ready queue
    bool closing = false;
};

struct Done {
    bool finished = false;
    kkt_step_result r{};
};

}  // namespace

struct kkt_server {
    kkt_server_opts o{};
    int dev = 0;
    int64_t budget = 0;
    int64_t held = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // workers: a ready instance or stop
    std::condition_variable cv_done;   // waiters: a step finished
    std::unordered_map<int64_t, std::unique_ptr<Instance>> inst;
    std::deque<Instance*> ready;
    std::unordered_map<int64_t, Done> done;
    int64_t next_id = 1, next_ticket = 1;
    int64_t submitted = 0, completed = 0;
    int in_flight = 0;
    bool stop = false;
    std::vector<std::thread> workers;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// refactor + solve as one kkt_step (the forward sweep fused into the
// refactorization; same results as the two calls)
void run_step(kkt_server* s, Instance* in, Step& st, kkt_step_result* r) {
    cudaSetDevice(s->dev);
    int it = 0;
    double nr = 0.0;
    r->status = kkt_step(in->ctx, st.values.data(), st.b.data(), st.x, 0, st.tol, &it, &nr);
    r->iters = it;
    r->nrbe = nr;
}

void worker_main(kkt_server* s) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->ready.empty(); });
        if (s->ready.empty()) {
            if (s->stop) return;
            continue;
        }
        Instance* in = s->ready.front();
        s->ready.pop_front();
        in->queued = false;
        in->running = true;
        Step st = std::move(in->pending.front());
        in->pending.pop_front();
        s->in_flight++;
        lk.unlock();
        kkt_step_result r{};
        const auto t0 = Clock::now();
        r.queue_ms = ms_between(st.submitted, t0);
        run_step(s, in, st, &r);
        r.run_ms = ms_between(t0, Clock::now());
        lk.lock();
        s->in_flight--;
        s->completed++;
        Done& d = s->done[st.ticket];
        d.finished = true;
        d.r = r;
        in->running = false;
        if (!in->pending.empty() && !in->queued) {
            in->queued = true;
            s->ready.push_back(in);
            s->cv_work.notify_one();
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

void kkt_server_default_opts(kkt_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->workers = 8;
    o->hbm_budget = 0;
    kkt_default_opts(&o->opts);
}

int kkt_server_create(kkt_server** out, const kkt_server_opts* o) {
    if (!out) return KKT_ERR_INVALID;
    *out = nullptr;
    kkt_server_opts opts;
    if (o) opts = *o;
    else kkt_server_default_opts(&opts);
    if (opts.workers < 1 || opts.workers > 256 || opts.hbm_budget < 0) return KKT_ERR_INVALID;
    auto* s = new kkt_server();
    s->o = opts;
    s->o.opts.create_stream = 1;
    s->o.opts.stream = nullptr;
    s->dev = opts.opts.device;
    if (cudaSetDevice(s->dev) != cudaSuccess) { delete s; return KKT_ERR_CUDA; }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { delete s; return KKT_ERR_CUDA; }
    s->budget = opts.hbm_budget > 0 ? opts.hbm_budget : (int64_t)(0.9 * (double)free_b);
    for (int i = 0; i < opts.workers; i++) s->workers.emplace_back(worker_main, s);
    *out = s;
    return KKT_OK;
}

int kkt_server_open(kkt_server* s, int32_t n, const int32_t* rowptr, const int32_t* colind,
                    const double* values0, int64_t* instance) {
    if (!s || !instance) return KKT_ERR_INVALID;
    *instance = 0;
    cudaSetDevice(s->dev);
    kkt_ctx* c = nullptr;
    int rc = kkt_create(&c, &s->o.opts);
    if (rc) return rc;
    rc = kkt_analyze(c, n, rowptr, colind, values0, nullptr, nullptr);
    if (rc) { kkt_destroy(c); return rc; }
    kkt_info info;
    kkt_query(c, &info);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->held + info.device_bytes > s->budget) {   // admission by device memory
        kkt_destroy(c);
        return KKT_ERR_OOM;
    }
    auto in = std::make_unique<Instance>();
    in->id = s->next_id++;
    in->ctx = c;
    in->n = n;
    in->nnz = info.nnz_a;
    in->bytes = info.device_bytes;
    s->held += in->bytes;
    *instance = in->id;
    s->inst[in->id] = std::move(in);
    return KKT_OK;
}

int kkt_server_submit(kkt_server* s, int64_t instance, const double* values, const double* b, double* x,
                      double tol, int64_t* ticket) {
    if (!s || !values || !b || !x || !ticket || !(tol > 0)) return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->inst.find(instance);
    if (it == s->inst.end() || it->second->closing) return KKT_ERR_INVALID;
    Instance* in = it->second.get();
    Step st;
    st.ticket = s->next_ticket++;
    st.values.assign(values, values + in->nnz);
    st.b.assign(b, b + in->n);
    st.x = x;
    st.tol = tol;
    st.submitted = Clock::now();
    *ticket = st.ticket;
    s->done[st.ticket] = Done{};
    in->pending.push_back(std::move(st));
    s->submitted++;
    if (!in->running && !in->queued) {
        in->queued = true;
        s->ready.push_back(in);
        s->cv_work.notify_one();
    }
    return KKT_OK;
}

int kkt_server_wait(kkt_server* s, int64_t ticket, kkt_step_result* r) {
    if (!s || !r) return KKT_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return KKT_ERR_INVALID;
    s->cv_done.wait(lk, [&] { return s->done[ticket].finished; });
    *r = s->done[ticket].r;
    s->done.erase(ticket);
    return KKT_OK;
}

int kkt_server_close(kkt_server* s, int64_t instance) {
    if (!s) return KKT_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->inst.find(instance);
    if (it == s->inst.end()) return KKT_ERR_INVALID;
    Instance* in = it->second.get();
    in->closing = true;
    s->cv_done.wait(lk, [&] { return in->pending.empty() && !in->running && !in->queued; });
    kkt_ctx* c = in->ctx;
    s->held -= in->bytes;
    s->inst.erase(it);
    lk.unlock();
    cudaSetDevice(s->dev);
    kkt_destroy(c);
    return KKT_OK;
}

int kkt_server_query(kkt_server* s, kkt_server_info* info) {
    if (!s || !info) return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    info->instances = (int32_t)s->inst.size();
    info->device_bytes = s->held;
    info->hbm_budget = s->budget;
    info->submitted = s->submitted;
    info->completed = s->completed;
    info->in_flight = s->in_flight;
    return KKT_OK;
}

void kkt_server_destroy(kkt_server* s) {
    if (!s) return;
    std::vector<int64_t> ids;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& kv : s->inst) ids.push_back(kv.first);
    }
    for (int64_t id : ids) kkt_server_close(s, id);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

}  // extern "C"
