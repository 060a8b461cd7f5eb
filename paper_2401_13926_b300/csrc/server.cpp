// Serving runtime: many resident KKT sequences ("instances") on one or more
// GPUs, their refactor + solve steps in flight together.
//
// The method solves a sequence of same-pattern KKT systems reusing the
// analysis, the factor storage and the Krylov space (Sections 2.1, 3.1.1);
// one such sequence keeps only part of a B300 busy (its refactorization and
// triangular solves are chains of dependent rows).  This runtime keeps many
// instances resident, each a context with its own stream placed whole on
// one device, and runs their steps together:
//   - batch > 0 (continuous batching): one dispatcher thread per device
//     takes up to `batch` instances that have a queued step and are not
//     running one, runs those steps as one kkt_batch_step (shared launches),
//     and re-queues instances with more steps; steps submitted while a batch
//     runs join the next one;
//   - batch == 0: a pool of workers runs each step as its own kkt_step.
// Steps of one instance run one at a time, in submission order.
// Admission: the host analysis runs in the opening thread (off the GPU
// path); the instance is placed on the device with the most budget left
// and waits, first come first served per device, until its device memory
// fits that device's budget.
#include <algorithm>
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
    int slot = 0;            // index of its device in the server's device list
    kkt_ctx* ctx = nullptr;
    int32_t n = 0;
    int64_t nnz = 0;
    int64_t bytes = 0;
    std::deque<Step> pending;
    bool running = false;    // a worker or dispatcher holds this instance
    bool queued = false;     // in a ready queue
    bool closing = false;
};

struct Done {
    bool finished = false;
    kkt_step_result r{};
};

struct DeviceSlot {
    int dev = 0;
    int64_t budget = 0;
    int64_t held = 0;        // admitted instances
    int64_t reserved = 0;    // opens waiting for admission (placement counts them)
    std::deque<int64_t> admit;   // waiting opens, first come first served
    std::deque<Instance*> ready; // instances with a queued step (batch mode)
    kkt_batch* batch = nullptr;
};

}  // namespace

struct kkt_server {
    kkt_server_opts o{};
    std::vector<DeviceSlot> slots;
    std::mutex mu;
    std::condition_variable cv_work;    // workers / dispatchers: a ready instance or stop
    std::condition_variable cv_done;    // waiters: a step finished
    std::condition_variable cv_admit;   // opens: device memory freed
    std::unordered_map<int64_t, std::unique_ptr<Instance>> inst;
    std::deque<Instance*> ready;        // batch == 0: every device's ready instances
    std::unordered_map<int64_t, Done> done;
    int64_t next_id = 1, next_ticket = 1, next_admit = 1;
    int64_t submitted = 0, completed = 0, batches = 0;
    int in_flight = 0, waiting = 0;
    bool stop = false;
    std::vector<std::thread> threads;
};

namespace {

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// The instance's next step is finished: record it and re-queue the instance
// if more steps wait.  Called with the lock held.
void finish_step(kkt_server* s, Instance* in, int64_t ticket, const kkt_step_result& r) {
    s->in_flight--;
    s->completed++;
    Done& d = s->done[ticket];
    d.finished = true;
    d.r = r;
    in->running = false;
    if (!in->pending.empty() && !in->queued) {
        in->queued = true;
        if (s->o.batch > 0) s->slots[in->slot].ready.push_back(in);
        else s->ready.push_back(in);
        s->cv_work.notify_all();
    }
    s->cv_done.notify_all();
}

// batch == 0: one step per worker, as its own kkt_step
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
        const int dev = s->slots[in->slot].dev;
        lk.unlock();
        kkt_step_result r{};
        const auto t0 = Clock::now();
        r.queue_ms = ms_between(st.submitted, t0);
        cudaSetDevice(dev);
        int it = 0;
        double nr = 0.0;
        r.status = kkt_step(in->ctx, st.values.data(), st.b.data(), st.x, 0, st.tol, &it, &nr);
        r.iters = it;
        r.nrbe = nr;
        r.run_ms = ms_between(t0, Clock::now());
        r.batch_size = 1;
        r.device = dev;
        lk.lock();
        finish_step(s, in, st.ticket, r);
    }
}

// batch > 0: the dispatcher of one device -- up to `batch` ready instances'
// next steps as one kkt_batch_step
void dispatcher_main(kkt_server* s, int slot_index) {
    DeviceSlot& slot = s->slots[slot_index];
    std::unique_lock<std::mutex> lk(s->mu);
    std::vector<Instance*> ins;
    std::vector<Step> steps;
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || !slot.ready.empty(); });
        if (slot.ready.empty()) {
            if (s->stop) return;
            continue;
        }
        ins.clear();
        steps.clear();
        while (!slot.ready.empty() && (int)ins.size() < s->o.batch) {
            Instance* in = slot.ready.front();
            slot.ready.pop_front();
            in->queued = false;
            in->running = true;
            steps.push_back(std::move(in->pending.front()));
            in->pending.pop_front();
            ins.push_back(in);
        }
        // one tolerance per call: steps with another tolerance wait for the next batch
        const double tol = steps[0].tol;
        for (size_t i = ins.size(); i-- > 1;) {
            if (steps[i].tol != tol) {
                ins[i]->pending.push_front(std::move(steps[i]));
                ins[i]->running = false;
                ins[i]->queued = true;
                slot.ready.push_front(ins[i]);
                ins.erase(ins.begin() + (long)i);
                steps.erase(steps.begin() + (long)i);
            }
        }
        const int k = (int)ins.size();
        s->in_flight += k;
        s->batches++;
        lk.unlock();
        std::vector<kkt_ctx*> ctxs(k);
        std::vector<const double*> vals(k), bs(k);
        std::vector<double*> xs(k);
        std::vector<int> it(k, 0), st(k, KKT_ERR_INVALID);
        std::vector<double> nr(k, 0.0);
        for (int i = 0; i < k; i++) {
            ctxs[i] = ins[i]->ctx;
            vals[i] = steps[i].values.data();
            bs[i] = steps[i].b.data();
            xs[i] = steps[i].x;
        }
        const auto t0 = Clock::now();
        cudaSetDevice(slot.dev);
        const int rc = kkt_batch_step(slot.batch, ctxs.data(), k, vals.data(), bs.data(), xs.data(), 0, tol,
                                      it.data(), nr.data(), st.data());
        const auto t1 = Clock::now();
        lk.lock();
        for (int i = 0; i < k; i++) {
            kkt_step_result r{};
            r.status = rc ? rc : st[i];
            r.iters = it[i];
            r.nrbe = nr[i];
            r.queue_ms = ms_between(steps[i].submitted, t0);
            r.run_ms = ms_between(t0, t1);
            r.batch_size = k;
            r.device = slot.dev;
            finish_step(s, ins[i], steps[i].ticket, r);
        }
    }
}

}  // namespace

extern "C" {

void kkt_server_default_opts(kkt_server_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->workers = 8;
    o->hbm_budget = 0;
    o->batch = 8;
    o->ndevices = 0;
    kkt_default_opts(&o->opts);
}

int kkt_server_create(kkt_server** out, const kkt_server_opts* o) {
    if (!out) return KKT_ERR_INVALID;
    *out = nullptr;
    kkt_server_opts opts;
    if (o) opts = *o;
    else kkt_server_default_opts(&opts);
    if (opts.workers < 1 || opts.workers > 256 || opts.hbm_budget < 0 || opts.batch < 0 || opts.batch > 4096 ||
        opts.ndevices < 0 || opts.ndevices > KKT_SERVER_MAX_DEVICES)
        return KKT_ERR_INVALID;
    auto* s = new kkt_server();
    s->o = opts;
    s->o.opts.create_stream = 1;
    s->o.opts.stream = nullptr;
    const int nd = opts.ndevices > 0 ? opts.ndevices : 1;
    s->slots.resize(nd);
    int rc = KKT_OK;
    for (int i = 0; i < nd && rc == KKT_OK; i++) {
        DeviceSlot& sl = s->slots[i];
        sl.dev = opts.ndevices > 0 ? opts.devices[i] : opts.opts.device;
        for (int j = 0; j < i; j++)
            if (s->slots[j].dev == sl.dev) rc = KKT_ERR_INVALID;   // each device once
        if (rc) break;
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(sl.dev) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            rc = KKT_ERR_CUDA;
            break;
        }
        sl.budget = opts.hbm_budget > 0 ? opts.hbm_budget : (int64_t)(0.9 * (double)free_b);
        if (opts.batch > 0) rc = kkt_batch_create(&sl.batch, opts.batch, sl.dev);
    }
    if (rc) {
        for (auto& sl : s->slots) kkt_batch_destroy(sl.batch);
        delete s;
        return rc;
    }
    if (opts.batch > 0)
        for (int i = 0; i < nd; i++) s->threads.emplace_back(dispatcher_main, s, i);
    else
        for (int i = 0; i < opts.workers; i++) s->threads.emplace_back(worker_main, s);
    *out = s;
    return KKT_OK;
}

int kkt_server_open(kkt_server* s, int32_t n, const int32_t* rowptr, const int32_t* colind,
                    const double* values0, int64_t* instance) {
    if (!s || !instance || !values0 || n < 1) return KKT_ERR_INVALID;
    *instance = 0;
    // the host analysis, in this thread
    std::vector<int32_t> P((size_t)n), Q((size_t)n);
    kkt_host_stats st{};
    int rc = kkt_host_analyze(n, rowptr, colind, values0, s->o.opts.pivot_tol, P.data(), Q.data(), &st);
    if (rc) return rc;
    int64_t need = 0;
    if ((rc = kkt_estimate_device_bytes(n, rowptr[n], &st, &s->o.opts, st.canonical_order, &need))) return rc;
    // placement, then admission in arrival order on that device
    std::unique_lock<std::mutex> lk(s->mu);
    const int nd = (int)s->slots.size();
    std::vector<int64_t> budget(nd), held(nd);
    for (int i = 0; i < nd; i++) {
        budget[i] = s->slots[i].budget;
        held[i] = s->slots[i].held + s->slots[i].reserved;
    }
    const int si = kkt_place_instance(nd, budget.data(), held.data(), need);
    if (si < 0) return KKT_ERR_OOM;   // more than a whole device's budget
    DeviceSlot& slot = s->slots[si];
    const int64_t me = s->next_admit++;
    slot.admit.push_back(me);
    slot.reserved += need;
    s->waiting++;
    s->cv_admit.wait(lk, [&] { return slot.admit.front() == me && slot.held + need <= slot.budget; });
    slot.admit.pop_front();
    slot.reserved -= need;
    slot.held += need;
    s->waiting--;
    s->cv_admit.notify_all();   // the next in line may fit too
    lk.unlock();
    kkt_opts o = s->o.opts;
    o.device = slot.dev;
    kkt_ctx* c = nullptr;
    cudaSetDevice(slot.dev);
    rc = kkt_create(&c, &o);
    if (rc == KKT_OK) rc = kkt_analyze(c, n, rowptr, colind, values0, Q.data(), P.data());
    kkt_info info{};
    if (rc == KKT_OK) rc = kkt_query(c, &info);
    lk.lock();
    if (rc) {
        slot.held -= need;
        s->cv_admit.notify_all();
        lk.unlock();
        kkt_destroy(c);
        return rc;
    }
    slot.held += info.device_bytes - need;   // the exact figure (the estimate equals it)
    auto in = std::make_unique<Instance>();
    in->id = s->next_id++;
    in->slot = si;
    in->ctx = c;
    in->n = n;
    in->nnz = info.nnz_a;
    in->bytes = info.device_bytes;
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
        if (s->o.batch > 0) s->slots[in->slot].ready.push_back(in);
        else s->ready.push_back(in);
        s->cv_work.notify_all();
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
    DeviceSlot& slot = s->slots[in->slot];
    slot.held -= in->bytes;
    s->inst.erase(it);
    s->cv_admit.notify_all();   // waiting opens may fit now
    const int dev = slot.dev;
    lk.unlock();
    cudaSetDevice(dev);
    kkt_destroy(c);
    return KKT_OK;
}

int kkt_server_query(kkt_server* s, kkt_server_info* info) {
    if (!s || !info) return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(info, 0, sizeof(*info));
    info->instances = (int32_t)s->inst.size();
    for (const auto& sl : s->slots) {
        info->device_bytes += sl.held;
        info->hbm_budget += sl.budget;
    }
    info->submitted = s->submitted;
    info->completed = s->completed;
    info->in_flight = s->in_flight;
    info->waiting = s->waiting;
    info->batches = s->batches;
    info->ndevices = (int32_t)s->slots.size();
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
    for (auto& t : s->threads) t.join();
    for (auto& sl : s->slots) {
        cudaSetDevice(sl.dev);
        kkt_batch_destroy(sl.batch);
    }
    delete s;
}

}  // extern "C"
