// Serving loop with continuous batching, on top of the public C ABI.
//
// Solve requests (problem description, initial state, step count) arrive at
// any time from any thread.  A scheduler thread owns the GPU work:
//  - admission: pending requests enter in arrival order while the server's
//    device-memory budget and its slot count allow (a request larger than the
//    whole budget fails with SWP_EBUDGET); an admitted request's state stays
//    resident on the device until it finishes;
//  - rounds: an admitted request's whole solve is one swept plan (node width
//    fixed at admission) run a few phases at a time, the open triangle
//    edges staying in its rows between rounds.  A round runs every request
//    whose remaining work (estimated FP64 work per point-update of its
//    equation) fits in a target round time to its end, and the long ones
//    shortest remaining work first, aged by their waiting time: the first
//    for a round's worth of phases, others beside it while the GPU has idle
//    blocks.  All of it goes
//    into one batched launch per group (a round of one request below 2^17
//    points, or in FP32, runs as that request's per-phase launches, as
//    swp_advance would run it alone); requests that arrive meanwhile join
//    the next round, so new and in-flight work overlap on the device;
//  - retirement: finished requests are copied back to host memory, their
//    device memory is freed, and waiters are woken.
// A request's phases are those of one swept advance of its whole step count,
// so its result is bit-identical to that advance, whatever else was in the
// mix.  The paper has no serving layer; this is the GB300 build's.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swept.h"
#include "launch.h"

namespace swp {
// Record `msg` as this thread's swp_last_error and return s (api.cu).
swp_status set_error(swp_status s, const char* msg);
}  // namespace swp

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    swp_desc desc{};
    std::vector<unsigned char> u0;       // host copy of the initial state
    std::vector<unsigned char> result;   // host copy of the final state
    int64_t steps_total = 0, steps_done = 0;
    int n = 0;                           // node width of the request's swept plan (classic: chunk width)
    int kind = swp::BATCH_SWEPT;         // BATCH_CLASSIC when N is too small for any node width
    int64_t n_phases = 0, phase_next = 0;
    double phase_cost = 0.0;             // estimated FP64 operations of one phase
    int64_t width = 0;                   // nodes (classic: chunks) per phase
    int state = 0;                       // 0 pending, 1 active, 2 done
    swp_status status = SWP_OK;
    std::string error;                   // why it failed (handed to the waiter)
    swp_problem* prob = nullptr;
    size_t bytes = 0;                    // device bytes while active
    Clock::time_point t_submit, t_admit, t_done;
};

size_t state_bytes(const swp_desc& d)
{
    return (size_t)(d.eq == SWP_EULER ? 3 : 1) * (size_t)d.n_points * (d.dtype == SWP_F32 ? 4 : 8);
}

// Estimated cost of one point-update, in units of which the device runs
// about 4e11 per second: calibrated from the swept rates measured on GB300 at
// N = 2^20 (FP64 heat 160, KS 37.9, Euler 2.57 G point-updates/s; FP32
// heat and KS about 9 and 13 times faster).
double cost_per_update(const swp_desc& d)
{
    if (d.dtype == SWP_F32) return d.eq == SWP_HEAT ? 0.28 : 0.8;
    return d.eq == SWP_HEAT ? 2.5 : (d.eq == SWP_KS ? 10.5 : 156.0);
}

}  // namespace

struct swp_server {
    swp_server_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    swp_batch* batch = nullptr;
    int64_t width_cap = 608;   // nodes in flight that fill the GPU: 4 per SM
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    int64_t next_id = 1;
    std::deque<std::shared_ptr<Request>> pending;
    std::vector<std::shared_ptr<Request>> active;
    std::map<int64_t, std::shared_ptr<Request>> all;
    size_t in_use = 0;
    // statistics
    int64_t rounds = 0, completed = 0, launches = 0;
    double point_updates = 0.0;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;

    void run();
    void admit();
    swp_status round();
    void retire_finished();
};

void swp_server::admit()
{
    // called with mu held
    while (!pending.empty() && (int)active.size() < cfg.max_active) {
        auto r = pending.front();
        const size_t need = 2 * state_bytes(r->desc);
        if (cfg.hbm_budget_bytes && need > cfg.hbm_budget_bytes) {
            pending.pop_front();
            r->status = SWP_EBUDGET;
            r->error = "the request needs " + std::to_string(need) + " device bytes, more than the server's budget of " +
                       std::to_string(cfg.hbm_budget_bytes);
            r->state = 2;
            r->t_done = Clock::now();
            r->u0.clear();
            cv_done.notify_all();
            continue;
        }
        if (cfg.hbm_budget_bytes && in_use + need > cfg.hbm_budget_bytes) break;
        pending.pop_front();
        swp_problem* p = nullptr;
        swp_status st = swp_create(&r->desc, r->u0.data(), 0, stream, &p);
        if (st != SWP_OK) {
            r->status = st;
            r->error = swp_last_error();
            r->state = 2;
            r->t_done = Clock::now();
            cv_done.notify_all();
            continue;
        }
        r->prob = p;
        r->n = swp::swept_width(p);
        r->kind = swp::BATCH_SWEPT;
        if (r->n == 0) {   // too few points for two swept nodes: the classic plan
            r->kind = swp::BATCH_CLASSIC;
            r->n = swp::classic_chunk(p);
        }
        r->n_phases = swp::phase_count(p, r->steps_total, r->kind, r->n);
        if (r->n_phases <= 0) {
            swp_destroy(p);
            r->prob = nullptr;
            r->status = SWP_EINVAL;
            r->error = "the request's plan has no phases";
            r->state = 2;
            r->t_done = Clock::now();
            cv_done.notify_all();
            continue;
        }
        r->phase_cost = (double)r->desc.n_points * (double)r->steps_total * cost_per_update(r->desc) /
                        (double)r->n_phases;
        r->width = r->kind == swp::BATCH_SWEPT ? r->desc.n_points / r->n
                                               : (r->desc.n_points + r->n - 1) / r->n;
        r->bytes = need;
        in_use += need;
        r->u0.clear();
        r->u0.shrink_to_fit();
        r->state = 1;
        r->t_admit = Clock::now();
        active.push_back(r);
    }
}

// The work rate (operations per second) the round budget and the aging of
// long requests are expressed in.
constexpr double kOpsPerSecond = 4.0e11;

swp_status swp_server::round()
{
    // called without mu: the active list only changes on this thread.
    // A request whose remaining work fits in one round's budget (a small one)
    // runs all its remaining phases now, so it never waits behind a long
    // solve.  Longer ones go in order of their remaining work less the work
    // the GPU does while they wait (remaining operations - age x the
    // operation rate): the first runs a round's budget of its phases, and
    // each next one joins only if its nodes fit in the blocks that those
    // already chosen leave idle (a narrow solve cannot fill the GPU by
    // itself), also with a round's budget.  Shorter solves thus pass longer
    // ones, which keeps the many mid-size solves from queueing behind the few
    // largest; a solve that has waited as long as its own remaining work
    // ranks ahead of every newer one, which bounds how long it can be passed.
    // When every active request is long and none is pending, rounds are four
    // times longer: fewer rounds, less host work between them, and a request
    // arriving meanwhile waits at most one such round.
    double budget_ops = cfg.round_target_ms * 1e-3 * kOpsPerSecond;
    bool all_long = true;
    for (auto& rq : active)
        if ((double)(rq->n_phases - rq->phase_next) * rq->phase_cost <= budget_ops) all_long = false;
    bool idle_queue;
    {
        std::lock_guard<std::mutex> lock(mu);
        idle_queue = pending.empty();
    }
    const double long_budget = all_long && idle_queue ? 4.0 * budget_ops : budget_ops;
    std::vector<swp::PhaseRange> ranges;
    std::vector<int64_t> take(active.size(), 0);
    int64_t width = 0;   // nodes (or chunks) per phase of the long solves chosen
    bool any_long = false;
    const auto now = Clock::now();
    std::vector<std::pair<double, size_t>> order(active.size());
    for (size_t i = 0; i < active.size(); ++i) {
        const Request& r = *active[i];
        const double age_s = std::chrono::duration<double>(now - r.t_submit).count();
        order[i] = {(double)(r.n_phases - r.phase_next) * r.phase_cost - age_s * kOpsPerSecond, i};
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, size_t>& a, const std::pair<double, size_t>& b) { return a.first < b.first; });
    for (const auto& o : order) {
        const size_t i = o.second;
        Request& r = *active[i];
        const int64_t left = r.n_phases - r.phase_next;
        if ((double)left * r.phase_cost <= budget_ops) {
            take[i] = left;
            continue;
        }
        if (any_long && width + r.width > width_cap) continue;   // only into idle blocks
        take[i] = std::min<int64_t>(left, std::max<int64_t>(1, (int64_t)(long_budget / r.phase_cost)));
        width += r.width;
        any_long = true;
    }
    for (size_t i = 0; i < active.size(); ++i) {
        if (take[i] <= 0) continue;
        Request& r = *active[i];
        ranges.push_back(swp::PhaseRange{r.prob, r.n, r.steps_total, r.phase_next, r.phase_next + take[i], r.kind});
    }
    const int64_t l0 = swp_batch_kernel_launches(batch);
    int64_t round_launches = 0;
    double round_updates = 0.0;
    swp_status st = SWP_OK;
    bool solo_phases = false;   // one request, of a size where per-phase launches beat the batched kernel
    if (ranges.size() == 1)
        for (auto& rq : active)
            if (rq->prob == ranges[0].p)
                solo_phases = rq->kind == swp::BATCH_SWEPT &&
                              (rq->desc.n_points < ((int64_t)1 << 17) || rq->desc.dtype == SWP_F32);
    if (solo_phases) {
        // as swp_advance would run it alone (SWP_LAUNCH_AUTO)
        const swp::PhaseRange& r = ranges[0];
        const int64_t k0 = swp_kernel_launches(r.p);
        st = swp::advance_phases(r.p, r.n, r.steps, r.p_lo, r.p_hi);
        if (st == SWP_OK) st = swp_synchronize(r.p);
        round_launches = swp_kernel_launches(r.p) - k0;
    } else {
        st = swp::batch_advance_phases(batch, ranges.data(), (int)ranges.size(), cfg.threads);
        if (st == SWP_OK) st = swp_batch_synchronize(batch);
        round_launches = swp_batch_kernel_launches(batch) - l0;
    }
    const std::string round_error = st != SWP_OK ? swp_last_error() : "";
    for (size_t i = 0; i < active.size(); ++i) {
        Request& r = *active[i];
        if (st != SWP_OK) {
            r.status = st;
            r.error = round_error;
            r.steps_done = r.steps_total;
            continue;
        }
        r.phase_next += take[i];
        if (r.phase_next >= r.n_phases) {
            r.steps_done = r.steps_total;
            round_updates += (double)r.steps_total * (double)r.desc.n_points;
        }
    }
    // the statistics are read by other threads under mu
    std::lock_guard<std::mutex> lock(mu);
    rounds++;
    launches += round_launches;
    point_updates += round_updates;
    return st;
}

void swp_server::retire_finished()
{
    std::vector<std::shared_ptr<Request>> keep;
    std::vector<std::shared_ptr<Request>> done;
    for (auto& r : active) (r->steps_done >= r->steps_total ? done : keep).push_back(r);
    for (auto& r : done) {
        if (r->status == SWP_OK) {
            r->result.resize(state_bytes(r->desc));
            r->status = swp_read(r->prob, r->result.data(), r->result.size(), 0);
            if (r->status != SWP_OK) r->error = swp_last_error();
        }
        swp_destroy(r->prob);
        r->prob = nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    const auto now = Clock::now();
    for (auto& r : done) {
        in_use -= r->bytes;
        r->state = 2;
        r->t_done = now;
        completed++;
        t_last_done = now;
    }
    active.swap(keep);
    if (!done.empty()) cv_done.notify_all();
}

void swp_server::run()
{
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait(lock, [&] { return stop || !pending.empty() || !active.empty(); });
            if (stop && pending.empty() && active.empty()) return;
            if (stop) {
                // shutting down: fail what has not started
                for (auto& r : pending) {
                    r->status = SWP_EINVAL;
                    r->error = "the server shut down before admitting the request";
                    r->state = 2;
                    r->t_done = Clock::now();
                }
                pending.clear();
                cv_done.notify_all();
            }
            admit();
        }
        if (active.empty()) continue;
        round();
        retire_finished();
    }
}

extern "C" {

swp_status swp_server_create(const swp_server_config* cfg, void* cuda_stream, swp_server** out)
{
    if (!cfg || !out) return swp::set_error(SWP_EINVAL, "server config or out is NULL");
    *out = nullptr;
    if (cfg->max_active <= 0 || !(cfg->round_target_ms > 0) || cfg->threads < 0)
        return swp::set_error(SWP_EINVAL, "server config: max_active and round_target_ms must be > 0, threads >= 0");
    swp_server* s = new (std::nothrow) swp_server();
    if (!s) return swp::set_error(SWP_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->stream = (cudaStream_t)cuda_stream;
    int sms = 0;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return swp::set_error(SWP_EDEVICE, "no usable CUDA device");
    }
    s->width_cap = 4 * (int64_t)sms;
    swp_status st = swp_batch_create(cuda_stream, &s->batch);
    if (st != SWP_OK) {
        delete s;
        return st;
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return SWP_OK;
}

swp_status swp_server_submit(swp_server* s, const swp_desc* desc, const void* u0_host, int64_t n_steps,
                             int64_t* request_id)
{
    if (!s || !desc || !u0_host || !request_id || n_steps < 1)
        return swp::set_error(SWP_EINVAL, "server, desc, u0_host or request_id is NULL, or n_steps < 1");
    size_t req = 0;
    swp_status st = swp_required_bytes(desc, &req);   // validates the description
    if (st != SWP_OK) return st;
    auto r = std::make_shared<Request>();
    r->desc = *desc;
    const size_t nb = state_bytes(*desc);
    r->u0.assign((const unsigned char*)u0_host, (const unsigned char*)u0_host + nb);
    r->steps_total = n_steps;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return swp::set_error(SWP_EINVAL, "the server is shutting down");
        r->id = s->next_id++;
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first_submit = r->t_submit;
        }
        s->pending.push_back(r);
        s->all[r->id] = r;
    }
    s->cv_work.notify_one();
    *request_id = r->id;
    return SWP_OK;
}

swp_status swp_server_poll(swp_server* s, int64_t id, int32_t* done)
{
    if (!s || !done) return swp::set_error(SWP_EINVAL, "server or done is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return swp::set_error(SWP_EINVAL, "unknown request id");
    *done = it->second->state == 2 ? 1 : 0;
    return SWP_OK;
}

swp_status swp_server_wait(swp_server* s, int64_t id, void* dst_host, size_t dst_bytes, double* latency_s)
{
    if (!s) return swp::set_error(SWP_EINVAL, "server is NULL");
    std::shared_ptr<Request> r;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        auto it = s->all.find(id);
        if (it == s->all.end()) return swp::set_error(SWP_EINVAL, "unknown request id (or already waited for)");
        r = it->second;
        s->cv_done.wait(lock, [&] { return r->state == 2; });
        s->all.erase(id);
    }
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    if (r->status != SWP_OK) return swp::set_error(r->status, r->error.c_str());
    if (dst_host) {
        if (dst_bytes < r->result.size()) return swp::set_error(SWP_EINVAL, "dst_bytes smaller than the state");
        std::memcpy(dst_host, r->result.data(), r->result.size());
    }
    return SWP_OK;
}

swp_status swp_server_stats(swp_server* s, swp_server_statistics* out)
{
    if (!s || !out) return swp::set_error(SWP_EINVAL, "server or out is NULL");
    std::lock_guard<std::mutex> lock(s->mu);
    out->completed = s->completed;
    out->rounds = s->rounds;
    out->kernel_launches = s->launches;
    out->pending = (int64_t)s->pending.size();
    out->active = (int64_t)s->active.size();
    out->device_bytes_in_use = s->in_use;
    out->point_updates = s->point_updates;
    out->busy_span_s = s->completed ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count() : 0.0;
    return SWP_OK;
}

swp_status swp_server_destroy(swp_server* s)
{
    if (!s) return SWP_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& r : s->active)
        if (r->prob) swp_destroy(r->prob);
    swp_batch_destroy(s->batch);
    delete s;
    return SWP_OK;
}

}  // extern "C"
