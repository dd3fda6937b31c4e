// Continuous-batching request server (lp_server_*).
//
// Requests (one graph each, host CSR) queue up as they are submitted.  An
// admission thread takes a queued request as soon as an active slot is free
// and its estimated device footprint fits the HBM budget, and ingests it on
// one of the server's CUDA streams.  A worker thread advances every ingested
// request one RAK iteration at a time: whenever a request's in-flight
// iteration has finished on the device (event query), the worker applies the
// tolerance test and either launches its next iteration or retires it
// (modularity, labels copied to the caller's buffer, result queued for
// lp_server_poll).  Requests therefore join and leave between iterations while
// the kernels of the others keep running on their streams, and ingest never
// holds up the launches; each result is the same as a lone lp_rak_run.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lp.h"
#include "lp_internal.cuh"

struct lp_graph;
namespace lp {
lp_status lp_fail(lp_status s, const std::string &msg);
lp_status graph_run_begin(lp_graph *g, const lp_rak_params *p);
bool graph_run_done(lp_graph *g);
lp_status graph_run_launch(lp_graph *g, cudaEvent_t *done_event);
lp_status graph_run_finish(lp_graph *g);
lp_status graph_run_end(lp_graph *g, lp_rak_result *r);
}  // namespace lp

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

struct Request {
    int64_t id = 0;
    int32_t n = 0;
    int64_t m = 0;
    const int32_t *off = nullptr, *idx = nullptr, *wts = nullptr;
    int32_t *labels_out = nullptr;
    int64_t footprint = 0;
    Clock::time_point t_submit, t_admit;
    lp_graph *g = nullptr;
    cudaEvent_t ev = nullptr;  // end of the in-flight iteration (owned by the graph)
    bool in_flight = false;
    lp_serve_result res{};
};

// device bytes a request may hold: CSR, two label buffers, bucket and wave
// lists, modularity scratch, majority flags (1 byte per vertex), hub
// fallback tables (at most 4 slots of 12 bytes per entry) and hub segment
// records (at most 32 bytes per entry)
int64_t footprint(int32_t n, int64_t m, bool weighted)
{
    return 4 * ((int64_t)n + 1) + (weighted ? 8 : 4) * m + 37 * (int64_t)n + 80 * m + (1 << 20);
}

}  // namespace

struct lp_server {
    lp_server_config cfg{};
    lp_rak_params params{};
    int device = 0;
    std::vector<cudaStream_t> streams;
    int next_stream = 0;
    Clock::time_point t0 = Clock::now();

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<std::unique_ptr<Request>> queue;    // submitted, not yet admitted
    std::deque<std::unique_ptr<Request>> ready;    // ingested, not yet picked up
    std::deque<lp_serve_result> results;
    int64_t outstanding = 0;  // submitted, result not yet queued
    int64_t slots_used = 0;   // admitted, not yet retired
    int64_t mem_used = 0;     // footprint of the admitted requests
    bool stop = false;
    std::thread worker, admitter;

    std::vector<std::unique_ptr<Request>> active;  // worker thread only

    void retire(std::unique_ptr<Request> r, lp_status st)
    {
        r->res.status = st;
        r->res.latency_ms = ms_since(r->t_submit);
        if (r->g) {
            lp_graph_destroy(r->g);
            r->g = nullptr;
        }
        std::lock_guard<std::mutex> lock(mu);
        mem_used -= r->footprint;
        --slots_used;
        results.push_back(r->res);
        --outstanding;
        cv_done.notify_all();
        cv_admit.notify_one();
    }

    // ingest and start a request; false if it failed (already retired)
    bool admit(std::unique_ptr<Request> &r)
    {
        r->t_admit = Clock::now();
        r->res.queued_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
        cudaStream_t st = streams[(size_t)next_stream];
        next_stream = (next_stream + 1) % (int)streams.size();
        lp_status s = lp_graph_create(r->n, r->m, r->off, r->idx, r->wts, 0, st, &r->g);
        if (s == LP_OK) s = lp::graph_run_begin(r->g, &params);
        if (s != LP_OK) {
            retire(std::move(r), s);
            return false;
        }
        return true;
    }

    // advance one request by at most one iteration; false once retired
    bool advance(std::unique_ptr<Request> &r, bool *progressed)
    {
        lp_status s = LP_OK;
        if (r->in_flight) {
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) return true;
            if (q != cudaSuccess) {
                retire(std::move(r), LP_ECUDA);
                return false;
            }
            r->in_flight = false;
            *progressed = true;
            s = lp::graph_run_finish(r->g);
        }
        if (s == LP_OK && !lp::graph_run_done(r->g)) {
            s = lp::graph_run_launch(r->g, &r->ev);
            if (s == LP_OK) {
                r->in_flight = true;
                *progressed = true;
                return true;
            }
        }
        if (s == LP_OK) {
            lp_rak_result rr{};
            s = lp::graph_run_end(r->g, &rr);
            r->res.iterations = rr.iterations;
            r->res.converged = rr.converged;
            if (s == LP_OK) s = lp_modularity(r->g, nullptr, 0, &r->res.modularity);
            if (s == LP_OK && r->labels_out) s = lp_labels_get(r->g, r->labels_out, 0);
        }
        *progressed = true;
        retire(std::move(r), s);
        return false;
    }

    // admission thread: slot and budget check, then ingest on a stream
    void admit_loop()
    {
        cudaSetDevice(device);
        for (;;) {
            std::unique_ptr<Request> r;
            {
                std::unique_lock<std::mutex> lock(mu);
                cv_admit.wait(lock, [this] {
                    return stop || (!queue.empty() && slots_used < cfg.max_active &&
                                    mem_used + queue.front()->footprint <= cfg.hbm_budget);
                });
                if (stop && queue.empty()) return;
                if (queue.empty()) continue;
                r = std::move(queue.front());
                queue.pop_front();
                mem_used += r->footprint;
                ++slots_used;
            }
            if (admit(r)) {
                std::lock_guard<std::mutex> lock(mu);
                ready.push_back(std::move(r));
                cv_work.notify_one();
            }
        }
    }

    // worker thread: advance every ingested request by iterations
    void run()
    {
        cudaSetDevice(device);
        for (;;) {
            {
                std::unique_lock<std::mutex> lock(mu);
                if (active.empty())
                    cv_work.wait(lock, [this] { return !ready.empty() || (stop && outstanding == 0); });
                if (active.empty() && ready.empty() && stop && outstanding == 0) return;
                while (!ready.empty()) {
                    active.push_back(std::move(ready.front()));
                    ready.pop_front();
                }
            }
            bool progressed = false;
            for (size_t i = 0; i < active.size();) {
                if (advance(active[i], &progressed)) {
                    ++i;
                } else {
                    active[i] = std::move(active.back());
                    active.pop_back();
                }
            }
            if (!progressed && !active.empty()) {
                // nothing finished: wait briefly for a newly ingested request
                std::unique_lock<std::mutex> lock(mu);
                cv_work.wait_for(lock, std::chrono::microseconds(20),
                                 [this] { return !ready.empty(); });
            }
        }
    }
};

extern "C" {

lp_status lp_server_config_default(lp_server_config *cfg)
{
    if (!cfg) return lp::lp_fail(LP_EINVAL, "cfg is NULL");
    cfg->hbm_budget = (int64_t)8 << 30;
    cfg->max_active = 64;
    cfg->streams = 8;
    return LP_OK;
}

lp_status lp_server_create(const lp_server_config *cfg, const lp_rak_params *p, lp_server **out)
{
    if (!out) return lp::lp_fail(LP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || !p) return lp::lp_fail(LP_EINVAL, "cfg or params is NULL");
    if (cfg->hbm_budget <= 0 || cfg->max_active < 1 || cfg->streams < 1 || cfg->streams > 64)
        return lp::lp_fail(LP_EINVAL, "hbm_budget > 0, max_active >= 1, 1 <= streams <= 64");
    if (p->init_labels) return lp::lp_fail(LP_EINVAL, "served requests start from unique labels");
    if (!(p->tolerance >= 0.0 && p->tolerance <= 1.0) || p->max_iter < 1 ||
        (p->mode != LP_SYNC && p->mode != LP_ASYNC) || (p->mode == LP_ASYNC && p->waves < 1))
        return lp::lp_fail(LP_EINVAL, "invalid RAK parameters");
    std::unique_ptr<lp_server> s(new (std::nothrow) lp_server);
    if (!s) return lp::lp_fail(LP_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    s->params = *p;
    if (cudaGetDevice(&s->device) != cudaSuccess) return lp::lp_fail(LP_ECUDA, "no CUDA device");
    for (int i = 0; i < cfg->streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            return lp::lp_fail(LP_ECUDA, "stream creation failed");
        }
        s->streams.push_back(st);
    }
    lp_server *raw = s.get();
    s->worker = std::thread([raw] { raw->run(); });
    s->admitter = std::thread([raw] { raw->admit_loop(); });
    *out = s.release();
    return LP_OK;
}

lp_status lp_server_submit(lp_server *s, int64_t request_id, int32_t n, int64_t m,
                           const int32_t *offsets, const int32_t *indices, const int32_t *weights,
                           int32_t *labels_out)
{
    if (!s) return lp::lp_fail(LP_EINVAL, "server is NULL");
    if (n < 0 || m < 0 || m > 2147483647LL || !offsets || (m > 0 && !indices))
        return lp::lp_fail(LP_EINVAL, "bad graph arguments");
    std::unique_ptr<Request> r(new (std::nothrow) Request);
    if (!r) return lp::lp_fail(LP_ENOMEM, "host allocation failed");
    r->id = request_id;
    r->n = n;
    r->m = m;
    r->off = offsets;
    r->idx = indices;
    r->wts = weights;
    r->labels_out = labels_out;
    r->footprint = footprint(n, m, weights != nullptr);
    r->t_submit = Clock::now();
    r->res.request_id = request_id;
    if (r->footprint > s->cfg.hbm_budget)
        return lp::lp_fail(LP_ENOMEM, "request does not fit the server's HBM budget");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return lp::lp_fail(LP_EINVAL, "server is shutting down");
        s->queue.push_back(std::move(r));
        ++s->outstanding;
    }
    s->cv_admit.notify_one();
    return LP_OK;
}

lp_status lp_server_poll(lp_server *s, lp_serve_result *out, int32_t capacity, int32_t *count,
                         int32_t wait_ms)
{
    if (!s || !count || (capacity > 0 && !out)) return lp::lp_fail(LP_EINVAL, "bad arguments");
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->results.empty() && wait_ms > 0)
        s->cv_done.wait_for(lock, std::chrono::milliseconds(wait_ms),
                            [s] { return !s->results.empty(); });
    int32_t k = 0;
    while (k < capacity && !s->results.empty()) {
        out[k++] = s->results.front();
        s->results.pop_front();
    }
    *count = k;
    return k > 0 ? LP_OK : LP_ENOTREADY;
}

lp_status lp_server_drain(lp_server *s)
{
    if (!s) return lp::lp_fail(LP_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv_done.wait(lock, [s] { return s->outstanding == 0; });
    return LP_OK;
}

lp_status lp_server_destroy(lp_server *s)
{
    if (!s) return LP_OK;
    {
        // every submitted request is finished first
        std::unique_lock<std::mutex> lock(s->mu);
        s->cv_done.wait(lock, [s] { return s->outstanding == 0; });
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_admit.notify_all();
    if (s->admitter.joinable()) s->admitter.join();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return LP_OK;
}

}  // extern "C"
