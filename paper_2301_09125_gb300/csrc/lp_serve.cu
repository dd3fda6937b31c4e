// Continuous-batching request server (lp_server_*).
//
// Requests (one graph each, host CSR) queue up as they are submitted.  An
// admission thread takes the requests queued at that moment, as many as the
// free active slots, the HBM budget and max_cohort allow (a graph of more
// than cohort_max_entries entries alone), and ingests them as one cohort on
// one of the server's CUDA streams: a lone request as a graph, several as
// one batch arena, whose iterations sweep every graph with one launch per
// degree bucket.  Several admission threads ingest cohorts side by side.  A worker thread advances every cohort one
// RAK iteration at a time: whenever a cohort's in-flight iteration has
// finished on the device (event query), it applies the tolerance test to
// each of its graphs (a converged graph is left out of later iterations) and
// either launches the next iteration or, once every graph has finished,
// retires the cohort's requests (modularity, labels copied to the callers'
// buffers, results queued for lp_server_poll).  Requests therefore join
// between iterations of the running cohorts, ingest never holds up their
// launches, and each result is the same as a lone lp_rak_run.
#include <algorithm>
#include <atomic>
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
lp_status batch_run_begin(lp_batch *b, const lp_rak_params *p);
bool batch_run_done(lp_batch *b);
lp_status batch_run_launch(lp_batch *b, cudaEvent_t *done_event);
lp_status batch_run_finish(lp_batch *b);
lp_status batch_run_end(lp_batch *b, lp_rak_result *per_graph);
int32_t batch_run_active(lp_batch *b);
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
    lp_serve_result res{};
};

// Requests ingested and iterated together: one graph, or one batch arena.
struct Cohort {
    std::vector<std::unique_ptr<Request>> reqs;
    lp_graph *g = nullptr;  // a lone request
    lp_batch *b = nullptr;  // several
    cudaEvent_t ev = nullptr;  // end of the in-flight iteration (owned by the graph set)
    bool in_flight = false;
    // requests still holding an active slot: a converged graph of a batch
    // gives its slot back at once (its memory stays counted until the cohort
    // retires), so that queued requests need not wait for the cohort's last one
    int64_t slots = 0;
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
    std::atomic<int> next_stream{0};
    Clock::time_point t0 = Clock::now();

    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_admit;
    std::deque<std::unique_ptr<Request>> queue;  // submitted, not yet admitted
    std::deque<std::unique_ptr<Cohort>> ready;   // ingested, not yet picked up
    std::deque<lp_serve_result> results;
    int64_t outstanding = 0;  // submitted, result not yet queued
    int64_t slots_used = 0;   // admitted and still iterating
    int64_t mem_used = 0;     // footprint of the admitted requests
    int64_t n_cohorts = 0, n_batched = 0, max_cohort_seen = 0;  // lp_server_stats
    bool stop = false;
    std::thread worker;
    std::vector<std::thread> admitters;

    std::vector<std::unique_ptr<Cohort>> active;  // worker thread only

    // give back active slots of requests whose graphs have finished
    void release_slots(int64_t k)
    {
        if (k <= 0) return;
        std::lock_guard<std::mutex> lock(mu);
        slots_used -= k;
        cv_admit.notify_one();
    }

    void retire(std::unique_ptr<Request> r, lp_status st)
    {
        r->res.status = st;
        r->res.latency_ms = ms_since(r->t_submit);
        std::lock_guard<std::mutex> lock(mu);
        mem_used -= r->footprint;
        results.push_back(r->res);
        --outstanding;
        cv_done.notify_all();
        cv_admit.notify_one();
    }

    // free a cohort's graph set, then retire its requests (st[i] per request)
    void retire_cohort(std::unique_ptr<Cohort> c, const std::vector<lp_status> &st)
    {
        if (c->g) lp_graph_destroy(c->g);
        if (c->b) lp_batch_destroy(c->b);
        c->g = nullptr;
        c->b = nullptr;
        release_slots(c->slots);
        c->slots = 0;
        for (size_t i = 0; i < c->reqs.size(); ++i) retire(std::move(c->reqs[i]), st[i]);
    }
    void retire_cohort(std::unique_ptr<Cohort> c, lp_status st)
    {
        const std::vector<lp_status> all(c->reqs.size(), st);
        retire_cohort(std::move(c), all);
    }

    cudaStream_t take_stream()
    {
        return streams[(size_t)(next_stream.fetch_add(1) % (int)streams.size())];
    }

    // ingest a lone request and start its run; null if it failed (retired)
    std::unique_ptr<Cohort> admit_one(std::unique_ptr<Request> r)
    {
        std::unique_ptr<Cohort> c(new Cohort);
        c->reqs.push_back(std::move(r));
        c->slots = 1;
        lp_status s = lp_graph_create(c->reqs[0]->n, c->reqs[0]->m, c->reqs[0]->off,
                                      c->reqs[0]->idx, c->reqs[0]->wts, 0, take_stream(), &c->g);
        if (s == LP_OK) s = lp::graph_run_begin(c->g, &params);
        if (s != LP_OK) {
            retire_cohort(std::move(c), s);
            return nullptr;
        }
        return c;
    }

    // ingest requests taken from the queue together, as one cohort when
    // there are several and their batch ingests; otherwise one by one
    void admit(std::vector<std::unique_ptr<Request>> take)
    {
        const Clock::time_point now = Clock::now();
        for (auto &r : take) {
            r->t_admit = now;
            r->res.queued_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
        }
        std::vector<std::unique_ptr<Cohort>> made;
        if (take.size() > 1) {
            std::vector<lp_graph_desc> d(take.size());
            for (size_t i = 0; i < take.size(); ++i)
                d[i] = lp_graph_desc{take[i]->n, take[i]->m, take[i]->off, take[i]->idx,
                                     take[i]->wts};
            std::unique_ptr<Cohort> c(new Cohort);
            lp_status s = lp_batch_create((int32_t)take.size(), d.data(), 0, take_stream(), &c->b);
            if (s == LP_OK) s = lp::batch_run_begin(c->b, &params);
            if (s == LP_OK) {
                c->slots = (int64_t)take.size();
                c->reqs = std::move(take);
                take.clear();
                made.push_back(std::move(c));
            } else if (c->b) {
                lp_batch_destroy(c->b);
                c->b = nullptr;
            }
        }
        for (auto &r : take)  // a lone request, or a cohort that did not ingest
            if (r) {
                std::unique_ptr<Cohort> c = admit_one(std::move(r));
                if (c) made.push_back(std::move(c));
            }
        if (made.empty()) return;
        std::lock_guard<std::mutex> lock(mu);
        for (auto &c : made) {
            const int64_t k = (int64_t)c->reqs.size();
            ++n_cohorts;
            if (k > 1) n_batched += k;
            max_cohort_seen = std::max(max_cohort_seen, k);
            ready.push_back(std::move(c));
        }
        cv_work.notify_one();
    }

    // advance a cohort by at most one iteration; false once retired
    bool advance(std::unique_ptr<Cohort> &c, bool *progressed)
    {
        lp_status s = LP_OK;
        if (c->in_flight) {
            const cudaError_t q = cudaEventQuery(c->ev);
            if (q == cudaErrorNotReady) return true;
            c->in_flight = false;
            *progressed = true;
            if (q != cudaSuccess) {
                retire_cohort(std::move(c), LP_ECUDA);
                return false;
            }
            s = c->g ? lp::graph_run_finish(c->g) : lp::batch_run_finish(c->b);
            if (s == LP_OK && c->b) {
                const int64_t left = lp::batch_run_active(c->b);
                if (left < c->slots) {
                    release_slots(c->slots - left);
                    c->slots = left;
                }
            }
        }
        if (s == LP_OK && !(c->g ? lp::graph_run_done(c->g) : lp::batch_run_done(c->b))) {
            s = c->g ? lp::graph_run_launch(c->g, &c->ev) : lp::batch_run_launch(c->b, &c->ev);
            if (s == LP_OK) {
                c->in_flight = true;
                *progressed = true;
                return true;
            }
        }
        *progressed = true;
        std::vector<lp_status> st(c->reqs.size(), s);
        if (s == LP_OK && c->g) {
            lp_rak_result rr{};
            Request &r = *c->reqs[0];
            lp_status e = lp::graph_run_end(c->g, &rr);
            r.res.iterations = rr.iterations;
            r.res.converged = rr.converged;
            if (e == LP_OK) e = lp_modularity(c->g, nullptr, 0, &r.res.modularity);
            if (e == LP_OK && r.labels_out) e = lp_labels_get(c->g, r.labels_out, 0);
            st[0] = e;
        } else if (s == LP_OK) {
            std::vector<lp_rak_result> rr(c->reqs.size());
            lp_status e = lp::batch_run_end(c->b, rr.data());
            for (size_t i = 0; i < c->reqs.size(); ++i) {
                Request &r = *c->reqs[i];
                lp_status ei = e;
                r.res.iterations = rr[i].iterations;
                r.res.converged = rr[i].converged;
                if (ei == LP_OK) ei = lp_batch_modularity(c->b, (int32_t)i, &r.res.modularity);
                if (ei == LP_OK && r.labels_out)
                    ei = lp_batch_labels_get(c->b, (int32_t)i, r.labels_out, 0);
                st[i] = ei;
            }
        }
        retire_cohort(std::move(c), st);
        return false;
    }

    // admission threads: slot and budget checks, then ingest on a stream
    void admit_loop()
    {
        cudaSetDevice(device);
        for (;;) {
            std::vector<std::unique_ptr<Request>> take;
            {
                std::unique_lock<std::mutex> lock(mu);
                cv_admit.wait(lock, [this] {
                    return stop || (!queue.empty() && slots_used < cfg.max_active &&
                                    mem_used + queue.front()->footprint <= cfg.hbm_budget);
                });
                if (stop && queue.empty()) return;
                // the requests queued now, in order, while slots and budget last:
                // a large request alone, else the small ones up to the next large
                // one (and a batch's vertex ids stay below 2^31)
                int64_t nv = 0;
                const bool alone = queue.front()->m > cfg.cohort_max_entries;
                while (!queue.empty() && (int64_t)take.size() < (alone ? 1 : cfg.max_cohort) &&
                       slots_used < cfg.max_active &&
                       mem_used + queue.front()->footprint <= cfg.hbm_budget &&
                       (alone || queue.front()->m <= cfg.cohort_max_entries) &&
                       nv + queue.front()->n + (int64_t)take.size() + 1 < 2147483647LL) {
                    nv += queue.front()->n;
                    mem_used += queue.front()->footprint;
                    ++slots_used;
                    take.push_back(std::move(queue.front()));
                    queue.pop_front();
                }
                if (!queue.empty()) cv_admit.notify_one();  // another admitter may go on
            }
            if (!take.empty()) admit(std::move(take));
        }
    }

    // worker thread: advance every ingested cohort by iterations
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
                // nothing finished: wait briefly for a newly ingested cohort
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
    cfg->max_cohort = 16;
    cfg->admitters = 2;
    cfg->cohort_max_entries = (int64_t)1 << 18;
    return LP_OK;
}

lp_status lp_server_create(const lp_server_config *cfg, const lp_rak_params *p, lp_server **out)
{
    if (!out) return lp::lp_fail(LP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg || !p) return lp::lp_fail(LP_EINVAL, "cfg or params is NULL");
    if (cfg->hbm_budget <= 0 || cfg->max_active < 1 || cfg->streams < 1 || cfg->streams > 64 ||
        cfg->max_cohort < 1 || cfg->admitters < 1 || cfg->admitters > 16 ||
        cfg->cohort_max_entries < 0)
        return lp::lp_fail(LP_EINVAL, "hbm_budget > 0, max_active >= 1, 1 <= streams <= 64, "
                                      "max_cohort >= 1, 1 <= admitters <= 16, "
                                      "cohort_max_entries >= 0");
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
    for (int i = 0; i < cfg->admitters; ++i)
        s->admitters.emplace_back([raw] { raw->admit_loop(); });
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

lp_status lp_server_stats(lp_server *s, int64_t *cohorts, int64_t *batched, int64_t *largest)
{
    if (!s || !cohorts || !batched || !largest) return lp::lp_fail(LP_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lock(s->mu);
    *cohorts = s->n_cohorts;
    *batched = s->n_batched;
    *largest = s->max_cohort_seen;
    return LP_OK;
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
    for (std::thread &t : s->admitters)
        if (t.joinable()) t.join();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
    return LP_OK;
}

}  // extern "C"
