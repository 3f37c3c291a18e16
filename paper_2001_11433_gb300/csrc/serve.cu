// Serving loop for incremental maximal cliques: continuous batching of edge
// batches over device-resident graphs and clique indexes.
//
// Section 5 defines the incremental step for a graph G and a batch H, so the
// batches of one graph form a total order (G, G+H1, G+H1+H2, ...): a tenant
// (one graph with its clique index) runs at most one batch at a time, in
// submission order.  Batches of different tenants run side by side, one per
// slot; a slot is a worker thread with its own CUDA stream.  A batch is
// admitted when it has arrived, its tenant is idle, a slot is free and its
// projected device memory fits the budget next to the batches in flight.  The
// oldest arrived batch that does not fit holds back every later one, so large
// batches are not starved; a batch is always admitted when nothing is in
// flight.
//
// Latency of a batch = completion - arrival on the server clock; the stats
// report nearest-rank p50/p99 of latency and of the admission wait.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "mce_host.h"

using namespace mce;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int32_t tenant = 0;
    std::vector<int32_t> u, v;
    int64_t k = 0;
    uint64_t reserve = 0;
    Clock::time_point arrival, admit, done;
    bool finished = false;
    mce_status status = MCE_OK;
    imce_delta delta{};
};

struct Tenant {
    imce_state *st = nullptr;
    int64_t n = 0, nnz = 0;
    bool busy = false;
    std::deque<int64_t> fifo;   // submitted, not yet admitted
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// nearest-rank percentile of sorted values
double pct(const std::vector<double> &s, double q) {
    if (s.empty()) return 0.0;
    size_t r = (size_t)std::ceil(q * (double)s.size());
    if (r < 1) r = 1;
    return s[r - 1];
}

}  // namespace

struct imce_server {
    imce_server_opts o{};
    std::mutex mu;
    std::condition_variable cv_work;   // a request arrived or finished, or stop
    std::condition_variable cv_done;   // a request finished
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    cudaStream_t admin = nullptr;
    std::vector<std::unique_ptr<Tenant>> tenants;
    std::vector<std::unique_ptr<Request>> reqs;   // by id
    std::deque<int64_t> queue;                    // not admitted, by arrival time
    uint64_t reserved = 0, peak_reserved = 0;
    int32_t in_flight = 0, max_in_flight = 0;
    Clock::time_point t0;
    int64_t stats_from = 0;
    bool stop = false;
};

namespace {

uint64_t projected_bytes(const imce_server *S, const Tenant &t, int64_t k) {
    // queue ring and per-warp search state (fixed), batch keys and adjacency,
    // the merged graph G' and the new-clique lists
    return S->o.mem_fixed + 16ULL * (uint64_t)(t.n + 1) + 8ULL * (uint64_t)(t.nnz + 2 * k) + 96ULL * (uint64_t)k;
}

void worker(imce_server *S, int slot) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->stop) return;
        const Clock::time_point now = Clock::now();
        Clock::time_point next = Clock::time_point::max();
        int64_t pick = -1;
        bool held = false;
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
            Request &r = *S->reqs[*it];
            if (r.arrival > now) {
                next = std::min(next, r.arrival);
                continue;
            }
            Tenant &t = *S->tenants[r.tenant];
            if (t.busy || t.fifo.front() != *it) continue;
            if (held) continue;
            if (S->in_flight > 0 && S->reserved + r.reserve > S->o.mem_budget) {
                held = true;   // the oldest arrived batch that does not fit waits first
                continue;
            }
            pick = *it;
            S->queue.erase(it);
            break;
        }
        if (pick < 0) {
            if (next != Clock::time_point::max()) S->cv_work.wait_until(lk, next);
            else S->cv_work.wait(lk);
            continue;
        }
        Request &r = *S->reqs[pick];
        Tenant &t = *S->tenants[r.tenant];
        t.busy = true;
        t.fifo.pop_front();
        S->reserved += r.reserve;
        S->peak_reserved = std::max(S->peak_reserved, S->reserved);
        S->in_flight += 1;
        S->max_in_flight = std::max(S->max_in_flight, S->in_flight);
        r.admit = Clock::now();
        lk.unlock();
        mce_status st;
        if (S->o.execute) {
            st = S->o.execute(S->o.execute_ctx, r.tenant, r.u.data(), r.v.data(), r.k, &r.delta);
        } else {
            // the tenant's previous batch has completed, so its state may
            // move to this slot's stream
            mce::imce_set_stream(t.st, S->streams[slot]);
            st = imce_add_edges(t.st, r.u.data(), r.v.data(), r.k, 0, &r.delta);
        }
        lk.lock();
        r.status = st;
        r.done = Clock::now();
        r.finished = true;
        std::vector<int32_t>().swap(r.u);
        std::vector<int32_t>().swap(r.v);
        if (st == MCE_OK) t.nnz += 2 * r.delta.applied;
        t.busy = false;
        S->reserved -= r.reserve;
        S->in_flight -= 1;
        S->cv_work.notify_all();
        S->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

void imce_server_opts_init(imce_server_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->slots = 4;
}

mce_status imce_server_create(const imce_server_opts *opts, imce_server **out) {
    if (!out) return MCE_EINVAL;
    imce_server_opts o;
    if (opts) o = *opts;
    else imce_server_opts_init(&o);
    if (o.slots < 1 || o.slots > 64) {
        g_last_error = "imce_server_create: slots must be in [1, 64]";
        return MCE_EINVAL;
    }
    if (o.mem_fixed == 0) o.mem_fixed = 384ULL << 20;
    if (o.mem_budget == 0) {
        if (o.execute) {
            o.mem_budget = ~0ULL;
        } else {
            size_t fr = 0, tot = 0;
            MCE_CUDA(cudaMemGetInfo(&fr, &tot));
            o.mem_budget = (uint64_t)((double)fr * 0.8);
        }
    }
    std::unique_ptr<imce_server> S(new imce_server());
    S->o = o;
    if (!o.execute) {
        MCE_CUDA(cudaStreamCreateWithFlags(&S->admin, cudaStreamNonBlocking));
        for (int i = 0; i < o.slots; ++i) {
            cudaStream_t s = nullptr;
            const cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
                cudaStreamDestroy(S->admin);
                return cuda_status(e, "imce_server_create");
            }
            S->streams.push_back(s);
        }
    }
    S->t0 = Clock::now();
    for (int i = 0; i < o.slots; ++i) S->workers.emplace_back(worker, S.get(), i);
    *out = S.release();
    return MCE_OK;
}

mce_status imce_server_add_tenant(imce_server *S, const mce_graph *g, const mce_opts *opts, int32_t *tenant) {
    if (!S || !tenant || (!S->o.execute && (!g || !opts))) {
        g_last_error = "imce_server_add_tenant: bad arguments";
        return MCE_EINVAL;
    }
    std::unique_ptr<Tenant> t(new Tenant());
    if (!S->o.execute) {
        mce_opts o = *opts;
        o.stream = S->admin;
        MCE_TRY(imce_open(g, &o, &t->st));
        t->n = g->n;
        t->nnz = g->nnz;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    *tenant = (int32_t)S->tenants.size();
    S->tenants.push_back(std::move(t));
    return MCE_OK;
}

mce_status imce_server_submit(imce_server *S, int32_t tenant, const int32_t *u, const int32_t *v, int64_t k,
                              double arrival_ms, int64_t *id) {
    if (!S || k < 0 || (k > 0 && (!u || !v))) {
        g_last_error = "imce_server_submit: bad arguments";
        return MCE_EINVAL;
    }
    std::unique_ptr<Request> r(new Request());
    r->tenant = tenant;
    r->k = k;
    r->u.assign(u, u + k);
    r->v.assign(v, v + k);
    std::lock_guard<std::mutex> lk(S->mu);
    if (tenant < 0 || tenant >= (int32_t)S->tenants.size()) {
        g_last_error = "imce_server_submit: unknown tenant";
        return MCE_EINVAL;
    }
    const Clock::time_point now = Clock::now();
    r->arrival = now;
    if (arrival_ms >= 0) {
        const auto at = S->t0 + std::chrono::duration_cast<Clock::duration>(
                                    std::chrono::duration<double, std::milli>(arrival_ms));
        if (at > now) r->arrival = at;
    }
    Tenant &t = *S->tenants[tenant];
    r->reserve = projected_bytes(S, t, k);
    const int64_t rid = (int64_t)S->reqs.size();
    t.fifo.push_back(rid);
    // keep the queue sorted by arrival (stable for equal times)
    auto pos = std::upper_bound(S->queue.begin(), S->queue.end(), r->arrival,
                                [&](const Clock::time_point &a, int64_t x) { return a < S->reqs[x]->arrival; });
    S->reqs.push_back(std::move(r));
    S->queue.insert(pos, rid);
    if (id) *id = rid;
    S->cv_work.notify_all();
    return MCE_OK;
}

mce_status imce_server_wait(imce_server *S, int64_t id, imce_request_info *info) {
    if (!S) return MCE_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (id < 0 || id >= (int64_t)S->reqs.size()) {
        g_last_error = "imce_server_wait: unknown request";
        return MCE_EINVAL;
    }
    S->cv_done.wait(lk, [&] { return S->reqs[id]->finished; });
    const Request &r = *S->reqs[id];
    if (info) {
        info->id = id;
        info->tenant = r.tenant;
        info->status = r.status;
        info->edges = r.k;
        info->arrival_ms = ms_between(S->t0, r.arrival);
        info->admit_ms = ms_between(S->t0, r.admit);
        info->done_ms = ms_between(S->t0, r.done);
        info->reserved = r.reserve;
        info->delta = r.delta;
    }
    return r.status;
}

mce_status imce_server_drain(imce_server *S) {
    if (!S) return MCE_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->in_flight == 0; });
    return MCE_OK;
}

mce_status imce_server_reset_clock(imce_server *S) {
    if (!S) return MCE_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->queue.empty() && S->in_flight == 0; });
    S->t0 = Clock::now();
    S->stats_from = (int64_t)S->reqs.size();
    S->peak_reserved = 0;
    S->max_in_flight = 0;
    return MCE_OK;
}

mce_status imce_server_stats_get(imce_server *S, imce_server_stats *st) {
    if (!S || !st) return MCE_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof(*st));
    std::vector<double> lat, wait;
    Clock::time_point first = Clock::time_point::max(), last = Clock::time_point::min();
    for (int64_t i = S->stats_from; i < (int64_t)S->reqs.size(); ++i) {
        const Request &r = *S->reqs[i];
        if (!r.finished) continue;
        if (r.status != MCE_OK) {
            st->failed += 1;
            continue;
        }
        st->completed += 1;
        st->edges += r.k;
        st->applied += r.delta.applied;
        st->new_cliques += r.delta.new_count;
        st->subsumed_cliques += r.delta.sub_count;
        lat.push_back(ms_between(r.arrival, r.done));
        wait.push_back(ms_between(r.arrival, r.admit));
        first = std::min(first, r.arrival);
        last = std::max(last, r.done);
    }
    std::sort(lat.begin(), lat.end());
    std::sort(wait.begin(), wait.end());
    st->p50_ms = pct(lat, 0.50);
    st->p99_ms = pct(lat, 0.99);
    st->max_ms = lat.empty() ? 0.0 : lat.back();
    st->wait_p50_ms = pct(wait, 0.50);
    st->wait_p99_ms = pct(wait, 0.99);
    st->span_ms = lat.empty() ? 0.0 : ms_between(first, last);
    st->edges_per_s = st->span_ms > 0 ? (double)st->edges / (st->span_ms * 1e-3) : 0.0;
    st->max_in_flight = S->max_in_flight;
    st->peak_reserved = S->peak_reserved;
    st->mem_budget = S->o.mem_budget;
    return MCE_OK;
}

imce_state *imce_server_tenant(imce_server *S, int32_t tenant) {
    if (!S) return nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    if (tenant < 0 || tenant >= (int32_t)S->tenants.size()) return nullptr;
    return S->tenants[tenant]->st;
}

void imce_server_free(imce_server *S) {
    if (!S) return;
    imce_server_drain(S);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (std::thread &w : S->workers) w.join();
    for (auto &t : S->tenants)
        if (t->st) imce_close(t->st);
    for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
    if (S->admin) cudaStreamDestroy(S->admin);
    delete S;
}

}  // extern "C"
