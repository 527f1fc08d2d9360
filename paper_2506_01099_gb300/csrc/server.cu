// Serving loop (continuous batching of interval requests) and the autotuner.
//
// Serving: a host thread owns the context while it runs.  Every iteration it
//   1. admits waiting requests (first come, first served) while a slot is free
//      and the workspace of an iteration that gives every admitted request a
//      slice of `slice` integers fits the memory budget; a request that does
//      not fit waits for memory (and is counted once as deferred);
//   2. cuts the next slice of every active request and runs all slices as one
//      batched pipeline (one persistent sieve launch over the shared queue), so
//      the work of requests that arrived at different times overlaps on the GPU.
//      An iteration covers as many integers as an equal share eq of slice * max_active
//      (at least `slice` per request) would: a request with at most eq left finishes
//      in it, as with equal shares; every other active request gets `slice`, and the
//      rest go to those in order of arrival, so that a long request that is the
//      oldest gets most of the GPU (close to first come, first served) instead of an
//      equal share that stretches it over many iterations.  Iterations stay as long
//      as with equal shares.
//      While the iteration's workspace exceeds the budget the extra share is halved,
//      then the per-request `slice` (down to one queue segment); the workspace is
//      sized under the same budget, so the budget bounds the device memory the loop
//      holds;
//   3. appends each slice's pairs to its request and retires finished requests
//      (and cancelled ones, whose pairs are discarded).
// The workspace bytes of an iteration come from the same function that sizes the
// workspace (ws_need_bytes), so admission and allocation agree.  Results are
// exact, so a request's pairs are the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "benelux.h"
#include "bnx_ctx.cuh"

namespace bnx {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    bnx_interval iv{};
    uint64_t cursor = 0;
    std::vector<bnx_pair> pairs;
    Clock::time_point t_submit, t_done;
    bool done = false;
    bool deferred = false;  // waited for memory at least once
    bool cancelled = false;  // bnx_server_cancel: retire at the end of the current iteration
    int status = BNX_OK;
};

struct Server {
    bnx_server_cfg cfg{};
    uint64_t budget = 0;
    std::thread th;
    std::mutex m;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<std::shared_ptr<Request>> pending;
    std::vector<std::shared_ptr<Request>> active;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    std::vector<bnx_pair> buf;
    std::vector<uint64_t> offs;
    std::vector<IvDev> plan_tmp;
    bnx_server_stats st{};
};

// End of a request's next slice of `per` integers (no overflow for any per).
static uint64_t slice_end(const Request &r, uint64_t per) {
    return per >= r.iv.hi - r.cursor ? r.iv.hi : r.cursor + per;
}

// Workspace bytes of an iteration in which request i runs [cursor, ends[i]).
static uint64_t iteration_bytes(bnx_ctx *c, const std::vector<std::shared_ptr<Request>> &rs,
                                const std::vector<uint64_t> &ends, std::vector<IvDev> &tmp) {
    tmp.assign(rs.size(), IvDev{});
    for (size_t i = 0; i < rs.size(); i++) {
        tmp[i].lo = rs[i]->cursor;
        tmp[i].hi = ends[i];
    }
    PlanTotals t;
    plan_host(c, tmp.data(), rs.size(), &t);
    return ws_need_bytes(c, t, rs.size());
}

// ... in which each request runs its next `per` integers.
static uint64_t iteration_bytes(bnx_ctx *c, const std::vector<std::shared_ptr<Request>> &rs, uint64_t per,
                                std::vector<uint64_t> &ends, std::vector<IvDev> &tmp) {
    ends.resize(rs.size());
    for (size_t i = 0; i < rs.size(); i++) ends[i] = slice_end(*rs[i], per);
    return iteration_bytes(c, rs, ends, tmp);
}

// Slice ends of an iteration: a request with at most `fin` integers left runs all of
// them; every other request up to `base` integers; then up to `cap` integers in all, the
// rest going to the requests in the order given (arrival).  Returns the integers of the
// first two parts.
static uint64_t cut_slices(const std::vector<std::shared_ptr<Request>> &rs, uint64_t fin, uint64_t base,
                           uint64_t cap, std::vector<uint64_t> &ends) {
    ends.resize(rs.size());
    uint64_t used = 0;
    for (size_t i = 0; i < rs.size(); i++) {
        const uint64_t rem = rs[i]->iv.hi - rs[i]->cursor;
        ends[i] = rem <= fin ? rs[i]->iv.hi : slice_end(*rs[i], base);
        const uint64_t a = ends[i] - rs[i]->cursor;
        used = a > UINT64_MAX - used ? UINT64_MAX : used + a;
    }
    uint64_t left = cap > used ? cap - used : 0;
    for (size_t i = 0; i < rs.size() && left > 0; i++) {
        const uint64_t more = std::min<uint64_t>(rs[i]->iv.hi - ends[i], left);
        ends[i] += more;
        left -= more;
    }
    return used;
}

static void publish_stats(bnx_ctx *c, const Server &S) {
    std::lock_guard<std::mutex> g(c->stats_mu);
    c->srv_stats = S.st;
}

static void serve(bnx_ctx *c) {
    Server &S = *c->server;
    cudaSetDevice(c->device);
    std::vector<uint64_t> ends;
    for (;;) {
        std::vector<std::shared_ptr<Request>> batch;
        {
            std::unique_lock<std::mutex> lk(S.m);
            if (S.stop) break;
            while (!S.pending.empty() && S.active.size() < S.cfg.max_active) {
                auto r = S.pending.front();
                auto trial = S.active;
                trial.push_back(r);
                if (iteration_bytes(c, trial, S.cfg.slice, ends, S.plan_tmp) > S.budget) {
                    if (S.active.empty()) {  // its first slice does not fit even alone: it never will
                        r->status = BNX_E_NOMEM;
                        r->done = true;
                        r->t_done = Clock::now();
                        S.pending.pop_front();
                        S.st.rejected++;
                        S.st.completed++;
                        continue;
                    }
                    if (!r->deferred) {
                        r->deferred = true;
                        S.st.deferred++;
                    }
                    break;  // wait for memory: first come, first served
                }
                S.active.push_back(r);
                S.pending.pop_front();
            }
            {  // requests cancelled while waiting between iterations
                std::vector<std::shared_ptr<Request>> keep;
                for (auto &r : S.active) {
                    if (r->cancelled) {
                        r->status = BNX_E_CANCELLED;
                        r->done = true;
                        r->t_done = Clock::now();
                        S.st.completed++;
                        S.st.cancelled++;
                    } else {
                        keep.push_back(r);
                    }
                }
                S.active.swap(keep);
            }
            publish_stats(c, S);
            if (S.active.empty()) {
                S.cv.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            batch = S.active;
        }
        const size_t k = batch.size();
        NvtxRange r_it("bnx.serve.iteration");
        // this iteration's slices: as many integers in all as an equal share eq of
        // slice * max_active (at least `slice` each) would give; a request with at most eq
        // left finishes, every other one gets `slice`, and the rest go to those in arrival
        // order.  While the workspace exceeds the budget, halve the total down to no extra
        // share, then the per-request slice (and the finishing bound) down to one queue
        // segment
        const uint64_t share = S.cfg.slice > UINT64_MAX / S.cfg.max_active ? UINT64_MAX : S.cfg.slice * S.cfg.max_active;
        const uint64_t eq = std::max<uint64_t>(S.cfg.slice, share / k);
        uint64_t cap = 0;
        for (size_t i = 0; i < k; i++) {
            const uint64_t a = slice_end(*batch[i], eq) - batch[i]->cursor;
            cap = a > UINT64_MAX - cap ? UINT64_MAX : cap + a;
        }
        const uint64_t seg = 1ull << c->seg_log2();
        uint64_t base = S.cfg.slice, fin = eq;
        for (;;) {
            const uint64_t used = cut_slices(batch, fin, base, cap, ends);
            if (iteration_bytes(c, batch, ends, S.plan_tmp) <= S.budget) break;
            if (cap > used) {
                cap = std::max(used, cap / 2);
            } else if (fin > base) {
                fin = base;
                cap = 0;
            } else if (base > seg) {
                base = fin = std::max(seg, base / 2);
                cap = 0;
            } else {
                break;  // one segment each still does not fit: the run reports BNX_E_NOMEM
            }
        }
        int rc = ensure_staging(c, k);
        if (rc == BNX_OK) {
            for (size_t i = 0; i < k; i++) {
                const Request &r = *batch[i];
                IvDev &d = c->h_ivs[i];
                memset(&d, 0, sizeof d);
                d.lo = r.cursor;
                d.hi = ends[i];
                d.kinds = r.iv.kinds;
                d.id = (uint32_t)i;
            }
            S.offs.assign(k + 1, 0);
            size_t np = 0;
            rc = search_staged(c, k, S.buf.data(), S.buf.size(), &np, S.offs.data(), S.budget);
            if (rc == BNX_E_TRUNCATED) {
                S.buf.resize(np + 64);
                rc = search_staged(c, k, S.buf.data(), S.buf.size(), &np, S.offs.data(), S.budget);
            }
        }
        std::lock_guard<std::mutex> lk(S.m);
        S.st.iterations++;
        S.st.ws_peak_bytes = std::max<uint64_t>(S.st.ws_peak_bytes, ws_footprint(c));
        std::vector<std::shared_ptr<Request>> still;
        for (size_t i = 0; i < k; i++) {
            Request &r = *batch[i];
            if (r.cancelled) {  // cancelled during this iteration: its slice's pairs are dropped
                r.status = BNX_E_CANCELLED;
                r.done = true;
                r.t_done = Clock::now();
                S.st.completed++;
                S.st.cancelled++;
                continue;
            }
            if (rc == BNX_OK) {
                for (uint64_t e = S.offs[i]; e < S.offs[i + 1]; e++) {
                    bnx_pair p = S.buf[e];
                    p.iv = r.iv.id;
                    r.pairs.push_back(p);
                }
                r.cursor = ends[i];
            } else {
                r.status = rc;
                r.cursor = r.iv.hi;
            }
            if (r.cursor >= r.iv.hi) {
                r.done = true;
                r.t_done = Clock::now();
                S.st.completed++;
            } else {
                still.push_back(batch[i]);
            }
        }
        // requests admitted during this iteration are appended after `batch`
        for (size_t i = k; i < S.active.size(); i++) still.push_back(S.active[i]);
        S.active.swap(still);
        publish_stats(c, S);
    }
}

// The loop thread: a C++ exception in it (a failed host allocation) fails every request
// not yet finished and ends the loop, instead of terminating the process.
static void serve_guarded(bnx_ctx *c) {
    try {
        serve(c);
    } catch (...) {
        const bool oom = [] {
            try {
                throw;
            } catch (const std::bad_alloc &) {
                return true;
            } catch (...) {
                return false;
            }
        }();
        Server &S = *c->server;
        std::lock_guard<std::mutex> lk(S.m);
        for (auto &kv : S.all) {
            Request &r = *kv.second;
            if (!r.done) {
                r.status = oom ? BNX_E_NOMEM : BNX_E_STATE;
                r.done = true;
                r.t_done = Clock::now();
                S.st.completed++;
            }
        }
        S.pending.clear();
        S.active.clear();
        S.stop = true;
        c->serving.store(false);  // later submits are refused; bnx_server_stop still joins and frees
        publish_stats(c, S);
    }
}

}  // namespace bnx

using namespace bnx;

extern "C" {

static int bnx_server_start_impl(bnx_ctx *c, const bnx_server_cfg *cfg) {
    if (!c || !cfg) return fail(BNX_E_ARG, "NULL argument");
    if (cfg->max_active < 1 || cfg->slice < 1) return fail(BNX_E_ARG, "max_active and slice must be >= 1");
    if (cfg->max_active > (1u << 24)) return fail(BNX_E_ARG, "max_active must be <= 2^24 (a batch's interval limit)");
    std::lock_guard<std::mutex> g(c->mu);
    if (c->serving.load() || c->server)
        return fail(BNX_E_STATE, "already serving (a loop that ended on an error is released by bnx_server_stop)");
    cudaSetDevice(c->device);
    Server *S = new (std::nothrow) Server();
    if (!S) return fail(BNX_E_NOMEM, "host allocation failed");
    S->cfg = *cfg;
    if (cfg->mem_budget) {
        S->budget = cfg->mem_budget;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return fail(BNX_E_CUDA, "cudaMemGetInfo failed");
        }
        S->budget = (uint64_t)(0.9 * (double)fr);
    }
    S->st.budget_bytes = S->budget;
    publish_stats(c, *S);  // this loop's counters from the start
    S->buf.resize(4096);
    c->server = S;
    c->serving.store(true);
    S->th = std::thread(serve_guarded, c);
    return BNX_OK;
}

int bnx_server_start(bnx_ctx *c, const bnx_server_cfg *cfg) {
    return guarded([&] { return bnx_server_start_impl(c, cfg); });
}

static int bnx_server_submit_impl(bnx_ctx *c, const bnx_interval *iv, uint64_t *ticket) {
    if (!c || !iv || !ticket) return fail(BNX_E_ARG, "NULL argument");
    if (!c->serving.load() || !c->server) return fail(BNX_E_STATE, "not serving");
    int rc = validate_interval(c, iv->lo, iv->hi, iv->kinds);
    if (rc) return rc;
    Server &S = *c->server;
    auto r = std::make_shared<Request>();
    r->iv = *iv;
    r->cursor = iv->lo;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S.m);
        r->ticket = S.next_ticket++;
        S.pending.push_back(r);
        S.all[r->ticket] = r;
        S.st.submitted++;
        publish_stats(c, S);
    }
    S.cv.notify_one();
    *ticket = r->ticket;
    return BNX_OK;
}

int bnx_server_submit(bnx_ctx *c, const bnx_interval *iv, uint64_t *ticket) {
    return guarded([&] { return bnx_server_submit_impl(c, iv, ticket); });
}

int bnx_server_cancel(bnx_ctx *c, uint64_t ticket) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (!c->serving.load() || !c->server) return fail(BNX_E_STATE, "not serving");
    Server &S = *c->server;
    std::lock_guard<std::mutex> lk(S.m);
    auto it = S.all.find(ticket);
    if (it == S.all.end()) return fail(BNX_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request &r = *it->second;
    if (r.done || r.cancelled) return BNX_OK;
    r.cancelled = true;
    for (auto p = S.pending.begin(); p != S.pending.end(); ++p) {
        if (p->get() == &r) {  // not admitted yet: drop it now
            S.pending.erase(p);
            r.status = BNX_E_CANCELLED;
            r.done = true;
            r.t_done = Clock::now();
            S.st.completed++;
            S.st.cancelled++;
            publish_stats(c, S);
            break;
        }
    }
    return BNX_OK;
}

int bnx_server_poll(bnx_ctx *c, uint64_t ticket, bnx_pair *out, size_t cap, size_t *n_out, double *latency_s) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (!c->server) return fail(BNX_E_STATE, "not serving");
    Server &S = *c->server;
    std::lock_guard<std::mutex> lk(S.m);
    auto it = S.all.find(ticket);
    if (it == S.all.end()) return fail(BNX_E_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request &r = *it->second;
    if (!r.done) return BNX_E_BUSY;
    if (r.status != BNX_OK) {
        const int st = r.status;
        S.all.erase(it);
        return fail(st, "request failed: %s", bnx_strerror(st));
    }
    const size_t np = r.pairs.size();
    if (n_out) *n_out = np;
    if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    if (np > cap) return fail(BNX_E_TRUNCATED, "%zu pairs, buffer holds %zu", np, cap);
    if (np && !out) return fail(BNX_E_ARG, "out is NULL");
    if (np) memcpy(out, r.pairs.data(), np * sizeof(bnx_pair));
    S.all.erase(it);
    return BNX_OK;
}

int bnx_server_stop(bnx_ctx *c) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    Server *S = c->server;
    if (!S) return BNX_OK;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    c->serving.store(false);
    c->server = nullptr;
    delete S;
    return BNX_OK;
}

int bnx_server_get_stats(bnx_ctx *c, bnx_server_stats *out) {
    if (!c || !out) return fail(BNX_E_ARG, "NULL argument");
    std::lock_guard<std::mutex> g(c->stats_mu);
    *out = c->srv_stats;
    return BNX_OK;
}

static int bnx_workspace_bytes_impl(bnx_ctx *c, const bnx_interval *iv, size_t k, uint64_t *bytes) {
    if (!c || !bytes || (!iv && k)) return fail(BNX_E_ARG, "NULL argument");
    if (k > (1u << 24)) return fail(BNX_E_ARG, "at most 2^24 intervals per batch");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::vector<IvDev> d(k);
    for (size_t i = 0; i < k; i++) {
        int rc = validate_interval(c, iv[i].lo, iv[i].hi, iv[i].kinds);
        if (rc) return rc;
        memset(&d[i], 0, sizeof d[i]);
        d[i].lo = iv[i].lo;
        d[i].hi = iv[i].hi;
    }
    std::lock_guard<std::mutex> g(c->mu);
    PlanTotals t;
    plan_host(c, d.data(), k, &t);
    *bytes = ws_need_bytes(c, t, k);
    return BNX_OK;
}

int bnx_workspace_bytes(bnx_ctx *c, const bnx_interval *iv, size_t k, uint64_t *bytes) {
    return guarded([&] { return bnx_workspace_bytes_impl(c, iv, k, bytes); });
}

static int bnx_autotune_impl(bnx_ctx *c, const bnx_interval *iv, size_t k, int rounds, char *json_out, size_t json_cap) {
    if (!c || !iv || k == 0) return fail(BNX_E_ARG, "need a context and at least one sample interval");
    if (rounds < 1) rounds = 1;
    bnx_tune best;
    bnx_get_tune(c, &best);
    std::vector<bnx_pair> buf(1024);
    std::vector<uint64_t> offs(k + 1);
    auto time_of = [&](const bnx_tune &t, float *ms) -> int {
        int rc = bnx_set_tune(c, &t);
        if (rc) return rc;
        float bestms = 1e30f;
        for (int r = 0; r < rounds + 1; r++) {  // the first run builds the graph
            size_t np = 0;
            rc = bnx_batch(c, iv, k, buf.data(), buf.size(), &np, offs.data());
            if (rc == BNX_E_TRUNCATED) {
                buf.resize(np + 64);
                rc = bnx_batch(c, iv, k, buf.data(), buf.size(), &np, offs.data());
            }
            if (rc) return rc;
            if (r > 0) bestms = std::min(bestms, c->stats.ms_total);
        }
        *ms = bestms;
        return BNX_OK;
    };
    float best_ms = 0;
    int rc = time_of(best, &best_ms);
    if (rc) return rc;
    const uint32_t tiles[] = {13, 14, 15, 16};
    const uint32_t segt[] = {2, 4, 8, 16, 32};
    const uint32_t thr[] = {128, 256, 512, 1024};
    const uint32_t qs[] = {12, 13, 14, 15, 16};
    const uint32_t ctas[] = {0, 1, 2};
    const uint32_t kinds[] = {0, 2, 3};
    for (int pass = 0; pass < 2; pass++) {
        for (int field = 0; field < 6; field++) {
            const uint32_t *vals;
            int nv;
            switch (field) {
                case 0: vals = tiles; nv = 4; break;
                case 1: vals = segt; nv = 5; break;
                case 2: vals = thr; nv = 4; break;
                case 3: vals = qs; nv = 5; break;
                case 4: vals = ctas; nv = 3; break;
                default: vals = kinds; nv = 3; break;
            }
            for (int v = 0; v < nv; v++) {
                bnx_tune t = best;
                uint32_t *f = field == 0   ? &t.tile_log2
                              : field == 1 ? &t.seg_tiles
                              : field == 2 ? &t.threads
                              : field == 3 ? &t.small_q_log2
                              : field == 4 ? &t.ctas_per_sm
                                           : &t.tile_kind;
                if (*f == vals[v]) continue;
                *f = vals[v];
                float ms = 0;
                if (time_of(t, &ms) != BNX_OK) continue;  // a tuning that does not fit is skipped
                if (ms < best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
        }
    }
    rc = bnx_set_tune(c, &best);
    if (rc) return rc;
    if (json_out && json_cap) {
        snprintf(json_out, json_cap,
                 "{\"tile_log2\": %u, \"seg_tiles\": %u, \"threads\": %u, \"ctas_per_sm\": %u, "
                 "\"small_q_log2\": %u, \"tile_kind\": %u, \"ms\": %.4f}",
                 best.tile_log2, best.seg_tiles, best.threads, best.ctas_per_sm, best.small_q_log2, best.tile_kind,
                 best_ms);
    }
    return BNX_OK;
}

int bnx_autotune(bnx_ctx *c, const bnx_interval *iv, size_t k, int rounds, char *json_out, size_t json_cap) {
    return guarded([&] { return bnx_autotune_impl(c, iv, k, rounds, json_out, json_cap); });
}

}  // extern "C"
