// Serving loop: continuous batching of active-region requests over one phmm context.
//
// The paper scores a batch of independent read-haplotype pairs (Section 3: the pairs of
// an active region are independent); it has no request layer.  This file is a client of
// the public batch ABI only (phmm_submit_batch / phmm_poll / phmm_batch_footprint): a
// scheduler thread joins waiting requests into epochs (one batch each), admits them by
// device footprint, keeps up to max_inflight_epochs epochs on the device at once and
// hands each request its own results when its epoch finishes.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "phmm.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int status = PHMM_PENDING;
    uint32_t nr = 0, nh = 0, np = 0;
    std::vector<uint8_t> bases, bq, iq, dq, gq, hap;
    std::vector<uint64_t> roff, hoff;
    std::vector<uint32_t> pr, ph;
    std::vector<uint64_t> pcells;  // l * k of each pair
    double* out = nullptr;
    uint8_t* out_flags = nullptr;
    uint64_t foot = 0, cells = 0;
    bool small = false;
    uint32_t next = 0;        // first pair not yet given to an epoch
    uint32_t done = 0;        // pairs whose epoch has finished
    bool started = false;     // a first chunk was admitted
    bool any_error = false;   // a pair came back with PHMM_PAIR_ERROR
    int fail = PHMM_OK;       // status of a failed epoch, if any
    Clock::time_point t_in, t_done;
};

// A slice of one request's pairs inside an epoch (the whole request, or one chunk of a
// request larger than the epoch cell budget).
struct Segment {
    Request* r = nullptr;
    uint32_t p0 = 0, p1 = 0;  // the request's pairs [p0, p1)
    uint32_t first = 0;       // index of pair p0 in the epoch's batch
};

struct Epoch {
    uint64_t ticket = 0;
    std::vector<Segment> segs;
    std::vector<double> out;
    std::vector<uint8_t> flags;
    uint64_t foot = 0;
    bool large = false;
};

}  // namespace

struct phmm_server {
    phmm_ctx* ctx = nullptr;
    phmm_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;  // scheduler: new request or stop
    std::condition_variable cv_done;  // pollers: a request finished
    std::deque<Request*> pending;     // requests with pairs not yet in an epoch, by arrival
    std::unordered_map<uint64_t, Request*> live;  // enqueued, not yet retired by poll
    std::vector<Epoch*> inflight;                  // touched by the scheduler thread only
    uint64_t next_id = 0;
    bool stop = false;
    bool single = false;  // after an ENOMEM epoch: admit one request at a time once
    phmm_server_stats st{};
    std::thread th;

    // default budget: about 15 ms of one GB300 per epoch (measured: small requests' p99 at
    // 8 req/s fell from 208 ms at 1e11 cells to 57 ms at 2e10, same throughput)
    uint64_t epoch_cells() const { return cfg.epoch_cells ? cfg.epoch_cells : 20000000000ull; }
    uint64_t small_cells() const { return cfg.small_cells ? cfg.small_cells : epoch_cells() / 20; }

    void finish(Request* r, int status) {  // with mu held
        r->status = status;
        r->t_done = Clock::now();
        if (status == PHMM_OK || status == PHMM_EINVAL) {
            st.completed++;
            st.cells_completed += r->cells;
        } else {
            st.failed++;
        }
        st.inflight--;
    }

    // Copy an epoch's results to its requests; complete the requests whose last pairs
    // these were.
    void retire(Epoch* e, int rc) {
        std::lock_guard<std::mutex> lk(mu);
        for (const Segment& g : e->segs) {
            Request* r = g.r;
            const uint32_t n = g.p1 - g.p0;
            if (rc == PHMM_OK || rc == PHMM_EINVAL) {
                const double* src = e->out.data() + g.first;
                const uint8_t* fl = e->flags.data() + g.first;
                memcpy(r->out + g.p0, src, n * sizeof(double));
                if (r->out_flags) memcpy(r->out_flags + g.p0, fl, n);
                for (uint32_t p = 0; p < n; ++p)
                    if (fl[p] & PHMM_PAIR_ERROR) r->any_error = true;
            } else if (r->fail == PHMM_OK) {
                r->fail = rc;
            }
            r->done += n;
            if (r->done == r->np)
                finish(r, r->fail != PHMM_OK ? r->fail : (r->any_error ? PHMM_EINVAL : PHMM_OK));
        }
        st.bytes_inflight -= e->foot;
        cv_done.notify_all();
    }

    // Join the segments' requests into one host batch (every read and haplotype of each
    // request, the segment's pairs) and submit it.  Returns the submit status.
    int submit(Epoch* e) {
        uint64_t nb = 0, nhb = 0;
        uint32_t nr = 0, nh = 0, np = 0;
        for (const Segment& g : e->segs) {
            nb += g.r->roff[g.r->nr];
            nhb += g.r->hoff[g.r->nh];
            nr += g.r->nr;
            nh += g.r->nh;
            np += g.p1 - g.p0;
        }
        std::vector<uint8_t> bases(nb), bq(nb), iq(nb), dq(nb), gq(nb), hap(nhb);
        std::vector<uint64_t> roff(nr + 1), hoff(nh + 1);
        std::vector<uint32_t> pr(np), ph(np);
        uint64_t ob = 0, oh = 0;
        uint32_t orr = 0, ohh = 0, op = 0;
        for (Segment& g : e->segs) {
            const Request* r = g.r;
            const uint64_t rb = r->roff[r->nr], hb = r->hoff[r->nh];
            memcpy(&bases[ob], r->bases.data(), rb);
            memcpy(&bq[ob], r->bq.data(), rb);
            memcpy(&iq[ob], r->iq.data(), rb);
            memcpy(&dq[ob], r->dq.data(), rb);
            memcpy(&gq[ob], r->gq.data(), rb);
            memcpy(&hap[oh], r->hap.data(), hb);
            for (uint32_t i = 0; i < r->nr; ++i) roff[orr + i] = ob + r->roff[i];
            for (uint32_t i = 0; i < r->nh; ++i) hoff[ohh + i] = oh + r->hoff[i];
            g.first = op;
            for (uint32_t p = g.p0; p < g.p1; ++p, ++op) {
                pr[op] = orr + r->pr[p];
                ph[op] = ohh + r->ph[p];
            }
            ob += rb;
            oh += hb;
            orr += r->nr;
            ohh += r->nh;
        }
        roff[nr] = nb;
        hoff[nh] = nhb;
        e->out.assign(np, 0.0);
        e->flags.assign(np, 0);
        phmm_batch b{};
        b.n_reads = nr;
        b.read_bases = bases.data();
        b.read_off = roff.data();
        b.base_q = bq.data();
        b.ins_q = iq.data();
        b.del_q = dq.data();
        b.gcp_q = gq.data();
        b.n_haps = nh;
        b.hap_bases = hap.data();
        b.hap_off = hoff.data();
        b.n_pairs = np;
        b.pair_read = pr.data();
        b.pair_hap = ph.data();
        b.out_log10 = e->out.data();
        b.out_flags = e->flags.data();
        // host inputs are copied to the device before submit returns
        return phmm_submit_batch(ctx, &b, &e->ticket);
    }

    // Gives the epoch the next pairs of r: all of them, or for a request larger than
    // the cell budget the pairs up to that budget (at least one).  With mu held.
    void take(Epoch* e, Request* r, uint64_t& cells, uint32_t& pairs, uint32_t max_pairs) {
        Segment g;
        g.r = r;
        g.p0 = r->next;
        uint64_t c = 0;
        uint32_t p = r->next;
        const uint64_t cap = epoch_cells() > cells ? epoch_cells() - cells : 0;
        while (p < r->np && (p == r->next || (c + r->pcells[p] <= cap && pairs + (p - r->next) < max_pairs)))
            c += r->pcells[p++];
        g.p1 = p;
        r->next = p;
        if (!r->started) {
            r->started = true;
            st.admitted++;
            st.inflight++;
        }
        e->segs.push_back(g);
        e->foot += r->foot;
        cells += c;
        pairs += g.p1 - g.p0;
    }

    // Forms the next epoch (with mu held).  Small requests (at most small_cells) go first,
    // in arrival order, into epochs of their own; then larger requests in arrival order,
    // split into chunks of at most epoch_cells, so no epoch holds the device for long and
    // small requests that arrive meanwhile start within about one epoch.  A large request
    // that has waited longer than max_wait_ms goes ahead of small ones.  Large epochs use
    // at most max_inflight_epochs - 1 slots, leaving one for small requests.
    Epoch* form(uint32_t max_pairs, uint32_t max_ep, uint64_t budget, size_t large_inflight) {
        const auto now = Clock::now();
        const double max_wait = cfg.max_wait_ms ? (double)cfg.max_wait_ms : 2000.0;
        bool have_small = false, aged = false;
        for (Request* r : pending) {
            if (r->small) have_small = true;
            else if (std::chrono::duration<double, std::milli>(now - r->t_in).count() > max_wait) aged = true;
        }
        const bool large_slot = max_ep < 2 || large_inflight + 1 < max_ep;
        const bool want_large = large_slot && (aged || !have_small);
        Epoch* e = new Epoch();
        e->large = want_large;
        uint64_t cells = 0;
        uint32_t pairs = 0;
        for (auto it = pending.begin(); it != pending.end();) {
            Request* r = *it;
            if (r->small == want_large) {
                ++it;
                continue;
            }
            if (st.bytes_inflight + e->foot + r->foot > budget) break;  // wait for memory
            if (!e->segs.empty() && (single || pairs + (r->np - r->next) > max_pairs || cells >= epoch_cells()))
                break;
            take(e, r, cells, pairs, max_pairs);
            if (r->next == r->np) {
                it = pending.erase(it);
                st.pending--;
            } else {
                break;  // a chunk of a large request fills the epoch
            }
        }
        if (e->segs.empty()) {
            delete e;
            return nullptr;
        }
        return e;
    }

    // Puts an epoch that could not be submitted back: its requests' cursors move back and
    // requests that had left the queue return to its front.  With mu held.
    void unform(Epoch* e) {
        for (auto it = e->segs.rbegin(); it != e->segs.rend(); ++it) {
            Request* r = it->r;
            const bool was_out = r->next == r->np;
            r->next = it->p0;
            if (r->next == 0 && r->done == 0 && r->started) {
                r->started = false;
                st.admitted--;
                st.inflight--;
            }
            if (was_out) {
                pending.push_front(r);
                st.pending++;
            }
        }
    }

    void run() {
        const uint32_t max_pairs = cfg.max_epoch_pairs ? cfg.max_epoch_pairs : (1u << 20);
        const uint32_t max_ep = cfg.max_inflight_epochs ? cfg.max_inflight_epochs : 2;
        const uint64_t budget = cfg.mem_budget_bytes ? cfg.mem_budget_bytes : (40ull << 30);
        for (;;) {
            // retire finished epochs
            for (size_t i = 0; i < inflight.size();) {
                Epoch* e = inflight[i];
                const int rc = phmm_poll(ctx, e->ticket, 0);
                if (rc == PHMM_PENDING) {
                    ++i;
                    continue;
                }
                retire(e, rc);
                delete e;
                inflight.erase(inflight.begin() + i);
            }
            // admit waiting requests into new epochs while a slot and memory are free
            bool blocked = false;
            while (!blocked && inflight.size() < max_ep) {
                Epoch* e = nullptr;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (stop || pending.empty()) break;
                    size_t large = 0;
                    for (Epoch* x : inflight) large += x->large ? 1 : 0;
                    e = form(max_pairs, max_ep, budget, large);
                    if (!e) break;  // the head waits for memory or a slot held by running epochs
                    st.bytes_inflight += e->foot;
                }
                const int rc = submit(e);
                if (rc == PHMM_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    st.epochs++;
                    single = false;
                    inflight.push_back(e);
                    continue;
                }
                std::lock_guard<std::mutex> lk(mu);
                st.bytes_inflight -= e->foot;
                if ((rc == PHMM_EBUSY || rc == PHMM_ENOMEM) && (rc == PHMM_EBUSY || e->segs.size() > 1)) {
                    // retry after a retirement (EBUSY) or one request at a time (ENOMEM of
                    // a joined epoch)
                    unform(e);
                    if (rc == PHMM_ENOMEM) single = true;
                    blocked = rc == PHMM_EBUSY;
                } else {
                    for (const Segment& g : e->segs) {
                        Request* r = g.r;
                        if (r->fail == PHMM_OK) r->fail = rc;
                        r->done += g.p1 - g.p0;
                        if (r->done == r->np) finish(r, r->fail);
                    }
                    cv_done.notify_all();
                }
                delete e;
                if (blocked && inflight.empty()) {
                    // nothing to wait for: the context has no room even when idle
                    Request* r = pending.front();
                    pending.pop_front();
                    st.pending--;
                    if (!r->started) st.inflight++;
                    r->fail = PHMM_ENOMEM;
                    r->done += r->np - r->next;
                    r->next = r->np;
                    if (r->done == r->np) finish(r, PHMM_ENOMEM);
                    cv_done.notify_all();
                    blocked = false;
                }
            }
            std::unique_lock<std::mutex> lk(mu);
            if (stop && inflight.empty()) break;
            if (inflight.empty() && pending.empty() && !stop)
                cv_work.wait(lk);
            else
                cv_work.wait_for(lk, std::chrono::microseconds(100));
        }
        // cancel what was never admitted (or not completely)
        std::lock_guard<std::mutex> lk(mu);
        while (!pending.empty()) {
            Request* r = pending.front();
            pending.pop_front();
            st.pending--;
            if (!r->started) st.inflight++;
            r->done += r->np - r->next;
            r->next = r->np;
            if (r->fail == PHMM_OK) r->fail = PHMM_ECANCELED;
            if (r->done == r->np) finish(r, r->fail);
        }
        cv_done.notify_all();
    }
};

extern "C" {

int phmm_server_create(phmm_ctx* ctx, const phmm_server_config* cfg, phmm_server** out) {
    if (!ctx || !out) return PHMM_EINVAL;
    *out = nullptr;
    phmm_server* s = new phmm_server();
    s->ctx = ctx;
    if (cfg) s->cfg = *cfg;
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return PHMM_OK;
}

int phmm_server_enqueue(phmm_server* s, const phmm_batch* b, uint64_t* req_id) {
    if (!s || !b || !req_id || b->inputs_on_device || b->outputs_on_device) return PHMM_EINVAL;
    if (b->n_pairs == 0 || !b->read_bases || !b->base_q || !b->ins_q || !b->del_q || !b->gcp_q ||
        !b->hap_bases || !b->out_log10)
        return PHMM_EINVAL;
    uint64_t foot = 0;
    const int rc = phmm_batch_footprint(s->ctx, b, &foot);  // also validates offsets and indices
    if (rc != PHMM_OK) return rc;
    const uint64_t budget = s->cfg.mem_budget_bytes ? s->cfg.mem_budget_bytes : (40ull << 30);
    if (foot > budget) return PHMM_ENOMEM;
    Request* r = new Request();
    r->nr = b->n_reads;
    r->nh = b->n_haps;
    r->np = b->n_pairs;
    const uint64_t nb = b->read_off[r->nr], nhb = b->hap_off[r->nh];
    r->bases.assign(b->read_bases, b->read_bases + nb);
    r->bq.assign(b->base_q, b->base_q + nb);
    r->iq.assign(b->ins_q, b->ins_q + nb);
    r->dq.assign(b->del_q, b->del_q + nb);
    r->gq.assign(b->gcp_q, b->gcp_q + nb);
    r->hap.assign(b->hap_bases, b->hap_bases + nhb);
    r->roff.assign(b->read_off, b->read_off + r->nr + 1);
    r->hoff.assign(b->hap_off, b->hap_off + r->nh + 1);
    r->pr.assign(b->pair_read, b->pair_read + r->np);
    r->ph.assign(b->pair_hap, b->pair_hap + r->np);
    r->pcells.resize(r->np);
    for (uint32_t p = 0; p < r->np; ++p) {
        r->pcells[p] = (r->roff[r->pr[p] + 1] - r->roff[r->pr[p]]) * (r->hoff[r->ph[p] + 1] - r->hoff[r->ph[p]]);
        r->cells += r->pcells[p];
    }
    r->small = r->cells <= s->small_cells();
    r->out = b->out_log10;
    r->out_flags = b->out_flags;
    r->foot = foot;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return PHMM_ECANCELED;
        }
        if (s->cfg.max_pending && s->pending.size() >= s->cfg.max_pending) {
            delete r;
            return PHMM_EBUSY;
        }
        r->id = ++s->next_id;
        r->t_in = Clock::now();
        s->pending.push_back(r);
        s->live[r->id] = r;
        s->st.enqueued++;
        s->st.pending++;
        *req_id = r->id;
    }
    s->cv_work.notify_one();
    return PHMM_OK;
}

int phmm_server_poll(phmm_server* s, uint64_t id, int timeout_ms, double* latency_ms) {
    if (!s) return PHMM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->live.find(id) == s->live.end()) return PHMM_ENOTFOUND;
    // look the request up again after every wake-up: another poller may have retired it
    auto done = [s, id] {
        auto f = s->live.find(id);
        return f == s->live.end() || f->second->status != PHMM_PENDING;
    };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    auto it = s->live.find(id);
    if (it == s->live.end()) return PHMM_ENOTFOUND;
    Request* r = it->second;
    if (r->status == PHMM_PENDING) return PHMM_PENDING;
    const int rc = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_in).count();
    s->live.erase(it);
    delete r;
    return rc;
}

int phmm_server_get_stats(phmm_server* s, phmm_server_stats* out) {
    if (!s || !out) return PHMM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return PHMM_OK;
}

void phmm_server_destroy(phmm_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& kv : s->live) delete kv.second;
    delete s;
}

}  // extern "C"
