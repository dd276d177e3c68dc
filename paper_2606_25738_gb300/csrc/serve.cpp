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
    double* out = nullptr;
    uint8_t* out_flags = nullptr;
    uint64_t foot = 0, cells = 0;
    Clock::time_point t_in, t_done;
};

struct Epoch {
    uint64_t ticket = 0;
    std::vector<Request*> reqs;
    std::vector<uint32_t> first;  // index of each request's first pair in the epoch
    std::vector<double> out;
    std::vector<uint8_t> flags;
    uint64_t foot = 0;
};

}  // namespace

struct phmm_server {
    phmm_ctx* ctx = nullptr;
    phmm_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work;  // scheduler: new request or stop
    std::condition_variable cv_done;  // pollers: a request finished
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> live;  // enqueued, not yet retired by poll
    std::vector<Epoch*> inflight;                  // touched by the scheduler thread only
    uint64_t next_id = 0;
    bool stop = false;
    bool single = false;  // after an ENOMEM epoch: admit one request at a time once
    phmm_server_stats st{};
    std::thread th;

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

    // Copy an epoch's results to its requests and complete them.
    void retire(Epoch* e, int rc) {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t q = 0; q < e->reqs.size(); ++q) {
            Request* r = e->reqs[q];
            int s = rc;
            if (rc == PHMM_OK || rc == PHMM_EINVAL) {
                const double* src = e->out.data() + e->first[q];
                const uint8_t* fl = e->flags.data() + e->first[q];
                memcpy(r->out, src, r->np * sizeof(double));
                if (r->out_flags) memcpy(r->out_flags, fl, r->np);
                s = PHMM_OK;
                for (uint32_t p = 0; p < r->np; ++p)
                    if (fl[p] & PHMM_PAIR_ERROR) s = PHMM_EINVAL;
            }
            finish(r, s);
        }
        st.bytes_inflight -= e->foot;
        cv_done.notify_all();
    }

    // Join requests into one host batch and submit it.  Returns the submit status.
    int submit(Epoch* e) {
        uint64_t nb = 0, nhb = 0;
        uint32_t nr = 0, nh = 0, np = 0;
        for (Request* r : e->reqs) {
            nb += r->roff[r->nr];
            nhb += r->hoff[r->nh];
            nr += r->nr;
            nh += r->nh;
            np += r->np;
        }
        std::vector<uint8_t> bases(nb), bq(nb), iq(nb), dq(nb), gq(nb), hap(nhb);
        std::vector<uint64_t> roff(nr + 1), hoff(nh + 1);
        std::vector<uint32_t> pr(np), ph(np);
        uint64_t ob = 0, oh = 0;
        uint32_t orr = 0, ohh = 0, op = 0;
        e->first.clear();
        for (Request* r : e->reqs) {
            const uint64_t rb = r->roff[r->nr], hb = r->hoff[r->nh];
            memcpy(&bases[ob], r->bases.data(), rb);
            memcpy(&bq[ob], r->bq.data(), rb);
            memcpy(&iq[ob], r->iq.data(), rb);
            memcpy(&dq[ob], r->dq.data(), rb);
            memcpy(&gq[ob], r->gq.data(), rb);
            memcpy(&hap[oh], r->hap.data(), hb);
            for (uint32_t i = 0; i < r->nr; ++i) roff[orr + i] = ob + r->roff[i];
            for (uint32_t i = 0; i < r->nh; ++i) hoff[ohh + i] = oh + r->hoff[i];
            e->first.push_back(op);
            for (uint32_t p = 0; p < r->np; ++p) {
                pr[op + p] = orr + r->pr[p];
                ph[op + p] = ohh + r->ph[p];
            }
            ob += rb;
            oh += hb;
            orr += r->nr;
            ohh += r->nh;
            op += r->np;
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
                Epoch* e = new Epoch();
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (stop || pending.empty()) {
                        delete e;
                        break;
                    }
                    uint64_t pairs = 0;
                    while (!pending.empty()) {
                        Request* r = pending.front();
                        if (st.bytes_inflight + e->foot + r->foot > budget) break;
                        if (!e->reqs.empty() && (pairs + r->np > max_pairs || single)) break;
                        e->reqs.push_back(r);
                        e->foot += r->foot;
                        pairs += r->np;
                        pending.pop_front();
                    }
                    if (e->reqs.empty()) {  // the head waits for memory held by running epochs
                        delete e;
                        break;
                    }
                    st.pending -= e->reqs.size();
                    st.admitted += e->reqs.size();
                    st.inflight += e->reqs.size();
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
                if ((rc == PHMM_EBUSY || rc == PHMM_ENOMEM) && (rc == PHMM_EBUSY || e->reqs.size() > 1)) {
                    // put the requests back in order; retry after a retirement (EBUSY) or
                    // one request at a time (ENOMEM of a joined epoch)
                    for (auto it = e->reqs.rbegin(); it != e->reqs.rend(); ++it) pending.push_front(*it);
                    st.pending += e->reqs.size();
                    st.admitted -= e->reqs.size();
                    st.inflight -= e->reqs.size();
                    st.bytes_inflight -= e->foot;
                    if (rc == PHMM_ENOMEM) single = true;
                    blocked = rc == PHMM_EBUSY;
                } else {
                    for (Request* r : e->reqs) finish(r, rc);
                    st.bytes_inflight -= e->foot;
                    cv_done.notify_all();
                }
                delete e;
                if (blocked && inflight.empty()) {
                    // nothing to wait for: the context has no room even when idle
                    Request* r = pending.front();
                    pending.pop_front();
                    st.pending--;
                    st.inflight++;
                    finish(r, PHMM_ENOMEM);
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
        // cancel what was never admitted
        std::lock_guard<std::mutex> lk(mu);
        while (!pending.empty()) {
            Request* r = pending.front();
            pending.pop_front();
            st.pending--;
            st.inflight++;
            finish(r, PHMM_ECANCELED);
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
    for (uint32_t p = 0; p < r->np; ++p)
        r->cells += (r->roff[r->pr[p] + 1] - r->roff[r->pr[p]]) * (r->hoff[r->ph[p] + 1] - r->hoff[r->ph[p]]);
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
