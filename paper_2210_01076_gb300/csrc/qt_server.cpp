// qt_server.cpp -- serving loop over many resident circuits (C ABI qt_server_*).
//
// Requests (a few circuit edits followed by an incremental update of one
// circuit) are queued and run by a pool of host worker threads.  Each circuit
// owns a CUDA stream, so requests on different circuits that run at the same
// time overlap on the GPU; a request that arrives while others are running
// starts as soon as a worker (a slot) and device memory free up -- continuous
// batching rather than a queue drained in rounds.  Device memory is admitted
// against a budget that counts every resident circuit's state and
// checkpoints: when a request's circuit is not resident and does not fit,
// idle circuits are evicted least-recently-used first (their next update is a
// full one); a request that cannot fit yet waits without blocking others.
// Requests on one circuit run in submission order, so a circuit's results do
// not depend on what else is in the mix.
//
// With a budget, the server also sizes every circuit's checkpoints to its
// share of the budget (the circuit's ckpt_budget option): the budget minus
// one spare state vector per circuit is divided in proportion to the
// circuits' state sizes, each getting room for its state and at least one
// checkpoint.  An evicted circuit's next request re-simulates it in full,
// which costs far more than the longer segments of fewer checkpoints, so
// the circuits stay resident whenever their states fit together.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qt_internal.h"

using namespace qt;

namespace {
using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int32_t slot = 0;
    std::vector<qt_edit> edits;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    qt_request_result result;
};

struct Slot {
    qt_circuit* c = nullptr;
    bool busy = false;
    uint64_t last_used = 0;
    size_t bytes = 0;          // device bytes held (as of its last request)
    size_t state_bytes = 0;    // one state vector
    int64_t ckpt_budget = 0;   // its share of the budget (0: no budget), applied before its next request
};
}  // namespace

struct qt_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::map<uint64_t, Request*> requests;
    std::vector<Slot> slots;
    std::vector<std::thread> workers;
    int64_t budget = 0;
    size_t resident = 0;
    int32_t evictions = 0;
    uint64_t next_ticket = 1, clock = 0;
    bool stopping = false;
    std::string err;
};

namespace {

qt_status apply_edits(qt_circuit* c, const std::vector<qt_edit>& edits, qt_request_result* res) {
    res->n_new_ids = 0;
    for (const qt_edit& e : edits) {
        qt_status s = QT_OK;
        qt_gate_id id = 0;
        switch (e.kind) {
            case QT_EDIT_INSERT_LEVEL: s = qt_insert_level(c, e.level); break;
            case QT_EDIT_REMOVE_LEVEL: s = qt_remove_level(c, e.level); break;
            case QT_EDIT_INSERT_GATE: s = qt_insert_gate(c, e.level, &e.gate, &id); break;
            case QT_EDIT_REMOVE_GATE: s = qt_remove_gate(c, e.level, e.id); break;
            case QT_EDIT_REPLACE_GATE: s = qt_replace_gate(c, e.level, e.id, &e.gate, &id); break;
            default: s = QT_ERR_ARG; break;
        }
        if (s != QT_OK) return s;
        if (id && res->n_new_ids < int32_t(sizeof(res->new_ids) / sizeof(res->new_ids[0])))
            res->new_ids[res->n_new_ids++] = id;
    }
    return QT_OK;
}

// Next runnable request: the oldest request of a circuit that is idle and has
// no older request waiting, whose memory fits the budget (after evicting idle
// circuits if needed).  Called with the lock held.
Request* pick(qt_server* s) {
    std::vector<char> seen(s->slots.size(), 0);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Request* r = *it;
        Slot& sl = s->slots[r->slot];
        if (seen[r->slot]) continue;
        seen[r->slot] = 1;
        if (sl.busy) continue;
        const size_t need = circuit_device_need(sl.c);
        if (s->budget > 0 && int64_t(need) > s->budget) {  // can never fit: fail it now
            r->result.status = QT_ERR_OOM;
            r->t_start = r->t_done = Clock::now();
            r->done = true;
            s->queue.erase(it);
            s->cv_done.notify_all();
            return pick(s);
        }
        if (s->budget > 0) {
            size_t others = s->resident - sl.bytes;
            while (int64_t(others + need) > s->budget) {
                // evict the least recently used idle resident circuit
                int victim = -1;
                for (size_t k = 0; k < s->slots.size(); ++k) {
                    const Slot& o = s->slots[k];
                    if (int(k) == r->slot || o.busy || o.bytes == 0) continue;
                    if (victim < 0 || o.last_used < s->slots[victim].last_used) victim = int(k);
                }
                if (victim < 0) break;
                Slot& v = s->slots[victim];
                circuit_release_device(v.c);
                s->resident -= v.bytes;
                others -= v.bytes;
                v.bytes = 0;
                s->evictions += 1;
            }
            if (int64_t(others + need) > s->budget) continue;  // wait for memory; try the next circuit
            // reserve the circuit's memory now so concurrent admissions see it
            s->resident = others + need;
            sl.bytes = need;
        }
        s->queue.erase(it);
        sl.busy = true;
        return r;
    }
    return nullptr;
}

void worker_main(qt_server* s) {
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        Request* r = nullptr;
        s->cv_work.wait(lk, [&] { return (r = pick(s)) != nullptr || (s->stopping && s->queue.empty()); });
        if (!r) return;
        Slot& sl = s->slots[r->slot];
        qt_circuit* c = sl.c;
        const int64_t ckpt_budget = sl.ckpt_budget;
        lk.unlock();
        r->t_start = Clock::now();
        qt_status st = QT_OK;
        if (ckpt_budget > 0) st = qt_set_option(c, "ckpt_budget", ckpt_budget);
        if (st == QT_OK) st = apply_edits(c, r->edits, &r->result);
        if (st == QT_OK) st = qt_update_state(c, 0, &r->result.stats);
        r->t_done = Clock::now();
        lk.lock();
        r->result.status = st;
        const size_t held = circuit_device_bytes(c);
        s->resident = s->resident - sl.bytes + held;
        sl.bytes = held;
        sl.busy = false;
        sl.last_used = ++s->clock;
        r->done = true;
        s->cv_done.notify_all();
        s->cv_work.notify_all();  // memory or a circuit may have freed up
    }
}

double ms(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double, std::milli>(b - a).count(); }

}  // namespace

extern "C" {

qt_status qt_server_create(int32_t workers, int64_t hbm_budget_bytes, qt_server** out) {
    if (!out || workers < 1 || workers > 256 || hbm_budget_bytes < 0) {
        set_thread_error("qt_server_create: workers in [1, 256], budget >= 0, out not NULL");
        return QT_ERR_ARG;
    }
    try {
        qt_server* s = new qt_server();
        s->budget = hbm_budget_bytes;
        for (int i = 0; i < workers; ++i) s->workers.emplace_back(worker_main, s);
        *out = s;
        return QT_OK;
    } catch (...) {
        set_thread_error("qt_server_create: could not start the workers");
        return QT_ERR_OOM;
    }
}

qt_status qt_server_destroy(qt_server* s) {
    if (!s) return QT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->requests) delete kv.second;
    delete s;
    return QT_OK;
}

qt_status qt_server_add_circuit(qt_server* s, qt_circuit* c, int32_t* slot) {
    if (!s || !c || !slot) return QT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    Slot sl;
    sl.c = c;
    sl.bytes = circuit_device_bytes(c);
    sl.state_bytes = circuit_state_bytes(c);
    sl.last_used = ++s->clock;
    s->resident += sl.bytes;
    s->slots.push_back(sl);
    *slot = int32_t(s->slots.size()) - 1;
    if (s->budget > 0) {
        // checkpoint shares: (budget - one spare state per circuit) split by
        // state size, at least the state and one checkpoint each
        double states = 0.0;
        for (const Slot& o : s->slots) states += double(o.state_bytes);
        const double pool = double(s->budget) - states;
        for (Slot& o : s->slots) {
            const double share = pool > 0.0 ? pool * double(o.state_bytes) / states : 0.0;
            o.ckpt_budget = int64_t(std::max(share, 2.0 * double(o.state_bytes)));
            // an idle circuit takes its share now (admission sizes its need
            // from it); a busy one from its worker before its next request
            if (!o.busy) qt_set_option(o.c, "ckpt_budget", o.ckpt_budget);
        }
    }
    return QT_OK;
}

qt_status qt_server_submit(qt_server* s, int32_t slot, int32_t nedits, const qt_edit* edits, uint64_t* ticket) {
    if (!s || !ticket || nedits < 0 || (nedits > 0 && !edits)) return QT_ERR_ARG;
    try {
        Request* r = new Request();
        r->slot = slot;
        r->edits.assign(edits, edits + nedits);
        std::memset(&r->result, 0, sizeof r->result);
        r->result.circuit = slot;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (slot < 0 || slot >= int32_t(s->slots.size())) {
                delete r;
                s->err = "no such circuit slot";
                return QT_ERR_RANGE;
            }
            r->ticket = s->next_ticket++;
            r->t_submit = Clock::now();
            s->requests[r->ticket] = r;
            s->queue.push_back(r);
            *ticket = r->ticket;
        }
        s->cv_work.notify_one();
        return QT_OK;
    } catch (...) {
        return QT_ERR_OOM;
    }
}

qt_status qt_server_wait(qt_server* s, uint64_t ticket, qt_request_result* out) {
    if (!s || !out) return QT_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(ticket);
    if (it == s->requests.end()) {
        s->err = "unknown ticket";
        return QT_ERR_NOT_FOUND;
    }
    Request* r = it->second;
    s->cv_done.wait(lk, [&] { return r->done; });
    *out = r->result;
    out->queue_ms = ms(r->t_submit, r->t_start);
    out->latency_ms = ms(r->t_submit, r->t_done);
    out->service_ms = ms(r->t_start, r->t_done);
    s->requests.erase(it);
    delete r;
    return QT_OK;
}

qt_status qt_server_info(qt_server* s, int64_t* resident_bytes, int32_t* evictions, int32_t* queued) {
    if (!s) return QT_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (resident_bytes) *resident_bytes = int64_t(s->resident);
    if (evictions) *evictions = s->evictions;
    if (queued) *queued = int32_t(s->queue.size());
    return QT_OK;
}

}  // extern "C"
