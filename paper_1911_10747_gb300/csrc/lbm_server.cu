// Continuous-batching request loop for boiling runs (host code on top of the
// public C ABI).  Requests (a run configuration and a step count) queue in
// arrival order; each tick admits queued requests while the device-memory
// budget and the slot limit allow, advances every active run together by
// one chunk through a concurrent batch graph, and retires the runs that
// reached their step count (their diagnostics, and optionally rho and T, are
// kept on the host and their device memory is freed for the next
// admissions).  lbm_server_poll does the same without waiting: requests that
// arrive while a chunk runs are admitted at once and join at the next chunk.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_launch.h"

namespace {

struct Request {
    int64_t id = 0;
    lbm_domain_t d{};
    lbm_heater_t ht{};
    lbm_eos_t eo{};
    lbm_bc_t bc{};
    lbm_opts_t op{};
    int64_t steps = 0, done = 0;
    uint64_t bytes = 0;
    int keep = 0;
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    double t_submit = 0, t_start = 0, t_done = 0;
    lbm_handle h = nullptr;
    double diag[4] = {0, 0, 0, 0};
    std::vector<double> rho, T;
    std::string err;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct lbm_server_s {
    uint64_t budget = 0, used = 0;
    int max_active = 0, chunk = 0, device = 0;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::vector<int64_t> active;
    lbm_batch batch = nullptr;
    bool dirty = true;
    bool inflight = false;   // a chunk of inflight_k steps is queued on the batch
    int64_t inflight_k = 0;
    std::vector<int64_t> inflight_ids;  // the runs in that chunk (later admissions are not)
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    std::string msg;
};

static int sfail(lbm_server_s *s, int code, const std::string &m) {
    if (s) s->msg = m; else lbmgb::set_global_error(m);
    return code;
}

static void retire(lbm_server_s *s, Request &r, int state, const std::string &err) {
    if (r.h) lbm_destroy(r.h);
    r.h = nullptr;
    s->used -= std::min(s->used, r.bytes);
    r.state = state;
    r.err = err;
    r.t_done = seconds_since(s->t0);
    s->dirty = true;
}

extern "C" {

int lbm_server_create(uint64_t hbm_budget_bytes, int32_t max_active, int32_t chunk_steps, int32_t device,
                      lbm_server *out) {
    if (!out) return sfail(nullptr, LBM_E_INVAL, "out is NULL");
    *out = nullptr;
    if (hbm_budget_bytes == 0 || max_active < 1 || chunk_steps < 1)
        return sfail(nullptr, LBM_E_INVAL, "budget, max_active and chunk_steps must be positive");
    lbm_server_s *s = new (std::nothrow) lbm_server_s();
    if (!s) return sfail(nullptr, LBM_E_NOMEM, "host allocation failed");
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    s->chunk = chunk_steps;
    s->device = device;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return LBM_OK;
}

int lbm_server_destroy(lbm_server s) {
    if (!s) return LBM_OK;
    if (s->batch && s->inflight) lbm_batch_sync(s->batch);
    if (s->batch) lbm_batch_destroy(s->batch);
    for (auto &kv : s->reqs)
        if (kv.second->h) lbm_destroy(kv.second->h);
    delete s;
    return LBM_OK;
}

const char *lbm_server_last_error(lbm_server s) { return s ? s->msg.c_str() : lbm_last_error(nullptr); }

int lbm_server_submit(lbm_server s, const lbm_domain_t *domain, const lbm_heater_t *heater, const lbm_eos_t *eos,
                      const lbm_bc_t *bc, const lbm_opts_t *opts, int64_t steps, int32_t keep_fields, int64_t *id) {
    if (!s || !domain || !heater || !eos || !bc || !opts || !id)
        return sfail(s, LBM_E_INVAL, "NULL argument");
    if (steps < 1) return sfail(s, LBM_E_INVAL, "steps must be >= 1");
    uint64_t bytes = 0;
    int rc = lbm_device_bytes(domain, heater, opts, &bytes);
    if (rc != LBM_OK) return sfail(s, rc, lbm_last_error(nullptr));
    if (bytes > s->budget) return sfail(s, LBM_E_INVAL, "request needs more device memory than the whole budget");
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->d = *domain; r->ht = *heater; r->eo = *eos; r->bc = *bc; r->op = *opts;
    r->op.stream = nullptr;        // each run gets its own stream
    r->op.device = s->device;
    r->steps = steps;
    r->bytes = bytes;
    r->keep = keep_fields != 0;
    r->t_submit = seconds_since(s->t0);
    *id = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    return LBM_OK;
}

// Admission: arrival order, while slots and memory allow.
static void admit(lbm_server_s *s, int &nfin) {
    while (!s->queue.empty() && (int)s->active.size() < s->max_active) {
        Request &r = *s->reqs[s->queue.front()];
        if (s->used + r.bytes > s->budget) break;
        s->queue.pop_front();
        int rc = lbm_create(&r.d, &r.ht, &r.eo, &r.bc, &r.op, &r.h);
        if (rc != LBM_OK) {
            r.h = nullptr;
            r.state = 3;
            r.err = lbm_last_error(nullptr);
            r.t_done = seconds_since(s->t0);
            nfin++;
            continue;
        }
        s->used += r.bytes;
        r.state = 1;
        r.t_start = seconds_since(s->t0);
        s->active.push_back(r.id);
        s->dirty = true;
    }
}

// Queue the next chunk over every active run (no wait).
static int launch_chunk(lbm_server_s *s) {
    if (s->inflight || s->active.empty()) return LBM_OK;
    if (s->dirty) {
        if (s->batch) lbm_batch_destroy(s->batch);
        s->batch = nullptr;
        std::vector<lbm_handle> hs;
        for (int64_t id : s->active) hs.push_back(s->reqs[id]->h);
        int rc = lbm_batch_create(hs.data(), (int32_t)hs.size(), &s->batch);
        if (rc != LBM_OK) return sfail(s, rc, lbm_batch_last_error(nullptr));
        s->dirty = false;
    }
    int64_t k = s->chunk;
    for (int64_t id : s->active) k = std::min(k, s->reqs[id]->steps - s->reqs[id]->done);
    int rc = lbm_batch_step(s->batch, k);
    if (rc != LBM_OK) return sfail(s, rc, lbm_batch_last_error(s->batch));
    s->inflight = true;
    s->inflight_k = k;
    s->inflight_ids = s->active;
    return LBM_OK;
}

// Finish the chunk in flight (waiting for it, or only if it is done) and
// retire the runs that reached their step count or faulted.
static int complete_chunk(lbm_server_s *s, bool wait, int &nfin) {
    if (!s->inflight) return LBM_OK;
    if (!wait) {
        int32_t done = 0;
        int rc = lbm_batch_query(s->batch, &done);
        if (rc != LBM_OK) return sfail(s, rc, lbm_batch_last_error(s->batch));
        if (!done) return LBM_OK;
    }
    int rc = lbm_batch_sync(s->batch);
    if (rc != LBM_OK && rc != LBM_E_NUMERIC) return sfail(s, rc, lbm_batch_last_error(s->batch));
    const int64_t k = s->inflight_k;
    s->inflight = false;
    std::vector<int64_t> still;
    for (int64_t id : s->active) {
        Request &r = *s->reqs[id];
        if (std::find(s->inflight_ids.begin(), s->inflight_ids.end(), id) == s->inflight_ids.end()) {
            still.push_back(id);  // admitted after the chunk was launched
            continue;
        }
        r.done += k;
        int src = lbm_sync(r.h);
        if (src != LBM_OK) {  // a faulted run is retired alone; the others go on
            retire(s, r, 3, lbm_last_error(r.h));
            nfin++;
            continue;
        }
        if (r.done < r.steps) {
            still.push_back(id);
            continue;
        }
        double row[4];
        src = lbm_series(r.h, r.steps - 1, 1, row);
        if (src == LBM_OK) std::memcpy(r.diag, row, sizeof(row));
        if (src == LBM_OK && r.keep) {
            // T rows: the heater's and the fluid's, or for model A (no heater,
            // walls) the heated wall's Dirichlet row and the fluid's
            const bool model_a = r.ht.ny_solid == 0 && !(r.d.flags & LBM_PERIODIC_Y);
            const size_t nfl = (size_t)r.d.nx * r.d.ny_fluid,
                         ntl = (size_t)r.d.nx * (r.d.ny_fluid + (model_a ? 1 : r.ht.ny_solid));
            r.rho.resize(nfl);
            r.T.resize(ntl);
            double *dst[2] = {r.rho.data(), r.T.data()};
            src = lbm_fields(r.h, LBM_FIELD_RHO | LBM_FIELD_T, dst, 0);
        }
        retire(s, r, src == LBM_OK ? 2 : 3, src == LBM_OK ? "" : lbm_last_error(r.h));
        nfin++;
    }
    s->active.swap(still);
    return LBM_OK;
}

int lbm_server_tick(lbm_server s, int32_t *finished) {
    if (!s) return LBM_E_INVAL;
    int nfin = 0, rc;
    if ((rc = complete_chunk(s, true, nfin)) != LBM_OK) return rc;
    admit(s, nfin);
    if ((rc = launch_chunk(s)) != LBM_OK) return rc;
    if ((rc = complete_chunk(s, true, nfin)) != LBM_OK) return rc;
    if (finished) *finished = nfin;
    return LBM_OK;
}

int lbm_server_poll(lbm_server s, int32_t *finished) {
    if (!s) return LBM_E_INVAL;
    int nfin = 0, rc;
    if ((rc = complete_chunk(s, false, nfin)) != LBM_OK) return rc;
    admit(s, nfin);
    if ((rc = launch_chunk(s)) != LBM_OK) return rc;
    if (finished) *finished = nfin;
    return LBM_OK;
}

int lbm_server_status(lbm_server s, int64_t id, int32_t *state, double *times) {
    if (!s) return LBM_E_INVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_E_INVAL, "unknown request id");
    const Request &r = *it->second;
    if (state) *state = r.state;
    if (times) { times[0] = r.t_submit; times[1] = r.t_start; times[2] = r.t_done; }
    return LBM_OK;
}

int lbm_server_result(lbm_server s, int64_t id, double *diag4, double *rho, double *T) {
    if (!s) return LBM_E_INVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(s, LBM_E_INVAL, "unknown request id");
    const Request &r = *it->second;
    if (r.state == 3) return sfail(s, LBM_E_NUMERIC, "request failed: " + r.err);
    if (r.state != 2) return sfail(s, LBM_E_STATE, "request not finished");
    if (diag4) std::memcpy(diag4, r.diag, sizeof(r.diag));
    if ((rho || T) && !r.keep) return sfail(s, LBM_E_STATE, "fields were not kept for this request");
    if (rho) std::memcpy(rho, r.rho.data(), r.rho.size() * sizeof(double));
    if (T) std::memcpy(T, r.T.data(), r.T.size() * sizeof(double));
    return LBM_OK;
}

int lbm_server_counts(lbm_server s, int32_t *queued, int32_t *active, uint64_t *bytes_in_use) {
    if (!s) return LBM_E_INVAL;
    if (queued) *queued = (int32_t)s->queue.size();
    if (active) *active = (int32_t)s->active.size();
    if (bytes_in_use) *bytes_in_use = s->used;
    return LBM_OK;
}

}  // extern "C"
