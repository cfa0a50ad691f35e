// Serving loop with continuous batching (included by sbpsat.cu).
//
// One scheduler thread per server owns every device call: it admits
// requests in arrival order while a slot and enough of the HBM budget are
// free (device memory comes from the stream-ordered pool, so neither
// allocation nor release synchronises the device; set-up runs on a separate
// admission stream joined to the batch stream by an event), lets admitted
// requests join the running sbp_batch at the next chunk boundary, advances
// the batch one chunk at a time (at most two chunks in flight; a chunk is a
// captured graph, updated in place when the membership changes), and
// retires finished requests: their probe samples are copied to pinned host
// memory behind an event and their memory goes back to the pool.  Requests
// with an energy monitor (energy_every > 0) are sampled at chunk boundaries
// (sbp_batch_step); the sample is mirrored to pinned host memory and checked
// after each chunk, so a request that goes unstable leaves the batch with
// SBP_EUNSTABLE while the others run on unchanged.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct ServerRequest {
    uint64_t ticket = 0;
    sbp_grid_desc desc{};
    std::vector<float> eps, mu;
    int64_t nsteps = 0;
    std::vector<sbp_source_desc> src;
    std::vector<sbp_probe_desc> prb;
    size_t ws_bytes = 0, probe_bytes = 0, energy_bytes = 0;
    double submit_s = 0, admit_s = 0, done_s = 0;
    int status = SBP_OK;
    bool done = false;
    int64_t steps = 0;
    sbp_sim *sim = nullptr;
    void *ws = nullptr;
    void *probe_dev = nullptr;
    float *probe_host = nullptr;
    double *energy_dev = nullptr;        // energy series (stream-ordered pool)
    double *energy_host = nullptr;       // pinned mirror of the latest energy sample
    double energy_max = 0.0;             // largest sample seen so far
    int pending_status = SBP_OK;         // status to report once the retirement copy has landed
    cudaEvent_t done_ev = nullptr;
};

// Stability check of a monitored request: the latest energy sample is not
// finite, or exceeds kEnergyGrowth times the largest earlier sample.  The
// requests are driven by sources from zero fields, so the energy legitimately
// grows while a source injects it; an unstable scheme grows it exponentially
// (a mode amplified by |lambda| > 1 per step gains many orders of magnitude
// over a chunk) and soon overflows; a source ramping up stays far below 1e6 per
// chunk.
constexpr double kEnergyGrowth = 1e6;
bool energy_unstable(ServerRequest &r)
{
    if (!r.energy_host) return false;
    const double v = *static_cast<volatile double *>(r.energy_host);
    if (!std::isfinite(v) || (r.energy_max > 0.0 && v > kEnergyGrowth * r.energy_max)) return true;
    r.energy_max = std::max(r.energy_max, v);
    return false;
}

// Release what a simulation created without waiting for the device: its side
// stream and events are destroyed (freed once their work completes); the
// workspace and probe buffer belong to the server and return to the pool.
void destroy_sim_async(sbp_sim *s)
{
    if (!s) return;
    if (s->side) cudaStreamDestroy(s->side);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->eseries) cudaFreeAsync(s->eseries, s->stream);
    delete s;
}

}  // namespace

struct sbp_server {
    cudaStream_t stream = nullptr;
    cudaStream_t adm = nullptr;           // admissions: allocation, material upload, set-up kernels
    int device = 0;
    size_t budget = 0, used = 0;
    int max_slots = 1, chunk = 32;
    sbp_batch *batch = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<ServerRequest>> pending;
    std::vector<std::shared_ptr<ServerRequest>> active, retiring;
    std::map<uint64_t, std::shared_ptr<ServerRequest>> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    double first_submit = -1.0, last_done = 0.0, cell_updates = 0.0;
    std::deque<cudaEvent_t> chunks;
};

namespace {

long long cells_of(const sbp_grid_desc &d) { return (long long)d.nx * d.ny * d.nz; }

void finish(sbp_server *S, const std::shared_ptr<ServerRequest> &r, int status)
{
    r->status = status;
    r->done = true;
    r->done_s = now_s();
    S->last_done = r->done_s;
    S->cv_done.notify_all();
}

// Create the request's simulation on the admission stream (its pageable
// material upload waits only for that stream), then hand it to the batch
// stream, which waits for the set-up to finish before the next chunk.
int admit(sbp_server *S, const std::shared_ptr<ServerRequest> &r)
{
    Trace trace("sbp_server_admit");
    cudaError_t e = cudaMallocAsync(&r->ws, r->ws_bytes, S->adm);
    if (e != cudaSuccess) { (void)cudaGetLastError(); r->ws = nullptr; return cuda_fail(e); }
    sbp_sim *s = nullptr;
    int rc = create_common(&r->desc, S->adm, r->ws, r->ws_bytes, false, &s, true, true);
    if (rc) return rc;
    r->sim = s;
    for (const auto &q : r->src) {
        int id = sbp_add_source(s, q.comp, q.i, q.j, q.k, q.waveform, q.amp, q.tw, q.t0, q.f);
        if (id < 0) return id;
    }
    for (const auto &q : r->prb) {
        int id;
        if ((rc = sbp_add_probe(s, q.comp, q.i, q.j, q.k, &id))) return rc;
    }
    if (r->probe_bytes) {
        e = cudaMallocAsync(&r->probe_dev, r->probe_bytes, S->adm);
        if (e != cudaSuccess) { (void)cudaGetLastError(); r->probe_dev = nullptr; return cuda_fail(e); }
        SBP_CUDA(cudaMemsetAsync(r->probe_dev, 0, r->probe_bytes, S->adm));
        s->probe_buf = r->probe_dev;
        s->probe_cap = r->nsteps;
        s->probe_base = s->step;
    }
    if (r->energy_bytes) {
        // the energy series from the pool (zeroed: samples not taken read 0), so
        // that joining the batch allocates nothing on the batch's stream
        e = cudaMallocAsync((void **)&r->energy_dev, r->energy_bytes, S->adm);
        if (e != cudaSuccess) { (void)cudaGetLastError(); r->energy_dev = nullptr; return cuda_fail(e); }
        SBP_CUDA(cudaMemsetAsync(r->energy_dev, 0, r->energy_bytes, S->adm));
        s->eseries = r->energy_dev;
        s->eseries_cap = (long long)(r->energy_bytes / sizeof(double));
        if (!r->energy_host) {
            if (cudaHostAlloc((void **)&r->energy_host, sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
                (void)cudaGetLastError();
                r->energy_host = nullptr;
                return SBP_ENOMEM;
            }
        }
        *r->energy_host = 0.0;
    }
    cudaEvent_t ready;
    SBP_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    SBP_CUDA(cudaEventRecord(ready, S->adm));
    SBP_CUDA(cudaStreamWaitEvent(S->stream, ready, 0));
    cudaEventDestroy(ready);
    s->stream = S->stream;
    rc = sbp_batch_add(S->batch, s, r->nsteps);
    if (rc) return rc;
    if (r->energy_host) S->batch->m.back().mirror = r->energy_host;
    return SBP_OK;
}

void release_device(sbp_server *S, const std::shared_ptr<ServerRequest> &r)
{
    if (r->sim) {
        r->sim->eseries = nullptr;        // the series belongs to the request (pool memory)
        destroy_sim_async(r->sim);
        r->sim = nullptr;
    }
    if (r->energy_dev) { cudaFreeAsync(r->energy_dev, S->stream); r->energy_dev = nullptr; }
    if (r->probe_dev) { cudaFreeAsync(r->probe_dev, S->stream); r->probe_dev = nullptr; }
    if (r->ws) { cudaFreeAsync(r->ws, S->stream); r->ws = nullptr; }
    S->used -= r->ws_bytes + r->probe_bytes + r->energy_bytes;
}

void server_loop(sbp_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // 1. completions: probe copies that have landed
        for (auto it = S->retiring.begin(); it != S->retiring.end();) {
            auto r = *it;
            if (cudaEventQuery(r->done_ev) == cudaSuccess) {
                cudaEventDestroy(r->done_ev);
                r->done_ev = nullptr;
                // the last energy sample has landed with the retirement copy
                int st = r->pending_status;
                if (!st && energy_unstable(*r)) st = SBP_EUNSTABLE;
                if (!st) S->cell_updates += (double)cells_of(r->desc) * (double)r->steps;
                finish(S, r, st);
                it = S->retiring.erase(it);
            } else {
                ++it;
            }
        }
        (void)cudaGetLastError();
        // 2. admission in arrival order while a slot and the budget allow
        while (!S->pending.empty() && (int)S->active.size() < S->max_slots) {
            auto r = S->pending.front();
            const size_t need = r->ws_bytes + r->probe_bytes + r->energy_bytes;
            if (S->used + need > S->budget && !S->active.empty()) break;   // wait for memory to free up
            S->pending.pop_front();
            S->used += need;
            r->admit_s = now_s();
            lk.unlock();
            int rc = admit(S, r);
            lk.lock();
            if (rc) {
                if (r->sim) sbp_batch_remove(S->batch, r->sim);
                release_device(S, r);
                finish(S, r, rc);
                continue;
            }
            S->active.push_back(r);
        }
        // 3. one chunk of the batch, then retire the members that finished
        if (!S->active.empty()) {
            lk.unlock();
            while (S->chunks.size() >= 2) {
                cudaEventSynchronize(S->chunks.front());
                cudaEventDestroy(S->chunks.front());
                S->chunks.pop_front();
            }
            int rc = sbp_batch_step(S->batch, S->chunk);
            cudaEvent_t ev = nullptr;
            if (!rc && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(ev, S->stream);
                S->chunks.push_back(ev);
            }
            lk.lock();
            for (auto it = S->active.begin(); it != S->active.end();) {
                auto r = *it;
                int64_t rem = 0;
                sbp_batch_remaining(S->batch, r->sim, &rem);
                // a monitored request whose energy (mirrored from a chunk that
                // has completed) shows instability leaves the batch now
                const bool unstable = rc == SBP_OK && energy_unstable(*r);
                if (rc == SBP_OK && rem > 0 && !unstable) { ++it; continue; }
                r->steps = r->nsteps - rem;
                sbp_batch_remove(S->batch, r->sim);
                int st = rc;
                if (unstable) r->pending_status = SBP_EUNSTABLE;
                if (!st && !unstable && r->probe_bytes) {
                    if (cudaHostAlloc((void **)&r->probe_host, r->probe_bytes, cudaHostAllocDefault) != cudaSuccess) {
                        (void)cudaGetLastError();
                        r->probe_host = nullptr;
                        st = SBP_ENOMEM;
                    } else if (cudaMemcpyAsync(r->probe_host, r->probe_dev, r->probe_bytes, cudaMemcpyDeviceToHost,
                                               S->stream) != cudaSuccess) {
                        (void)cudaGetLastError();
                        st = SBP_ECUDA;
                    }
                }
                if (!st && cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming) != cudaSuccess) st = SBP_ECUDA;
                if (!st) cudaEventRecord(r->done_ev, S->stream);
                release_device(S, r);
                it = S->active.erase(it);
                if (st) finish(S, r, st);
                else S->retiring.push_back(r);
            }
            continue;
        }
        if (!S->retiring.empty()) {
            auto r = S->retiring.front();
            lk.unlock();
            cudaEventSynchronize(r->done_ev);
            lk.lock();
            continue;
        }
        if (S->stop && S->pending.empty()) break;
        S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
    }
    while (!S->chunks.empty()) {
        cudaEventSynchronize(S->chunks.front());
        cudaEventDestroy(S->chunks.front());
        S->chunks.pop_front();
    }
}

}  // namespace

extern "C" {

int sbp_server_create(void *cuda_stream, size_t hbm_budget_bytes, int max_slots, int chunk_steps, sbp_server **out)
{
    if (!out || max_slots <= 0 || chunk_steps <= 0) return SBP_EINVAL;
    sbp_server *S = new (std::nothrow) sbp_server();
    if (!S) return SBP_ENOMEM;
    cudaGetDevice(&S->device);
    S->stream = static_cast<cudaStream_t>(cuda_stream);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { (void)cudaGetLastError(); delete S; return SBP_ECUDA; }
    const size_t cap = (size_t)(0.9 * (double)free_b);
    S->budget = hbm_budget_bytes ? std::min(hbm_budget_bytes, cap) : cap;
    S->max_slots = max_slots;
    S->chunk = chunk_steps;
    int rc = sbp_batch_create(cuda_stream, 1, &S->batch);
    if (rc) { delete S; return rc; }
    if (cudaStreamCreateWithFlags(&S->adm, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        sbp_batch_destroy(S->batch);
        delete S;
        return SBP_ECUDA;
    }
    S->worker = std::thread(server_loop, S);
    *out = S;
    return SBP_OK;
}

int sbp_server_submit(sbp_server *S, const sbp_request *req, uint64_t *ticket)
{
    if (!S || !req || req->nsteps < 0 || req->nsources < 0 || req->nprobes < 0) return SBP_EINVAL;
    if ((req->nsources && !req->sources) || (req->nprobes && !req->probes)) return SBP_EINVAL;
    const sbp_grid_desc &d = req->grid;
    if (d.precision != SBP_FP32 || d.mu_r || d.nx < 8 || d.ny < 8 || d.nz < 8) return SBP_EINVAL;
    for (int f = 0; f < 6; f++)
        if (d.face[f] == SBP_INTERFACE) return SBP_EINVAL;
    if (!desc_valid(&d)) return SBP_EINVAL;
    if (req->nsources > sbp::kMaxSources || req->nprobes > sbp::kMaxProbes) return SBP_ECAPACITY;
    auto r = std::make_shared<ServerRequest>();
    r->desc = d;
    if (d.eps_r) r->eps.assign(d.eps_r, d.eps_r + cells_of(d));
    r->desc.eps_r = d.eps_r ? r->eps.data() : nullptr;
    r->desc.mu_r = nullptr;
    r->nsteps = req->nsteps;
    if (req->nsources) r->src.assign(req->sources, req->sources + req->nsources);
    if (req->nprobes) r->prb.assign(req->probes, req->probes + req->nprobes);
    r->ws_bytes = sbp_workspace_bytes(&r->desc);
    r->probe_bytes = (size_t)req->nprobes * (size_t)req->nsteps * sizeof(float);
    if (d.energy_every > 0) r->energy_bytes = (size_t)(req->nsteps / d.energy_every + 2) * sizeof(double);
    if (r->ws_bytes + r->probe_bytes + r->energy_bytes > S->budget) return SBP_ENOMEM;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return SBP_ESTATE;
    r->ticket = S->next_ticket++;
    r->submit_s = now_s();
    if (S->first_submit < 0) S->first_submit = r->submit_s;
    S->all[r->ticket] = r;
    S->pending.push_back(r);
    if (ticket) *ticket = r->ticket;
    S->cv_work.notify_one();
    return SBP_OK;
}

int sbp_server_poll(sbp_server *S, uint64_t ticket, sbp_result *res)
{
    if (!S) return SBP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SBP_EINVAL;
    const auto &r = it->second;
    if (!r->done) return SBP_EAGAIN;
    if (res) {
        res->status = r->status;
        res->steps = r->steps;
        res->submit_s = r->submit_s;
        res->admit_s = r->admit_s;
        res->done_s = r->done_s;
        res->nprobes = (int32_t)r->prb.size();
    }
    return SBP_OK;
}

int sbp_server_probes(sbp_server *S, uint64_t ticket, double *out, int64_t cap)
{
    if (!S || cap < 0 || (!out && cap > 0)) return SBP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return SBP_EINVAL;
    const auto &r = it->second;
    if (!r->done) return SBP_EAGAIN;
    if (r->status) return r->status;
    const int64_t m = std::min<int64_t>(cap, r->nsteps);
    for (size_t q = 0; q < r->prb.size(); q++)
        for (int64_t t = 0; t < m; t++) out[q * cap + t] = r->probe_host ? (double)r->probe_host[q * r->nsteps + t] : 0.0;
    return SBP_OK;
}

int sbp_server_release(sbp_server *S, uint64_t ticket)
{
    if (!S) return SBP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end() || !it->second->done) return SBP_EINVAL;
    if (it->second->probe_host) cudaFreeHost(it->second->probe_host);
    it->second->probe_host = nullptr;
    if (it->second->energy_host) cudaFreeHost(it->second->energy_host);
    it->second->energy_host = nullptr;
    S->all.erase(it);
    return SBP_OK;
}

int sbp_server_drain(sbp_server *S)
{
    if (!S) return SBP_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] {
        if (!S->pending.empty() || !S->active.empty() || !S->retiring.empty()) return false;
        for (auto &kv : S->all)
            if (!kv.second->done) return false;
        return true;
    });
    return SBP_OK;
}

int sbp_server_stats(sbp_server *S, double *cell_updates, double *span_s)
{
    if (!S) return SBP_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (cell_updates) *cell_updates = S->cell_updates;
    if (span_s) *span_s = S->first_submit < 0 ? 0.0 : S->last_done - S->first_submit;
    return SBP_OK;
}

int sbp_server_destroy(sbp_server *S)
{
    if (!S) return SBP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    sbp_server_drain(S);
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->all) {
        if (kv.second->probe_host) cudaFreeHost(kv.second->probe_host);
        if (kv.second->energy_host) cudaFreeHost(kv.second->energy_host);
    }
    cudaStreamSynchronize(S->stream);
    cudaStreamSynchronize(S->adm);
    cudaStreamDestroy(S->adm);
    sbp_batch_destroy(S->batch);
    delete S;
    return SBP_OK;
}

}  // extern "C"
