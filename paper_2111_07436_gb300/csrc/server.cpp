// Continuous-batching request loop over the batched solve (camp_server_*).
//
// A host model emits chunks of grid cells every time step (CAMP paper
// Sect. 2.4.2: the host iterates over its domain and hands each air mass to
// the solver); here chunks of any size and mechanism arrive while others are
// on the GPU.  A worker thread admits pending chunks in arrival order as soon
// as a stream slot and enough of the device-memory budget are free, stages
// each chunk on its own stream (copy in, solve, copy out), and retires
// chunks as their completion events fire, so admitted chunks overlap on the
// device and memory is recycled continuously.  Mechanism tables stay resident
// on the device for the server's life, and so, for resident cell sets, does a
// chunk's state across the host's consecutive steps: a step of such a set
// moves only its env in (and, optionally, its status out).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "camp.h"
#include "launch.h"

struct camp_resident {
    const camp_mech *mech = nullptr;
    int64_t n_cells = 0;
    int n = 0, n_env = 0;
    bool warm = false;
    size_t bytes = 0;
    void *dev = nullptr;
    double *d_state = nullptr, *d_env = nullptr, *d_step = nullptr, *d_atol = nullptr;
    int32_t *d_status = nullptr;
    cudaEvent_t last = nullptr;  // the latest enqueued operation on the set's memory
    int queued = 0;              // steps submitted and not yet finished (server lock)
};

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    const camp_mech *mech = nullptr;
    int64_t n_cells = 0;
    double *state = nullptr;
    const double *env = nullptr;
    int32_t *status = nullptr;
    double dt = 0, rtol = 0, atol = 0;
    camp_solve_opts opts{};
    size_t bytes = 0;
    int n = 0, n_env = 0;
    camp_resident *res = nullptr;  // a step of a resident set (state stays on the device)
    // progress
    int slot = -1;
    void *dev = nullptr;
    cudaEvent_t done_ev = nullptr;
    camp_request_info info{};
    bool finished = false;
};

}  // namespace

struct camp_server {
    size_t budget = 0;
    size_t used = 0;
    int device = 0;
    std::vector<cudaStream_t> streams;
    cudaStream_t res_stream = nullptr;  // creation, reads and writes of resident sets
    std::vector<camp_resident *> residents;
    std::vector<void *> workspaces;
    std::vector<char> slot_busy;
    std::deque<Request *> pending;
    std::vector<Request *> inflight;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    std::string err;
    double t0 = 0;

    size_t request_bytes(const Request &r) const {
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        return al((size_t)r.n_cells * r.n * 8) + al((size_t)r.n_cells * r.n_env * 8) +
               al((size_t)r.n_cells * 4) + 256;
    }

    // a step of a resident set: wait for the set's previous operation, copy
    // env (and atol) in, solve in place, optionally copy the status out
    void issue_resident(Request *r) {
        CampRange range_("camp_server: step a resident set");
        cudaStream_t s = streams[r->slot];
        camp_resident *R = r->res;
        cudaError_t e = cudaStreamWaitEvent(s, R->last, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(R->d_env, r->env, (size_t)r->n_cells * r->n_env * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(R->d_atol, &r->atol, 8, cudaMemcpyHostToDevice, s);
        int rc = CAMP_OK;
        if (e == cudaSuccess) {
            camp_solve_opts o = r->opts;
            o.workspace = workspaces[r->slot];
            o.stats = nullptr;
            o.step = R->warm ? R->d_step : nullptr;
            rc = camp_solve(r->mech, r->n_cells, R->d_state, R->d_env, r->dt, r->rtol, R->d_atol, 1, R->d_status,
                            &o, s);
        }
        if (e == cudaSuccess && rc == CAMP_OK && r->status)
            e = cudaMemcpyAsync(r->status, R->d_status, (size_t)r->n_cells * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(R->last, s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, s);
        r->info.rc = (e != cudaSuccess) ? CAMP_E_CUDA : rc;
    }

    void issue(Request *r) {
        if (r->res) return issue_resident(r);
        CampRange range_("camp_server: stage and launch a chunk");
        cudaStream_t s = streams[r->slot];
        const size_t bs = (size_t)r->n_cells * r->n * 8, be = (size_t)r->n_cells * r->n_env * 8;
        const size_t bst = (size_t)r->n_cells * 4;
        auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
        cudaError_t e = cudaMallocAsync(&r->dev, r->bytes, s);
        char *base = (char *)r->dev;
        double *d_state = (double *)base;
        double *d_env = (double *)(base + al(bs));
        int32_t *d_status = (int32_t *)(base + al(bs) + al(be));
        double *d_atol = (double *)(base + al(bs) + al(be) + al(bst));
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_state, r->state, bs, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_env, r->env, be, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_atol, &r->atol, 8, cudaMemcpyHostToDevice, s);
        int rc = CAMP_OK;
        if (e == cudaSuccess) {
            camp_solve_opts o = r->opts;
            o.workspace = workspaces[r->slot];
            o.stats = nullptr;
            o.step = nullptr;  // chunks are independent: always a cold start
            rc = camp_solve(r->mech, r->n_cells, d_state, d_env, r->dt, r->rtol, d_atol, 1, d_status, &o, s);
        }
        if (e == cudaSuccess && rc == CAMP_OK) e = cudaMemcpyAsync(r->state, d_state, bs, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && rc == CAMP_OK) e = cudaMemcpyAsync(r->status, d_status, bst, cudaMemcpyDeviceToHost, s);
        if (r->dev) cudaFreeAsync(r->dev, s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r->done_ev, s);
        r->info.rc = (e != cudaSuccess) ? CAMP_E_CUDA : rc;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (true) {
            bool progressed = false;
            // admit in arrival order while a slot and the budget allow
            while (!pending.empty()) {
                Request *r = pending.front();
                if (r->bytes > budget) {  // can never fit
                    pending.pop_front();
                    r->info.rc = CAMP_E_BUDGET;
                    r->info.t_admit = r->info.t_done = now_s() - t0;
                    r->finished = true;
                    progressed = true;
                    continue;
                }
                int slot = -1;
                for (size_t i = 0; i < slot_busy.size(); i++)
                    if (!slot_busy[i]) { slot = (int)i; break; }
                if (slot < 0 || used + r->bytes > budget) break;
                pending.pop_front();
                slot_busy[slot] = 1;
                used += r->bytes;
                r->slot = slot;
                r->info.t_admit = now_s() - t0;
                lk.unlock();
                issue(r);
                lk.lock();
                inflight.push_back(r);
                progressed = true;
            }
            // retire finished requests
            for (size_t i = 0; i < inflight.size();) {
                Request *r = inflight[i];
                cudaError_t q = r->done_ev ? cudaEventQuery(r->done_ev) : cudaSuccess;
                if (q == cudaErrorNotReady) { i++; continue; }
                if (q != cudaSuccess && r->info.rc == CAMP_OK) r->info.rc = CAMP_E_CUDA;
                if (r->done_ev) cudaEventDestroy(r->done_ev);
                r->done_ev = nullptr;
                r->info.t_done = now_s() - t0;
                r->finished = true;
                used -= r->bytes;
                if (r->res) r->res->queued--;
                slot_busy[r->slot] = 0;
                inflight[i] = inflight.back();
                inflight.pop_back();
                progressed = true;
            }
            if (progressed) cv_done.notify_all();
            if (stop && pending.empty() && inflight.empty()) break;
            if (!progressed) {
                if (inflight.empty())
                    cv_work.wait_for(lk, std::chrono::milliseconds(5));
                else
                    cv_work.wait_for(lk, std::chrono::microseconds(50));
            }
        }
    }
};

extern "C" {

int camp_server_create(const camp_server_opts *o, camp_server **out) {
    if (!o || !out || o->hbm_budget_bytes == 0) return CAMP_E_INVAL;
    *out = nullptr;
    camp_server *s = new camp_server();
    s->budget = o->hbm_budget_bytes;
    int slots = o->max_inflight > 0 ? o->max_inflight : 8;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return CAMP_E_CUDA; }
    if (cudaStreamCreateWithFlags(&s->res_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return CAMP_E_CUDA;
    }
    for (int i = 0; i < slots; i++) {
        cudaStream_t st;
        void *ws = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&ws, camp_workspace_bytes()) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto w : s->workspaces) cudaFree(w);
            cudaStreamDestroy(s->res_stream);
            delete s;
            return CAMP_E_CUDA;
        }
        s->streams.push_back(st);
        s->workspaces.push_back(ws);
        s->slot_busy.push_back(0);
    }
    // keep freed chunk memory in the pool instead of returning it to the driver
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t thr = (uint64_t)s->budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    s->t0 = now_s();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return CAMP_OK;
}

int camp_server_submit(camp_server *s, const camp_mech *m, int64_t n_cells, double *state,
                       const double *env, double dt, double rtol, double atol, int32_t *status,
                       const camp_solve_opts *opts, uint64_t *req_id) {
    if (!s || !m || n_cells <= 0 || !state || !env || !status || !req_id) return CAMP_E_INVAL;
    if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0)) return CAMP_E_INVAL;
    camp_mech_info inf;
    if (camp_mech_info_get(m, &inf) != CAMP_OK) return CAMP_E_INVAL;
    Request *r = new Request();
    r->mech = m;
    r->n_cells = n_cells;
    r->state = state;
    r->env = env;
    r->status = status;
    r->dt = dt;
    r->rtol = rtol;
    r->atol = atol;
    r->n = inf.n_species;
    r->n_env = inf.n_env;
    camp_solve_opts_default(&r->opts, opts ? opts->variant : CAMP_VARIANT_MIXED);
    if (opts) r->opts = *opts;
    r->bytes = s->request_bytes(*r);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete r; return CAMP_E_INVAL; }
        r->id = s->next_id++;
        r->info.n_cells = n_cells;
        r->info.t_submit = now_s() - s->t0;
        r->info.rc = CAMP_OK;
        s->all[r->id] = r;
        s->pending.push_back(r);
        *req_id = r->id;
    }
    s->cv_work.notify_one();
    return CAMP_OK;
}

static int finish_locked(camp_server *s, uint64_t id, camp_request_info *info) {
    Request *r = s->all[id];
    if (info) *info = r->info;
    s->all.erase(id);
    delete r;
    return CAMP_OK;
}

int camp_server_poll(camp_server *s, uint64_t id, int32_t *done, camp_request_info *info) {
    if (!s || !done) return CAMP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return CAMP_E_INVAL;
    *done = it->second->finished ? 1 : 0;
    if (*done) return finish_locked(s, id, info);
    return CAMP_OK;
}

int camp_server_wait(camp_server *s, uint64_t id, int32_t timeout_ms, camp_request_info *info) {
    if (!s) return CAMP_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return CAMP_E_INVAL;
    Request *r = it->second;
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (!r->finished) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->finished)
            return CAMP_E_TIMEOUT;
    }
    return finish_locked(s, id, info);
}

int camp_server_cancel(camp_server *s, uint64_t id) {
    if (!s) return CAMP_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(id);
        if (it == s->all.end()) return CAMP_E_INVAL;
        Request *r = it->second;
        auto pos = std::find(s->pending.begin(), s->pending.end(), r);
        if (pos == s->pending.end()) return CAMP_E_UNSUPPORTED;  // admitted or finished
        s->pending.erase(pos);
        if (r->res) r->res->queued--;
        r->info.rc = CAMP_E_CANCELLED;
        r->info.t_admit = r->info.t_done = now_s() - s->t0;
        r->finished = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
    return CAMP_OK;
}

int camp_server_stats(camp_server *s, int32_t *pending, int32_t *inflight, size_t *bytes_in_use) {
    if (!s) return CAMP_E_INVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (pending) *pending = (int32_t)s->pending.size();
    if (inflight) *inflight = (int32_t)s->inflight.size();
    if (bytes_in_use) *bytes_in_use = s->used;
    return CAMP_OK;
}

int camp_server_destroy(camp_server *s) {
    if (!s) return CAMP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto w : s->workspaces) cudaFree(w);
    for (auto &kv : s->all) delete kv.second;
    for (camp_resident *R : s->residents) {
        cudaStreamWaitEvent(s->res_stream, R->last, 0);
        cudaFreeAsync(R->dev, s->res_stream);
        cudaStreamSynchronize(s->res_stream);
        cudaEventDestroy(R->last);
        delete R;
    }
    cudaStreamDestroy(s->res_stream);
    delete s;
    return CAMP_OK;
}

// ---- resident cell sets ------------------------------------------------------
static int resident_wait_idle(camp_server *s, camp_resident *r, int32_t timeout_ms,
                              std::unique_lock<std::mutex> &lk) {
    auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (r->queued > 0) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->queued > 0) return CAMP_E_TIMEOUT;
    }
    return CAMP_OK;
}

static bool known_resident(camp_server *s, camp_resident *r) {
    return std::find(s->residents.begin(), s->residents.end(), r) != s->residents.end();
}

int camp_server_resident_create(camp_server *s, const camp_mech *m, int64_t n_cells, const double *state,
                                int32_t warm_start, camp_resident **out) {
    if (!s || !m || n_cells <= 0 || !state || !out) return CAMP_E_INVAL;
    *out = nullptr;
    camp_mech_info inf;
    if (camp_mech_info_get(m, &inf) != CAMP_OK) return CAMP_E_INVAL;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t C = (size_t)n_cells;
    const size_t b_state = al(C * inf.n_species * 8), b_env = al(C * inf.n_env * 8), b_st = al(C * 4);
    const size_t b_step = warm_start ? al(C * 8) : 0;
    camp_resident *R = new camp_resident();
    R->mech = m;
    R->n_cells = n_cells;
    R->n = inf.n_species;
    R->n_env = inf.n_env;
    R->warm = warm_start != 0;
    R->bytes = b_state + b_env + b_st + b_step + 256;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete R; return CAMP_E_INVAL; }
        if (s->used + R->bytes > s->budget) { delete R; return CAMP_E_BUDGET; }
        s->used += R->bytes;
    }
    cudaStream_t st = s->res_stream;
    cudaError_t e = cudaMallocAsync(&R->dev, R->bytes, st);
    if (e == cudaSuccess) {
        char *base = (char *)R->dev;
        R->d_state = (double *)base;
        R->d_env = (double *)(base + b_state);
        R->d_status = (int32_t *)(base + b_state + b_env);
        R->d_step = warm_start ? (double *)(base + b_state + b_env + b_st) : nullptr;
        R->d_atol = (double *)(base + b_state + b_env + b_st + b_step);
        e = cudaMemcpyAsync(R->d_state, state, C * inf.n_species * 8, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(R->d_status, 0, C * 4, st);
    if (e == cudaSuccess && R->d_step) e = cudaMemsetAsync(R->d_step, 0, C * 8, st);  // the first step starts cold
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->last, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(R->last, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        if (R->dev) {
            cudaFreeAsync(R->dev, st);
            cudaStreamSynchronize(st);
        }
        if (R->last) cudaEventDestroy(R->last);
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= R->bytes;
        delete R;
        return e == cudaErrorMemoryAllocation ? CAMP_E_NOMEM : CAMP_E_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->residents.push_back(R);
    }
    *out = R;
    return CAMP_OK;
}

int camp_server_resident_step(camp_server *s, camp_resident *R, const double *env, double dt, double rtol,
                              double atol, int32_t *status, const camp_solve_opts *opts, uint64_t *req_id) {
    if (!s || !R || !env || !req_id) return CAMP_E_INVAL;
    if (!(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0)) return CAMP_E_INVAL;
    Request *r = new Request();
    r->mech = R->mech;
    r->n_cells = R->n_cells;
    r->env = env;
    r->status = status;
    r->dt = dt;
    r->rtol = rtol;
    r->atol = atol;
    r->n = R->n;
    r->n_env = R->n_env;
    r->res = R;
    camp_solve_opts_default(&r->opts, opts ? opts->variant : CAMP_VARIANT_MIXED);
    if (opts) r->opts = *opts;
    r->bytes = 0;  // the set's memory is already counted
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop || !known_resident(s, R)) { delete r; return CAMP_E_INVAL; }
        r->id = s->next_id++;
        r->info.n_cells = R->n_cells;
        r->info.t_submit = now_s() - s->t0;
        r->info.rc = CAMP_OK;
        s->all[r->id] = r;
        s->pending.push_back(r);
        R->queued++;
        *req_id = r->id;
    }
    s->cv_work.notify_one();
    return CAMP_OK;
}

int camp_server_resident_read(camp_server *s, camp_resident *R, double *state, int32_t *status, double *step,
                              int32_t timeout_ms) {
    if (!s || !R || !state) return CAMP_E_INVAL;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!known_resident(s, R)) return CAMP_E_INVAL;
        if (int rc = resident_wait_idle(s, R, timeout_ms, lk)) return rc;
    }
    cudaStream_t st = s->res_stream;
    const size_t C = (size_t)R->n_cells;
    cudaError_t e = cudaStreamWaitEvent(st, R->last, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(state, R->d_state, C * R->n * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, R->d_status, C * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && step) {
        if (R->d_step) e = cudaMemcpyAsync(step, R->d_step, C * 8, cudaMemcpyDeviceToHost, st);
        else std::fill(step, step + C, 0.0);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CAMP_OK : CAMP_E_CUDA;
}

int camp_server_resident_write(camp_server *s, camp_resident *R, const double *state, int32_t timeout_ms) {
    if (!s || !R || !state) return CAMP_E_INVAL;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!known_resident(s, R)) return CAMP_E_INVAL;
        if (int rc = resident_wait_idle(s, R, timeout_ms, lk)) return rc;
    }
    cudaStream_t st = s->res_stream;
    cudaError_t e = cudaStreamWaitEvent(st, R->last, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R->d_state, state, (size_t)R->n_cells * R->n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(R->last, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CAMP_OK : CAMP_E_CUDA;
}

int camp_server_resident_destroy(camp_server *s, camp_resident *R) {
    if (!s || !R) return CAMP_E_INVAL;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (!known_resident(s, R)) return CAMP_E_INVAL;
        while (R->queued > 0) s->cv_done.wait(lk);
        s->residents.erase(std::find(s->residents.begin(), s->residents.end(), R));
    }
    cudaStream_t st = s->res_stream;
    cudaStreamWaitEvent(st, R->last, 0);
    cudaFreeAsync(R->dev, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaEventDestroy(R->last);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= R->bytes;
    }
    s->cv_work.notify_one();  // freed budget may admit a waiting chunk
    delete R;
    return e == cudaSuccess ? CAMP_OK : CAMP_E_CUDA;
}

}  // extern "C"
