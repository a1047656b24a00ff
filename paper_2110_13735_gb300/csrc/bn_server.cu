// bn_server.cu -- continuous-batching solve server over the C ABI.
//
// Requests (homogeneous Boltzmann-Nordheim solves: operator, initial state, dt, t_end) are
// queued by any thread.  One worker thread owns the GPU work: at every tick it admits
// queued requests, the one with the least estimated work first (a request queued for longer
// than kMaxWait seconds goes first), while slots and the device-memory budget allow (kernel-mode
// tables are shared by requests with the same operator and counted once), advances every
// active request by a few RK steps in shared launches (bn_step_rk_batch: one captured graph
// for the whole active set), and retires finished requests, copying their final state to
// host memory.  Requests that arrive while others run join at the next tick.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "bn_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct ServerReq {
    long long id = 0;
    bn_request r{};
    std::vector<double> f0, result;
    int state = 0;   // 0 queued, 1 running, 2 done, 3 failed
    double t_submit = 0, t_admit = 0, t_done = 0;
    double t_escalated = -1;   // solve time of the switch to FP64 (escalate_at), -1 if none
    long long steps_total = 0, steps_done = 0;
    double work = 0;   // estimated work: steps x terms of one evaluation
    bn_solver* s = nullptr;
    size_t bytes = 0;
    std::string err;
};

thread_local std::string g_srv_err;

bn_status sfail(bn_status st, const std::string& m) {
    g_srv_err = m;
    return st;
}

// Device bytes of one solver apart from its kernel-mode tables (mirrors bn_create_solver).
size_t solver_bytes(const bn_request& r) {
    const size_t N = (size_t)r.N, nm = r.d == 2 ? N * N : N * N * N, nExt = r.d == 2 ? 4 * N * N : 8 * N * N * N;
    const size_t parts = 152 * 4;   // upper bound of the CTA partials
    size_t b = nm * (6 * sizeof(double) + 7 * sizeof(double2) + sizeof(float2)) + nExt * sizeof(double2) +
               parts * nm * sizeof(double2) + (1 << 16);
    if (r.d == 2 && r.opt.beta_split && r.opt.precision == BN_MIXED)   // the residual-table pass's buffers
        b += parts * nm * sizeof(double2) + nExt * sizeof(double2) + nm * sizeof(double2);
    if (r.d == 3)   // the kernel-mode slices of one round: the slice budget (default at most 40 GiB)
        b += r.opt.beta_budget_mb > 0 ? (size_t)r.opt.beta_budget_mb << 20 : (size_t)40 << 30;
    return b;
}

// Bytes of the kernel-mode tables of an operator (mirrors acquire_tables).
size_t table_bytes(const bn_request& r) {
    const size_t N = (size_t)r.N, nExt = r.d == 2 ? 4 * N * N : 8 * N * N * N, nm = r.d == 2 ? N * N : N * N * N;
    const size_t M2d = (size_t)(r.opt.M > 0 ? r.opt.M : 2 * r.N);
    const size_t P = r.d == 2 ? (r.kernel == BN_HARD_SPHERE ? M2d * (size_t)(r.opt.M1 > 0 ? r.opt.M1 : r.N + 8) : M2d)
                              : (size_t)(r.opt.M1 > 0 ? r.opt.M1 : r.N / 2) * (r.opt.M2 > 0 ? r.opt.M2 : r.N / 2);
    size_t b = 2 * P * nExt * sizeof(double);
    if (r.d == 2) {
        // beta in FP64 and FP32, the reducible and quadratic weights, and the rounding residuals of the
        // FP32 tables (kernel-mode rounding correction)
        b += nExt * nExt * (sizeof(double) + 2 * sizeof(float));
        b += nExt * nm * (sizeof(double) + 4 * sizeof(float));
        if (r.N <= 32) b += 2 * nExt * nExt * sizeof(float);   // transposed FP32 table and its residuals
    }
    return b;
}

std::string table_key(const bn_request& r) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "%d:%d:%.17g:%.17g:%d:%d:%d:%d:%d:%.17g", r.d, r.N, r.T, r.R, r.kernel, r.opt.M,
                  r.opt.M1, r.opt.M2, r.opt.quad3d, r.opt.c_phi);
    return buf;
}

}  // namespace

struct bn_server {
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    int max_active = 0;
    int steps_per_tick = 8;
    std::deque<ServerReq*> pending;
    std::vector<ServerReq*> active;
    std::map<long long, ServerReq*> all;
    std::map<std::string, int> table_refs;   // operator key -> active requests using it
    long long next_id = 1;
    int in_flight = 0;   // requests being admitted or retired outside the lock
    size_t bytes_in_use = 0;
    long long ticks = 0, admitted = 0, done = 0, failed = 0, max_seen_active = 0;
    Clock::time_point t0 = Clock::now();

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    void run();
    void admit_locked(std::unique_lock<std::mutex>& lock);
    void retire(ServerReq* q, bool ok, const std::string& err);
};

void bn_server::retire(ServerReq* q, bool ok, const std::string& err) {
    // called without the lock; q is no longer in `active`
    double t_esc = -1;
    if (ok && q->s) {
        q->result.resize(q->f0.size());
        if (bn_get_state(q->s, q->result.data(), q->result.size()) != BN_OK) {
            ok = false;
        }
        bn_precision_state(q->s, nullptr, &t_esc, nullptr);
    }
    if (q->s) bn_destroy_solver(q->s);
    std::lock_guard<std::mutex> lock(mu);
    q->s = nullptr;
    q->t_done = now();
    q->t_escalated = t_esc;
    q->state = ok ? 2 : 3;
    q->err = ok ? "" : (err.empty() ? std::string(bn_last_error()) : err);
    q->f0.clear();
    q->f0.shrink_to_fit();
    bytes_in_use -= q->bytes;
    const std::string key = table_key(q->r);
    if (--table_refs[key] == 0) {
        table_refs.erase(key);
        bytes_in_use -= table_bytes(q->r);
    }
    if (ok) done++;
    else failed++;
    in_flight--;
    cv.notify_all();
}

// Queued requests older than this are admitted before any shorter one (no starvation).
constexpr double kMaxWait = 60.0;

void bn_server::admit_locked(std::unique_lock<std::mutex>& lock) {
    while (!pending.empty() && (int)active.size() < max_active) {
        // the least estimated work first (ties: arrival order), unless the oldest waited too long
        auto pick = pending.begin();
        if (now() - pending.front()->t_submit <= kMaxWait)
            for (auto it = pending.begin(); it != pending.end(); ++it)
                if ((*it)->work < (*pick)->work) pick = it;
        ServerReq* q = *pick;
        const std::string key = table_key(q->r);
        const size_t need = solver_bytes(q->r) + (table_refs.count(key) ? 0 : table_bytes(q->r));
        if (bytes_in_use + need > budget && !active.empty()) break;   // wait for memory to free up
        pending.erase(pick);
        in_flight++;
        q->bytes = solver_bytes(q->r);
        bytes_in_use += need;
        table_refs[key]++;
        lock.unlock();
        bn_solver* s = nullptr;
        bn_status st = bn_create_solver(q->r.d, q->r.N, q->r.T, q->r.R, q->r.kernel, q->r.eps, &q->r.opt, stream, &s);
        if (st == BN_OK) st = bn_set_state(s, q->f0.data(), q->f0.size());
        lock.lock();
        if (st != BN_OK) {
            q->s = s;
            const std::string e = bn_last_error();
            lock.unlock();
            retire(q, false, e);   // leaves in_flight to retire()
            lock.lock();
            continue;
        }
        q->s = s;
        q->state = 1;
        q->t_admit = now();
        admitted++;
        active.push_back(q);
        in_flight--;
        if ((long long)active.size() > max_seen_active) max_seen_active = (long long)active.size();
    }
}

void bn_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (true) {
        if (stop) break;   // bn_server_destroy: abandon what is queued or running
        admit_locked(lock);
        if (active.empty()) {
            cv.wait_for(lock, std::chrono::milliseconds(1));
            continue;
        }
        // advance the active set together by the smallest remaining step count (at most steps_per_tick)
        std::vector<ServerReq*> act = active;
        long long k = steps_per_tick;
        for (ServerReq* q : act) k = std::min(k, q->steps_total - q->steps_done);
        if (!pending.empty()) k = 1;   // let queued requests join quickly
        lock.unlock();
        std::vector<bn_solver*> ss;
        std::vector<double> dts;
        for (ServerReq* q : act) {
            ss.push_back(q->s);
            dts.push_back(q->r.dt);
        }
        int bad = -1;
        bn_status st = k > 0 ? bn_step_rk_batch(ss.data(), (int)ss.size(), dts.data(), (int)k, &bad) : BN_OK;
        const std::string err = st == BN_OK ? "" : bn_last_error();
        lock.lock();
        ticks++;
        std::vector<std::pair<ServerReq*, bool>> finished;
        for (size_t i = 0; i < act.size(); ++i) {
            ServerReq* q = act[i];
            if (st != BN_OK && (bad < 0 || (int)i == bad)) {
                finished.push_back({q, false});
                continue;
            }
            q->steps_done += k;
            if (q->steps_done >= q->steps_total) finished.push_back({q, true});
        }
        for (auto& fq : finished) active.erase(std::find(active.begin(), active.end(), fq.first));
        in_flight += (int)finished.size();
        lock.unlock();
        for (auto& fq : finished) retire(fq.first, fq.second, fq.second ? "" : err);
        lock.lock();
    }
}

extern "C" {

bn_status bn_server_create(size_t device_bytes, int max_active, void* cuda_stream, bn_server** out) {
    if (!out) return sfail(BN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (max_active <= 0) return sfail(BN_ERR_ARG, "max_active must be > 0");
    bn_server* S = new bn_server();
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        cudaGetLastError();
        return sfail(BN_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    if (cuda_stream) {
        S->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete S;
            return sfail(BN_ERR_CUDA, "stream create failed");
        }
        S->own_stream = true;
    }
    if (device_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        device_bytes = fr / 10 * 8;
    }
    S->budget = device_bytes;
    S->max_active = max_active;
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return BN_OK;
}

bn_status bn_server_submit(bn_server* S, const bn_request* r, const double* f0, size_t count, long long* id) {
    if (!S || !r || !f0 || !id) return sfail(BN_ERR_ARG, "null argument");
    if (r->d != 2 && r->d != 3) return sfail(BN_ERR_ARG, "d must be 2 or 3");
    if (r->N < 4 || r->N % 2) return sfail(BN_ERR_ARG, "N must be even and >= 4");
    const size_t nm = r->d == 2 ? (size_t)r->N * r->N : (size_t)r->N * r->N * r->N;
    if (count != nm) return sfail(BN_ERR_ARG, "count must be N^d");
    if (!(r->dt > 0) || !(r->t_end > 0)) return sfail(BN_ERR_ARG, "dt and t_end must be > 0");
    ServerReq* q = new ServerReq();
    q->r = *r;
    q->f0.assign(f0, f0 + count);
    q->steps_total = (long long)std::llround(r->t_end / r->dt);
    if (q->steps_total < 1) q->steps_total = 1;
    {
        // terms of one evaluation: the Q_{1,q} sum when eps != 0, else the quadratic sum; FP64 runs
        // count 32 times (the FP64 pipe's rate against FP32)
        const double n = r->N;
        const double c = r->eps != 0.0 ? std::pow(2.0 * (n * n * n - n) / 3.0, r->d) : std::pow(0.75 * n * n, r->d);
        q->work = (double)q->steps_total * c * (r->opt.precision == BN_MIXED ? 1.0 : 32.0);
    }
    std::lock_guard<std::mutex> lock(S->mu);
    q->id = S->next_id++;
    q->t_submit = S->now();
    S->pending.push_back(q);
    S->all[q->id] = q;
    *id = q->id;
    S->cv.notify_all();
    return BN_OK;
}

bn_status bn_server_poll(bn_server* S, long long id, int* state, double* f_out, size_t count, double* times,
                         size_t ntimes) {
    if (!S || !state) return sfail(BN_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return sfail(BN_ERR_ARG, "unknown request id");
    ServerReq* q = it->second;
    *state = q->state;
    if (times && ntimes >= 3) {
        times[0] = q->t_submit;
        times[1] = q->t_admit;
        times[2] = q->t_done;
        if (ntimes >= 4) times[3] = q->t_escalated;
    }
    if (q->state == 2 && f_out) {
        if (count != q->result.size()) return sfail(BN_ERR_ARG, "count must be N^d");
        std::memcpy(f_out, q->result.data(), count * sizeof(double));
    }
    if (q->state == 3) return sfail(BN_ERR_STATE, "request failed: " + q->err);
    return BN_OK;
}

bn_status bn_server_wait_idle(bn_server* S, double timeout_s) {
    if (!S) return sfail(BN_ERR_ARG, "null server");
    std::unique_lock<std::mutex> lock(S->mu);
    const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!(S->pending.empty() && S->active.empty() && S->in_flight == 0)) {
        if (S->cv.wait_until(lock, limit) == std::cv_status::timeout && Clock::now() >= limit)
            return sfail(BN_ERR_TIMEOUT, "server still busy at the timeout");
    }
    return BN_OK;
}

bn_status bn_server_stats(bn_server* S, double* out, size_t count) {
    if (!S || !out || count < 8) return sfail(BN_ERR_ARG, "out needs 8 entries");
    std::lock_guard<std::mutex> lock(S->mu);
    out[0] = (double)S->all.size();
    out[1] = (double)S->admitted;
    out[2] = (double)S->done;
    out[3] = (double)S->failed;
    out[4] = (double)S->ticks;
    out[5] = (double)S->max_seen_active;
    out[6] = (double)S->bytes_in_use;
    out[7] = (double)S->budget;
    return BN_OK;
}

const char* bn_server_last_error(void) { return g_srv_err.c_str(); }

void bn_server_destroy(bn_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        // drop what has not started
        for (ServerReq* q : S->pending) q->state = 3;
        S->pending.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->all) {
        if (kv.second->s) bn_destroy_solver(kv.second->s);
        delete kv.second;
    }
    if (S->own_stream) cudaStreamDestroy(S->stream);
    delete S;
}

}  // extern "C"
