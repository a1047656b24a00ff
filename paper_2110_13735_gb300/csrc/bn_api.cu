// bn_api.cu -- the C ABI of libbn (include/bn.h): solver lifecycle, evaluation of
// Q_eps(f) (Mouton & Rey, Sec. 3.3 step 2, classical method of Sec. 3.2) and
// Runge-Kutta time stepping with one captured CUDA graph per step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <mutex>

#include "bn_internal.cuh"

namespace {

thread_local std::string g_err;

// cache of captured batched steps (a few recent solver sets)
std::mutex g_plan_mu;
std::vector<bn::BatchPlan*> g_plans;

void drop_plans_with(const bn_solver* s) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (bn::plan_contains(*it, s)) {
            bn::destroy_plan(*it);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

bn_status fail(bn_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

bn_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? BN_ERR_NOMEM : BN_ERR_CUDA, m);
}

void free_buffers(bn_solver* s) {
    void* ptrs[] = {s->f, s->f_prev, s->y, s->kacc, s->Qv, s->Ghat, s->Ghat32, s->work_c, s->twiddle, s->S2, s->quad,
                    s->red, s->q1q, s->partials, s->Qhat, s->partials_lo, s->S2lo, s->Qlo, s->resc_H, s->resc_M,
                    s->resc_acc, s->resc_div, s->resc_mom, s->resc_G0, s->moments, s->flags,
                    s->work.items, s->work_quad.items,
                    s->work.meta[0], s->work.meta[1], s->work.meta[2], s->work.meta[3]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (s->flags_host) cudaFreeHost(s->flags_host);
    if (s->resc_mom_host) cudaFreeHost(s->resc_mom_host);
    bn::free_nd(s);
}

// One evaluation Q = Q_eps(f_in) in velocity units, entirely on the solver's stream.
void eval_device(bn_solver* s, const double* f_in, double* Q_out) {
    bn::launch_dft_forward(s, f_in, s->Ghat);   // also writes the FP32 copy in mixed precision
    if (!s->nd) {
        // the whole 2-D operator in one pass over b (quadratic + reducible + Q_{1,q})
        const int slot = s->prof_slot;
        if (s->prof && slot < 8) cudaEventRecord(s->prof_ev[2 * slot], s->stream);
        bn::launch_fused2d(s);
        if (s->prof && slot < 8) {
            cudaEventRecord(s->prof_ev[2 * slot + 1], s->stream);
            s->prof_slot = slot + 1;
        }
        bn::launch_dft_inverse_real(s, s->Qhat, Q_out, s->scale);
        if (s->opt.conserve) bn::launch_conserve(s, Q_out);
        return;
    }
    // 3-D and CIRCULAR: kernel-mode slices recomputed per evaluation (bn_opnd.cu); with live
    // profiling the whole operator is timed per slot, and its phases by bn_profile_nd
    const int slot = s->prof_slot;
    if (s->prof && slot < 8) cudaEventRecord(s->prof_ev[2 * slot], s->stream);
    bn::launch_nd(s, s->prof ? slot : -1);
    if (s->prof && slot < 8) {
        cudaEventRecord(s->prof_ev[2 * slot + 1], s->stream);
        s->prof_slot = slot + 1;
    }
    bn::launch_dft_inverse_real(s, s->Qhat, Q_out, s->scale);
    if (s->opt.conserve) bn::launch_conserve(s, Q_out);
}

// One time step of the chosen integrator on s->f (state committed only if finite).
// The kernel-mode rounding correction (opt.beta_split) is formed at the first stage and reused by
// the later stages of the step.
void record_step(bn_solver* s, double dt) {
    s->lo_refresh = true;
    if (s->opt.integrator == 0) {
        // classical RK4: K1..K4, f += dt/6 (K1 + 2 K2 + 2 K3 + K4)
        eval_device(s, s->f, s->Qv);
        s->lo_refresh = false;
        bn::launch_rk_stage(s, s->f, s->Qv, s->kacc, s->y, 1.0, 0.5, dt, 1);
        eval_device(s, s->y, s->Qv);
        bn::launch_rk_stage(s, s->f, s->Qv, s->kacc, s->y, 2.0, 0.5, dt, 0);
        eval_device(s, s->y, s->Qv);
        bn::launch_rk_stage(s, s->f, s->Qv, s->kacc, s->y, 2.0, 1.0, dt, 0);
        eval_device(s, s->y, s->Qv);
        bn::launch_rk_final(s, s->f, s->kacc, s->Qv, 1.0, dt, s->f_prev, s->flags);
    } else {
        // SSP-RK2 (Heun): y = f + dt K(f); f = (f + y + dt K(y)) / 2
        eval_device(s, s->f, s->Qv);
        s->lo_refresh = false;
        bn::launch_rk_stage(s, s->f, s->Qv, s->kacc, s->y, 0.0, 1.0, dt, 1);
        eval_device(s, s->y, s->Qv);
        bn::launch_heun_final(s, s->f, s->y, s->Qv, dt, s->f_prev, s->flags);
    }
    s->lo_refresh = true;
}

bn_status ensure_graph(bn_solver* s, double dt) {
    if (s->step_graph && s->graph_dt == dt) return BN_OK;
    if (s->step_graph) {
        cudaGraphExecDestroy(s->step_graph);
        s->step_graph = nullptr;
    }
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "stream capture");
    long long before = s->launches;
    s->prof_slot = 0;
    record_step(s, dt);
    s->prof_slots_used = s->prof_slot;
    s->graph_launches = s->launches - before;
    s->launches = before;   // captured launches are counted when the graph runs
    e = cudaStreamEndCapture(s->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "stream capture end");
    e = cudaGraphInstantiate(&s->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    s->graph_dt = dt;
    return BN_OK;
}

bool valid_solver(const bn_solver* s) { return s != nullptr; }

// After a stepping call: read max f; switch a mixed-precision solver to FP64 for good when
// |eps| max f reaches opt.escalate_at (its captured step graphs are rebuilt on the next call).
void check_escalation(bn_solver* s) {
    unsigned long long bits;
    std::memcpy(&bits, s->flags_host + 4, sizeof bits);
    double mf;
    std::memcpy(&mf, &bits, sizeof mf);
    if (s->flags_host[1] > 0) s->last_max_f = mf;
    if (s->opt.precision == BN_MIXED && s->opt.escalate_at > 0 && std::fabs(s->eps) * s->last_max_f >= s->opt.escalate_at) {
        s->opt.precision = BN_FP64;
        s->t_escalated = s->t;
        if (s->nd) {
            // the slice buffers and kernel shapes depend on the precision
            cudaStreamSynchronize(s->stream);
            bn::free_nd(s);
            std::string err;
            if (bn::plan_nd(s, &err) != BN_OK || bn::prepare_nd(s) != BN_OK) {
                // no FP64 plan for this size (e.g. 3-D N > 32 exceeds the FP64 kernel's shared
                // memory): stay in mixed precision and stop trying
                bn::free_nd(s);
                s->opt.precision = BN_MIXED;
                s->opt.escalate_at = 0;
                s->t_escalated = -1;
                std::string err2;
                bn::plan_nd(s, &err2);
                bn::prepare_nd(s);
            }
            s->n_partials = bn::nd_ctas(s);
        }
        if (s->step_graph) {
            cudaGraphExecDestroy(s->step_graph);
            s->step_graph = nullptr;
        }
        drop_plans_with(s);
    }
}

// Accumulate the durations of the triple-sum launches recorded by the last graph replay
// or direct evaluation (the stream has been synchronised).
void harvest_profile(bn_solver* s, int slots) {
    if (!s->prof) return;
    bn::nd_profile_harvest(s, slots);
    if (s->prof_stamps && slots > 0) {
        unsigned long long st[16];
        if (cudaMemcpy(st, s->prof_stamps, sizeof(st), cudaMemcpyDeviceToHost) == cudaSuccess) {
            for (int i = 0; i < slots && i < 8; ++i)
                if (st[2 * i + 1] > st[2 * i] && st[2 * i] != ~0ull) {
                    s->prof_ns_total += (double)(st[2 * i + 1] - st[2 * i]);
                    s->prof_ns_count += 1;
                }
        } else {
            cudaGetLastError();
        }
    }
    for (int i = 0; i < slots && i < 8; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->prof_ev[2 * i], s->prof_ev[2 * i + 1]) == cudaSuccess) {
            s->prof_ms += ms;
            s->prof_count += 1;
        } else {
            cudaGetLastError();
        }
    }
}

}  // namespace

namespace bn {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace bn

extern "C" {

bn_status bn_default_options(bn_options* opt) {
    if (!opt) return fail(BN_ERR_ARG, "opt is NULL");
    std::memset(opt, 0, sizeof(*opt));
    return BN_OK;
}

size_t bn_options_bytes(void) { return sizeof(bn_options); }
size_t bn_request_bytes(void) { return sizeof(bn_request); }

const char* bn_last_error(void) { return g_err.c_str(); }

bn_status bn_create_solver(int d, int N, double T, double R, int kernel, double eps, const bn_options* opt,
                           void* cuda_stream, bn_solver** out) {
    if (!out) return fail(BN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (d != 2 && d != 3) return fail(BN_ERR_ARG, "d must be 2 or 3");
    if (N < 4 || N % 2 != 0) return fail(BN_ERR_ARG, "N must be even and >= 4");
    if ((d == 2 && N > 64) || (d == 3 && N > 48))
        return fail(BN_ERR_UNSUPPORTED, d == 2 ? "2-D N > 64 is not supported" : "3-D N > 48 is not supported");
    if (!(T > 0) || !(R > 0) || !std::isfinite(T) || !std::isfinite(R)) return fail(BN_ERR_ARG, "T and R must be > 0");
    if (!std::isfinite(eps)) return fail(BN_ERR_ARG, "eps must be finite");
    if (kernel != BN_MAXWELL && kernel != BN_HARD_SPHERE) return fail(BN_ERR_ARG, "unknown kernel");
    if (d == 3 && kernel != BN_HARD_SPHERE) return fail(BN_ERR_UNSUPPORTED, "3-D supports hard spheres only");
    const double Rxi = M_PI * R / T;
    if (Rxi * (3.0 + std::sqrt(2.0)) > 2.0 * M_PI * (1.0 + 1e-12))
        return fail(BN_ERR_ALIAS, "anti-aliasing: pi R / T (3 + sqrt 2) must not exceed 2 pi");

    bn_solver* s = new bn_solver();
    s->g.d = d;
    s->g.N = N;
    s->g.nModes = d == 2 ? N * N : N * N * N;
    s->g.E = 2 * N;
    s->g.nExt = d == 2 ? 4 * N * N : 8 * N * N * N;
    s->T = T;
    s->R = R;
    s->Rxi = Rxi;
    s->eps = eps;
    s->kernel = kernel;
    if (opt) s->opt = *opt;
    else bn_default_options(&s->opt);
    if (s->opt.precision != BN_FP64 && s->opt.precision != BN_MIXED) {
        delete s;
        return fail(BN_ERR_ARG, "precision must be BN_FP64 or BN_MIXED");
    }
    if (s->opt.integrator != 0 && s->opt.integrator != 1) {
        delete s;
        return fail(BN_ERR_ARG, "integrator must be 0 (RK4) or 1 (SSP-RK2)");
    }
    if (!(s->opt.escalate_at >= 0.0) || !std::isfinite(s->opt.escalate_at)) {
        delete s;
        return fail(BN_ERR_ARG, "escalate_at must be finite and >= 0");
    }
    if (s->opt.mixed_rw != 0 && s->opt.mixed_rw != 8 && s->opt.mixed_rw != 16) {
        delete s;
        return fail(BN_ERR_ARG, "mixed_rw must be 0, 8 or 16");
    }
    if (s->opt.mixed_variant < 0 || s->opt.mixed_variant > 4) {
        delete s;
        return fail(BN_ERR_ARG, "mixed_variant must be in 0..4");
    }
    if (s->opt.wrap != 0 && s->opt.wrap != 1) {
        delete s;
        return fail(BN_ERR_ARG, "wrap must be 0 (LINEAR) or 1 (CIRCULAR)");
    }
    if (s->opt.shard_count < 0 || (s->opt.shard_count > 1 && (d != 3 || s->opt.shard_index < 0 ||
                                                                s->opt.shard_index >= s->opt.shard_count ||
                                                                s->opt.shard_count > N))) {
        delete s;
        return fail(BN_ERR_ARG, "shards: 3-D only, 0 <= shard_index < shard_count <= N");
    }
    if (s->opt.debug_wait_giveup != 0 && s->opt.debug_wait_giveup != 1) {
        delete s;
        return fail(BN_ERR_ARG, "debug_wait_giveup must be 0 or 1");
    }
    if (s->opt.beta_split != 0 && s->opt.beta_split != 1) {
        delete s;
        return fail(BN_ERR_ARG, "beta_split must be 0 or 1");
    }
    if (s->opt.beta_budget_mb < 0 || (s->opt.beta_resident != 0 && s->opt.beta_resident != 1) ||
        (s->opt.pair_weights != 0 && s->opt.pair_weights != 1)) {
        delete s;
        return fail(BN_ERR_ARG, "beta_budget_mb must be >= 0, beta_resident and pair_weights 0 or 1");
    }
    if (s->opt.M <= 0) s->opt.M = 2 * N;
    if (s->opt.c_phi <= 0) s->opt.c_phi = d == 2 ? 1.0 / (2.0 * M_PI) : 1.0 / (4.0 * M_PI);
    if (d == 2) {
        // 2-D hard spheres: M1 = Gauss-Legendre points per radius (default N + 8)
        s->opt.M1 = kernel == BN_HARD_SPHERE ? (s->opt.M1 > 0 ? s->opt.M1 : N + 8) : 0;
        s->opt.M2 = 0;
        s->opt.quad3d = 0;
    } else {
        if (s->opt.M1 <= 0) s->opt.M1 = N / 2;
        if (s->opt.M2 <= 0) s->opt.M2 = N / 2;
        s->opt.M = 0;
    }
    s->scale = std::pow(T / M_PI, d + (kernel == BN_HARD_SPHERE ? 1 : 0));

    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { delete s; return cuda_fail(e, "no CUDA device"); }
    if (cuda_stream) {
        s->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete s; return cuda_fail(e, "stream create"); }
        s->own_stream = true;
    }
    std::string err;
    bn_status st = bn::acquire_tables(s, &err);
    if (st != BN_OK) {
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return fail(st, err);
    }
    const bool nd = bn::use_nd(s);
    if (nd) {
        st = bn::plan_nd(s, &err);
        s->n_partials = bn::nd_ctas(s);
    } else {
        st = bn::build_work_list(s, &err);
        if (st == BN_OK) {
            s->n_partials = bn::triple_partials(s);
            st = bn::balance_work_lists(s, &err);
        }
    }
    if (st != BN_OK) {
        free_buffers(s);   // the work lists / operator plan (the other buffers are not allocated yet)
        bn::release_tables(s->tabs);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return fail(st, err);
    }
    const size_t n = s->g.nModes;
    e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    alloc((void**)&s->f, n * sizeof(double));
    alloc((void**)&s->f_prev, n * sizeof(double));
    alloc((void**)&s->y, n * sizeof(double));
    alloc((void**)&s->kacc, n * sizeof(double));
    alloc((void**)&s->Qv, n * sizeof(double));
    alloc((void**)&s->Ghat, n * sizeof(double2));
    alloc((void**)&s->Ghat32, n * sizeof(float2));
    alloc((void**)&s->work_c, n * sizeof(double2));
    alloc((void**)&s->twiddle, (size_t)N * sizeof(double2));
    alloc((void**)&s->S2, (size_t)s->g.nExt * sizeof(double2));
    alloc((void**)&s->quad, n * sizeof(double2));
    alloc((void**)&s->red, n * sizeof(double2));
    alloc((void**)&s->q1q, n * sizeof(double2));
    if (!nd) alloc((void**)&s->partials, (size_t)s->n_partials * n * sizeof(double2));
    alloc((void**)&s->Qhat, n * sizeof(double2));
    if (!nd && d == 2 && s->opt.beta_split && s->opt.precision == BN_MIXED) {
        alloc((void**)&s->partials_lo, (size_t)s->n_partials * n * sizeof(double2));
        alloc((void**)&s->S2lo, (size_t)s->g.nExt * sizeof(double2));
        alloc((void**)&s->Qlo, n * sizeof(double2));
    }
    alloc((void**)&s->moments, 16 * sizeof(double));
    alloc((void**)&s->flags, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s->flags_host, 8 * sizeof(int));
    if (e != cudaSuccess) {
        bn_status r = cuda_fail(e, "device buffers");
        free_buffers(s);
        bn::release_tables(s->tabs);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return r;
    }
    cudaMemsetAsync(s->flags, 0, 8 * sizeof(int), s->stream);
    cudaMemsetAsync(s->Qhat, 0, n * sizeof(double2), s->stream);
    if (s->Qlo) {
        cudaMemsetAsync(s->Qlo, 0, n * sizeof(double2), s->stream);
        cudaMemsetAsync(s->S2lo, 0, (size_t)s->g.nExt * sizeof(double2), s->stream);
    }
    st = nd ? bn::prepare_nd(s) : bn::tune_mixed2d(s, &err);
    if (st != BN_OK) {
        if (nd) err = "kernel-mode slice production failed";
        free_buffers(s);
        bn::release_tables(s->tabs);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return fail(st, err);
    }
    {
        // twiddles e^{-2 i pi m / N} in FP64 on the host (one table per solver)
        std::vector<double2> tw(N);
        for (int m = 0; m < N; ++m) tw[m] = make_double2(std::cos(2.0 * M_PI * m / N), -std::sin(2.0 * M_PI * m / N));
        cudaMemcpyAsync(s->twiddle, tw.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
    }
    cudaMemsetAsync(s->S2, 0, (size_t)s->g.nExt * sizeof(double2), s->stream);
    cudaMemsetAsync(s->q1q, 0, n * sizeof(double2), s->stream);
    cudaMemsetAsync(s->red, 0, n * sizeof(double2), s->stream);
    *out = s;
    return BN_OK;
}

void bn_destroy_solver(bn_solver* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    drop_plans_with(s);
    if (s->step_graph) cudaGraphExecDestroy(s->step_graph);
    for (cudaEvent_t ev : s->prof_ev)
        if (ev) cudaEventDestroy(ev);
    if (s->prof_stamps) cudaFree(s->prof_stamps);
    free_buffers(s);
    bn::release_tables(s->tabs);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

bn_status bn_set_state(bn_solver* s, const double* f, size_t count) {
    if (!valid_solver(s) || !f) return fail(BN_ERR_ARG, "null argument");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    cudaError_t e = cudaMemcpyAsync(s->f, f, count * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state");
    s->has_state = true;
    s->t = 0;
    return BN_OK;
}

bn_status bn_set_state_device(bn_solver* s, const double* f_dev, size_t count) {
    if (!valid_solver(s) || !f_dev) return fail(BN_ERR_ARG, "null argument");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    cudaError_t e = cudaMemcpyAsync(s->f, f_dev, count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state_device");
    s->has_state = true;
    s->t = 0;
    return BN_OK;
}

bn_status bn_get_state(bn_solver* s, double* f, size_t count) {
    if (!valid_solver(s) || !f) return fail(BN_ERR_ARG, "null argument");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    cudaError_t e = cudaMemcpyAsync(f, s->f, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state");
    return BN_OK;
}

bn_status bn_get_state_device(bn_solver* s, double* f_dev, size_t count) {
    if (!valid_solver(s) || !f_dev) return fail(BN_ERR_ARG, "null argument");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    cudaError_t e = cudaMemcpyAsync(f_dev, s->f, count * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state_device");
    return BN_OK;
}

bn_status bn_eval_collision_device(bn_solver* s, const double* f_dev, double* Q_dev, size_t count) {
    if (!valid_solver(s) || !f_dev || !Q_dev) return fail(BN_ERR_ARG, "null argument");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    s->prof_slot = 0;
    eval_device(s, f_dev, Q_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "eval_collision launch");
    return BN_OK;
}

bn_status bn_eval_collision(bn_solver* s, double* Q, size_t count) {
    if (!valid_solver(s) || !Q) return fail(BN_ERR_ARG, "null argument");
    if (s->opt.shard_count > 1) return fail(BN_ERR_UNSUPPORTED, "a shard solver returns modes only (bn_eval_collision_modes)");
    if (count != (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be N^d");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    s->prof_slot = 0;
    cudaMemsetAsync(s->flags + 2, 0, sizeof(int), s->stream);   // the wait-timeout flag of this call
    eval_device(s, s->f, s->Qv);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(Q, s->Qv, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->flags_host, s->flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "eval_collision");
    harvest_profile(s, s->prof_slot);
    if (s->flags_host[2] != 0) return fail(BN_ERR_TIMEOUT, "a bounded device wait gave up during eval_collision");
    return BN_OK;
}

bn_status bn_eval_collision_modes(bn_solver* s, double* Qhat, size_t count) {
    if (!valid_solver(s) || !Qhat) return fail(BN_ERR_ARG, "null argument");
    if (count != 2 * (size_t)s->g.nModes) return fail(BN_ERR_ARG, "count must be 2 N^d");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    s->prof_slot = 0;
    cudaMemsetAsync(s->flags + 2, 0, sizeof(int), s->stream);   // the wait-timeout flag of this call
    eval_device(s, s->f, s->Qv);   // leaves the combined modes in s->Qhat
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(Qhat, s->Qhat, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->flags_host, s->flags, 3 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "eval_collision_modes");
    harvest_profile(s, s->prof_slot);
    if (s->flags_host[2] != 0) return fail(BN_ERR_TIMEOUT, "a bounded device wait gave up during eval_collision_modes");
    return BN_OK;
}

bn_status bn_step_rk(bn_solver* s, double dt, int nsteps) {
    if (!valid_solver(s)) return fail(BN_ERR_ARG, "null solver");
    if (s->opt.shard_count > 1) return fail(BN_ERR_UNSUPPORTED, "a shard solver does not step on its own");
    if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return fail(BN_ERR_ARG, "dt must be > 0 and nsteps >= 0");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    if (nsteps == 0) return BN_OK;
    bn_status st = ensure_graph(s, dt);
    if (st != BN_OK) return st;
    cudaError_t e = cudaMemsetAsync(s->flags, 0, 3 * sizeof(int), s->stream);   // incl. the wait-timeout flag
    if (e == cudaSuccess) e = cudaMemsetAsync(s->flags + 4, 0, 2 * sizeof(int), s->stream);
    for (int i = 0; i < nsteps && e == cudaSuccess; ++i) {
        e = cudaGraphLaunch(s->step_graph, s->stream);
        s->launches += s->graph_launches;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->flags_host, s->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step_rk");
    harvest_profile(s, s->prof_slots_used);
    if (s->flags_host[2] != 0) return fail(BN_ERR_TIMEOUT, "a bounded device wait gave up during step_rk");
    const int committed = s->flags_host[1];
    s->t += committed * dt;
    check_escalation(s);
    if (s->flags_host[0] != 0) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "state became non-finite at step %d of %d; state kept at t = %.17g", committed + 1,
                      nsteps, s->t);
        return fail(BN_ERR_NONFINITE, buf);
    }
    return BN_OK;
}

bn_status bn_moments(bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out) return fail(BN_ERR_ARG, "null argument");
    if (count < (size_t)(s->g.d + 6)) return fail(BN_ERR_ARG, "count must be >= d + 6");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    bn::launch_moments(s, s->f, s->moments);
    double h[16];
    cudaError_t e = cudaMemcpyAsync(h, s->moments, (s->g.d + 5) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moments");
    for (int i = 0; i < s->g.d + 5; ++i) out[i] = h[i];
    out[s->g.d + 5] = s->t;
    return BN_OK;
}

bn_status bn_work_counts(const bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out) return fail(BN_ERR_ARG, "null argument");
    if (count < 4) return fail(BN_ERR_ARG, "count must be >= 4");
    if (s->opt.wrap) {
        // CIRCULAR: every pair (x, y) and triple of I_N contributes
        const double nm = (double)s->g.nModes;
        out[0] = nm * nm;
        out[1] = s->eps != 0.0 ? 2.0 * nm * nm : 0.0;
        out[2] = s->eps != 0.0 ? nm * nm * nm : 0.0;
    } else {
        out[0] = bn::count_pair_terms(s->g.d, s->g.N);
        out[1] = s->eps != 0.0 ? bn::count_reducible_terms(s->g.d, s->g.N) : 0.0;
        out[2] = s->eps != 0.0 ? bn::count_triple_terms(s->g.d, s->g.N) : 0.0;
    }
    out[3] = s->g.nModes;
    return BN_OK;
}

long long bn_kernel_launches(const bn_solver* s) { return s ? s->launches : 0; }

bn_status bn_kernel_config(const bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out || count < 7) return fail(BN_ERR_ARG, "null solver/out or count < 7");
    const bool mixed2d = s->g.d == 2 && s->opt.precision == BN_MIXED && s->g.N <= 32;
    out[0] = mixed2d ? s->mixed_rw : 0;
    out[1] = s->n_partials;
    out[2] = mixed2d ? (s->mixed_v & 1) : 0;
    for (int v = 0; v < 4; ++v) out[3 + v] = s->tune_ms[v];
    return BN_OK;
}

bn_status bn_precision_state(const bn_solver* s, int* precision, double* t_escalated, double* max_f) {
    if (!valid_solver(s)) return fail(BN_ERR_ARG, "null solver");
    if (precision) *precision = s->opt.precision;
    if (t_escalated) *t_escalated = s->t_escalated;
    if (max_f) *max_f = s->last_max_f;
    return BN_OK;
}

bn_status bn_profile_enable(bn_solver* s, int enable) {
    if (!valid_solver(s)) return fail(BN_ERR_ARG, "null solver");
    const bool on = enable != 0;
    if (on && !s->prof_ev[0]) {
        for (cudaEvent_t& ev : s->prof_ev) {
            cudaError_t e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return cuda_fail(e, "profile events");
        }
        cudaError_t e = cudaMalloc(&s->prof_stamps, 16 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(e, "profile stamps");
    }
    if (s->nd) {
        bn_status st = bn::nd_profile_enable(s, on);
        if (st != BN_OK) return fail(st, "profile events");
    }
    if (on != s->prof && s->step_graph) {
        cudaStreamSynchronize(s->stream);
        cudaGraphExecDestroy(s->step_graph);
        s->step_graph = nullptr;
    }
    s->prof = on;
    s->prof_ms = 0;
    s->prof_count = 0;
    s->prof_ns_total = 0;
    s->prof_ns_count = 0;
    return BN_OK;
}

bn_status bn_profile_read(bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out) return fail(BN_ERR_ARG, "null argument");
    if (count < 2) return fail(BN_ERR_ARG, "count must be >= 2");
    out[0] = s->prof_ms;
    out[1] = (double)s->prof_count;
    if (count >= 4) {
        out[2] = s->prof_ns_total * 1e-6;
        out[3] = (double)s->prof_ns_count;
    }
    s->prof_ms = 0;
    s->prof_count = 0;
    s->prof_ns_total = 0;
    s->prof_ns_count = 0;
    return BN_OK;
}

bn_status bn_step_rk_batch(bn_solver** solvers, int n, const double* dts, int nsteps, int* failed) {
    if (failed) *failed = -1;
    if (!solvers || n <= 0 || !dts || nsteps < 0) return fail(BN_ERR_ARG, "invalid batch arguments");
    bool shared = true;   // every request 2-D with one integrator and no live profiling: one graph for all
    for (int i = 0; i < n; ++i) {
        if (!solvers[i]) return fail(BN_ERR_ARG, "null solver in batch");
        if (!solvers[i]->has_state) return fail(BN_ERR_STATE, "solver in batch has no state");
        if (solvers[i]->opt.shard_count > 1) return fail(BN_ERR_UNSUPPORTED, "a shard solver does not step on its own");
        if (!(dts[i] > 0) || !std::isfinite(dts[i])) return fail(BN_ERR_ARG, "dt must be > 0");
        for (int j = 0; j < i; ++j)
            if (solvers[j] == solvers[i]) return fail(BN_ERR_ARG, "a solver appears twice in the batch");
        if (solvers[i]->nd || solvers[i]->opt.integrator != solvers[0]->opt.integrator) shared = false;
    }
    if (nsteps == 0) return BN_OK;
    cudaStream_t st0 = solvers[0]->stream;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n; ++i)
        if (solvers[i]->stream != st0) {
            // order each solver's own stream before the shared stream
            cudaEvent_t ev;
            cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            cudaEventRecord(ev, solvers[i]->stream);
            cudaStreamWaitEvent(st0, ev, 0);
            cudaEventDestroy(ev);
        }
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaMemsetAsync(solvers[i]->flags, 0, 3 * sizeof(int), st0);
        if (e == cudaSuccess) e = cudaMemsetAsync(solvers[i]->flags + 4, 0, 2 * sizeof(int), st0);
    }
    if (e != cudaSuccess) return cuda_fail(e, "step_rk_batch");
    const bool timed = solvers[0]->prof;
    bn::BatchPlan* plan = nullptr;
    if (shared) {
        {
            std::lock_guard<std::mutex> lock(g_plan_mu);
            for (bn::BatchPlan* p : g_plans)
                if (bn::plan_matches(p, solvers, n, dts, timed)) { plan = p; break; }
        }
        if (!plan) {
            std::string err;
            bn_status st = bn::build_plan(solvers, n, dts, timed, st0, &plan, &err);
            if (st != BN_OK) return fail(st, err);
            std::lock_guard<std::mutex> lock(g_plan_mu);
            g_plans.push_back(plan);
            while (g_plans.size() > 4) {
                bn::destroy_plan(g_plans.front());
                g_plans.erase(g_plans.begin());
            }
        }
        if (bn::replay_plan(plan, st0, nsteps) != BN_OK) return cuda_fail(cudaGetLastError(), "batch replay");
    } else {
        for (int i = 0; i < n; ++i) {
            bn_status st = ensure_graph(solvers[i], dts[i]);
            if (st != BN_OK) return st;
        }
        for (int k = 0; k < nsteps && e == cudaSuccess; ++k)
            for (int i = 0; i < n && e == cudaSuccess; ++i) {
                e = cudaGraphLaunch(solvers[i]->step_graph, st0);
                solvers[i]->launches += solvers[i]->graph_launches;
            }
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(solvers[i]->flags_host, solvers[i]->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, st0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st0);
    if (e != cudaSuccess) return cuda_fail(e, "step_rk_batch");
    if (shared && timed) {
        double ns = 0;
        long long cnt = 0;
        if (bn::plan_read_spans(plan, st0, &ns, &cnt)) {
            solvers[0]->prof_ns_total += ns;
            solvers[0]->prof_ns_count += cnt;
        }
    }
    bn_status result = BN_OK;
    for (int i = 0; i < n; ++i) {
        bn_solver* s = solvers[i];
        if (!shared) harvest_profile(s, s->prof_slots_used);
        s->t += s->flags_host[1] * dts[i];
        check_escalation(s);
        if (s->flags_host[2] != 0 && result == BN_OK) {
            if (failed) *failed = i;
            result = fail(BN_ERR_TIMEOUT, "a bounded device wait gave up in the batch");
        }
        if (s->flags_host[0] != 0 && result == BN_OK) {
            if (failed) *failed = i;
            result = fail(BN_ERR_NONFINITE, "a solver in the batch became non-finite");
        }
    }
    return result;
}

}  // extern "C"

extern "C" bn_status bn_plan_mixed2d(int N, int rw, int oriented, int nblk, int* out, size_t count, int* n_items) {
    if (N < 2 || N > 32 || (N & 1) || (rw != 8 && rw != 16) || nblk < 1 || !n_items)
        return fail(BN_ERR_ARG, "bn_plan_mixed2d: N even in [2, 32], rw 8 or 16, nblk >= 1, n_items non-null");
    const std::vector<int> rows = bn::plan_mixed2d_rows(N, rw, oriented != 0, nblk);
    *n_items = (int)(rows.size() / bn::kPlanCols);
    if (out) {
        if (count < rows.size()) return fail(BN_ERR_ARG, "bn_plan_mixed2d: out too small");
        std::copy(rows.begin(), rows.end(), out);
    }
    return BN_OK;
}

extern "C" bn_status bn_profile_nd(bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out || count < 8) return fail(BN_ERR_ARG, "null solver/out or count < 8");
    if (!s->nd) return fail(BN_ERR_UNSUPPORTED, "bn_profile_nd: not a 3-D or CIRCULAR solver");
    return bn::nd_profile_read(s, out, count);
}

extern "C" bn_status bn_plan_shards(int d, int N, int wrap, int count, int* bounds, size_t nbounds) {
    if (d != 3 || N < 4 || N > 48 || (N & 1) || (wrap != 0 && wrap != 1) || count < 1 || count > N || !bounds ||
        nbounds < (size_t)count + 1)
        return fail(BN_ERR_ARG, "bn_plan_shards: d = 3, N even in [4, 48], wrap 0/1, 1 <= count <= N, nbounds >= count + 1");
    const std::vector<int> b = bn::shard_bounds_for(d, N, wrap, count);
    for (int i = 0; i <= count; ++i) bounds[i] = b[i];
    return BN_OK;
}

// ------------------------------------------------------------------ velocity rescaling (Sec. 3)
extern "C" bn_status bn_rescale_set(bn_solver* s, double L, double omega, const double* u, size_t du, double rho, double e) {
    if (!valid_solver(s) || !u) return fail(BN_ERR_ARG, "null solver or u");
    if (s->opt.wrap || s->opt.shard_count > 1)
        return fail(BN_ERR_UNSUPPORTED, "velocity rescaling: LINEAR truncation, unsharded solvers only");
    if (std::fabs(s->T - M_PI) > 1e-12 * M_PI)
        return fail(BN_ERR_ARG, "velocity rescaling: the solver's box must be T = pi (the rescaled variable xi)");
    if (du != (size_t)s->g.d) return fail(BN_ERR_ARG, "velocity rescaling: u needs d components");
    bool ufin = true;
    for (int c = 0; c < s->g.d; ++c) ufin = ufin && std::isfinite(u[c]);
    if (!(L > 0) || !(omega > 0) || !(rho > 0) || !(e > 0) || !std::isfinite(L) || !std::isfinite(omega) ||
        !std::isfinite(rho) || !std::isfinite(e) || !ufin)
        return fail(BN_ERR_ARG, "velocity rescaling: L, omega, rho, e must be finite and > 0, u finite");
    const size_t n = s->g.nModes;
    if (!s->resc_H) {
        cudaError_t e2 = cudaMalloc((void**)&s->resc_H, n * sizeof(double));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&s->resc_M, n * sizeof(double2));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&s->resc_acc, n * sizeof(double2));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&s->resc_div, n * sizeof(double));
        if (e2 == cudaSuccess) e2 = cudaMalloc((void**)&s->resc_mom, 5 * sizeof(double));
        if (e2 == cudaSuccess) e2 = cudaMallocHost((void**)&s->resc_mom_host, 5 * sizeof(double));
        if (e2 != cudaSuccess) return cuda_fail(e2, "velocity rescaling buffers");
    }
    double T = 0, z = 0;
    std::string err;
    const bn_status st = bn::rescale_temperature(s->g.d, s->eps, rho, e, &T, &z, &err);
    if (st != BN_OK) return fail(st, err);
    s->resc = true;
    s->resc_L = L;
    s->resc_w = omega;
    for (int c = 0; c < 3; ++c) s->resc_u[c] = c < s->g.d ? u[c] : 0.0;
    s->resc_rho = rho;
    s->resc_e = e;
    s->resc_T = T;
    s->resc_z = z;
    return BN_OK;
}

extern "C" bn_status bn_equilibrium_temperature(int d, double eps, double rho, double e, double* T, double* z) {
    if (!T || !z || (d != 2 && d != 3)) return fail(BN_ERR_ARG, "T, z must be non-null and d 2 or 3");
    std::string err;
    const bn_status st = bn::rescale_temperature(d, eps, rho, e, T, z, &err);
    if (st != BN_OK) return fail(st, err);
    return BN_OK;
}

extern "C" bn_status bn_rescale_get(const bn_solver* s, double* out, size_t count) {
    if (!valid_solver(s) || !out || count < 9) return fail(BN_ERR_ARG, "null solver/out or count < 9");
    if (!s->resc) return fail(BN_ERR_STATE, "velocity rescaling not set (bn_rescale_set)");
    const double v[9] = {s->resc_w, s->resc_u[0], s->resc_u[1], s->resc_u[2], s->resc_rho, s->resc_e, s->resc_T,
                         s->resc_z, s->t};
    std::copy(v, v + 9, out);
    return BN_OK;
}

namespace {

// Step 2 and 3(a) of Sec. 3.3 for the rescaled solve: Q of s->f (the solver's operator with eps0 times
// the scale^d) into s->Qv, and rho, u, e advanced by dt with its moments from the stored macroscopic
// state.  Nothing of the state changes.
bn_status resc_eval_moments(bn_solver* s, double dt, double eps0, double* rho1, double* u1, double* e1) {
    const int d = s->g.d, N = s->g.N;
    const double gamma = s->kernel == BN_HARD_SPHERE ? 1.0 : 0.0;
    const double dxi = std::pow(2.0 * M_PI / N, d);
    const double sc = M_PI * s->resc_w / s->resc_L;
    s->eps = eps0 * std::pow(sc, d);
    s->lo_refresh = true;
    eval_device(s, s->f, s->Qv);
    s->eps = eps0;
    bn::launch_resc_moments(s, s->Qv, s->resc_mom);
    cudaMemcpyAsync(s->resc_mom_host, s->resc_mom, (d + 2) * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaMemcpyAsync(s->flags_host, s->flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "rescaled step");
    if (s->flags_host[2]) {
        cudaMemsetAsync(s->flags + 2, 0, sizeof(int), s->stream);
        return fail(BN_ERR_TIMEOUT, "a bounded device wait gave up during the rescaled step");
    }
    const double* S = s->resc_mom_host;   // [sum Q, sum xi_c Q (c < d), sum |xi|^2 Q]
    bool fin = true;
    for (int c = 0; c < d + 2; ++c) fin = fin && std::isfinite(S[c]);
    if (!fin) return fail(BN_ERR_NONFINITE, "rescaled step: non-finite collision moments (state kept)");
    const double coef = dxi * std::pow(sc, -gamma);
    *rho1 = s->resc_rho + dt * coef * S[0];
    for (int c = 0; c < 3; ++c)
        u1[c] = c < d ? (s->resc_rho * s->resc_u[c] + dt * coef * (S[1 + c] / sc + s->resc_u[c] * S[0])) / *rho1 : 0.0;
    *e1 = (s->resc_rho * s->resc_e + dt * 0.5 * coef * S[1 + d] / (sc * sc)) / *rho1;
    return BN_OK;
}

double resc_omega(int d, double eps0, double T, const double* u) {
    double u2 = 0;
    for (int c = 0; c < d; ++c) u2 += u[c] * u[c];
    return eps0 != 0.0 ? std::sqrt(T) : std::sqrt(T + u2 / d);
}

// One forward Euler step of Sec. 3.3 (steps 2 to 5), in place on s->f and the macroscopic state;
// a_used, b_used (d values) receive the dilation rate and drift of its divergence term.  On an error
// the state is that of the start of the step.
bn_status resc_euler_step(bn_solver* s, double dt, double eps0, double* a_used, double* b_used) {
    const int d = s->g.d;
    const double gamma = s->kernel == BN_HARD_SPHERE ? 1.0 : 0.0;
    const double sc = M_PI * s->resc_w / s->resc_L;
    double rho1 = 0, u1[3] = {0, 0, 0}, e1 = 0;
    bn_status st = resc_eval_moments(s, dt, eps0, &rho1, u1, &e1);
    if (st != BN_OK) return st;
    // step 3(b), (c): temperature, fugacity, scale
    double T1 = 0, z1 = 0;
    std::string err;
    st = bn::rescale_temperature(d, eps0, rho1, e1, &T1, &z1, &err);
    if (st != BN_OK) return fail(st, err + " (state kept)");
    const double w1 = resc_omega(d, eps0, T1, u1);
    // steps 4, 5: the divergence term and G^{n+1}
    const double a = (w1 - s->resc_w) / (dt * s->resc_w);
    double b[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) b[c] = sc * (u1[c] - s->resc_u[c]) / dt;
    bn::launch_resc_advance(s, s->f, s->Qv, a, b, dt, std::pow(sc, -gamma), s->resc_H, s->resc_M, s->resc_acc,
                            s->resc_div);
    if (a_used) *a_used = a;
    if (b_used)
        for (int c = 0; c < d; ++c) b_used[c] = b[c];
    s->resc_rho = rho1;
    for (int c = 0; c < 3; ++c) s->resc_u[c] = u1[c];
    s->resc_e = e1;
    s->resc_T = T1;
    s->resc_z = z1;
    s->resc_w = w1;
    return BN_OK;
}

bn_status resc_check(bn_solver* s, double dt, int nsteps) {
    if (!valid_solver(s)) return fail(BN_ERR_ARG, "null solver");
    if (!s->resc) return fail(BN_ERR_STATE, "velocity rescaling not set (bn_rescale_set)");
    if (!s->has_state) return fail(BN_ERR_STATE, "no state set");
    if (!(dt > 0) || !std::isfinite(dt) || nsteps < 0) return fail(BN_ERR_ARG, "dt must be > 0 and nsteps >= 0");
    return BN_OK;
}

}  // namespace

extern "C" bn_status bn_step_rescaled(bn_solver* s, double dt, int nsteps) {
    bn_status st = resc_check(s, dt, nsteps);
    if (st != BN_OK) return st;
    const double eps0 = s->eps;
    cudaMemsetAsync(s->flags + 2, 0, sizeof(int), s->stream);
    for (int step = 0; step < nsteps; ++step) {
        st = resc_euler_step(s, dt, eps0, nullptr, nullptr);
        if (st != BN_OK) return st;
        s->t += dt;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rescaled step");
    return BN_OK;
}

extern "C" bn_status bn_step_rescaled_rk2(bn_solver* s, double dt, int nsteps) {
    bn_status st = resc_check(s, dt, nsteps);
    if (st != BN_OK) return st;
    const int d = s->g.d;
    const size_t n = s->g.nModes;
    const double gamma = s->kernel == BN_HARD_SPHERE ? 1.0 : 0.0;
    if (!s->resc_G0) {
        cudaError_t e0 = cudaMalloc((void**)&s->resc_G0, n * sizeof(double));
        if (e0 != cudaSuccess) return cuda_fail(e0, "rescaled RK2 buffer");
    }
    const double eps0 = s->eps;
    cudaMemsetAsync(s->flags + 2, 0, sizeof(int), s->stream);
    for (int step = 0; step < nsteps; ++step) {
        // Y^n: G^n and the macroscopic state
        cudaMemcpyAsync(s->resc_G0, s->f, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
        const double rho0 = s->resc_rho, e0 = s->resc_e, w0 = s->resc_w, T0 = s->resc_T, z0 = s->resc_z;
        const double s0 = M_PI * w0 / s->resc_L;
        double u0[3];
        for (int c = 0; c < 3; ++c) u0[c] = s->resc_u[c];
        auto restore = [&]() {
            cudaMemcpyAsync(s->f, s->resc_G0, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream);
            s->resc_rho = rho0;
            s->resc_e = e0;
            s->resc_w = w0;
            s->resc_T = T0;
            s->resc_z = z0;
            for (int c = 0; c < 3; ++c) s->resc_u[c] = u0[c];
            cudaStreamSynchronize(s->stream);
        };
        // predictor: the forward Euler step (G^(1) in s->f; its rates a1, b1)
        double a1 = 0, b1[3] = {0, 0, 0};
        st = resc_euler_step(s, dt, eps0, &a1, b1);
        if (st != BN_OK) {
            restore();
            return st;
        }
        // second stage: Q1 = Q(G^(1)) at the scale of G^(1) and the Euler moment update Y^(2)
        const double s1 = M_PI * s->resc_w / s->resc_L;
        double rho2 = 0, u2[3] = {0, 0, 0}, e2 = 0;
        st = resc_eval_moments(s, dt, eps0, &rho2, u2, &e2);
        if (st != BN_OK) {
            restore();
            return st;
        }
        // Y^{n+1} = (Y^n + Y^(2)) / 2 for rho, rho u, rho e; T, z, w from them
        const double rhoN = 0.5 * (rho0 + rho2);
        double uN[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) uN[c] = 0.5 * (rho0 * u0[c] + rho2 * u2[c]) / rhoN;
        const double eN = 0.5 * (rho0 * e0 + rho2 * e2) / rhoN;
        double TN = 0, zN = 0;
        std::string err;
        st = bn::rescale_temperature(d, eps0, rhoN, eN, &TN, &zN, &err);
        if (st != BN_OK) {
            restore();
            return fail(st, err + " (state kept)");
        }
        const double wN = resc_omega(d, eps0, TN, uN);
        // G^{n+1} = G0 + dt/2 [F(G0) + F(G1)] with the midpoint rates a = ln(wN / w0) / dt and
        // u' = (uN - u0) / dt, each F at its stage's scale.  With the predictor G1 = G0 + dt F(G0; a1, b1):
        // G^{n+1} = (Z + W) / 2, Z = G1 + dt F(G1; a, s1 u'), W = G0 + dt T(G0; a - a1, s0 u' - b1),
        // T the divergence part of F alone
        const double a = std::log(wN / w0) / dt;
        double bZ[3] = {0, 0, 0}, bW[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) {
            const double du = (uN[c] - u0[c]) / dt;
            bZ[c] = s1 * du;
            bW[c] = s0 * du - b1[c];
        }
        bn::launch_resc_advance(s, s->f, s->Qv, a, bZ, dt, std::pow(s1, -gamma), s->resc_H, s->resc_M, s->resc_acc,
                                s->resc_div);
        bn::launch_resc_advance(s, s->resc_G0, s->Qv, a - a1, bW, dt, 0.0, s->resc_H, s->resc_M, s->resc_acc,
                                s->resc_div);
        bn::launch_resc_average(s, s->f, s->resc_G0);
        s->resc_rho = rhoN;
        for (int c = 0; c < 3; ++c) s->resc_u[c] = uN[c];
        s->resc_e = eN;
        s->resc_T = TN;
        s->resc_z = zN;
        s->resc_w = wN;
        s->t += dt;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "rescaled step");
    return BN_OK;
}
