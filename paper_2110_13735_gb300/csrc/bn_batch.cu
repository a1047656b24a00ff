// bn_batch.cu -- many 2-D requests advanced together: every stage of one RK step of all
// requests runs as a fixed set of shared launches, captured once per set of requests as one CUDA
// graph.  Per evaluation: the second forward transform pass, the fused operator per
// precision/size group, the partial sums, the first inverse pass, and one row kernel
// with the last inverse pass, the RK update and the first forward pass of the next stage.  Each request keeps its own CTA partition and every output keeps the arithmetic of
// the single-request kernels, so its result is identical to the one it gets alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kThreads = 256;

// one request in the batched element-wise / transform launches
struct ElemJob {
    int N, nm;
    double* f;          // state
    double* y;          // stage argument
    double* kacc;       // RK accumulator
    double* Qv;         // stage derivative in velocity units
    double* cand;       // candidate state
    int* flags;         // [0] non-finite, [1] committed steps
    double2* Ghat;
    float2* Ghat32;     // null in FP64 mode
    double2* work_c;
    const double2* tw;
    double2* Qhat;
    double2* partials;  // FP64 pairs, or FP32 (sum, compensation) quadruples when part32
    int nPart;
    int part32;
    double dt, scale;
    const float2* Sb;   // mixed N <= 32 with eps != 0: S(b) from the operator kernel (else null)
    float eps;
    const double2* Qlo; // kernel-mode rounding correction: its modes, added to Q^ (else null)
};

__device__ __forceinline__ double2 warp_sum2(double sr, double si) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    return make_double2(sr, si);
}

__device__ __forceinline__ double2 tw_at(const double2* tw, int k, int j, int N, int sign) {
    int m;
    if ((N & (N - 1)) == 0) {
        m = (k * j) & (N - 1);
    } else {
        m = (k * j) % N;
        if (m < 0) m += N;
    }
    double2 w = __ldg(tw + m);
    if (sign > 0) w.y = -w.y;
    return w;
}

// Pass `pass` of the 2-D transforms for job blockIdx.y, one warp per output:
//   0: real stage input (f or y) along n_2 -> work_c         (forward)
//   1: work_c along n_1 -> Ghat (and Ghat32), scale N^-2      (forward)
//   2: Qhat along n_1 -> work_c                               (inverse)
//   3: work_c along n_2 -> Qv = scale * Re                    (inverse)
// In pass 3 the Runge-Kutta update of the same entry can follow (rk: 0 none; 1 RK4 stage
// acc = (first ? 0 : acc) + w_acc K, y = f + c dt K; 2 RK4 final, candidate = f + dt/6 (acc + K);
// 3 SSP-RK2 final, candidate = (f + y + dt K) / 2), non-finite candidates flagged.
__global__ void k_dft_batch(const ElemJob* __restrict__ jobs, int pass, int stage_in, int rk = 0, double w_acc = 0.0,
                            double c_next = 0.0, int first = 0) {
    const ElemJob J = jobs[blockIdx.y];
    const int N = J.N, nm = J.nm, lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int stride = (pass == 0 || pass == 3) ? 1 : N;
    const int sign = pass < 2 ? -1 : +1;
    const double* rin = stage_in == 0 ? J.f : J.y;
    for (int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < nm; idx += warps) {
        const int c = (idx / stride) % N, base = idx - c * stride, k = c - N / 2;
        double sr = 0.0, si = 0.0;
        for (int jj = lane; jj < N; jj += 32) {
            const double2 w = tw_at(J.tw, k, jj - N / 2, N, sign);
            if (pass == 0) {
                const double x = rin[base + jj * stride];
                sr = fma(x, w.x, sr);
                si = fma(x, w.y, si);
            } else {
                const double2 x = (pass == 2 ? J.Qhat : J.work_c)[base + jj * stride];
                sr = fma(x.x, w.x, fma(-x.y, w.y, sr));
                si = fma(x.x, w.y, fma(x.y, w.x, si));
            }
        }
        const double2 sum = warp_sum2(sr, si);
        if (lane == 0) {
            if (pass == 0 || pass == 2) {
                J.work_c[idx] = sum;
            } else if (pass == 1) {
                const double sc = 1.0 / nm;
                J.Ghat[idx] = make_double2(sum.x * sc, sum.y * sc);
                if (J.Ghat32) J.Ghat32[idx] = make_float2((float)(sum.x * sc), (float)(sum.y * sc));
            } else {
                const double K = sum.x * J.scale;
                J.Qv[idx] = K;
                if (rk == 1) {
                    J.kacc[idx] = first ? w_acc * K : fma(w_acc, K, J.kacc[idx]);
                    J.y[idx] = fma(c_next * J.dt, K, J.f[idx]);
                } else if (rk >= 2) {
                    const double v = rk == 2 ? fma(J.dt / 6.0, J.kacc[idx] + K, J.f[idx])
                                             : 0.5 * (J.f[idx] + fma(J.dt, K, J.y[idx]));
                    J.cand[idx] = v;
                    if (!isfinite(v)) atomicOr(&J.flags[0], 1);
                }
            }
        }
    }
}

// The RK update of one entry after its stage derivative K (as in k_dft_batch, pass 3).
__device__ __forceinline__ void rk_entry(const ElemJob& J, int idx, double K, int rk, double w_acc, double c_next,
                                         int first) {
    J.Qv[idx] = K;
    if (rk == 1) {
        J.kacc[idx] = first ? w_acc * K : fma(w_acc, K, J.kacc[idx]);
        J.y[idx] = fma(c_next * J.dt, K, J.f[idx]);
    } else if (rk >= 2) {
        const double v = rk == 2 ? fma(J.dt / 6.0, J.kacc[idx] + K, J.f[idx]) : 0.5 * (J.f[idx] + fma(J.dt, K, J.y[idx]));
        J.cand[idx] = v;
        if (!isfinite(v)) atomicOr(&J.flags[0], 1);
    }
}

// Row j1 = blockIdx.x of job blockIdx.y: the last inverse pass (work_c along n_2 -> Q), the RK update
// of the row and, for an RK stage (rk == 1), the first forward pass of the next evaluation on the
// new stage argument y (along n_2 -> work_c).  Each output is one warp with the lanes over the
// summation index and the same butterfly as k_dft_batch, so the values are bitwise those of the
// separate launches.  N <= 64.
__global__ void __launch_bounds__(256) k_row_inv_rk_fwd(const ElemJob* __restrict__ jobs, int rk, double w_acc,
                                                       double c_next, int first) {
    __shared__ double ysh[64];
    const ElemJob J = jobs[blockIdx.y];
    const int N = J.N, j1 = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (j1 >= N) return;   // uniform per block
    const int base = j1 * N;
    for (int c = warp; c < N; c += 8) {   // pass 3: output (j1, c)
        const int k = c - N / 2;
        double sr = 0.0, si = 0.0;
        for (int jj = lane; jj < N; jj += 32) {
            const double2 w = tw_at(J.tw, k, jj - N / 2, N, +1);
            const double2 x = J.work_c[base + jj];
            sr = fma(x.x, w.x, fma(-x.y, w.y, sr));
            si = fma(x.x, w.y, fma(x.y, w.x, si));
        }
        const double2 sum = warp_sum2(sr, si);
        if (lane == 0) {
            rk_entry(J, base + c, sum.x * J.scale, rk, w_acc, c_next, first);
            if (rk == 1) ysh[c] = J.y[base + c];
        }
    }
    if (rk != 1) return;   // uniform
    __syncthreads();
    for (int c = warp; c < N; c += 8) {   // pass 0 of the next evaluation: output (j1, c)
        const int k = c - N / 2;
        double sr = 0.0, si = 0.0;
        for (int jj = lane; jj < N; jj += 32) {
            const double2 w = tw_at(J.tw, k, jj - N / 2, N, -1);
            const double x = ysh[jj];
            sr = fma(x, w.x, sr);
            si = fma(x, w.y, si);
        }
        const double2 sum = warp_sum2(sr, si);
        if (lane == 0) J.work_c[base + c] = sum;
    }
}

// Fixed-order sum of each job's partials into its Q^ (same order as the single-request kernel).
// With `tm` (a timed plan), thread 0 of the first block also closes the timing of the fused
// launches of this evaluation: tm[0..1] = (min start, max end) stamped by their CTAs are added to
// the running total tm[2] and count tm[3], then reset for the next evaluation.  The fused kernels
// have completed (stream order) and no other thread touches tm.
__global__ void __launch_bounds__(256) k_sum_partials_batch(const ElemJob* __restrict__ jobs,
                                                            unsigned long long* __restrict__ tm) {
    if (tm && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        const unsigned long long t0 = tm[0], t1 = tm[1];
        if (t1 > t0) {
            tm[2] += t1 - t0;
            tm[3] += 1;
        }
        tm[0] = ~0ull;
        tm[1] = 0;
    }
    const ElemJob J = jobs[blockIdx.y];
    if (!J.Qhat) return;   // a job without a residual-table pass (uniform per block)
    if (J.part32) {
        if (blockIdx.x * kPartModes >= J.nm) return;   // uniform per block
        sum_partials_f32_block(J.nm, J.nPart, reinterpret_cast<const float4*>(J.partials), J.Qhat, blockIdx.x, J.N,
                               J.Ghat32, J.Sb, J.eps);
        return;
    }
    if (blockIdx.x * 8 >= J.nm) return;   // uniform per block
    __shared__ double2 sh[32][8];
    const int m = threadIdx.x & 7, w = threadIdx.x >> 3;
    const int i = blockIdx.x * 8 + m;
    double x = 0, y = 0;
    if (i < J.nm) {
        for (int c = w; c < J.nPart; c += 32) {
            const double2 v = J.partials[(size_t)c * J.nm + i];
            x += v.x;
            y += v.y;
        }
    }
    sh[w][m] = make_double2(x, y);
    __syncthreads();
    if (threadIdx.x < 8 && i < J.nm) {
        double sx = 0, sy = 0;
        for (int k = 0; k < 32; ++k) { sx += sh[k][m].x; sy += sh[k][m].y; }
        J.Qhat[i] = make_double2(sx, sy);
    }
}

// Q^ += the modes of the kernel-mode rounding correction, for the jobs that have it.
__global__ void k_add_lo_batch(const ElemJob* __restrict__ jobs) {
    const ElemJob J = jobs[blockIdx.y];
    if (!J.Qlo) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nm; i += gridDim.x * blockDim.x) {
        const double2 a = J.Qlo[i];
        double2 q = J.Qhat[i];
        q.x += a.x;
        q.y += a.y;
        J.Qhat[i] = q;
    }
}

// RK4 stage update for every job: acc = (first ? 0 : acc) + w_acc K;  y = f + c dt K
__global__ void k_rk_stage_batch(const ElemJob* __restrict__ jobs, double w_acc, double c, int first) {
    const ElemJob J = jobs[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nm; i += gridDim.x * blockDim.x) {
        const double k = J.Qv[i];
        J.kacc[i] = first ? w_acc * k : fma(w_acc, k, J.kacc[i]);
        J.y[i] = fma(c * J.dt, k, J.f[i]);
    }
}

// candidate = f + dt/6 (acc + K); non-finite -> flags[0]
__global__ void k_rk_final_batch(const ElemJob* __restrict__ jobs) {
    const ElemJob J = jobs[blockIdx.y];
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nm; i += gridDim.x * blockDim.x) {
        const double v = fma(J.dt / 6.0, J.kacc[i] + J.Qv[i], J.f[i]);
        J.cand[i] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&J.flags[0], 1);
}

// SSP-RK2: candidate = (f + y + dt K) / 2
__global__ void k_heun_final_batch(const ElemJob* __restrict__ jobs) {
    const ElemJob J = jobs[blockIdx.y];
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nm; i += gridDim.x * blockDim.x) {
        const double v = 0.5 * (J.f[i] + fma(J.dt, J.Qv[i], J.y[i]));
        J.cand[i] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&J.flags[0], 1);
}

__global__ void k_commit_batch(const ElemJob* __restrict__ jobs) {
    const ElemJob J = jobs[blockIdx.y];
    if (J.flags[0] != 0) return;
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.nm; i += gridDim.x * blockDim.x) {
        const double v = J.cand[i];
        J.f[i] = v;
        m = fmax(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(J.flags + 4), (unsigned long long)__double_as_longlong(m));
    if (blockIdx.x == 0 && threadIdx.x == 0) J.flags[1] += 1;
}

}  // namespace

// A captured batched step for a fixed list of 2-D solvers.
struct BatchPlan {
    std::vector<bn_solver*> solvers;
    std::vector<double> dts;
    int integrator = 0;
    ElemJob* d_elem = nullptr;
    struct Group {
        int variant = 0, njobs = 0, total = 0, maxN = 0, maxCount = 0;
        void* d_jobs = nullptr;
        int* d_cta = nullptr;
    };
    std::vector<Group> groups;
    // kernel-mode rounding correction: the residual-table pass of the jobs that have it (its own
    // groups, and job records whose Q^, partials and S(b) are that pass's buffers)
    std::vector<Group> lo_groups;
    ElemJob* d_elem_lo = nullptr;
    int maxN = 0, maxNm = 0;
    bool timed = false;
    unsigned long long* d_time = nullptr;   // [min start, max end, total ns, count] (timed plans)
    cudaGraphExec_t graph = nullptr;
    long long launches = 0;   // kernels per replay
};

void destroy_plan(BatchPlan* p) {
    if (!p) return;
    if (p->graph) cudaGraphExecDestroy(p->graph);
    cudaFree(p->d_elem);
    cudaFree(p->d_elem_lo);
    cudaFree(p->d_time);
    for (auto* gs : {&p->groups, &p->lo_groups})
        for (auto& g : *gs) {
            cudaFree(g.d_jobs);
            cudaFree(g.d_cta);
        }
    delete p;
}

// One evaluation of every request's operator; with rk != 0 (no request projects Q) the RK update
// that follows is fused into the last transform pass (arguments as for k_dft_batch): per row, the
// last inverse pass, the RK update and, for an RK stage, the first forward pass of the next
// evaluation run as one launch (fwd0_done: this evaluation's first pass was done that way).
// With lo_pass (the first evaluation of a step) the residual-table pass of the kernel-mode rounding
// correction runs first; every evaluation then adds its modes to Q^.
static void record_batched_eval(BatchPlan* p, cudaStream_t st, int stage_in, int rk = 0, double w_acc = 0.0,
                                double c_next = 0.0, int first = 0, bool fwd0_done = false, bool lo_pass = false) {
    const int nj = (int)p->solvers.size();
    const dim3 gw((p->maxNm * 32 + kThreads - 1) / kThreads, nj);
    const dim3 gp((p->maxNm + kPartModes - 1) / kPartModes, nj);
    if (!fwd0_done) {
        k_dft_batch<<<gw, kThreads, 0, st>>>(p->d_elem, 0, stage_in);
        p->launches++;
    }
    k_dft_batch<<<gw, kThreads, 0, st>>>(p->d_elem, 1, stage_in);
    p->launches++;
    if (lo_pass && !p->lo_groups.empty()) {
        for (auto& g : p->lo_groups) launch_fused2d_group(st, g.variant, g.d_jobs, g.d_cta, g.njobs, g.total, g.maxN);
        k_sum_partials_batch<<<gp, 256, 0, st>>>(p->d_elem_lo, nullptr);
        p->launches += (long long)p->lo_groups.size() + 1;
    }
    for (auto& g : p->groups) launch_fused2d_group(st, g.variant, g.d_jobs, g.d_cta, g.njobs, g.total, g.maxN);
    p->launches += (long long)p->groups.size();
    k_sum_partials_batch<<<gp, 256, 0, st>>>(p->d_elem, p->d_time);
    p->launches++;
    if (!p->lo_groups.empty()) {
        k_add_lo_batch<<<dim3((p->maxNm + kThreads - 1) / kThreads, nj), kThreads, 0, st>>>(p->d_elem);
        p->launches++;
    }
    k_dft_batch<<<gw, kThreads, 0, st>>>(p->d_elem, 2, stage_in);
    p->launches++;
    if (rk == 0) {   // requests project Q: the last pass, the projection, then the RK kernels
        k_dft_batch<<<gw, kThreads, 0, st>>>(p->d_elem, 3, stage_in);
        p->launches++;
        for (bn_solver* s : p->solvers)
            if (s->opt.conserve) {
                cudaStream_t own = s->stream;   // the projection kernel joins the capture on the shared stream
                s->stream = st;
                launch_conserve(s, s->Qv);
                s->stream = own;
            }
        return;
    }
    k_row_inv_rk_fwd<<<dim3(p->maxN, nj), 256, 0, st>>>(p->d_elem, rk, w_acc, c_next, first);
    p->launches++;
}

bn_status build_plan(bn_solver** solvers, int n, const double* dts, bool timed, cudaStream_t st, BatchPlan** out,
                     std::string* err) {
    BatchPlan* p = new BatchPlan();
    p->integrator = solvers[0]->opt.integrator;
    p->timed = timed;
    std::vector<ElemJob> elem;
    std::map<int, std::vector<int>> by_variant;
    for (int i = 0; i < n; ++i) {
        bn_solver* s = solvers[i];
        p->solvers.push_back(s);
        p->dts.push_back(dts[i]);
        ElemJob J{};
        J.N = s->g.N;
        J.nm = s->g.nModes;
        J.f = s->f;
        J.y = s->y;
        J.kacc = s->kacc;
        J.Qv = s->Qv;
        J.cand = s->f_prev;
        J.flags = s->flags;
        J.Ghat = s->Ghat;
        J.Ghat32 = s->opt.precision == BN_MIXED ? s->Ghat32 : nullptr;
        J.work_c = s->work_c;
        J.tw = s->twiddle;
        J.Qhat = s->Qhat;
        J.partials = s->partials;
        J.nPart = std::max(1, std::min(s->eps != 0.0 ? s->work.count : s->work_quad.count, s->n_partials));
        J.part32 = fused2d_partials_f32(s) ? 1 : 0;
        J.Sb = J.part32 && s->eps != 0.0 && s->work.count > 0 ? reinterpret_cast<const float2*>(s->S2) : nullptr;
        J.eps = (float)s->eps;
        J.dt = dts[i];
        J.scale = s->scale;
        J.Qlo = beta_split_on(s) ? s->Qlo : nullptr;
        elem.push_back(J);
        p->maxN = std::max(p->maxN, s->g.N);
        p->maxNm = std::max(p->maxNm, s->g.nModes);
        by_variant[fused2d_variant(s)].push_back(i);
    }
    cudaError_t e = cudaMalloc(&p->d_elem, sizeof(ElemJob) * elem.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_elem, elem.data(), sizeof(ElemJob) * elem.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && timed) {
        const unsigned long long init[4] = {~0ull, 0ull, 0ull, 0ull};
        e = cudaMalloc((void**)&p->d_time, sizeof init);
        if (e == cudaSuccess) e = cudaMemcpy(p->d_time, init, sizeof init, cudaMemcpyHostToDevice);
    }
    for (auto& kv : by_variant) {
        if (e != cudaSuccess) break;
        BatchPlan::Group g;
        g.variant = kv.first;
        const bool mixed = kv.first <= 1 || kv.first == 4;
        // heaviest requests first: their CTAs take the SMs at the start of the launch and the CTAs of
        // light requests (e.g. eps = 0, quadratic part only) fill the tail; a request's CTAs compute
        // the same whatever their position in the grid
        std::stable_sort(kv.second.begin(), kv.second.end(), [&](int x, int y) {
            const bn_solver* a = solvers[x];
            const bn_solver* b = solvers[y];
            const double wa = a->eps != 0.0 ? a->work.terms : (double)a->work_quad.count;
            const double wb = b->eps != 0.0 ? b->work.terms : (double)b->work_quad.count;
            return wa > wb;
        });
        const size_t asz = mixed ? sizeof(FusedArgs<float>) : sizeof(FusedArgs<double>);
        std::vector<unsigned char> args(asz * kv.second.size());
        std::vector<int> cta(1, 0);
        for (size_t k = 0; k < kv.second.size(); ++k) {
            bn_solver* s = solvers[kv.second[k]];
            fill_fused_args(s, args.data() + asz * k);
            if (mixed) reinterpret_cast<FusedArgs<float>*>(args.data() + asz * k)->stamps = p->d_time;
            else reinterpret_cast<FusedArgs<double>*>(args.data() + asz * k)->stamps = p->d_time;
            cta.push_back(cta.back() + elem[kv.second[k]].nPart);
            g.maxN = std::max(g.maxN, s->g.N);
            g.maxCount = std::max(g.maxCount, s->eps != 0.0 ? s->work.count : 0);
        }
        g.njobs = (int)kv.second.size();
        g.total = cta.back();
        e = cudaMalloc(&g.d_jobs, args.size());
        if (e == cudaSuccess) e = cudaMalloc((void**)&g.d_cta, sizeof(int) * cta.size());
        if (e == cudaSuccess) e = cudaMemcpy(g.d_jobs, args.data(), args.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g.d_cta, cta.data(), sizeof(int) * cta.size(), cudaMemcpyHostToDevice);
        p->groups.push_back(g);
        // the residual-table pass of the same jobs that have the kernel-mode rounding correction (same
        // order, same CTAs per job), untimed
        if (!mixed || e != cudaSuccess) continue;
        std::vector<int> lo_jobs;
        for (int j : kv.second)
            if (beta_split_on(solvers[j])) lo_jobs.push_back(j);
        if (lo_jobs.empty()) continue;
        BatchPlan::Group gl;
        gl.variant = kv.first;
        std::vector<unsigned char> largs(sizeof(FusedArgs<float>) * lo_jobs.size());
        std::vector<int> lcta(1, 0);
        for (size_t k = 0; k < lo_jobs.size(); ++k) {
            bn_solver* s = solvers[lo_jobs[k]];
            fill_fused_args_lo(s, largs.data() + sizeof(FusedArgs<float>) * k);
            reinterpret_cast<FusedArgs<float>*>(largs.data() + sizeof(FusedArgs<float>) * k)->stamps = nullptr;
            lcta.push_back(lcta.back() + elem[lo_jobs[k]].nPart);
            gl.maxN = std::max(gl.maxN, s->g.N);
        }
        gl.njobs = (int)lo_jobs.size();
        gl.total = lcta.back();
        e = cudaMalloc(&gl.d_jobs, largs.size());
        if (e == cudaSuccess) e = cudaMalloc((void**)&gl.d_cta, sizeof(int) * lcta.size());
        if (e == cudaSuccess) e = cudaMemcpy(gl.d_jobs, largs.data(), largs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(gl.d_cta, lcta.data(), sizeof(int) * lcta.size(), cudaMemcpyHostToDevice);
        p->lo_groups.push_back(gl);
    }
    if (e == cudaSuccess && !p->lo_groups.empty()) {
        std::vector<ElemJob> lo = elem;
        for (int i = 0; i < n; ++i) {
            bn_solver* s = solvers[i];
            ElemJob& J = lo[i];
            J.Qlo = nullptr;
            if (!beta_split_on(s)) {
                J.Qhat = nullptr;   // no residual-table pass for this job
                continue;
            }
            J.Qhat = s->Qlo;
            J.partials = s->partials_lo;
            if (J.Sb) J.Sb = reinterpret_cast<const float2*>(s->S2lo);
        }
        e = cudaMalloc(&p->d_elem_lo, sizeof(ElemJob) * lo.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->d_elem_lo, lo.data(), sizeof(ElemJob) * lo.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        *err = std::string("batch plan: ") + cudaGetErrorString(e);
        cudaGetLastError();
        destroy_plan(p);
        return e == cudaErrorMemoryAllocation ? BN_ERR_NOMEM : BN_ERR_CUDA;
    }
    // capture one step of every request
    cudaGraph_t graph;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        *err = std::string("batch capture: ") + cudaGetErrorString(e);
        destroy_plan(p);
        return BN_ERR_CUDA;
    }
    const int nj = n;
    const dim3 ge((p->maxNm + kThreads - 1) / kThreads, nj);
    bool fuse_rk = true;   // the projection of Q must run between the transform and the RK update
    for (int i = 0; i < n; ++i)
        if (solvers[i]->opt.conserve) fuse_rk = false;
    if (p->integrator == 0) {
        const double wacc[4] = {1.0, 2.0, 2.0, 1.0}, cnext[3] = {0.5, 0.5, 1.0};
        for (int stage = 0; stage < 4; ++stage) {
            if (fuse_rk) {
                record_batched_eval(p, st, stage == 0 ? 0 : 1, stage < 3 ? 1 : 2, stage < 3 ? wacc[stage] : 0.0,
                                    stage < 3 ? cnext[stage] : 0.0, stage == 0, stage > 0, stage == 0);
                continue;
            }
            record_batched_eval(p, st, stage == 0 ? 0 : 1, 0, 0.0, 0.0, 0, false, stage == 0);
            if (stage < 3) {
                k_rk_stage_batch<<<ge, kThreads, 0, st>>>(p->d_elem, wacc[stage], cnext[stage], stage == 0);
                p->launches++;
            }
        }
        if (!fuse_rk) {
            k_rk_final_batch<<<ge, kThreads, 0, st>>>(p->d_elem);
            p->launches++;
        }
    } else if (fuse_rk) {
        record_batched_eval(p, st, 0, 1, 0.0, 1.0, 1, false, true);
        record_batched_eval(p, st, 1, 3, 0.0, 0.0, 0, true);
    } else {
        record_batched_eval(p, st, 0, 0, 0.0, 0.0, 0, false, true);
        k_rk_stage_batch<<<ge, kThreads, 0, st>>>(p->d_elem, 0.0, 1.0, 1);
        record_batched_eval(p, st, 1);
        k_heun_final_batch<<<ge, kThreads, 0, st>>>(p->d_elem);
        p->launches += 2;
    }
    k_commit_batch<<<ge, kThreads, 0, st>>>(p->d_elem);
    p->launches += 1;
    e = cudaStreamEndCapture(st, &graph);
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&p->graph, graph, 0);
        cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) {
        *err = std::string("batch graph: ") + cudaGetErrorString(e);
        cudaGetLastError();
        destroy_plan(p);
        return BN_ERR_CUDA;
    }
    *out = p;
    return BN_OK;
}

bool plan_matches(const BatchPlan* p, bn_solver** solvers, int n, const double* dts, bool timed) {
    if (!p || (int)p->solvers.size() != n || p->timed != timed) return false;
    for (int i = 0; i < n; ++i)
        if (p->solvers[i] != solvers[i] || p->dts[i] != dts[i]) return false;
    return true;
}

bn_status replay_plan(BatchPlan* p, cudaStream_t st, int nsteps) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(p->graph, st);
    if (e != cudaSuccess) return BN_ERR_CUDA;
    for (bn_solver* s : p->solvers) s->launches += p->launches * nsteps / (long long)p->solvers.size();
    return BN_OK;
}

long long plan_launches(const BatchPlan* p) { return p ? p->launches : 0; }

bool plan_read_spans(BatchPlan* p, cudaStream_t st, double* ns_total, long long* count) {
    *ns_total = 0;
    *count = 0;
    if (!p || !p->d_time) return false;
    unsigned long long h[4];
    if (cudaMemcpyAsync(h, p->d_time, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return false;
    if (cudaMemsetAsync(p->d_time + 2, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(st) != cudaSuccess) return false;
    *ns_total = (double)h[2];
    *count = (long long)h[3];
    return true;
}

bool plan_contains(const BatchPlan* p, const bn_solver* s) {
    return p && std::find(p->solvers.begin(), p->solvers.end(), s) != p->solvers.end();
}

}  // namespace bn
