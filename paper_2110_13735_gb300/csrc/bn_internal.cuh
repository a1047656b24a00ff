// bn_internal.cuh -- declarations shared by the translation units of libbn.
// Fourier-Galerkin Boltzmann-Nordheim operator (Mouton & Rey, arXiv:2110.13735).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bn.h"

namespace bn {

// ---------------------------------------------------------------- complex helpers
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im) {
    C c; c.x = re; c.y = im; return c;
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- index geometry
// Modes k in I_N = [-N/2, N/2-1]^d are stored row-major at k_i + N/2 (last fastest).
// Kernel-mode arguments a in the extended box [-N, N-1]^d are stored at a_i + N.
struct Geometry {
    int d = 2;
    int N = 16;
    int nModes = 0;   // N^d
    int E = 0;        // 2N
    int nExt = 0;     // (2N)^d
};

// ---------------------------------------------------------------- shared tables
// Kernel modes beta(a,b) for one (d, N, R_xi, kernel, quadrature).
struct KernelTables {
    std::string key;
    int refcount = 0;
    Geometry g;
    int P = 0;                    // quadrature terms
    double* alpha64 = nullptr;    // [P][nExt]  (weights folded in)
    double* alphap64 = nullptr;   // [P][nExt]
    double* beta64 = nullptr;     // [nExt(b)][nExt(a)] = beta(a, b)  (b-major)
    float* beta32 = nullptr;      // same, rounded to FP32
    float* beta32T = nullptr;     // 2-D N <= 32: [b][a2][a1] (the FP32 table with the two a axes swapped)
    double* sw64 = nullptr;       // 2-D: [b (ext)][s in I_N] = beta(s,b-s) - beta(b,s) - beta(s,b) (0 off box_s(b))
    float* sw32 = nullptr;
    float* dq32 = nullptr;        // 2-D: [b in I_N][a (ext)] = beta(a, b) - beta(b, b), formed in FP64, rounded once
    // 2-D: the rounding residuals of the four FP32 tables, x - fl32(x) rounded to FP32 (x the FP64
    // value), laid out as their FP32 tables: the second pass of the kernel-mode rounding correction
    float* beta32lo = nullptr;
    float* beta32Tlo = nullptr;
    float* sw32lo = nullptr;
    float* dq32lo = nullptr;
    float* alpha32 = nullptr;     // FP32 copies of alpha64 / alphap64 ([P][nExt])
    float* alphap32 = nullptr;
    double* alphaI64 = nullptr;   // alpha, alpha' restricted to a in I_N ([P][N^d]), FP64 and FP32
    double* alphapI64 = nullptr;
    float* alphaI32 = nullptr;
    float* alphapI32 = nullptr;
    size_t bytes = 0;
};

// ---------------------------------------------------------------- fused 2-D operator arguments
// One request of the fused 2-D kernel (bn_fused2d.cu).
template <typename Real>
struct FusedArgs {
    int N;
    double eps;              // 0: quadratic part only
    const cplx<Real>* G;     // modes (N^2)
    const Real* beta;        // [b][a] kernel-mode table
    const int* items;        // b (flat extended index), descending work
    int count;
    double2* partials;       // [gridDim.x][N^2]
    int* err;                // [0] set to 1 if a bounded wait gave up
    int giveup_first;        // testing: 1 = the first bounded wait gives up at once (0 = the normal wait)
    unsigned long long* stamps;  // optional [2]: min start / max end %globaltimer (ns) over CTAs
    const Real* sw;          // [b][s in I_N] reducible weights beta(s,b-s) - beta(b,s) - beta(s,b)
    void* Sb;                // mixed N <= 32: [b] S(b) (float2), written by the operator kernel
    const void* meta;        // mixed N <= 32: ItemMeta per item (same order as items)
    const float* dq;         // mixed N <= 32: quadratic weights beta(a, b) - beta(b, b), [b in I_N][a]
    const float* betaT;      // mixed N <= 32: [b][a2][a1]
};

// Fixed-order sum of the FP32 (sum, compensation) partials of the mixed 2-D kernel into Q^: a
// block of 256 threads owns the kPartModes modes [kPartModes bx, kPartModes (bx + 1)); each of its
// 256 / kPartModes thread groups adds the partials c = w, w + groups, ... with FP32 compensated
// (Kahan) summation, and the group results meet in a fixed FP64 tree (deterministic).
constexpr int kPartModes = 4;
// Packed FP32 pairs (sm_100 family): a 64-bit register holding two floats, and the paired FMA
// fma.rn.f32x2, which rounds each half exactly as fmaf does and issues once for both.
__device__ __forceinline__ uint64_t dup2(float x) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ void split2(uint64_t v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t pack2(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void kahan_add_f(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}
// With Sb (mixed 2-D, eps != 0) the reducible part eps sum_b G^_{n-b} S(b) is added as well: S(b) for
// every b with a non-empty box_s (b_d <= N - 2) was written by the operator kernel, G32 = G^ in FP32.
__device__ __forceinline__ void sum_partials_f32_block(int nm, int nPart, const float4* __restrict__ partials,
                                                       double2* __restrict__ out, int bx, int N = 0,
                                                       const float2* __restrict__ G32 = nullptr,
                                                       const float2* __restrict__ Sb = nullptr, float eps = 0.f) {
    constexpr int G = 256 / kPartModes;
    __shared__ double2 sh[256];
    const int m = threadIdx.x % kPartModes, w = threadIdx.x / kPartModes;
    const int i = bx * kPartModes + m;
    float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
    if (i < nm) {
        int c = w;
        for (; c + 3 * G < nPart; c += 4 * G) {   // four loads in flight, added in order
            float4 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = partials[(size_t)(c + q * G) * nm + i];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                kahan_add_f(sx, cx, v[q].x);
                kahan_add_f(sx, cx, -v[q].z);
                kahan_add_f(sy, cy, v[q].y);
                kahan_add_f(sy, cy, -v[q].w);
            }
        }
        for (; c < nPart; c += G) {
            const float4 v = partials[(size_t)c * nm + i];
            kahan_add_f(sx, cx, v.x);
            kahan_add_f(sx, cx, -v.z);
            kahan_add_f(sy, cy, v.y);
            kahan_add_f(sy, cy, -v.w);
        }
        if (Sb) {
            // eps sum over k in I_N of G^_k S(n - k), k = w, w + G, ...: eight terms' loads in flight,
            // then added in order; terms with an empty box_s(b) (b_d = N - 1: S(b) = 0) are skipped
            const int h = N / 2, E = 2 * N, n1 = i / N - h, n2 = i % N - h;
            for (int kf = w; kf < nm; kf += 8 * G) {
                float2 g[8], sb[8];
                bool ok[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = kf + q * G, b1 = n1 - (k / N - h), b2 = n2 - (k % N - h);
                    ok[q] = k < nm && b1 <= N - 2 && b2 <= N - 2;
                    g[q] = ok[q] ? G32[k] : make_float2(0.f, 0.f);
                    sb[q] = ok[q] ? Sb[(b1 + N) * E + (b2 + N)] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (ok[q]) {
                        kahan_add_f(sx, cx, eps * fmaf(g[q].x, sb[q].x, -g[q].y * sb[q].y));
                        kahan_add_f(sy, cy, eps * fmaf(g[q].x, sb[q].y, g[q].y * sb[q].x));
                    }
            }
        }
    }
    sh[threadIdx.x] = make_double2((double)sx - (double)cx, (double)sy - (double)cy);
    __syncthreads();
    for (int st = G / 2; st >= 1; st >>= 1) {
        if (w < st) {
            const double2 a = sh[threadIdx.x], b = sh[threadIdx.x + st * kPartModes];
            sh[threadIdx.x] = make_double2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
    }
    if (w == 0 && i < nm) out[i] = sh[m];
}

struct BatchPlan;
struct NdPlan;

// ---------------------------------------------------------------- triple-sum work list
// Geometry of one b of the 2-D mixed kernel, derived once on the host (64 bytes).  The sweep runs
// its register window along dimension w and splits dimension u (orient 0: u = 1, w = 2; orient 1:
// u = 2, w = 1, chosen per b for the better warp mapping).  Outputs n in box_n(b) = [nlo, nlo + L),
// inner s in box_s(b) = [slo, slo + S) per dimension; the beta rectangle a = n - s is staged as rows
// [a_ulo, a_ulo + Au) x columns [a_wlo, a_wlo + Aw) (one spare column on the left); Gg groups of RW
// outputs along w; the warp split: J chunks of the s_u range (chunk rows each), tpw = 32 / J tasks
// per warp unit (lanes >= J tpw idle), `units` warp units covering base = L_u Gg tasks, numbered with
// the group fastest (orient 0) or the row fastest (orient 1) so that the lanes of a warp touch
// distinct shared-memory banks; ginv = ceil(2^16 / Gg), linv = ceil(2^16 / L_u) (division by
// multiply-shift).
struct ItemMeta {
    int ib, ginv, linv;
    short orient, b1, b2, nlo_u, nlo_w, Lu, Lw, slo_u, Su, slo_w, Sw, Gg, Au, Aw, a_ulo, a_wlo, quad, J, tpw, chunk,
        units, base;
    // the last, partial round of units may use a finer split: units2 units of 32/J2 tasks x J2
    // chunks (of chunk2 rows) covering the tasks [tail0, base); units then counts full rounds only
    short J2, chunk2, units2, tail0;
};
static_assert(sizeof(ItemMeta) == 64, "ItemMeta is 64 bytes");

struct WorkList {
    int* items = nullptr;   // flat extended index of b, sorted by descending work
    int count = 0;
    double terms = 0;       // sum over items of |box_n| |box_s|
    // 2-D: per item (same order) for the mixed kernel: RW = 8, 8 with the per-b orientation choice,
    // 16, 16 with orientation
    ItemMeta* meta[4] = {nullptr, nullptr, nullptr, nullptr};
};

// The warp split of one b for a CTA of `warps` warps: J in {1, 2, 4, 8} chunks of the S_u rows,
// tpw = 32 / J tasks per warp unit, units dealt to the warps round-robin.  When the unit count is
// not a multiple of `warps`, the tasks of the last round may be re-split with J2 in {J .. 32}
// chunks, so that its work spreads over more warps instead of leaving most of them idle at the
// barrier that ends the b.  Minimises the issue cost of the busiest warp: per round, chunk rows x
// (Sw steps x kStepInstr + kRowInstr) + kUnitInstr (+ kStageInstr per butterfly stage when the
// chunks outnumber the RW outputs of a task), instruction counts per lane of one sweep step (8
// paired FMA + 2 shared loads + the window duplication), of the per-row work (window load, loop
// tail) and of the per-unit work (task decode, reduce-scatter, epilogue); the overheads were
// calibrated by timing the kernel at N = 32.  Returns that cost.
constexpr int kStepInstr = 18, kRowInstr = 150, kUnitInstr = 400, kStageInstr = 20;
struct SplitChoice {
    int J, chunk, units, J2, chunk2, units2, tail0;
};
inline int unit_cost_host(int J, int Su, int Sw, int RW) {
    int c = ((Su + J - 1) / J) * (Sw * kStepInstr + kRowInstr) + kUnitInstr;
    for (int j = RW; j < J; j <<= 1) c += kStageInstr;
    return c;
}
inline int choose_split_host(int base, int Su, int Sw, int RW, int warps, SplitChoice* out) {
    int best = 0x7fffffff;
    for (int j = 1; j <= 8; j <<= 1) {
        const int tpw = 32 / j;
        const int u = (base + tpw - 1) / tpw;
        const int tj = unit_cost_host(j, Su, Sw, RW);
        const int full = u / warps;
        SplitChoice c{j, (Su + j - 1) / j, u, j, (Su + j - 1) / j, 0, 0};
        int cost = ((u + warps - 1) / warps) * tj;
        if (u % warps != 0 && full > 0) {
            // re-split the tasks of the last round
            const int tail0 = full * warps * tpw, T = base - tail0;
            for (int j2 = 2 * j; j2 <= 32; j2 <<= 1) {
                const int u2 = (T + 32 / j2 - 1) / (32 / j2);
                const int c2 = full * tj + ((u2 + warps - 1) / warps) * unit_cost_host(j2, Su, Sw, RW);
                if (c2 < cost) {
                    cost = c2;
                    c = SplitChoice{j, (Su + j - 1) / j, full * warps, j2, (Su + j2 - 1) / j2, u2, tail0};
                }
            }
        }
        if (cost < best) {
            best = cost;
            *out = c;
        }
    }
    return best;
}

}  // namespace bn

// ---------------------------------------------------------------- solver object
struct bn_solver {
    bn::Geometry g;
    double T = 0, R = 0, Rxi = 0, eps = 0;
    int kernel = 0;
    bn_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    double scale = 1.0;          // (T/pi)^{d+gamma}
    bn::KernelTables* tabs = nullptr;
    bn::NdPlan* nd = nullptr;    // 3-D and CIRCULAR operator path (bn_opnd.cu)
    bn::WorkList work;           // b with non-empty triple-sum boxes (eps != 0)
    bn::WorkList work_quad;      // b in I_N (quadratic part only, eps == 0)
    int n_partials = 0;          // CTAs of the triple-sum kernel (rows of the partial buffer)
    int mixed_rw = 8;            // outputs per thread of the mixed 2-D kernel (N <= 32)
    int mixed_v = 0;             // its metadata variant (index into work.meta)
    float tune_ms[4] = {0, 0, 0, 0};   // autotuner timings of the four variants (0 = not timed)

    // device buffers
    double* f = nullptr;         // state, N^d
    double* f_prev = nullptr;    // last finite state
    double* y = nullptr;         // RK stage argument
    double* kacc = nullptr;      // RK accumulator
    double* Qv = nullptr;        // Q in velocity units (stage derivative)
    double2* Ghat = nullptr;     // modes of the stage argument (FP64)
    float2* Ghat32 = nullptr;    // same in FP32 (mixed precision)
    double2* work_c = nullptr;   // transform scratch, N^d
    double2* twiddle = nullptr;  // e^{-2 i pi m / N}, m = 0..N-1
    double2* S2 = nullptr;       // reducible pair sums S(t), t in ext box
    double2* quad = nullptr;     // quadratic modes, N^d
    double2* red = nullptr;      // reducible cubic modes, N^d
    double2* q1q = nullptr;      // Q_{1,q} modes, N^d
    double2* partials = nullptr; // [n_partials][N^d]
    double2* Qhat = nullptr;     // combined modes
    // kernel-mode rounding correction (opt.beta_split, mixed 2-D): the residual-table pass's own
    // partials and S(b) sums, and its modes, added to Q^ by every evaluation
    double2* partials_lo = nullptr;
    double2* S2lo = nullptr;
    double2* Qlo = nullptr;
    bool lo_refresh = true;      // recompute Qlo in the next evaluation (cleared for RK stages 2..4)
    // velocity rescaling (bn_rescale_set, bn_step_rescaled): the state is G on the grid of [-pi, pi]^d;
    // L the velocity box of scale 1, w the velocity scale, u the mean velocity, rho, e, T, z the
    // moments, temperature and fugacity; scratch for the divergence term and the moments of Q
    bool resc = false;
    double resc_L = 0, resc_w = 1, resc_u[3] = {0, 0, 0}, resc_rho = 0, resc_e = 0, resc_T = 0, resc_z = 0;
    double* resc_H = nullptr;
    double2* resc_M = nullptr;
    double2* resc_acc = nullptr;
    double* resc_div = nullptr;
    double* resc_mom = nullptr;       // device [5]
    double* resc_mom_host = nullptr;  // pinned [5]
    double* resc_G0 = nullptr;        // G at the start of an RK2 step (bn_step_rescaled_rk2)
    double* moments = nullptr;   // d+6
    int* flags = nullptr;        // [0] non-finite, [1] committed steps, [2] wait timeout, [4..5] max f (u64 bits)
    int* flags_host = nullptr;   // pinned copy of the 8 flag words
    double t_escalated = -1;     // time of the switch to FP64 (escalate_at), -1 if none
    double last_max_f = 0;

    bool has_state = false;
    double t = 0;
    long long launches = 0;

    // captured step graphs
    cudaGraphExec_t step_graph = nullptr;
    double graph_dt = 0;
    long long graph_launches = 0;  // kernels in one captured step

    // live timing of the triple-sum kernel
    bool prof = false;
    cudaEvent_t prof_ev[16] = {};   // pairs (start, stop) per evaluation slot
    int prof_slot = 0;              // next slot while recording
    int prof_slots_used = 0;        // slots recorded by the current graph / last eval
    double prof_ms = 0;
    long long prof_count = 0;
    unsigned long long* prof_stamps = nullptr;  // device [16]: per slot (start, end) %globaltimer
    double prof_ns_total = 0;                   // kernel-span time from the device stamps
    long long prof_ns_count = 0;
};

namespace bn {

// tables (bn_tables.cu)
bn_status acquire_tables(bn_solver* s, std::string* err);
void release_tables(KernelTables* t);
bn_status build_work_list(bn_solver* s, std::string* err);
bn_status balance_work_lists(bn_solver* s, std::string* err);   // after n_partials is set
constexpr int kPlanCols = 14;   // columns of a bn_plan_mixed2d row
std::vector<int> plan_mixed2d_rows(int N, int rw, bool oriented, int nblk);
double count_triple_terms(int d, int N);
double count_pair_terms(int d, int N);
double count_reducible_terms(int d, int N);

// transforms and stage kernels (bn_transform.cu)
void launch_dft_forward(bn_solver* s, const double* f, double2* out);
void launch_dft_inverse_real(bn_solver* s, const double2* in, double* out, double scale);
void launch_to_fp32(bn_solver* s, const double2* in, float2* out, int n);
void launch_rk_stage(bn_solver* s, const double* f, const double* K, double* acc, double* y, double w_acc,
                     double c_next, double dt, int first);
void launch_rk_final(bn_solver* s, double* f, const double* acc, const double* K, double w_last, double dt,
                     double* f_prev, int* flags);
void launch_heun_final(bn_solver* s, double* f, const double* y, const double* K, double dt, double* f_prev,
                       int* flags);
void launch_moments(bn_solver* s, const double* f, double* out);
void launch_conserve(bn_solver* s, double* Q);
void launch_conserve_on(const bn_solver* s, double* Q, cudaStream_t st);
void dft2_forward_into(const bn_solver* s, cudaStream_t st, const double* f, double2* work, double2* out, float2* out32);
void dft2_inverse_real_into(const bn_solver* s, cudaStream_t st, const double2* in, double2* work, double* out);

// 3-D and CIRCULAR operator (bn_opnd.cu)
bool use_nd(const bn_solver* s);
std::vector<int> shard_bounds_for(int d, int N, int wrap, int count);   // host only
bn_status plan_nd(bn_solver* s, std::string* err);
bn_status build_nd_tables(bn_solver* s, KernelTables* t, std::string* err);
bn_status prepare_nd(bn_solver* s);
void launch_nd(bn_solver* s, int slot);   // slot: live phase-timing slot, -1 = none
bn_status nd_profile_enable(bn_solver* s, bool on);
void nd_profile_harvest(bn_solver* s, int slots);
bn_status nd_profile_read(bn_solver* s, double* out, size_t count);
void free_nd(bn_solver* s);
double nd_triple_terms(const bn_solver* s);
int nd_rounds(const bn_solver* s);
int nd_ctas(const bn_solver* s);
size_t nd_slice_bytes(const bn_solver* s);

// CTAs of the 2-D fused operator launch (bn_sums.cu)
int triple_partials(const bn_solver* s);

// batched stepping of 2-D solvers (bn_batch.cu)
// mixed-precision 2-D kernel for N <= 32 (bn_fused2d_mixed.cu)
// rw = outputs per thread (8 or 16)
size_t mixed2d_smem(int N, int rw);
void configure_mixed2d();
int mixed2d_ctas_per_sm(int N, int rw);
void launch_mixed2d_kernel(const FusedArgs<float>& A, int grid, int rw, cudaStream_t st);
int launch_mixed2d(const FusedArgs<float>& A, int grid, int rw, double2* Qhat, cudaStream_t st);   // returns launches
void launch_mixed2d_group(cudaStream_t st, int rw, const void* d_jobs, const int* d_cta, int njobs, int total,
                          int maxN);
// Chooses the outputs per thread of the mixed 2-D kernel for this solver (option, cache, or timing
// both candidates on the solver's stream) and sets s->mixed_rw and s->n_partials.
bn_status tune_mixed2d(bn_solver* s, std::string* err);
// true when the fused partials of this solver are FP32 (sum, compensation) pairs
bool fused2d_partials_f32(const bn_solver* s);

bn_status build_plan(bn_solver** solvers, int n, const double* dts, bool timed, cudaStream_t st, BatchPlan** out,
                     std::string* err);
void destroy_plan(BatchPlan* p);
bool plan_matches(const BatchPlan* p, bn_solver** solvers, int n, const double* dts, bool timed);
// Summed fused-kernel spans (ns) and their count since the last read of a timed plan; resets them.
bool plan_read_spans(BatchPlan* p, cudaStream_t st, double* ns_total, long long* count);
bn_status replay_plan(BatchPlan* p, cudaStream_t st, int nsteps);
long long plan_launches(const BatchPlan* p);
bool plan_contains(const BatchPlan* p, const bn_solver* s);

// error message reported by bn_last_error() for the calling thread (bn_api.cu)
void set_last_error(const std::string& msg);

// fused 2-D operator (bn_fused2d.cu)
void configure_fused2d();
size_t fused2d_smem(int N, int precision);
void launch_fused2d(bn_solver* s);   // s->Qhat from s->Ghat / s->Ghat32
bool beta_split_on(const bn_solver* s);   // the kernel-mode rounding correction applies to this solver
// the fused-kernel arguments of the residual-table pass (tables, partials and S(b) buffers swapped)
void fill_fused_args_lo(const bn_solver* s, void* out);
void launch_add_modes(int nm, double2* Q, const double2* add, cudaStream_t st);   // Q += add
// velocity rescaling (bn_rescale.cu)
bn_status rescale_temperature(int d, double eps, double rho, double e, double* T, double* z, std::string* err);
void launch_resc_moments(bn_solver* s, const double* Q, double* out_dev);
void launch_resc_advance(bn_solver* s, double* G, const double* Q, double a, const double* b, double dt, double qc,
                         double* H, double2* M, double2* acc, double* div);
// G = (G0 + G) / 2 (the last stage of the RK2 rescaled step)
void launch_resc_average(bn_solver* s, double* G, const double* G0);

// batched launches (bn_fused2d.cu): variant 0 = mixed N <= 32, 1 = mixed N = 64,
// 2 = FP64 N <= 32, 3 = FP64 N = 64
int fused2d_variant(const bn_solver* s);
int fused2d_partials(const bn_solver* s);   // CTAs (partial sums) of the solver's fused launch
// sb: scratch of nExt float2 for S(b) (mixed N <= 32; may alias nothing else)
void fused2d_into(const bn_solver* s, cudaStream_t st, const void* G, double2* partials, double2* Qhat, int* err,
                  void* sb, bool lo = false);   // lo: the residual-table pass
void fill_fused_args(const bn_solver* s, void* out);   // FusedArgs<float> or <double> by precision
size_t fused2d_variant_smem(int variant, int N);
void launch_fused2d_group(cudaStream_t st, int variant, const void* d_jobs, const int* d_cta, int njobs, int total,
                          int maxN);

}  // namespace bn

#define BN_CUDA_LAUNCH_CHECK() ((void)0)
