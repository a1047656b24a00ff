// bn_fused2d.cu -- the whole 2-D Fourier-Galerkin operator (Mouton & Rey, Lemma of
// Sec. 2.3 combined as in Sec. 3.3 step 2(c)) in one pass over b on CUDA cores.
//
// Every term of Q^_n carries the factor G^_{n-b} for one b:
//   quadratic   k+l = n:    [beta(k,l) - beta(l,l)] G^_k G^_l           with b = l, k = n-b
//   reducible   Q2q-Q3q-Q4q: G^_k S(b),  S(b) = sum_s [beta(s,b-s) - beta(b,s) - beta(s,b)] G^_s G^_{b-s}
//   Q_{1,q}     a = n-s:    G^_{n-b} sum_s beta(n-s, b) G^_s G^_{b-s}   (b = l+m, s = l)
// so Q^_n = sum_b G^_{n-b} D_b(n) with
//   D_b(n) = eps [C_b(n) + S(b)] + [b in I_N] (beta(n-b, b) - beta(b,b)) G^_b,
//   C_b(n) = sum_{s in box_s(b)} beta(n-s, b) P_b(s),   P_b(s) = G^_s G^_{b-s},
// over n in box_n(b) = {n : n, n-b in I_N}, box_s(b) = {s : s, b-s in I_N}.
//
// One CTA walks a static share of the b values (descending work).  For each b it
// stages the kernel-mode slice beta(., b) (the rectangle a in box_n - box_s) in shared
// memory with a padded row stride, forms P_b, reduces S(b), and computes C_b with each
// thread owning RW consecutive outputs along n_2: along the inner loop over s_2 the
// weights beta(n-s, b) form a sliding register window, so each step costs one shared
// load of beta, one broadcast load of P_b and RW complex-by-real multiply-adds.  The
// s_1 range is split over threads when the box is small; partial sums are combined in a
// fixed order.  G^_{n-b} D_b(n) is accumulated in FP64 in shared memory (one owner per
// output per b) and each CTA writes its partial Q^ once; a second kernel sums the
// partials in a fixed order (deterministic results).
#include <cmath>
#include <cstdint>

#include "bn_internal.cuh"

namespace bn {

namespace {

// ------------------------------------------------------------------ bulk copy (TMA) helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared completing on an mbarrier (size and addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after `limit` polls and reports false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr uint32_t kWaitLimit = 1u << 22;

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
    unsigned long long* stamps;  // optional [2]: min start / max end %globaltimer (ns) over CTAs
    const Real* sw;          // [b][s in I_N] reducible weights beta(s,b-s) - beta(b,s) - beta(s,b)
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double2 cfma_d(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    return acc;
}

template <typename Real>
__device__ __forceinline__ double2 to_d2(cplx<Real> c) { return make_double2((double)c.x, (double)c.y); }

// Per-output accumulator of G^_{n-b} D_b(n) over b in shared memory: FP64 in FP64 mode;
// in mixed mode an FP32 Kahan pair (sum, compensation), so that no FP64 arithmetic (1/64
// of the FP32 rate on GB300) runs per (n, b).
template <typename Real> struct Acc;
template <> struct Acc<double> {
    static constexpr bool kComp = false;
    static __device__ __forceinline__ void add(double2* s, double2*, double2 x) { s->x += x.x; s->y += x.y; }
};
template <> struct Acc<float> {
    static constexpr bool kComp = true;
    static __device__ __forceinline__ void kahan(float& s, float& c, float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    static __device__ __forceinline__ void add(float2* s, float2* c, float2 x) {
        kahan(s->x, c->x, x.x);
        kahan(s->y, c->y, x.y);
    }
};

// Shared-memory layout (bytes) for a given N, thread count and staging choice.
template <typename Real, int RW, bool STAGE>
struct Layout2D {
    // padded row stride of the staged beta rectangle: >= RW ceil(N/RW) + N columns and
    // congruent to 1 mod 32, so lanes on 8 consecutive rows x 4 groups of RW columns hit
    // 32 distinct banks
    static __host__ __device__ int stride(int N) {
        const int w = RW * ((N + RW - 1) / RW) + N;
        return 32 * ((w - 1 + 31) / 32) + 1;
    }
    static __host__ __device__ size_t region(int N, int nt) {   // beta rectangle, reused for split sums
        const size_t bs = STAGE ? (size_t)(2 * N) * stride(N) * sizeof(Real) : 0;
        const size_t cp = (size_t)nt * RW * sizeof(cplx<Real>);
        return ((bs > cp ? bs : cp) + 15) / 16 * 16;
    }
    static __host__ __device__ size_t bytes(int N, int nt) {
        const size_t nm = (size_t)N * N;
        size_t b = nm * sizeof(cplx<Real>) * (Acc<Real>::kComp ? 2 : 1);   // Q accumulator (+ compensation)
        b += 2 * nm * sizeof(cplx<Real>);                                    // Gs, Pb
        b += region(N, nt);                                                  // beta rectangle / split sums
        b += 64 * sizeof(double2);                                           // S(b) warp partials
        b += 16;                                                             // mbarrier
        return b;
    }
};

// Lane -> (row, group) of the tasks of one b, row-major: with Gg = 4 a warp covers 8 rows x 4
// groups of RW columns, i.e. 32 distinct banks for the padded stride; Gg = 2, 3 give at most
// 2-way conflicts on the beta loads.
__device__ __forceinline__ void task_rc(int rem, int Gg, int& i, int& g) {
    i = rem / Gg;
    g = rem % Gg;
}
__device__ __forceinline__ int rc_task(int i, int g, int Gg) { return i * Gg + g; }

// One s_1 row of the Toeplitz product: ar/ai[r] += sum_{s2} beta(c0 + r - s2) P(s2), with the
// weights held in a register window whose slots rotate (slot of offset x is x mod RW), so that
// every step costs one load of beta, one load of P and 2 RW FMA, with no register moves.
template <typename Real, int RW, typename LoadB>
__device__ __forceinline__ void row_sweep(LoadB ldb, int c0, const cplx<Real>* __restrict__ prow, int S2,
                                          Real (&ar)[RW], Real (&ai)[RW]) {
    Real w[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) w[r] = ldb(c0 + r);
    int sl = 0;
    for (; sl + RW <= S2; sl += RW) {
#pragma unroll
        for (int k = 0; k < RW; ++k) {
            if (k == 0) {
                if (sl > 0) w[0] = ldb(c0 - sl);
            } else {
                w[RW - k] = ldb(c0 - sl - k);
            }
            const cplx<Real> p = prow[sl + k];
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const Real wr = w[(r - k + RW) % RW];
                ar[r] = fma(wr, p.x, ar[r]);
                ai[r] = fma(wr, p.y, ai[r]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < RW; ++k) {
        if (sl + k >= S2) break;
        if (k == 0) {
            if (sl > 0) w[0] = ldb(c0 - sl);
        } else {
            w[RW - k] = ldb(c0 - sl - k);
        }
        const cplx<Real> p = prow[sl + k];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const Real wr = w[(r - k + RW) % RW];
            ar[r] = fma(wr, p.x, ar[r]);
            ai[r] = fma(wr, p.y, ai[r]);
        }
    }
}

template <typename Real, int RW, int NT, bool STAGE>
__global__ void __launch_bounds__(NT) k_fused2d(FusedArgs<Real> A) {
    using C = cplx<Real>;
    using AC = Acc<Real>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = A.N, E = 2 * N, nExt = E * E, nm = N * N;
    const int WS = Layout2D<Real, RW, STAGE>::stride(N);
    C* Qs = reinterpret_cast<C*>(smem_raw);
    C* Qc = Qs + (AC::kComp ? nm : 0);
    C* Gs = Qc + nm;
    C* Pb = Gs + nm;
    unsigned char* region = reinterpret_cast<unsigned char*>(Pb + nm);
    Real* Bs = reinterpret_cast<Real*>(region);
    C* Cpart = reinterpret_cast<C*>(region);   // reused after the sweep (split sums)
    double2* Sred = reinterpret_cast<double2*>(region + Layout2D<Real, RW, STAGE>::region(N, NT));
    uint64_t* bar = reinterpret_cast<uint64_t*>(Sred + 64);
    const int tid = threadIdx.x;
    const bool cubic = A.eps != 0.0;
    const Real eps_r = (Real)A.eps;
    if (A.stamps && tid == 0) atomicMin(&A.stamps[0], global_ns());

    // G^ -> shared memory with one bulk copy (TMA engine), overlapped with zeroing the accumulator.
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, (uint32_t)(nm * sizeof(C)));
        bulk_g2s(Gs, A.G, (uint32_t)(nm * sizeof(C)), bar);
    }
    for (int i = tid; i < nm; i += NT) {
        Qs[i] = cmake<C>(0.0, 0.0);
        if (AC::kComp) Qc[i] = cmake<C>(0.0, 0.0);
    }
    __syncthreads();
    if (!mbar_wait_bounded(bar, 0, kWaitLimit)) {
        // the copy did not complete in time: record it, wait (bounded) once more for the
        // copy in flight, and give up
        atomicOr(A.err, 1);
        mbar_wait_bounded(bar, 0, kWaitLimit);
        return;
    }

    for (int item = blockIdx.x; item < A.count; item += gridDim.x) {
        const int ib = A.items[item];
        const int b1 = ib / E - N, b2 = ib % E - N;
        const int nlo1 = max(-N / 2, b1 - N / 2), L1 = min(N / 2 - 1, b1 + N / 2 - 1) - nlo1 + 1;
        const int nlo2 = max(-N / 2, b2 - N / 2), L2 = min(N / 2 - 1, b2 + N / 2 - 1) - nlo2 + 1;
        const int slo1 = max(-N / 2, b1 - N / 2 + 1), S1 = min(N / 2 - 1, b1 + N / 2) - slo1 + 1;
        const int slo2 = max(-N / 2, b2 - N / 2 + 1), S2 = min(N / 2 - 1, b2 + N / 2) - slo2 + 1;
        const bool quad = b1 >= -N / 2 && b1 < N / 2 && b2 >= -N / 2 && b2 < N / 2;
        const int Gg = (L2 + RW - 1) / RW;
        const Real* __restrict__ bsl = A.beta + (size_t)ib * nExt;   // beta(., b), [a1][a2]
        const C gb = quad ? Gs[(b1 + N / 2) * N + (b2 + N / 2)] : cmake<C>(0.0, 0.0);
        const Real wbb = quad ? __ldg(bsl + (b1 + N) * E + (b2 + N)) : Real(0);

        // D_b(n) = eps (C + S) + quadratic term; Qacc[n] += G^_{n-b} D
        auto epilogue = [&](int n1, int n2, Real cx, Real cy, Real Sx, Real Sy) {
            C D = cmake<C>(eps_r * (cx + Sx), eps_r * (cy + Sy));
            if (quad) {
                const Real wq = __ldg(bsl + (n1 - b1 + N) * E + (n2 - b2 + N)) - wbb;
                D.x = fma(wq, gb.x, D.x);
                D.y = fma(wq, gb.y, D.y);
            }
            const int on = (n1 + N / 2) * N + (n2 + N / 2);
            const C gk = Gs[(n1 - b1 + N / 2) * N + (n2 - b2 + N / 2)];
            AC::add(Qs + on, Qc + on, cmul(gk, D));
        };

        // staged beta rectangle: a1 in [a1lo, a1lo + A1), a2 in [a2lo, a2lo + A2)
        const int A1 = L1 + S1 - 1, a1lo = nlo1 - slo1 - S1 + 1;
        const int A2 = RW * Gg + S2, a2lo = nlo2 - slo2 - S2;   // one spare column on the left
        __syncthreads();   // readers of the previous item are done
        if (cubic) {
            if (STAGE) {
                for (int q = tid; q < A1 * A2; q += NT) {
                    const int r = q / A2, c = q % A2;
                    const int a1 = a1lo + r, a2 = a2lo + c;
                    Real v = 0;
                    if (a2 >= -N && a2 < N) v = __ldg(bsl + (a1 + N) * E + (a2 + N));
                    Bs[r * WS + c] = v;
                }
            }
            for (int q = tid; q < S1 * S2; q += NT) {
                const int s1 = slo1 + q / S2, s2 = slo2 + q % S2;
                const C x = Gs[(s1 + N / 2) * N + (s2 + N / 2)];
                const C y = Gs[(b1 - s1 + N / 2) * N + (b2 - s2 + N / 2)];
                Pb[q] = cmul(x, y);
            }
            __syncthreads();
            // S(b) = sum over box_s of W(b, s) P_b(s), W(b, s) = beta(s, b-s) - beta(b, s) - beta(s, b)
            Real sr = 0, si = 0;
            const Real* __restrict__ wrow = A.sw + (size_t)ib * nm;
            for (int q = tid; q < S1 * S2; q += NT) {
                const int s1 = slo1 + q / S2, s2 = slo2 + q % S2;
                const Real w = __ldg(wrow + (s1 + N / 2) * N + (s2 + N / 2));
                const C p = Pb[q];
                sr = fma(w, p.x, sr);
                si = fma(w, p.y, si);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if ((tid & 31) == 0) Sred[tid >> 5] = make_double2((double)sr, (double)si);
            __syncthreads();
            Real Sx = 0, Sy = 0;
            for (int w = 0; w < NT / 32; ++w) { Sx += (Real)Sred[w].x; Sy += (Real)Sred[w].y; }

            // C_b over (s_1 chunk, row, group) tasks
            const int base = L1 * Gg;
            int J = base >= NT ? 1 : min(S1, NT / base);
            const int chunk = (S1 + J - 1) / J;
            J = (S1 + chunk - 1) / chunk;
            const int ntask = base * J;   // <= NT whenever J > 1
            for (int task0 = 0; task0 < ntask; task0 += NT) {
                const int task = task0 + tid;
                Real ar[RW], ai[RW];
#pragma unroll
                for (int r = 0; r < RW; ++r) { ar[r] = 0; ai[r] = 0; }
                int i = 0, g = 0;
                if (task < ntask) {
                    const int j = task / base;
                    task_rc(task % base, Gg, i, g);
                    const int n1 = nlo1 + i, n20 = nlo2 + RW * g;
                    const int s1b = slo1 + j * chunk, s1e = min(slo1 + S1, s1b + chunk);
                    if (i < L1) {
                        for (int s1 = s1b; s1 < s1e; ++s1) {
                            const C* __restrict__ prow = Pb + (s1 - slo1) * S2;
                            if (STAGE) {
                                const Real* __restrict__ brow = Bs + (n1 - s1 - a1lo) * WS;
                                row_sweep<Real, RW>([&](int c) { return brow[c]; }, RW * g + S2, prow, S2, ar, ai);
                            } else {
                                const Real* __restrict__ brow = bsl + (n1 - s1 + N) * E;
                                row_sweep<Real, RW>([&](int c) { return __ldg(brow + min(max(c, 0), E - 1)); },
                                                    n20 - slo2 + N, prow, S2, ar, ai);
                            }
                        }
                    }
                }
                if (J == 1) {
                    if (task < ntask && i < L1) {
                        const int n1 = nlo1 + i, n20 = nlo2 + RW * g;
#pragma unroll
                        for (int r = 0; r < RW; ++r) {
                            if (n20 + r >= nlo2 + L2) break;
                            epilogue(n1, n20 + r, ar[r], ai[r], Sx, Sy);
                        }
                    }
                } else {
                    __syncthreads();   // every sweep is done with the staged rectangle: reuse it
                    if (task < ntask) {
#pragma unroll
                        for (int r = 0; r < RW; ++r) Cpart[(size_t)task * RW + r] = cmake<C>(ar[r], ai[r]);
                    }
                    __syncthreads();
                    for (int o = tid; o < L1 * L2; o += NT) {
                        const int ii = o / L2, c = o % L2, gg = c / RW, r = c % RW;
                        Real cx = 0, cy = 0;
                        for (int j = 0; j < J; ++j) {
                            const int t = j * base + rc_task(ii, gg, Gg);
                            const C v = Cpart[(size_t)t * RW + r];
                            cx += v.x;
                            cy += v.y;
                        }
                        epilogue(nlo1 + ii, nlo2 + c, cx, cy, Sx, Sy);
                    }
                }
            }
        } else if (quad) {
            for (int o = tid; o < L1 * L2; o += NT) epilogue(nlo1 + o / L2, nlo2 + o % L2, 0, 0, 0, 0);
        }
    }
    __syncthreads();
    double2* out = A.partials + (size_t)blockIdx.x * nm;
    for (int i = tid; i < nm; i += NT) {
        const C v = Qs[i];
        if (AC::kComp) {
            const C c = Qc[i];
            out[i] = make_double2((double)v.x - (double)c.x, (double)v.y - (double)c.y);
        } else {
            out[i] = make_double2((double)v.x, (double)v.y);
        }
    }
    if (A.stamps) {
        __syncthreads();
        if (tid == 0) atomicMax(&A.stamps[1], global_ns());
    }
}

// Fixed-order sum of the per-CTA partials into Q^ (deterministic): a block owns 32 modes; warp w
// sums the partials c = w, w+8, ... of its lane's mode, then the 8 warp sums combine in order.
__global__ void __launch_bounds__(256) k_sum_partials(int nm, int nPart, const double2* __restrict__ partials,
                                                      double2* __restrict__ out) {
    __shared__ double2 sh[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    double x = 0, y = 0;
    if (i < nm) {
        for (int c = w; c < nPart; c += 8) {
            const double2 v = partials[(size_t)c * nm + i];
            x += v.x;
            y += v.y;
        }
    }
    sh[w][lane] = make_double2(x, y);
    __syncthreads();
    if (w == 0 && i < nm) {
        double sx = 0, sy = 0;
        for (int k = 0; k < 8; ++k) { sx += sh[k][lane].x; sy += sh[k][lane].y; }
        out[i] = make_double2(sx, sy);
    }
}

template <typename Real, int RW, int NT, bool STAGE>
void launch_t(bn_solver* s, const cplx<Real>* G, const Real* beta) {
    FusedArgs<Real> A;
    A.N = s->g.N;
    A.eps = s->eps;
    A.G = G;
    A.beta = beta;
    A.items = s->eps != 0.0 ? s->work.items : s->work_quad.items;
    A.count = s->eps != 0.0 ? s->work.count : s->work_quad.count;
    A.partials = s->partials;
    A.err = s->flags + 2;
    A.sw = sizeof(Real) == 4 ? (const Real*)s->tabs->sw32 : (const Real*)s->tabs->sw64;
    A.stamps = nullptr;
    if (s->prof && s->prof_slot < 8 && s->prof_stamps) {
        A.stamps = s->prof_stamps + 2 * s->prof_slot;
        cudaMemsetAsync(A.stamps, 0xFF, sizeof(unsigned long long), s->stream);
        cudaMemsetAsync(A.stamps + 1, 0, sizeof(unsigned long long), s->stream);
    }
    const size_t smem = Layout2D<Real, RW, STAGE>::bytes(s->g.N, NT);
    const int grid = std::max(1, std::min(A.count, s->n_partials));
    k_fused2d<Real, RW, NT, STAGE><<<grid, NT, smem, s->stream>>>(A);
    k_sum_partials<<<(s->g.nModes + 31) / 32, 256, 0, s->stream>>>(s->g.nModes, grid, s->partials, s->Qhat);
    s->launches += 2;
}

template <typename Real, int RW, int NT, bool STAGE>
void configure_one() {
    cudaFuncSetAttribute(k_fused2d<Real, RW, NT, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

void configure_fused2d() {
    configure_one<float, 8, 128, true>();
    configure_one<float, 8, 256, true>();
    configure_one<double, 2, 128, true>();
    configure_one<double, 2, 256, false>();
}

size_t fused2d_smem(int N, int precision) {
    if (precision == BN_MIXED) return N > 32 ? Layout2D<float, 8, true>::bytes(N, 256) : Layout2D<float, 8, true>::bytes(N, 128);
    return N > 32 ? Layout2D<double, 2, false>::bytes(N, 256) : Layout2D<double, 2, true>::bytes(N, 128);
}

// The 2-D operator: Q^ (s->Qhat) from the modes of the stage argument.
void launch_fused2d(bn_solver* s) {
    const bool mixed = s->opt.precision == BN_MIXED;
    const bool big = s->g.N > 32;
    if (mixed) {
        if (big) launch_t<float, 8, 256, true>(s, s->Ghat32, s->tabs->beta32);
        else launch_t<float, 8, 128, true>(s, s->Ghat32, s->tabs->beta32);
    } else {
        if (big) launch_t<double, 2, 256, false>(s, s->Ghat, s->tabs->beta64);
        else launch_t<double, 2, 128, true>(s, s->Ghat, s->tabs->beta64);
    }
}

}  // namespace bn
