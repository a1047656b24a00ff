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
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <type_traits>

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

// threads per CTA of the mixed-precision kernel for N > 32 (one CTA per SM, limited by shared memory):
// 24 warps of up to 85 registers (N = 64 evaluation: 4.12, 3.61, 3.95, 4.08 ms at 640, 768, 896,
// 1024 threads; 1024 threads leave 64 registers, 512 hide the shared-load latency worse)
constexpr int kBigNT = 768;



__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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

// Shared-memory layout (bytes) for a given N, thread count, staging and double buffering.
template <typename Real, int RW, bool STAGE, bool DB>
struct Layout2D {
    // padded row stride of the staged beta rectangle: >= RW ceil(N/RW) + N columns and
    // congruent to 1 mod 32, so lanes on 8 consecutive rows x 4 groups of RW columns hit
    // 32 distinct banks
    static __host__ __device__ int stride(int N) {
        const int w = RW * ((N + RW - 1) / RW) + N;
        return 32 * ((w - 1 + 31) / 32) + 1;
    }
    // one buffer: the staged beta rectangle, reused for the split sums after the sweep
    static __host__ __device__ size_t slot(int N, int nt) {
        const size_t cp = (size_t)nt * RW * sizeof(cplx<Real>);
        const size_t bs = STAGE ? (size_t)(2 * N) * stride(N) * sizeof(Real) : cp;
        return ((bs > cp ? bs : cp) + 15) / 16 * 16;
    }
    static __host__ __device__ size_t bytes(int N, int nt) {
        const size_t nm = (size_t)N * N;
        size_t b = nm * sizeof(cplx<Real>) * (Acc<Real>::kComp ? 2 : 1);   // Q accumulator (+ compensation)
        b += nm * sizeof(cplx<Real>);                                        // Gs
        b += (size_t)N * (N + 2) * sizeof(cplx<Real>);                      // Pb (rows padded to even length)
        b += slot(N, nt) * (DB ? 2 : 1);                                     // beta rectangle(s) / split sums
        b += 32 * sizeof(cplx<Real>);                                        // S(b) warp sums
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

// 4- or 8-byte asynchronous copy global -> shared (zero-filled when !valid).
template <typename Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src, bool valid) {
    if (sizeof(Real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 4 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 8 : 0)
                     : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// Box geometry of one b (per dimension: outputs n with n, n-b in I_N; inner s with s, b-s in I_N)
// and the beta rectangle a = n - s that the sweep reads.
template <int RW>
struct ItemGeo {
    int b1, b2, nlo1, L1, nlo2, L2, slo1, S1, slo2, S2, Gg, A1, a1lo, A2, a2lo;
    bool quad;
    __device__ __forceinline__ ItemGeo(int ib, int N) {
        const int E = 2 * N;
        b1 = ib / E - N;
        b2 = ib % E - N;
        nlo1 = max(-N / 2, b1 - N / 2);
        L1 = min(N / 2 - 1, b1 + N / 2 - 1) - nlo1 + 1;
        nlo2 = max(-N / 2, b2 - N / 2);
        L2 = min(N / 2 - 1, b2 + N / 2 - 1) - nlo2 + 1;
        slo1 = max(-N / 2, b1 - N / 2 + 1);
        S1 = min(N / 2 - 1, b1 + N / 2) - slo1 + 1;
        slo2 = max(-N / 2, b2 - N / 2 + 1);
        S2 = min(N / 2 - 1, b2 + N / 2) - slo2 + 1;
        quad = b1 >= -N / 2 && b1 < N / 2 && b2 >= -N / 2 && b2 < N / 2;
        Gg = (L2 + RW - 1) / RW;
        A1 = L1 + S1 - 1;
        a1lo = nlo1 - slo1 - S1 + 1;
        A2 = RW * Gg + S2;            // one spare column on the left
        a2lo = nlo2 - slo2 - S2;
    }
};

// Issue the asynchronous copies of the beta rectangle of item `ib` into `Bs` (padded stride WS).
template <typename Real, int RW, int NT>
__device__ __forceinline__ void stage_rect(Real* Bs, const Real* __restrict__ beta, int ib, int N, int WS) {
    const ItemGeo<RW> g(ib, N);
    const int E = 2 * N, nExt = E * E;
    const Real* __restrict__ bsl = beta + (size_t)ib * nExt;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < g.A1; r += NT / 32) {
        const Real* __restrict__ src = bsl + (g.a1lo + r + N) * E + N;   // row a1, column a2 = 0
        Real* dst = Bs + r * WS;
        for (int c = lane; c < g.A2; c += 32) {
            const int a2 = g.a2lo + c;
            const bool ok = a2 >= -N && a2 < N;
            cp_async_elem(dst + c, src + (ok ? a2 : 0), ok);
        }
    }
}

// Two consecutive P_b entries (16 bytes; FP32 only).
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
    a = p[0];
    b = p[1];
}

// FP32 sweep of one s_1 row from the staged rectangle (the mixed N > 32 kernel): ar/ai[r] +=
// sum_{s2} beta(c0 + r - s2) P(s2) with the (real, imaginary) sums of an output and the duplicated
// weight held as packed pairs, so that one paired FMA (fma.rn.f32x2, rounded per half exactly as
// fmaf) serves both parts of P; the weights rotate through a register window (slot of offset x is
// x mod RW).  Per step: one load of beta, its duplication, one 64-bit load of P and RW paired FMA.
// The rectangle row is a plain pointer, so every load is addressed from one base (a form with a
// load functor and paired P loads issued ~7 register moves per step: 15 % slower at N = 64).
template <int RW>
__device__ __forceinline__ void row_sweep_p(const float* __restrict__ brow, int c0, const uint64_t* __restrict__ prow,
                                            int S2, float (&ar)[RW], float (&ai)[RW]) {
    uint64_t acc[RW], w[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        acc[r] = pack2(ar[r], ai[r]);
        w[r] = dup2(brow[c0 + r]);
    }
    int sl = 0;
    for (; sl + RW <= S2; sl += RW) {
#pragma unroll
        for (int kk = 0; kk < RW; ++kk) {
            if (kk == 0) {
                if (sl > 0) w[0] = dup2(brow[c0 - sl]);
            } else {
                w[RW - kk] = dup2(brow[c0 - sl - kk]);
            }
            const uint64_t p = prow[sl + kk];
#pragma unroll
            for (int r = 0; r < RW; ++r) acc[r] = fma2(w[(r - kk + RW) % RW], p, acc[r]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < RW; ++kk) {
        if (sl + kk >= S2) break;
        if (kk == 0) {
            if (sl > 0) w[0] = dup2(brow[c0 - sl]);
        } else {
            w[RW - kk] = dup2(brow[c0 - sl - kk]);
        }
        const uint64_t p = prow[sl + kk];
#pragma unroll
        for (int r = 0; r < RW; ++r) acc[r] = fma2(w[(r - kk + RW) % RW], p, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) split2(acc[r], ar[r], ai[r]);
}

// One s_1 row of the Toeplitz product in the generic form (FP64, and the unstaged path): ar/ai[r]
// += sum_{s2} beta(c0 + r - s2) P(s2), with the weights held in a register window whose slots
// rotate (slot of offset x is x mod RW), so that every step costs one load of beta, half a load
// of P (pairs, the row starts 16-byte aligned) and 2 RW FMA, with no register moves.
template <typename Real, int RW, typename LoadB>
__device__ __forceinline__ void row_sweep(LoadB ldb, int c0, const cplx<Real>* __restrict__ prow, int S2,
                                          Real (&ar)[RW], Real (&ai)[RW]) {
    static_assert(RW % 2 == 0, "RW must be even");
    Real w[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) w[r] = ldb(c0 + r);
    int sl = 0;
    for (; sl + RW <= S2; sl += RW) {
#pragma unroll
        for (int k = 0; k < RW; k += 2) {
            cplx<Real> p0, p1;
            ld_pair(prow + sl + k, p0, p1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kk = k + h;
                if (kk == 0) {
                    if (sl > 0) w[0] = ldb(c0 - sl);
                } else {
                    w[RW - kk] = ldb(c0 - sl - kk);
                }
                const cplx<Real> p = h == 0 ? p0 : p1;
#pragma unroll
                for (int r = 0; r < RW; ++r) {
                    const Real wr = w[(r - kk + RW) % RW];
                    ar[r] = fma(wr, p.x, ar[r]);
                    ai[r] = fma(wr, p.y, ai[r]);
                }
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

// The operator for one request, run by CTA `blk` of the `nblk` CTAs that serve it.
template <typename Real, int RW, int NT, bool STAGE, bool DB>
__device__ __forceinline__ void fused2d_body(const FusedArgs<Real>& A, int blk, int nblk) {
    using C = cplx<Real>;
    using AC = Acc<Real>;
    using LY = Layout2D<Real, RW, STAGE, DB>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = A.N, E = 2 * N, nExt = E * E, nm = N * N;
    const int WS = LY::stride(N);
    C* Qs = reinterpret_cast<C*>(smem_raw);
    C* Qc = Qs + (AC::kComp ? nm : 0);
    C* Gs = Qc + nm;
    C* Pb = Gs + nm;
    unsigned char* slots = reinterpret_cast<unsigned char*>(Pb + N * (N + 2));
    const size_t slot_bytes = LY::slot(N, NT);
    C* Sred = reinterpret_cast<C*>(slots + slot_bytes * (DB ? 2 : 1));
    uint64_t* bar = reinterpret_cast<uint64_t*>(Sred + 32);
    const int tid = threadIdx.x, lane = tid & 31;
    const bool cubic = A.eps != 0.0;
    const Real eps_r = (Real)A.eps;
    if (A.stamps && tid == 0) atomicMin(&A.stamps[0], global_ns());

    // G^ -> shared memory with one bulk copy (TMA engine); the first beta rectangle is requested
    // at the same time and the accumulator zeroed while both are in flight.
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, (uint32_t)(nm * sizeof(C)));
        bulk_g2s(Gs, A.G, (uint32_t)(nm * sizeof(C)), bar);
    }
    if (STAGE && cubic && blk < A.count)
        stage_rect<Real, RW, NT>(reinterpret_cast<Real*>(slots), A.beta, A.items[blk], N, WS);
    cp_async_commit();
    for (int i = tid; i < nm; i += NT) {
        Qs[i] = cmake<C>(0.0, 0.0);
        if (AC::kComp) Qc[i] = cmake<C>(0.0, 0.0);
    }
    __syncthreads();
    if (A.giveup_first || !mbar_wait_bounded(bar, 0, kWaitLimit)) {
        // the copy did not complete in time: record it, wait (bounded) once more for the
        // copy in flight, and give up
        atomicOr(A.err, 1);
        mbar_wait_bounded(bar, 0, kWaitLimit);
        cp_async_wait<0>();
        return;
    }

    int buf = 0;
    for (int item = blk; item < A.count; item += nblk, buf ^= (DB ? 1 : 0)) {
        const int ib = A.items[item];
        const ItemGeo<RW> g(ib, N);
        const Real* __restrict__ bsl = A.beta + (size_t)ib * nExt;   // beta(., b), [a1][a2]
        const C gb = g.quad ? Gs[(g.b1 + N / 2) * N + (g.b2 + N / 2)] : cmake<C>(0.0, 0.0);
        const Real wbb = g.quad ? __ldg(bsl + (g.b1 + N) * E + (g.b2 + N)) : Real(0);
        Real* Bs = reinterpret_cast<Real*>(slots + slot_bytes * buf);
        C* Cpart = reinterpret_cast<C*>(Bs);   // reused after the sweep (split sums)

        // D_b(n) = eps (C + S) + quadratic term; Qacc[n] += G^_{n-b} D
        auto epilogue = [&](int n1, int n2, Real cx, Real cy, Real Sx, Real Sy) {
            C D = cmake<C>(eps_r * (cx + Sx), eps_r * (cy + Sy));
            if (g.quad) {
                const Real wq = __ldg(bsl + (n1 - g.b1 + N) * E + (n2 - g.b2 + N)) - wbb;
                D.x = fma(wq, gb.x, D.x);
                D.y = fma(wq, gb.y, D.y);
            }
            const int on = (n1 + N / 2) * N + (n2 + N / 2);
            const C gk = Gs[(n1 - g.b1 + N / 2) * N + (n2 - g.b2 + N / 2)];
            AC::add(Qs + on, Qc + on, cmul(gk, D));
        };

        __syncthreads();   // [A] the previous item is done with Pb, its slot and the accumulator entries
        if (cubic && STAGE) {
            if (DB) {
                const int next = item + nblk;
                if (next < A.count)
                    stage_rect<Real, RW, NT>(reinterpret_cast<Real*>(slots + slot_bytes * (buf ^ 1)), A.beta,
                                             A.items[next], N, WS);
            } else if (item != blk) {
                stage_rect<Real, RW, NT>(Bs, A.beta, ib, N, WS);
            }
            cp_async_commit();
        }
        const int S2e = (g.S2 + 1) & ~1;   // P_b row stride (even: 16-byte aligned rows)
        if (cubic) {
            for (int r = tid >> 5; r < g.S1; r += NT / 32) {
                const int s1 = g.slo1 + r;
                const C* __restrict__ gx = Gs + (s1 + N / 2) * N + N / 2;
                const C* __restrict__ gy = Gs + (g.b1 - s1 + N / 2) * N + N / 2 + g.b2;
                for (int c = lane; c < g.S2; c += 32) {
                    const int s2 = g.slo2 + c;
                    Pb[r * S2e + c] = cmul(gx[s2], gy[-s2]);
                }
            }
            if (STAGE) {
                if (DB) cp_async_wait<1>();   // this thread's copies of the current rectangle have landed
                else cp_async_wait<0>();
            }
        }
        __syncthreads();   // [B] Pb and the staged rectangle are visible

        if (cubic) {
            // S(b) = sum over box_s of W(b, s) P_b(s): warp w takes the rows s_1 = slo1 + w, w + NW, ...;
            // the warp sums are combined after the next barrier
            {
                Real sr = 0, si = 0;
                const Real* __restrict__ wrow = A.sw + (size_t)ib * nm;
                for (int r = tid >> 5; r < g.S1; r += NT / 32) {
                    const Real* __restrict__ wr = wrow + (g.slo1 + r + N / 2) * N + N / 2;
                    for (int c = lane; c < g.S2; c += 32) {
                        const Real w = __ldg(wr + g.slo2 + c);
                        const C p = Pb[r * S2e + c];
                        sr = fma(w, p.x, sr);
                        si = fma(w, p.y, si);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                if (lane == 0) Sred[tid >> 5] = cmake<C>(sr, si);
            }
            Real Sx = 0, Sy = 0;   // read from Sred after the barrier that follows the sweeps

            // C_b over (s_1 chunk, row, group) tasks; lanes of a warp share the s_1 chunk (P_b loads
            // are broadcasts) and differ in (row, group) (beta loads on distinct banks)
            const int base = g.L1 * g.Gg;
            int J = base >= NT ? 1 : min(g.S1, NT / base);
            const int chunk = (g.S1 + J - 1) / J;
            J = (g.S1 + chunk - 1) / chunk;
            const int ntask = base * J;   // <= NT whenever J > 1
            for (int task0 = 0; task0 < ntask; task0 += NT) {
                const int task = task0 + tid;
                Real ar[RW], ai[RW];
#pragma unroll
                for (int r = 0; r < RW; ++r) { ar[r] = 0; ai[r] = 0; }
                int i = 0, gg = 0;
                if (task < ntask) {
                    const int j = task / base;
                    task_rc(task % base, g.Gg, i, gg);
                    const int n1 = g.nlo1 + i, n20 = g.nlo2 + RW * gg;
                    const int s1b = g.slo1 + j * chunk, s1e = min(g.slo1 + g.S1, s1b + chunk);
                    for (int s1 = s1b; s1 < s1e; ++s1) {
                        const C* __restrict__ prow = Pb + (s1 - g.slo1) * S2e;
                        if (STAGE) {
                            const Real* __restrict__ brow = Bs + (n1 - s1 - g.a1lo) * WS;
                            if constexpr (std::is_same<Real, float>::value)
                                row_sweep_p<RW>(brow, RW * gg + g.S2, reinterpret_cast<const uint64_t*>(prow), g.S2, ar, ai);
                            else
                                row_sweep<Real, RW>([&](int c) { return brow[c]; }, RW * gg + g.S2, prow, g.S2, ar, ai);
                        } else {
                            const Real* __restrict__ brow = bsl + (n1 - s1 + N) * E;
                            row_sweep<Real, RW>([&](int c) { return __ldg(brow + min(max(c, 0), E - 1)); },
                                                n20 - g.slo2 + N, prow, g.S2, ar, ai);
                        }
                    }
                }
                if (J == 1) {
                    __syncthreads();   // the warp sums of S(b) are visible
                    Sx = 0;
                    Sy = 0;
                    for (int w = 0; w < NT / 32; ++w) { Sx += Sred[w].x; Sy += Sred[w].y; }
                    if (task < ntask) {
                        const int n1 = g.nlo1 + i, n20 = g.nlo2 + RW * gg;
#pragma unroll
                        for (int r = 0; r < RW; ++r) {
                            if (n20 + r >= g.nlo2 + g.L2) break;
                            epilogue(n1, n20 + r, ar[r], ai[r], Sx, Sy);
                        }
                    }
                } else {
                    __syncthreads();   // every sweep is done with the staged rectangle: reuse its slot
                    if (task < ntask) {
#pragma unroll
                        for (int r = 0; r < RW; ++r) Cpart[(size_t)task * RW + r] = cmake<C>(ar[r], ai[r]);
                    }
                    __syncthreads();
                    for (int w = 0; w < NT / 32; ++w) { Sx += Sred[w].x; Sy += Sred[w].y; }
                    for (int ii = tid >> 5; ii < g.L1; ii += NT / 32) {
                        for (int c = lane; c < g.L2; c += 32) {
                            const int gq = c / RW, r = c % RW;
                            Real cx = 0, cy = 0;
                            for (int j = 0; j < J; ++j) {
                                const C v = Cpart[((size_t)(j * base + ii * g.Gg + gq)) * RW + r];
                                cx += v.x;
                                cy += v.y;
                            }
                            epilogue(g.nlo1 + ii, g.nlo2 + c, cx, cy, Sx, Sy);
                        }
                    }
                }
            }
        } else if (g.quad) {
            for (int ii = tid >> 5; ii < g.L1; ii += NT / 32)
                for (int c = lane; c < g.L2; c += 32) epilogue(g.nlo1 + ii, g.nlo2 + c, 0, 0, 0, 0);
        }
    }
    if (STAGE) cp_async_wait<0>();
    __syncthreads();
    double2* out = A.partials + (size_t)blk * nm;
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

template <typename Real, int RW, int NT, bool STAGE, bool DB>
__global__ void __launch_bounds__(NT) k_fused2d(FusedArgs<Real> A) {
    fused2d_body<Real, RW, NT, STAGE, DB>(A, blockIdx.x, gridDim.x);
}

// Many requests in one launch: CTAs [cta_begin[j], cta_begin[j+1]) serve request j with the same
// CTA count (and hence the same partial sums) as its own launch, so a request's result does not
// depend on what else is in the batch.  The dynamic shared memory is sized for the largest N.
template <typename Real, int RW, int NT, bool STAGE, bool DB>
__global__ void __launch_bounds__(NT) k_fused2d_batch(const FusedArgs<Real>* __restrict__ jobs,
                                                      const int* __restrict__ cta_begin, int njobs) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cta_begin[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const FusedArgs<Real> A = jobs[lo];
    fused2d_body<Real, RW, NT, STAGE, DB>(A, blockIdx.x - cta_begin[lo], cta_begin[lo + 1] - cta_begin[lo]);
}

// Fixed-order sum of the per-CTA partials into Q^ (deterministic): a block owns 8 modes; the 32
// thread groups sum the partials c = w, w + 32, ... of their mode, then combine in order.
__global__ void __launch_bounds__(256) k_sum_partials(int nm, int nPart, const double2* __restrict__ partials,
                                                      double2* __restrict__ out) {
    __shared__ double2 sh[32][8];
    const int m = threadIdx.x & 7, w = threadIdx.x >> 3;
    const int i = blockIdx.x * 8 + m;
    double x = 0, y = 0;
    if (i < nm) {
        for (int c = w; c < nPart; c += 32) {
            const double2 v = partials[(size_t)c * nm + i];
            x += v.x;
            y += v.y;
        }
    }
    sh[w][m] = make_double2(x, y);
    __syncthreads();
    if (threadIdx.x < 8 && i < nm) {
        double sx = 0, sy = 0;
        for (int k = 0; k < 32; ++k) { sx += sh[k][m].x; sy += sh[k][m].y; }
        out[i] = make_double2(sx, sy);
    }
}

template <typename Real>
void fill_args_t(const bn_solver* s, FusedArgs<Real>& A) {
    A.N = s->g.N;
    A.eps = s->eps;
    A.G = sizeof(Real) == 4 ? (const cplx<Real>*)(const void*)s->Ghat32 : (const cplx<Real>*)(const void*)s->Ghat;
    A.beta = sizeof(Real) == 4 ? (const Real*)(const void*)s->tabs->beta32 : (const Real*)(const void*)s->tabs->beta64;
    A.items = s->eps != 0.0 ? s->work.items : s->work_quad.items;
    A.count = s->eps != 0.0 ? s->work.count : s->work_quad.count;
    A.partials = s->partials;
    A.err = s->flags + 2;
    A.giveup_first = s->opt.debug_wait_giveup;
    A.sw = sizeof(Real) == 4 ? (const Real*)(const void*)s->tabs->sw32 : (const Real*)(const void*)s->tabs->sw64;
    A.stamps = nullptr;
    A.Sb = s->S2;
    A.meta = s->work.meta[s->mixed_v];
    A.dq = s->tabs->dq32;
    A.betaT = s->tabs->beta32T;
}

// The residual-table pass of the kernel-mode rounding correction: the same kernel over the
// rounding residuals of the FP32 tables, into its own partials and S(b) sums.
void fill_args_lo(const bn_solver* s, FusedArgs<float>& A) {
    fill_args_t<float>(s, A);
    A.beta = s->tabs->beta32lo;
    A.sw = s->tabs->sw32lo;
    A.dq = s->tabs->dq32lo;
    A.betaT = s->tabs->beta32Tlo;
    A.partials = s->partials_lo;
    A.Sb = s->S2lo;
}

__global__ void k_add_modes(int nm, double2* __restrict__ Q, const double2* __restrict__ add) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
        const double2 a = add[i];
        double2 q = Q[i];
        q.x += a.x;
        q.y += a.y;
        Q[i] = q;
    }
}

// Mixed precision N <= 32 (variant 0): k_mixed2d (which also forms S(b)) and the FP32-compensated
// partial sum with the S(b) convolution (bn_fused2d_mixed.cu).
void launch_mixed(bn_solver* s) {
    if (beta_split_on(s) && s->lo_refresh) {
        FusedArgs<float> L;
        fill_args_lo(s, L);
        s->launches += launch_mixed2d(L, std::max(1, std::min(L.count, s->n_partials)), s->mixed_rw, s->Qlo, s->stream);
    }
    FusedArgs<float> A;
    fill_args_t<float>(s, A);
    if (s->prof && s->prof_slot < 8 && s->prof_stamps) {
        A.stamps = s->prof_stamps + 2 * s->prof_slot;
        cudaMemsetAsync(A.stamps, 0xFF, sizeof(unsigned long long), s->stream);
        cudaMemsetAsync(A.stamps + 1, 0, sizeof(unsigned long long), s->stream);
    }
    const int grid = std::max(1, std::min(A.count, s->n_partials));
    s->launches += launch_mixed2d(A, grid, s->mixed_rw, s->Qhat, s->stream);
}

template <typename Real, int RW, int NT, bool STAGE, bool DB>
void launch_t(bn_solver* s, const cplx<Real>* G, const Real* beta) {
    if constexpr (sizeof(Real) == 4) {
        if (beta_split_on(s) && s->lo_refresh) {
            FusedArgs<float> L;
            fill_args_lo(s, L);
            L.G = G;
            const size_t smem = Layout2D<Real, RW, STAGE, DB>::bytes(s->g.N, NT);
            const int grid = std::max(1, std::min(L.count, s->n_partials));
            k_fused2d<Real, RW, NT, STAGE, DB><<<grid, NT, smem, s->stream>>>(L);
            k_sum_partials<<<(s->g.nModes + 7) / 8, 256, 0, s->stream>>>(s->g.nModes, grid, s->partials_lo, s->Qlo);
            s->launches += 2;
        }
    }
    FusedArgs<Real> A;
    fill_args_t<Real>(s, A);
    A.G = G;
    A.beta = beta;
    if (s->prof && s->prof_slot < 8 && s->prof_stamps) {
        A.stamps = s->prof_stamps + 2 * s->prof_slot;
        cudaMemsetAsync(A.stamps, 0xFF, sizeof(unsigned long long), s->stream);
        cudaMemsetAsync(A.stamps + 1, 0, sizeof(unsigned long long), s->stream);
    }
    const size_t smem = Layout2D<Real, RW, STAGE, DB>::bytes(s->g.N, NT);
    const int grid = std::max(1, std::min(A.count, s->n_partials));
    k_fused2d<Real, RW, NT, STAGE, DB><<<grid, NT, smem, s->stream>>>(A);
    k_sum_partials<<<(s->g.nModes + 7) / 8, 256, 0, s->stream>>>(s->g.nModes, grid, s->partials, s->Qhat);
    s->launches += 2;
}

template <typename Real, int RW, int NT, bool STAGE, bool DB>
void configure_one() {
    cudaFuncSetAttribute(k_fused2d<Real, RW, NT, STAGE, DB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_fused2d_batch<Real, RW, NT, STAGE, DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
}

template <typename Real, int RW, int NT, bool STAGE, bool DB>
void launch_group_t(cudaStream_t st, const void* d_jobs, const int* d_cta, int njobs, int total, int maxN) {
    const size_t smem = Layout2D<Real, RW, STAGE, DB>::bytes(maxN, NT);
    k_fused2d_batch<Real, RW, NT, STAGE, DB><<<total, NT, smem, st>>>((const FusedArgs<Real>*)d_jobs, d_cta, njobs);
}

}  // namespace

// Kernels: mixed precision N <= 32: k_mixed2d (bn_fused2d_mixed.cu); mixed N > 32: this file's
// kernel in FP32 with 8 outputs per thread, kBigNT threads per CTA, the paired-FMA sweep and a
// single staging buffer (shared memory); FP64: 2 outputs per thread (DFMA-bound), staged for
// N <= 32, read through L1 for N > 32.
void configure_fused2d() {
    configure_mixed2d();
    configure_one<float, 8, kBigNT, true, false>();
    configure_one<double, 2, 128, true, false>();
    configure_one<double, 2, 256, false, false>();
}

size_t fused2d_smem(int N, int precision) {
    if (precision == BN_MIXED) return N > 32 ? Layout2D<float, 8, true, false>::bytes(N, kBigNT) : mixed2d_smem(N, 8);
    return N > 32 ? Layout2D<double, 2, false, false>::bytes(N, 256) : Layout2D<double, 2, true, false>::bytes(N, 128);
}

// The fused operator into caller-chosen scratch on a given stream (used by the no-allocation
// entry point): G = the solver's precision copy of the modes, partials/Qhat/err in scratch.
template <typename Real, int RW, int NT, bool STAGE, bool DB>
void into_t(const bn_solver* s, cudaStream_t st, const void* G, double2* partials, double2* Qhat, int* err,
            bool lo = false) {
    FusedArgs<Real> A;
    if constexpr (sizeof(Real) == 4) {
        if (lo) fill_args_lo(s, A);
        else fill_args_t<Real>(s, A);
    } else {
        fill_args_t<Real>(s, A);
    }
    A.G = (const cplx<Real>*)G;
    A.partials = partials;
    A.err = err;
    const size_t smem = Layout2D<Real, RW, STAGE, DB>::bytes(s->g.N, NT);
    const int grid = std::max(1, std::min(A.count, s->n_partials));
    k_fused2d<Real, RW, NT, STAGE, DB><<<grid, NT, smem, st>>>(A);
    k_sum_partials<<<(s->g.nModes + 7) / 8, 256, 0, st>>>(s->g.nModes, grid, partials, Qhat);
}

void fused2d_into(const bn_solver* s, cudaStream_t st, const void* G, double2* partials, double2* Qhat, int* err,
                  void* sb, bool lo) {
    switch (fused2d_variant(s)) {
        case 0:
        case 4: {
            FusedArgs<float> A;
            if (lo) fill_args_lo(s, A);
            else fill_args_t<float>(s, A);
            A.G = (const float2*)G;
            A.partials = partials;
            A.err = err;
            A.Sb = sb;
            launch_mixed2d(A, std::max(1, std::min(A.count, s->n_partials)), s->mixed_rw, Qhat, st);
            break;
        }
        case 1: into_t<float, 8, kBigNT, true, false>(s, st, G, partials, Qhat, err, lo); break;
        case 2: into_t<double, 2, 128, true, false>(s, st, G, partials, Qhat, err); break;
        default: into_t<double, 2, 256, false, false>(s, st, G, partials, Qhat, err); break;
    }
}

int fused2d_partials(const bn_solver* s) {
    return std::max(1, std::min(s->eps != 0.0 ? s->work.count : s->work_quad.count, s->n_partials));
}

// ------------------------------------------------------------------ autotuner (mixed N <= 32)
// Four variants of the kernel: 8 or 16 outputs per thread (8: 3 CTAs per SM; 16: 2 CTAs per SM,
// fewer warp units and a longer register window, more padding on small boxes), each with the
// register window always along n_2 or with the orientation chosen per b by the host's mapping
// model.  The variant is chosen per (device, N, forced RW) by timing the candidates on the
// solver's stream: each runs twice untimed, then the candidates take turns for three rounds of one
// timed launch each (CUDA events) on the solver's own tables and buffers; the candidate with the
// fastest launch wins and is cached for the process.  opt.mixed_rw forces the
// outputs per thread (the orientation is still timed); opt.mixed_variant forces a variant.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;
}  // namespace

bn_status tune_mixed2d(bn_solver* s, std::string* err) {
    s->mixed_rw = 8;
    s->mixed_v = 0;
    if (s->g.d != 2 || s->opt.precision != BN_MIXED || s->g.N > 32) return BN_OK;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (sms <= 0) sms = 152;
    auto parts = [&](int rw) {
        return std::max(1, std::min(s->work.count, mixed2d_ctas_per_sm(s->g.N, rw) * sms));
    };
    const int forced = (s->opt.mixed_rw == 8 || s->opt.mixed_rw == 16) ? s->opt.mixed_rw : 0;
    const auto key = std::make_tuple(s->device, s->g.N, forced);
    int choice = s->opt.mixed_variant > 0 ? s->opt.mixed_variant - 1 : -1;
    if (choice < 0) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) choice = it->second;
    }
    if (choice < 0) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const int v0 = forced == 16 ? 2 : 0, v1 = forced == 8 ? 2 : 4;
        FusedArgs<float> A[4];
        int grid[4];
        for (int v = v0; v < v1; ++v) {
            const int rw = v < 2 ? 8 : 16;
            s->mixed_rw = rw;
            s->mixed_v = v;
            fill_args_t<float>(s, A[v]);
            A[v].items = s->work.items;   // the full cubic work list (timing does not depend on eps or values)
            A[v].count = s->work.count;
            A[v].eps = 1.0;
            grid[v] = std::min(parts(rw), s->n_partials);
        }
        // all candidates warm up first, then take turns: kRounds rounds of one timed launch each, the
        // fastest launch of a candidate counting (so a slow first launch or a transient on the GPU
        // does not decide)
        constexpr int kRounds = 3;
        for (int v = v0; v < v1; ++v)
            for (int i = 0; i < 2; ++i) launch_mixed2d_kernel(A[v], grid[v], v < 2 ? 8 : 16, s->stream);
        float tmin[4] = {1e30f, 1e30f, 1e30f, 1e30f};
        for (int round = 0; round < kRounds; ++round)
            for (int v = v0; v < v1; ++v) {
                cudaEventRecord(e0, s->stream);
                launch_mixed2d_kernel(A[v], grid[v], v < 2 ? 8 : 16, s->stream);
                cudaEventRecord(e1, s->stream);
                cudaError_t e = cudaEventSynchronize(e1);
                float ms = 0;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    cudaGetLastError();
                    *err = std::string("autotuner: ") + cudaGetErrorString(e);
                    return BN_ERR_CUDA;
                }
                tmin[v] = std::min(tmin[v], ms);
            }
        float best = 1e30f;
        for (int v = v0; v < v1; ++v) {
            s->tune_ms[v] = tmin[v];
            if (tmin[v] < best) {
                best = tmin[v];
                choice = v;
            }
            s->launches += 2 + kRounds;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaMemsetAsync(s->flags, 0, 8 * sizeof(int), s->stream);
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = choice;
    }
    s->mixed_v = choice;
    s->mixed_rw = choice < 2 ? 8 : 16;
    s->n_partials = std::min(s->n_partials, parts(s->mixed_rw));
    return BN_OK;
}

bool fused2d_partials_f32(const bn_solver* s) {
    return s->g.d == 2 && (fused2d_variant(s) == 0 || fused2d_variant(s) == 4);
}

// 0: mixed N <= 32 with 8 outputs per thread, 4: with 16; 1: mixed N > 32; 2, 3: FP64.
int fused2d_variant(const bn_solver* s) {
    const bool big = s->g.N > 32;
    if (s->opt.precision == BN_MIXED) return big ? 1 : (s->mixed_rw == 16 ? 4 : 0);
    return big ? 3 : 2;
}

void fill_fused_args(const bn_solver* s, void* out) {
    if (s->opt.precision == BN_MIXED) fill_args_t<float>(s, *(FusedArgs<float>*)out);
    else fill_args_t<double>(s, *(FusedArgs<double>*)out);
}

void fill_fused_args_lo(const bn_solver* s, void* out) { fill_args_lo(s, *(FusedArgs<float>*)out); }

bool beta_split_on(const bn_solver* s) {
    return s->opt.beta_split && s->opt.precision == BN_MIXED && s->g.d == 2 && !s->nd && s->Qlo && s->tabs &&
           s->tabs->beta32lo;
}

void launch_add_modes(int nm, double2* Q, const double2* add, cudaStream_t st) {
    k_add_modes<<<(nm + 255) / 256, 256, 0, st>>>(nm, Q, add);
}

size_t fused2d_variant_smem(int variant, int N) {
    switch (variant) {
        case 0: return mixed2d_smem(N, 8);
        case 4: return mixed2d_smem(N, 16);
        case 1: return Layout2D<float, 8, true, false>::bytes(N, kBigNT);
        case 2: return Layout2D<double, 2, true, false>::bytes(N, 128);
        default: return Layout2D<double, 2, false, false>::bytes(N, 256);
    }
}

// One launch for a group of requests of the same variant; CTAs [d_cta[j], d_cta[j+1]) serve job j.
void launch_fused2d_group(cudaStream_t st, int variant, const void* d_jobs, const int* d_cta, int njobs, int total,
                          int maxN) {
    switch (variant) {
        case 0: launch_mixed2d_group(st, 8, d_jobs, d_cta, njobs, total, maxN); break;
        case 4: launch_mixed2d_group(st, 16, d_jobs, d_cta, njobs, total, maxN); break;
        case 1: launch_group_t<float, 8, kBigNT, true, false>(st, d_jobs, d_cta, njobs, total, maxN); break;
        case 2: launch_group_t<double, 2, 128, true, false>(st, d_jobs, d_cta, njobs, total, maxN); break;
        default: launch_group_t<double, 2, 256, false, false>(st, d_jobs, d_cta, njobs, total, maxN); break;
    }
}

// The 2-D operator: Q^ (s->Qhat) from the modes of the stage argument.  With the kernel-mode
// rounding correction the residual-table pass runs first when s->lo_refresh is set (its modes
// kept in s->Qlo) and Qlo is added to Q^.
void launch_fused2d(bn_solver* s) {
    const bool mixed = s->opt.precision == BN_MIXED;
    const bool big = s->g.N > 32;
    if (mixed) {
        if (big) launch_t<float, 8, kBigNT, true, false>(s, s->Ghat32, s->tabs->beta32);
        else launch_mixed(s);
        if (beta_split_on(s)) {
            launch_add_modes(s->g.nModes, s->Qhat, s->Qlo, s->stream);
            s->launches++;
        }
    } else {
        if (big) launch_t<double, 2, 256, false, false>(s, s->Ghat, s->tabs->beta64);
        else launch_t<double, 2, 128, true, false>(s, s->Ghat, s->tabs->beta64);
    }
}

}  // namespace bn
