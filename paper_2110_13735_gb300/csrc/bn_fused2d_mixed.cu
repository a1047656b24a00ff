// bn_fused2d_mixed.cu -- the 2-D operator in mixed precision for N <= 32 (Mouton & Rey, Lemma of
// Sec. 2.3 combined as in Sec. 3.3 step 2(c)): FP32 sums with compensated accumulation.
//
// Same factorisation as the FP64 kernel (bn_fused2d.cu): with b = l + m and s = l,
//   Q^_n = sum_b G^_{n-b} D_b(n),
//   D_b(n) = eps [C_b(n) + S(b)] + [b in I_N] (beta(n-b, b) - beta(b,b)) G^_b,
//   C_b(n) = sum_{s in box_s(b)} beta(n-s, b) P_b(s),   P_b(s) = G^_s G^_{b-s},
//   S(b)   = sum_{s in box_s(b)} W(b, s) P_b(s),        W(b, s) = beta(s, b-s) - beta(b, s) - beta(s, b).
//
// Organisation (one CTA walks its share of the b values, dealt on the host by estimated cost,
// heaviest first):
//  * S(b) (the reducible part) is formed per b from the staged P_b by the warps once their sweep
//    units are done, summed in warp order and written out; its convolution with G^ is added by
//    the partial-sum kernel, so no output of this kernel waits on it.
//  * The beta rectangle (box_n - box_s) of the next b is copied into shared memory asynchronously
//    and its P_b formed while the current b is swept: one CTA barrier per b.
//  * The sweep is split into warp units.  A unit is 32/J (output row, group of 8 outputs along n_2)
//    tasks times J chunks of the s_1 range (J in {1, 2, 4, 8}, chosen per b from an issue-cost model
//    of the busiest warp; a last partial round of units may be re-split into up to 32 chunks so
//    that it spreads over all warps); the J partial sums of a task meet by a shuffle
//    reduce-scatter (then a butterfly past 8 chunks), so no shared-memory reduction or extra
//    barrier is needed, and each of the J lanes finishes 8/J of the task's outputs.
//  * Each thread keeps 8 outputs in registers as (real, imaginary) pairs; along s_2 the weights
//    beta(n-s, b) slide through a register window (one shared load of beta, its duplication into
//    a pair, one 64-bit load of P_b and 8 paired FMAs, fma.rn.f32x2, per step).
//  * G^_{n-b} D_b(n) is added to an FP32 (sum, compensation) pair per output in shared memory
//    (Kahan); each CTA writes both words, and the partials of all CTAs are summed in FP32 with
//    compensation in a fixed order, the group sums in FP64 (deterministic).
#include <algorithm>
#include <cstdint>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kNT = 256;            // threads per CTA
constexpr int kNW = kNT / 32;       // warps per CTA
constexpr int kWRows = 32 / kNW;    // P_b rows per warp in the S(b) sums (N <= 32)
constexpr uint32_t kWait = 1u << 22;  // polls of the bounded mbarrier wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bulk (TMA engine) copy of `bytes` (multiple of 16, both ends 16-byte aligned) completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
        "l"(src), "r"(bytes), "r"(su32(bar))
        : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWait; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(su32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void cp4(float* dst, const float* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(su32(dst)), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void kahan(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Shared-memory layout for N and RW outputs per thread: Q sums, Q compensations, G^, two P_b
// buffers, two beta rectangles, a ring of three item records and the copy barrier.
template <int RW>
struct MixedLayout {
    // beta row stride: >= the widest rectangle (RW ceil(N/RW) + N columns) and == 1 (mod 32), so
    // that consecutive rows of the lanes of a warp fall on distinct banks
    static __host__ __device__ int ws(int N) {
        const int w = RW * ((N + RW - 1) / RW) + N;
        return 32 * ((w - 1 + 31) / 32) + 1;
    }
    // P_b row stride (complex entries): odd, so that rows of different s_1 chunks read in one
    // 64-bit load fall on different banks
    static __host__ __device__ int ps(int N) { return N | 1; }
    static __host__ __device__ size_t bslot(int N) { return ((size_t)2 * N * ws(N) * 4 + 15) / 16 * 16; }
    static __host__ __device__ size_t pslot(int N) { return ((size_t)N * ps(N) * 8 + 15) / 16 * 16; }
    static __host__ __device__ size_t bytes(int N) {
        return (size_t)N * N * sizeof(float2) * 3 + 2 * pslot(N) + 2 * bslot(N) + 3 * sizeof(ItemMeta) + 16 +
               2 * 8 * sizeof(float2);
    }
};

// Asynchronous copy of the beta rectangle of one b into Bs (rows a_u by warp, columns a_w by lane)
// from the table whose rows run along u (beta for orient 0, the swapped table for orient 1);
// columns whose a_w falls outside [-N, N) are zero-filled.
__device__ __forceinline__ void stage_beta(float* Bs, const float* __restrict__ beta, const float* __restrict__ betaT,
                                           const ItemMeta& m, int N, int WS) {
    constexpr int kCB = 3;   // column blocks of 32: rectangles up to 96 columns wide (N <= 32 needs 64)
    const int E = 2 * N, Au = m.Au, Aw = m.Aw, lane = threadIdx.x & 31;
    const int clo = -N - m.a_wlo, chi = N - m.a_wlo;   // valid columns [clo, chi)
    const float* __restrict__ src0 =
        (m.orient ? betaT : beta) + (size_t)m.ib * E * E + (m.a_ulo + N) * E + N + m.a_wlo;
    // the column predicates and source offsets are the same in every row
    bool in[kCB], ok[kCB];
    int off[kCB];
#pragma unroll
    for (int q = 0; q < kCB; ++q) {
        const int c = lane + 32 * q;
        in[q] = c < Aw;
        ok[q] = c >= clo && c < chi;
        off[q] = ok[q] ? c : 0;
    }
    for (int r = threadIdx.x >> 5; r < Au; r += kNW) {
        const float* __restrict__ src = src0 + r * E;
        float* dst = Bs + r * WS + lane;
#pragma unroll
        for (int q = 0; q < kCB; ++q)
            if (in[q]) cp4(dst + 32 * q, src + off[q], ok[q]);
    }
}

// P_b(s) = G^_s G^_{b-s} over box_s(b): rows s_u, columns s_w, stride PS.  Lanes run along the
// dimension that is contiguous in G^ (s_w for orient 0, s_u for orient 1).
__device__ __forceinline__ void build_P(float2* Pb, const float2* Gs, const ItemMeta& m, int N, int PS) {
    const int h = N / 2, lane = threadIdx.x & 31, Su = m.Su, Sw = m.Sw;
    if (!m.orient) {
        for (int r = threadIdx.x >> 5; r < Su; r += kNW) {
            const int s1 = m.slo_u + r;
            const float2* gx = Gs + (s1 + h) * N + h + m.slo_w;
            const float2* gy = Gs + (m.b1 - s1 + h) * N + h + m.b2 - m.slo_w;
            float2* dst = Pb + r * PS;
            for (int c = lane; c < Sw; c += 32) dst[c] = cmulf(gx[c], gy[-c]);
        }
    } else {
        // u = dimension 2, w = dimension 1: s = (slo_w + c, slo_u + r)
        for (int c = threadIdx.x >> 5; c < Sw; c += kNW) {
            const int s1 = m.slo_w + c;
            const float2* gx = Gs + (s1 + h) * N + h + m.slo_u;
            const float2* gy = Gs + (m.b1 - s1 + h) * N + h + m.b2 - m.slo_u;
            for (int r = lane; r < Su; r += 32) Pb[r * PS + c] = cmulf(gx[r], gy[-r]);
        }
    }
}

// One s_1 row of the Toeplitz product: acc[r] += sum_{s2} beta[c0 + r - s2] P[s2] with acc[r] the
// (real, imaginary) pair of output r, the weights in a register window whose slots rotate (slot of
// column x is x mod RW) and hold each weight twice, so that one paired FMA serves both halves of
// P: per step one shared load of beta, one of P and RW paired FMA.  Columns read:
// c0 - S2 + 1 .. c0 + RW - 1.
template <int kRW>
__device__ __forceinline__ void row_sweep(const float* __restrict__ brow, int c0, const uint64_t* __restrict__ prow,
                                          int S2, uint64_t (&acc)[kRW]) {
    uint64_t w[kRW];
#pragma unroll
    for (int r = 0; r < kRW; ++r) w[r] = dup2(brow[c0 + r]);
    int sl = 0;
    for (; sl + kRW <= S2; sl += kRW) {
#pragma unroll
        for (int kk = 0; kk < kRW; ++kk) {
            if (kk == 0) {
                if (sl > 0) w[0] = dup2(brow[c0 - sl]);
            } else {
                w[kRW - kk] = dup2(brow[c0 - sl - kk]);
            }
            const uint64_t p = prow[sl + kk];
#pragma unroll
            for (int r = 0; r < kRW; ++r) acc[r] = fma2(w[(r - kk + kRW) % kRW], p, acc[r]);
        }
    }
#pragma unroll
    for (int kk = 0; kk < kRW; ++kk) {
        if (sl + kk >= S2) break;
        if (kk == 0) {
            if (sl > 0) w[0] = dup2(brow[c0 - sl]);
        } else {
            w[kRW - kk] = dup2(brow[c0 - sl - kk]);
        }
        const uint64_t p = prow[sl + kk];
#pragma unroll
        for (int r = 0; r < kRW; ++r) acc[r] = fma2(w[(r - kk + kRW) % kRW], p, acc[r]);
    }
}

// One halving step of the shuffle reduce-scatter over the first L of the kRW sums: the lane keeps
// entries [0, L/2) (hi false) or [L/2, L) (hi true), adds the partner's copy (lane ^ mk) of the same
// entries and stores them in [0, L/2).
template <int kRW, int L>
__device__ __forceinline__ void reduce_half(float (&ar)[kRW], float (&ai)[kRW], bool hi, int mk) {
#pragma unroll
    for (int i = 0; i < L / 2; ++i) {
        const float sr = hi ? ar[i] : ar[i + L / 2], si = hi ? ai[i] : ai[i + L / 2];
        const float kr = hi ? ar[i + L / 2] : ar[i], ki = hi ? ai[i + L / 2] : ai[i];
        ar[i] = kr + __shfl_xor_sync(0xffffffffu, sr, mk);
        ai[i] = ki + __shfl_xor_sync(0xffffffffu, si, mk);
    }
}

// Metadata of item `item` into a shared ring slot (4 threads, 16 bytes each, asynchronous).
__device__ __forceinline__ void fetch_meta(ItemMeta* slot, const ItemMeta* __restrict__ meta, int item, int count) {
    if (item < count && threadIdx.x < 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(su32(reinterpret_cast<int4*>(slot) + threadIdx.x)),
                     "l"(reinterpret_cast<const int4*>(meta + item) + threadIdx.x)
                     : "memory");
}

template <int kRW>
__device__ __forceinline__ void mixed_body(const FusedArgs<float>& A, int blk, int nblk) {
    using Lay = MixedLayout<kRW>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int N = A.N, E = 2 * N, nm = N * N, h = N / 2;
    const int WS = Lay::ws(N), PS = Lay::ps(N);
    float2* Qs = reinterpret_cast<float2*>(smem_raw);
    float2* Qc = Qs + nm;
    float2* Gs = Qc + nm;
    unsigned char* p = reinterpret_cast<unsigned char*>(Gs + nm);
    float2* const P0 = reinterpret_cast<float2*>(p);                       // P_b buffer k at P0 + k pstep
    const int pstep = (int)(Lay::pslot(N) / sizeof(float2));
    p += 2 * Lay::pslot(N);
    float* const B0 = reinterpret_cast<float*>(p);                         // rectangle k at B0 + k bstep
    const int bstep = (int)(Lay::bslot(N) / sizeof(float));
    p += 2 * Lay::bslot(N);
    ItemMeta* ring = reinterpret_cast<ItemMeta*>(p);                       // 3 slots
    uint64_t* bar = reinterpret_cast<uint64_t*>(p + 3 * sizeof(ItemMeta));
    float2* Sred = reinterpret_cast<float2*>(p + 3 * sizeof(ItemMeta) + 16);   // [2][kNW] warp sums of S(b)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool cubic = A.eps != 0.0;
    const float eps_r = (float)A.eps;
    float2* __restrict__ Sb = reinterpret_cast<float2*>(A.Sb);
    const float* __restrict__ Wt = A.sw;
    const ItemMeta* __restrict__ meta = reinterpret_cast<const ItemMeta*>(A.meta);
    if (A.stamps && tid == 0) atomicMin(&A.stamps[0], now_ns());

    if (!cubic) {
        // quadratic part only (b in I_N): each thread owns the outputs n == tid (mod NT) for every
        // b, so no barrier is needed between b values
        if (tid == 0) {
            bar_init(bar);
            bulk_load(Gs, A.G, (uint32_t)(nm * sizeof(float2)), bar);
        }
        for (int i = tid; i < nm; i += kNT) {
            Qs[i] = make_float2(0.f, 0.f);
            Qc[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        const bool landed = !A.giveup_first && bar_wait(bar, 0);
        if (__syncthreads_or(!landed)) {
            if (tid == 0) atomicOr(A.err, 1);
            bar_wait(bar, 0);
            return;
        }
        for (int item = blk; item < A.count; item += nblk) {
            const int ib = A.items[item], b1 = ib / E - N, b2 = ib % E - N;
            const float* __restrict__ dqb = A.dq + (size_t)((b1 + h) * N + (b2 + h)) * E * E;
            const float2 gb = Gs[(b1 + h) * N + (b2 + h)];
            for (int on = tid; on < nm; on += kNT) {
                const int n1 = on / N - h, n2 = on % N - h;
                const int k1 = n1 - b1, k2 = n2 - b2;
                if (k1 < -h || k1 >= h || k2 < -h || k2 >= h) continue;
                const float wq = __ldg(dqb + (k1 + N) * E + (k2 + N));
                const float2 x = cmulf(Gs[(k1 + h) * N + (k2 + h)], make_float2(wq * gb.x, wq * gb.y));
                kahan(Qs[on].x, Qc[on].x, x.x);
                kahan(Qs[on].y, Qc[on].y, x.y);
            }
        }
    } else {
        // G^ -> shared memory (one bulk copy); the metadata of the first two items and the first
        // rectangle are requested at the same time
        if (tid == 0) {
            bar_init(bar);
            bulk_load(Gs, A.G, (uint32_t)(nm * sizeof(float2)), bar);
        }
        fetch_meta(ring + 0, meta, blk, A.count);
        fetch_meta(ring + 1, meta, blk + nblk, A.count);
        cp_commit();
        for (int i = tid; i < nm; i += kNT) {
            Qs[i] = make_float2(0.f, 0.f);
            Qc[i] = make_float2(0.f, 0.f);
        }
        cp_wait_all();
        __syncthreads();
        if (blk < A.count) stage_beta(B0, A.beta, A.betaT, ring[0], N, WS);
        cp_commit();
        const bool landed = !A.giveup_first && bar_wait(bar, 0);
        if (__syncthreads_or(!landed)) {
            // the copy did not complete in time: record it, wait (bounded) for the copies in flight, give up
            if (tid == 0) atomicOr(A.err, 1);
            bar_wait(bar, 0);
            cp_wait_all();
            return;
        }
        if (blk < A.count) build_P(P0, Gs, ring[0], N, PS);
        cp_wait_all();
        __syncthreads();

        int k = 0, slot = 0, prev_ib = -1;
        for (int item = blk; item < A.count; item += nblk) {
            const ItemMeta& m = ring[slot];
            if (tid == 0 && prev_ib >= 0) {   // S(b) of the previous b: its warp sums, in warp order
                float2 t = Sred[(k ^ 1) * kNW];
                for (int w = 1; w < kNW; ++w) t = make_float2(t.x + Sred[(k ^ 1) * kNW + w].x, t.y + Sred[(k ^ 1) * kNW + w].y);
                Sb[prev_ib] = t;
            }
            const int nslot = slot == 2 ? 0 : slot + 1, n2slot = nslot == 2 ? 0 : nslot + 1;
            // the buffers and ring slot of the previous b are free (barrier at its end): fill them
            fetch_meta(ring + n2slot, meta, item + 2 * nblk, A.count);
            if (item + nblk < A.count) {
                stage_beta(B0 + (k ^ 1) * bstep, A.beta, A.betaT, ring[nslot], N, WS);
                build_P(P0 + (k ^ 1) * pstep, Gs, ring[nslot], N, PS);
            }
            cp_commit();
            const float* __restrict__ Bs = B0 + k * bstep;
            const float2* __restrict__ Pb = P0 + k * pstep;
            const int orient = m.orient, b1 = m.b1, b2 = m.b2;
            const int nlo_u = m.nlo_u, nlo_w = m.nlo_w, slo_u = m.slo_u, Su = m.Su, Sw = m.Sw;
            const int Gg = m.Gg, a_ulo = m.a_ulo, base = m.base;
            const int umain = m.units, uall = m.units + m.units2;
            // the weights W(b, s) of this warp's P_b rows for S(b), requested now and used after the
            // sweep (N <= 32: at most 4 rows of at most 32 entries per warp)
            float wv[kWRows];
#pragma unroll
            for (int j = 0; j < kWRows; ++j) {
                const int r = warp + kNW * j, su_ = m.slo_u + r, sw_ = m.slo_w + lane;
                const int s1 = orient ? sw_ : su_, s2 = orient ? su_ : sw_;
                wv[j] = r < Su && lane < Sw ? __ldg(Wt + (size_t)m.ib * nm + (s1 + h) * N + (s2 + h)) : 0.f;
            }
            const int nwend = nlo_w + m.Lw;
            const int su = orient ? 1 : N, sw = orient ? N : 1;   // flat strides of u and w (modes)
            const int eu = orient ? 1 : E, ew = orient ? E : 1;   // and in the extended box
            const bool quad = m.quad != 0;
            float2 gb = make_float2(0.f, 0.f);
            const float* __restrict__ dqb = A.dq;
            if (quad) {
                gb = Gs[(b1 + h) * N + (b2 + h)];
                dqb += (size_t)((b1 + h) * N + (b2 + h)) * E * E + (N - b1) * E + (N - b2);   // dq at a = n - b
            }
            const int bshift = b1 * N + b2;   // flat offset of n - b from n
            for (int u = warp; u < uall; u += kNW) {
                // units of the full rounds, then those of the re-split last round
                const bool tl = u >= umain;
                const int J = tl ? m.J2 : m.J, chunk = tl ? m.chunk2 : m.chunk;
                const int lgt = 5 - (31 - __clz(J)), tpw = 1 << lgt;   // tasks per unit, 32 / J
                const int jl = lane >> lgt, t = lane & (tpw - 1);
                const int s1b = slo_u + jl * chunk, s1e = min(slo_u + Su, s1b + chunk);
                const int tau = tl ? m.tail0 + ((u - umain) << lgt) + t : (u << lgt) + t;
                const bool valid = tau < base;
                int irow = 0, gg = 0;
                if (valid) {
                    if (orient) {   // row fastest
                        gg = (tau * m.linv) >> 16;
                        irow = tau - gg * m.Lu;
                    } else {        // group fastest
                        irow = (tau * m.ginv) >> 16;
                        gg = tau - irow * Gg;
                    }
                }
                uint64_t acc[kRW];
#pragma unroll
                for (int r = 0; r < kRW; ++r) acc[r] = 0ull;   // (+0.0f, +0.0f)
                const int n_u = nlo_u + irow;
                const int nw0 = nlo_w + kRW * gg;
                if (valid && quad) {
                    // the quadratic weights of this task's outputs are needed after the sweep
                    const float* pf = dqb + n_u * eu + nw0 * ew;
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(pf));
                }
                if (valid) {
                    const int c0 = kRW * gg + Sw;
                    const float* brow = Bs + (n_u - a_ulo - s1b) * WS;
                    const uint64_t* prow = reinterpret_cast<const uint64_t*>(Pb) + (s1b - slo_u) * PS;
                    for (int s1 = s1b; s1 < s1e; ++s1, brow -= WS, prow += PS)
                        row_sweep<kRW>(brow, c0, prow, Sw, acc);
                }
                float ar[kRW], ai[kRW];
#pragma unroll
                for (int r = 0; r < kRW; ++r) split2(acc[r], ar[r], ai[r]);
                // the J chunk sums of a task (lanes t + tpw j, J a power of two) meet by a shuffle
                // reduce-scatter: each halving step keeps half of the outputs, so that afterwards lane
                // j holds the complete sums of kRW / J outputs, starting at output `off`
                int off = 0;
                if (J >= 2) {
                    const bool hi = (lane & tpw) != 0;
                    reduce_half<kRW, kRW>(ar, ai, hi, tpw);
                    off += hi ? kRW / 2 : 0;
                }
                if (J >= 4) {
                    const bool hi = (lane & (2 * tpw)) != 0;
                    reduce_half<kRW, kRW / 2>(ar, ai, hi, 2 * tpw);
                    off += hi ? kRW / 4 : 0;
                }
                if (J >= 8) {
                    const bool hi = (lane & (4 * tpw)) != 0;
                    reduce_half<kRW, kRW / 4>(ar, ai, hi, 4 * tpw);
                    off += hi ? kRW / 8 : 0;
                }
                if constexpr (kRW >= 16) {
                    if (J >= 16) {
                        const bool hi = (lane & (8 * tpw)) != 0;
                        reduce_half<kRW, kRW / 8>(ar, ai, hi, 8 * tpw);
                        off += hi ? kRW / 16 : 0;
                    }
                }
                // more chunks than outputs (a re-split last round): each lane holds one output; the
                // copies of chunk groups jl, jl + RW, ... meet by a butterfly and group jl < RW stores it
                for (int mk = kRW * tpw; mk < 32; mk <<= 1) {
                    ar[0] += __shfl_xor_sync(0xffffffffu, ar[0], mk);
                    ai[0] += __shfl_xor_sync(0xffffffffu, ai[0], mk);
                }
                if (valid && jl < kRW) {
                    const int cnt = J >= kRW ? 1 : kRW / J;
                    const int nw1 = nw0 + off;
                    const float* qrow = dqb + n_u * eu + nw1 * ew;
                    const int on1 = (n_u + h) * su + h * sw + nw1 * sw;
#pragma unroll
                    for (int r = 0; r < kRW; ++r) {
                        if (r >= cnt || nw1 + r >= nwend) break;
                        float2 D = make_float2(eps_r * ar[r], eps_r * ai[r]);
                        if (quad) {
                            const float wq = __ldg(qrow + r * ew);
                            D.x = fmaf(wq, gb.x, D.x);
                            D.y = fmaf(wq, gb.y, D.y);
                        }
                        const int on = on1 + r * sw;
                        const float2 x = cmulf(Gs[on - bshift], D);
                        kahan(Qs[on].x, Qc[on].x, x.x);
                        kahan(Qs[on].y, Qc[on].y, x.y);
                    }
                }
            }
            {
                // S(b) = sum over box_s of W(b, s) P_b(s) (the reducible part; its convolution with
                // G^ is added by the partial-sum kernel): warp w takes the P_b rows w, w + 8, ...
                float sr = 0.f, si = 0.f;
#pragma unroll
                for (int j = 0; j < kWRows; ++j) {
                    const int r = warp + kNW * j;
                    if (r < Su && lane < Sw) {
                        const float2 pv = Pb[r * PS + lane];
                        sr = fmaf(wv[j], pv.x, sr);
                        si = fmaf(wv[j], pv.y, si);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                if (lane == 0) Sred[k * kNW + warp] = make_float2(sr, si);
            }
            prev_ib = m.ib;
            cp_wait_all();
            __syncthreads();
            k ^= 1;
            slot = nslot;
        }
        if (tid == 0 && prev_ib >= 0) {
            float2 t = Sred[(k ^ 1) * kNW];
            for (int w = 1; w < kNW; ++w) t = make_float2(t.x + Sred[(k ^ 1) * kNW + w].x, t.y + Sred[(k ^ 1) * kNW + w].y);
            Sb[prev_ib] = t;
        }
    }
    __syncthreads();
    float4* out = reinterpret_cast<float4*>(A.partials) + (size_t)blk * nm;
    for (int i = tid; i < nm; i += kNT) {
        const float2 v = Qs[i], c = Qc[i];
        out[i] = make_float4(v.x, v.y, c.x, c.y);
    }
    if (A.stamps) {
        __syncthreads();
        if (tid == 0) atomicMax(&A.stamps[1], now_ns());
    }
}

// RW = 8: 80 registers, 3 CTAs per SM; RW = 16: 2 CTAs per SM.
template <int RW>
__global__ void __launch_bounds__(kNT, RW == 8 ? 3 : 2) k_mixed2d(FusedArgs<float> A) {
    mixed_body<RW>(A, blockIdx.x, gridDim.x);
}

// Many requests in one launch: CTAs [cta_begin[j], cta_begin[j+1]) serve request j with its own CTA
// count, so that its result does not depend on the rest of the batch.
template <int RW>
__global__ void __launch_bounds__(kNT, RW == 8 ? 3 : 2) k_mixed2d_batch(const FusedArgs<float>* __restrict__ jobs,
                                                                        const int* __restrict__ cta_begin, int njobs) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cta_begin[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const FusedArgs<float> A = jobs[lo];
    mixed_body<RW>(A, blockIdx.x - cta_begin[lo], cta_begin[lo + 1] - cta_begin[lo]);
}

}  // namespace

namespace {
__global__ void __launch_bounds__(256) k_sum_partials_f32(int nm, int nPart, const float4* __restrict__ partials,
                                                          double2* __restrict__ out, int N, const float2* __restrict__ G32,
                                                          const float2* __restrict__ Sb, float eps) {
    sum_partials_f32_block(nm, nPart, partials, out, blockIdx.x, N, G32, Sb, eps);
}
}  // namespace

size_t mixed2d_smem(int N, int rw) { return rw == 16 ? MixedLayout<16>::bytes(N) : MixedLayout<8>::bytes(N); }

void configure_mixed2d() {
    cudaFuncSetAttribute(k_mixed2d<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_mixed2d_batch<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_mixed2d<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_mixed2d_batch<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

int mixed2d_ctas_per_sm(int N, int rw) {
    int n = 0;
    const size_t smem = mixed2d_smem(N, rw);
    if (rw == 16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mixed2d<16>, kNT, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mixed2d<8>, kNT, smem);
    cudaGetLastError();
    return std::max(1, n);
}

void launch_mixed2d_kernel(const FusedArgs<float>& A, int grid, int rw, cudaStream_t st) {
    if (rw == 16) k_mixed2d<16><<<grid, kNT, MixedLayout<16>::bytes(A.N), st>>>(A);
    else k_mixed2d<8><<<grid, kNT, MixedLayout<8>::bytes(A.N), st>>>(A);
}

int launch_mixed2d(const FusedArgs<float>& A, int grid, int rw, double2* Qhat, cudaStream_t st) {
    const int nm = A.N * A.N;
    const bool red = A.eps != 0.0 && A.count > 0;   // the kernel writes S(b); its convolution follows
    launch_mixed2d_kernel(A, grid, rw, st);
    k_sum_partials_f32<<<(nm + kPartModes - 1) / kPartModes, 256, 0, st>>>(
        nm, grid, reinterpret_cast<const float4*>(A.partials), Qhat, A.N, reinterpret_cast<const float2*>(A.G),
        red ? reinterpret_cast<const float2*>(A.Sb) : nullptr, (float)A.eps);
    return 2;
}

void launch_mixed2d_group(cudaStream_t st, int rw, const void* d_jobs, const int* d_cta, int njobs, int total,
                          int maxN) {
    const FusedArgs<float>* jobs = static_cast<const FusedArgs<float>*>(d_jobs);
    if (rw == 16) k_mixed2d_batch<16><<<total, kNT, MixedLayout<16>::bytes(maxN), st>>>(jobs, d_cta, njobs);
    else k_mixed2d_batch<8><<<total, kNT, MixedLayout<8>::bytes(maxN), st>>>(jobs, d_cta, njobs);
}

}  // namespace bn
