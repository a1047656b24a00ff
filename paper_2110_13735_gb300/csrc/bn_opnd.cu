// bn_opnd.cu -- the collision operator in 3-D (any N up to 48) and in the CIRCULAR truncation
// (2-D and 3-D), with the kernel modes beta recomputed from the quadrature factors at every
// evaluation (Mouton & Rey, Sec. 2.5, eq. betadD: beta(a,b) = sum_p alpha_p(a) alpha'_p(b)).
//
// The 2-D LINEAR operator has its own fused kernels (bn_fused2d*.cu) over a stored beta table.
// In 3-D that table would hold (2N)^6 entries (6.9e10 at N = 32), so this path never forms it.
// A 2-D problem is handled here as a 3-D one whose first axis is trivial (I = {0}).
//
// Factorisation (as in 2-D; b = l + m, s = l, every index sum reduced modulo N in CIRCULAR mode):
//   Q^_n   = quad(n) + eps [Q1q(n) + red(n)]                         (Sec. 3.3 step 2(c), alpha = -eps)
//   quad(n) = sum_{x+y=n} [beta(x,y) - beta(y,y)] G^_x G^_y          (Q_{1c} - Q_{2c})
//   S(t)    = sum_{x+y=t} [beta(x,y) - beta(t,x) - beta(x,t)] G^_x G^_y,   red(n) = sum_k G^_k S(n-k)
//                                                                     (Q_{2q} - Q_{3q} - Q_{4q})
//   Q1q(n)  = sum_b G^_{n-b} C_b(n),  C_b(n) = sum_{s} beta(n-s, b) P_b(s),  P_b(s) = G^_s G^_{b-s}
//                                                                     (Q_{1q}; Remark rem:computComplexity)
// with the Lemma's index sets: n, x, y, s, b-s, n-b in I_N.  For each b the inner sum of Q1q is a
// d-dimensional Toeplitz product of the kernel-mode slice beta(., b) with P_b.
//
// Kernels, per evaluation:
//  * k_pairw_nd (or k_pair_nd): quad and S.  Their weights over I_N x I_N, wq = beta(x,y) -
//    beta(y,y) and wr = beta(x,y) - beta(t,x) - beta(x,t), are formed once per solver by k_pair_nd
//    (a small dense contraction over the quadrature nodes per tile) into tables when they fit in
//    memory, and k_pairw_nd streams them; otherwise k_pair_nd forms them at every evaluation.
//    One CTA per row (t_0, t_1) of t = x + y; sums in a fixed order, accumulated in FP64.
//  * k_beta_slices: the slices beta(a, b) for a in the box A(b) of the differences n - s.  The b
//    whose boxes coincide in the first two axes (and nearly in the third) form groups of up to 64;
//    a group's slices are one contraction over the nodes (rows: a in the union box, columns: the
//    group's b), register-tiled 4 x 8 per thread, written to a slice buffer in global memory.
//    The slices of a "round" (as many groups as fit the buffer) are produced, then consumed.
//  * k_triple_nd: the Toeplitz products.  A work item is (b, T0 consecutive output planes n_0),
//    swept in tiles of output rows n_1; the host chooses per box the planes per item, the rows per
//    tile, the outputs per thread along axis 2 (RW = 4 or 8) and the split of the s_1 range over J
//    lanes (reduced by shuffles), by a cost model of the per-thread work.  The CTA walks the planes
//    a_0 of the slice: the rows a tile needs are copied into shared memory (odd row stride) while
//    the previous plane is swept, and each P_b plane is formed from two mode planes fetched by a
//    bulk (TMA) copy one step earlier.  Each thread sweeps its RW outputs with a register window of
//    weights and scalar FP32 FMA (FP64 in FP64 mode).  C_b(n) times G^_{n-b} is added to the CTA's
//    own partial sums in global memory (FP32 Kahan pairs or FP64); items are dealt to CTAs on the
//    host, so every sum has a fixed order.
//  * k_sum_partials_nd, then k_red_combine_nd: Q1q from the partials, red(n), and Q^.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kMaxGroup = 64;     // b per producer group
constexpr int kPA = 128;          // producer: a per CTA tile
constexpr int kPK = 16;           // producer: nodes per staged chunk
constexpr uint32_t kWaitNd = 1u << 22;   // polls of a bounded mbarrier wait

// ------------------------------------------------------------------ geometry (host and device)
// Axis x has n_x modes I_x = [lo_x, lo_x + n_x - 1] (n_x = 1: the trivial first axis of a 2-D
// problem).  All per-b boxes follow from the index sets of the Lemma (LINEAR) or are the whole
// I_x (CIRCULAR).
struct NdGeo {
    int d, N, wrap;
    int n[3], lo[3];
    int blo[3], nb[3];   // range of b per axis
    int nbTotal;
};

__host__ __device__ inline int red_mod(int x, int lo, int n) {
    int r = (x - lo) % n;
    if (r < 0) r += n;
    return r + lo;
}

struct Box3 { int nlo[3], L[3], slo[3], S[3], alo[3], A[3]; };

__host__ __device__ inline void box_of(const NdGeo& g, const int* b, Box3& B) {
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const int lo = g.lo[x], hi = g.lo[x] + g.n[x] - 1;
        if (g.wrap) {
            B.nlo[x] = lo; B.L[x] = g.n[x];
            B.slo[x] = lo; B.S[x] = g.n[x];
        } else {
            const int nlo = max(lo, b[x] + lo), nhi = min(hi, b[x] + hi);
            const int slo = max(lo, b[x] - hi), shi = min(hi, b[x] - lo);
            B.nlo[x] = nlo; B.L[x] = nhi - nlo + 1;
            B.slo[x] = slo; B.S[x] = shi - slo + 1;
        }
        B.alo[x] = B.nlo[x] - (B.slo[x] + B.S[x] - 1);
        B.A[x] = B.L[x] + B.S[x] - 1;
    }
}

__host__ __device__ inline void b_of_flat(const NdGeo& g, int f, int* b) {
    b[2] = f % g.nb[2] + g.blo[2];
    f /= g.nb[2];
    b[1] = f % g.nb[1] + g.blo[1];
    b[0] = f / g.nb[1] + g.blo[0];
}

// row stride of a slice (elements): the axis-2 length rounded up so that rows start 16-byte aligned
__host__ __device__ inline int slice_rs(int A2, int elem) { const int q = 16 / elem; return (A2 + q - 1) / q * q; }

// flat index of a mode (or I_N-table entry) and of an extended-box alpha entry
__host__ __device__ inline int mode_index(const NdGeo& g, int a0, int a1, int a2) {
    return ((a0 - g.lo[0]) * g.n[1] + (a1 - g.lo[1])) * g.n[2] + (a2 - g.lo[2]);
}
__host__ __device__ inline int ext_index(const NdGeo& g, int a0, int a1, int a2) {
    const int E = 2 * g.N;
    const int e0 = g.d == 3 ? a0 + g.N : 0;
    return (e0 * E + (a1 + g.N)) * E + (a2 + g.N);
}
// kernel-mode argument a (a difference n - s) as the alpha tables see it: reduced into I_N in
// CIRCULAR mode
__host__ __device__ inline int alpha_index(const NdGeo& g, int a0, int a1, int a2) {
    if (g.wrap) {
        a0 = red_mod(a0, g.lo[0], g.n[0]);
        a1 = red_mod(a1, g.lo[1], g.n[1]);
        a2 = red_mod(a2, g.lo[2], g.n[2]);
    }
    return ext_index(g, a0, a1, a2);
}

// ------------------------------------------------------------------ plan records
struct NdGroup {
    int ulo[3], uA[3];    // union box of the members' slice boxes (row-major order of a)
    int first, nb;        // members: group_b[first .. first + nb)
};

struct NdItem {
    uint32_t bflat;       // b (flat index over the b box)
    uint8_t t0i, T0;      // output planes n_0 in [nlo_0 + t0i, + T0)
    uint8_t L1t, J;       // output rows per tile along axis 1; lanes splitting the s_1 range
    uint8_t RW, pad0;     // outputs per thread along axis 2 (4 or 8)
    uint16_t pad1;
    uint32_t off16;       // slice offset in 16-byte units from the slice buffer
};
static_assert(sizeof(NdItem) == 16, "NdItem is 16 bytes");

template <typename Real> struct CT;
template <> struct CT<float> { using C = float2; using P4 = float4; };
template <> struct CT<double> { using C = double2; using P4 = double2; };

// ------------------------------------------------------------------ producer: beta slices
// CTA (group, tile): rows a = tile*kPA .. (the union box in row-major order), columns the group's
// b; beta(a, b_j) = sum_p alpha_p(a) alpha'_p(b_j), thread (tx, ty) owns a = tx + 32 q (q < 4) and
// j = 8 ty + r (r < 8); nodes staged kPK at a time.  Only a inside A(b_j) is stored.
template <typename Real>
__global__ void __launch_bounds__(256) k_beta_slices(NdGeo g, int P, const Real* __restrict__ alpha,
                                                     const Real* __restrict__ alphap, const NdGroup* __restrict__ groups,
                                                     const int* __restrict__ group_b, const uint32_t* __restrict__ off16,
                                                     const int2* __restrict__ work, Real* __restrict__ slices) {
    __shared__ __align__(16) Real As[kPK][kPA];
    __shared__ __align__(16) Real Bs[kPK][kMaxGroup];
    const int2 wk = work[blockIdx.x];
    const NdGroup G = groups[wk.x];
    const int tile0 = wk.y * kPA;
    const int uTot = G.uA[0] * G.uA[1] * G.uA[2];
    const size_t nE = (size_t)(g.d == 3 ? 8 : 4) * g.N * g.N * (g.d == 3 ? g.N : 1);
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    // staging assignments: As element (k, c) for c = tid & 127, k = (tid >> 7) + 2 i; Bs (k, j) for
    // j = tid & 63, k = (tid >> 6) + 4 i
    const int ca = tid & (kPA - 1);
    int ia_ext = -1;
    {
        const int u = tile0 + ca;
        if (u < uTot) {
            const int a2 = u % G.uA[2] + G.ulo[2], r = u / G.uA[2];
            const int a1 = r % G.uA[1] + G.ulo[1], a0 = r / G.uA[1] + G.ulo[0];
            ia_ext = alpha_index(g, a0, a1, a2);
        }
    }
    const int cb = tid & (kMaxGroup - 1);
    int ib_ext = -1;
    if (cb < G.nb) {
        int b[3];
        b_of_flat(g, group_b[G.first + cb], b);
        ib_ext = ext_index(g, b[0], b[1], b[2]);
    }
    Real acc[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[q][r] = 0;
    for (int p0 = 0; p0 < P; p0 += kPK) {
#pragma unroll
        for (int i = 0; i < kPK / 2; ++i) {
            const int k = (tid >> 7) + 2 * i, p = p0 + k;
            As[k][ca] = (ia_ext >= 0 && p < P) ? alpha[(size_t)p * nE + ia_ext] : Real(0);
        }
#pragma unroll
        for (int i = 0; i < kPK / 4; ++i) {
            const int k = (tid >> 6) + 4 * i, p = p0 + k;
            Bs[k][cb] = (ib_ext >= 0 && p < P) ? alphap[(size_t)p * nE + ib_ext] : Real(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kPK; ++k) {
            Real av[4], bv[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) av[q] = As[k][tx + 32 * q];
#pragma unroll
            for (int r = 0; r < 8; ++r) bv[r] = Bs[k][8 * ty + r];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[q][r] = fma(av[q], bv[r], acc[q][r]);
        }
        __syncthreads();
    }
    // store the entries inside each member's own box
    const int elem = (int)sizeof(Real);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int j = 8 * ty + r;
        if (j >= G.nb) continue;
        int b[3];
        b_of_flat(g, group_b[G.first + j], b);
        Box3 B;
        box_of(g, b, B);
        const int RS = slice_rs(B.A[2], elem);
        Real* __restrict__ dst = slices + (size_t)off16[j + G.first] * (16 / elem);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = tile0 + tx + 32 * q;
            if (u >= uTot) continue;
            const int a2 = u % G.uA[2] + G.ulo[2], rr = u / G.uA[2];
            const int a1 = rr % G.uA[1] + G.ulo[1], a0 = rr / G.uA[1] + G.ulo[0];
            const int i0 = a0 - B.alo[0], i1 = a1 - B.alo[1], i2 = a2 - B.alo[2];
            if (i0 < 0 || i0 >= B.A[0] || i1 < 0 || i1 >= B.A[1] || i2 < 0 || i2 >= B.A[2]) continue;
            dst[((size_t)i0 * B.A[1] + i1) * RS + i2] = acc[q][r];
        }
    }
}

// ------------------------------------------------------------------ consumer: Toeplitz sweeps
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void nd_bar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool nd_bar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitNd; ++i) {
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

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// One row of the Toeplitz product in FP32: acc[r] += sum_{sl < S2} w[c0 + r - sl] P[sl] for the RW
// outputs r of a thread (acc[r] holds (re, im) as two floats), the weights of the row in a
// rotating register window (slot of column x is x mod RW): per step one shared load of a weight,
// one 64-bit load of P and 2 RW scalar FMAs.  (A paired-FMA form with the weights duplicated
// into register pairs measured 14 % slower here: the duplication moves cost more issue slots
// than the pairing saves.)
template <int RW>
__device__ __forceinline__ void sweep_row_f32s(const float* __restrict__ brow, int c0, const float2* __restrict__ prow,
                                               int S2, uint64_t (&accp)[RW]) {
    float re[RW], im[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) split2(accp[r], re[r], im[r]);
    float w[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) w[r] = brow[c0 + r];
    int sl = 0;
    for (; sl + RW <= S2; sl += RW) {
#pragma unroll
        for (int kk = 0; kk < RW; ++kk) {
            if (kk == 0) {
                if (sl > 0) w[0] = brow[c0 - sl];
            } else {
                w[RW - kk] = brow[c0 - sl - kk];
            }
            const float2 p = prow[sl + kk];
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const float ww = w[(r - kk + RW) % RW];
                re[r] = fmaf(ww, p.x, re[r]);
                im[r] = fmaf(ww, p.y, im[r]);
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < RW; ++kk) {
        if (sl + kk >= S2) break;
        if (kk == 0) {
            if (sl > 0) w[0] = brow[c0 - sl];
        } else {
            w[RW - kk] = brow[c0 - sl - kk];
        }
        const float2 p = prow[sl + kk];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const float ww = w[(r - kk + RW) % RW];
            re[r] = fmaf(ww, p.x, re[r]);
            im[r] = fmaf(ww, p.y, im[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) accp[r] = pack2(re[r], im[r]);
}

// The same in FP64 (acc[r] = (re, im)).
template <int RW>
__device__ __forceinline__ void sweep_row_f64(const double* __restrict__ brow, int c0, const double2* __restrict__ prow,
                                              int S2, double2 (&acc)[RW]) {
    double w[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) w[r] = brow[c0 + r];
    int sl = 0;
    for (; sl + RW <= S2; sl += RW) {
#pragma unroll
        for (int kk = 0; kk < RW; ++kk) {
            if (kk == 0) {
                if (sl > 0) w[0] = brow[c0 - sl];
            } else {
                w[RW - kk] = brow[c0 - sl - kk];
            }
            const double2 p = prow[sl + kk];
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const double ww = w[(r - kk + RW) % RW];
                acc[r].x = fma(ww, p.x, acc[r].x);
                acc[r].y = fma(ww, p.y, acc[r].y);
            }
        }
    }
#pragma unroll
    for (int kk = 0; kk < RW; ++kk) {
        if (sl + kk >= S2) break;
        if (kk == 0) {
            if (sl > 0) w[0] = brow[c0 - sl];
        } else {
            w[RW - kk] = brow[c0 - sl - kk];
        }
        const double2 p = prow[sl + kk];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const double ww = w[(r - kk + RW) % RW];
            acc[r].x = fma(ww, p.x, acc[r].x);
            acc[r].y = fma(ww, p.y, acc[r].y);
        }
    }
}

struct TripleNdArgs {
    NdGeo g;
    const void* G;            // modes (float2 or double2), N^d
    const NdItem* items;      // per CTA: items[cta_off[c] .. cta_off[c+1])
    const int* cta_off;
    const void* slices;       // slice buffer (float or double)
    void* partials;           // [gridDim.x][N^d]: float4 (sum, compensation) or double2
    int* err;                 // [0] set when a bounded wait gives up
    int WS;                   // row stride (elements) of a staged slice plane: odd, >= widest row + RW - 1
    int PB;                   // elements per staged slice plane buffer (max rows x WS + RW slack)
    int PS;                   // P plane row stride (complex entries, odd)
    int PP;                   // complex entries per P plane buffer
    int GP;                   // complex entries per staged mode plane (n1 n2; 0 when axis 0 is trivial)
    int T0max;
    int gstage;               // 1: the two mode planes of each P plane are staged in shared memory by
                              // bulk copies one step ahead (kernel instance GS = true); 0: P planes are
                              // built from global memory (L2-resident), leaving that shared memory to
                              // more CTAs
    int giveup_first;             // testing: 1 = each tile's first bounded wait gives up at once
    unsigned long long* stamps;   // optional [2]: first CTA start / last CTA end (%globaltimer)
};

__device__ __forceinline__ unsigned long long nd_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename Real>
__device__ __forceinline__ typename CT<Real>::C load_mode(const TripleNdArgs& A, int m) {
    return reinterpret_cast<const typename CT<Real>::C*>(A.G)[m];
}

__device__ __forceinline__ void cp_async_el(void* dst, const void* src, int bytes) {
    if (bytes == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// generic-proxy accesses of shared memory before this point are ordered before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared memory: two slice-plane buffers (rows at the odd stride WS, so that the output rows a
// warp sweeps fall on distinct banks), T0max + 1 P planes (a ring, odd row stride), two slots of
// the two mode planes a P plane is built from (bulk copies, one mbarrier per slot).
struct NdShared {
    void* G;          // [2 slots][2 planes][GP] complex
    void* P;          // [T0max + 1][PP] complex
    void* B;          // [2][PB] real
    uint64_t* bar;    // [2]
};

// One work item: output planes n_0 in [t0, t0 + T0) of the box of b, in tiles of L1t output rows
// n_1; RW outputs per thread along axis 2 and the s_1 range split over J lanes.  For each tile the
// CTA walks the planes a_0 of the slice: the rows of plane a_0 the tile needs are copied into
// shared memory while the previous plane is swept, and the P plane first needed at the next step
// is built from mode planes fetched (bulk copy) one step earlier (GS), or from global memory.
template <typename Real, int RW, bool GS>
__device__ __forceinline__ void triple_item(const TripleNdArgs& A, const NdItem& item, const NdShared& sm,
                                            uint32_t& phases) {
    using C = typename CT<Real>::C;
    const NdGeo& g = A.g;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C* bufG = reinterpret_cast<C*>(sm.G);
    C* bufP = reinterpret_cast<C*>(sm.P);
    Real* bufB = reinterpret_cast<Real*>(sm.B);
    uint64_t* bar = sm.bar;
    const Real* slices = reinterpret_cast<const Real*>(A.slices);
    const C* Gm = reinterpret_cast<const C*>(A.G);
    const int planeG = g.n[1] * g.n[2];
    int b[3];
    b_of_flat(g, (int)item.bflat, b);
    Box3 B;
    box_of(g, b, B);
    const int RS = slice_rs(B.A[2], (int)sizeof(Real));
    const Real* __restrict__ slice = slices + (size_t)item.off16 * (16 / sizeof(Real));
    const int planeElems = B.A[1] * RS;
    const int T0 = item.T0, J = item.J, L1t = item.L1t;
    const int t0 = B.nlo[0] + item.t0i;
    const int G2 = (B.L[2] + RW - 1) / RW;
    const int aHi = t0 + T0 - 1 - B.slo[0];
    const int aLo = t0 - (B.slo[0] + B.S[0] - 1);
    const int shi0 = B.slo[0] + B.S[0] - 1;
    const int ringN = A.T0max + 1;
    const int task = tid / J, jj = tid % J;
    const int ch = (B.S[1] + J - 1) / J;
    const int s1a = B.slo[1] + jj * ch, s1b = min(B.slo[1] + B.S[1], s1a + ch);
    auto m0_of = [&](int s0) { return g.wrap ? red_mod(b[0] - s0, g.lo[0], g.n[0]) : b[0] - s0; };
    auto ring = [&](int s0) { return bufP + (size_t)(((s0 - B.slo[0]) % ringN + ringN) % ringN) * A.PP; };
    // mode planes s0 and b0 - s0 into slot k (one bulk copy each, completing on bar[k])
    auto fetch_modes = [&](int s0, int k) {
        if (tid == 0) {
            fence_proxy_async();
            C* dst = bufG + (size_t)k * 2 * A.GP;
            const uint32_t bytes = (uint32_t)(planeG * sizeof(C));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bar[k])), "r"(2 * bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
                "l"(Gm + (size_t)(s0 - g.lo[0]) * planeG), "r"(bytes), "r"(su32(&bar[k]))
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    su32(dst + A.GP)),
                "l"(Gm + (size_t)(m0_of(s0) - g.lo[0]) * planeG), "r"(bytes), "r"(su32(&bar[k]))
                : "memory");
        }
    };
    // P plane s0 from the staged mode planes of slot k, or from global memory (k < 0)
    auto build_P = [&](int s0, int k) {
        C* dst = ring(s0);
        const C* gs = bufG + (size_t)max(k, 0) * 2 * A.GP;
        const C* gm = gs + A.GP;
        const int m0 = m0_of(s0);
        const int tot = B.S[1] * B.S[2];
        for (int q = tid; q < tot; q += nthr) {
            const int r1 = q / B.S[2], r2 = q - r1 * B.S[2];
            const int s1 = B.slo[1] + r1, s2 = B.slo[2] + r2;
            int m1 = b[1] - s1, m2 = b[2] - s2;
            if (g.wrap) {
                m1 = red_mod(m1, g.lo[1], g.n[1]);
                m2 = red_mod(m2, g.lo[2], g.n[2]);
            }
            C v;
            if (k >= 0) v = cmul2(gs[(s1 - g.lo[1]) * g.n[2] + (s2 - g.lo[2])], gm[(m1 - g.lo[1]) * g.n[2] + (m2 - g.lo[2])]);
            else v = cmul2(Gm[mode_index(g, s0, s1, s2)], Gm[mode_index(g, m0, m1, m2)]);
            dst[r1 * A.PS + r2] = v;
        }
    };
    for (int n1i = 0; n1i < B.L[1]; n1i += L1t) {
        const int L1c = min(L1t, B.L[1] - n1i);
        const int R1 = L1c + B.S[1] - 1;   // slice rows this tile needs: [n1i, n1i + R1)
        const int tasks = T0 * L1c * G2;
        const bool active = task < tasks;
        const int g2 = task % G2, n1 = B.nlo[1] + n1i + (task / G2) % L1c, i0 = task / (G2 * L1c);
        const int n0 = t0 + i0;
        const int n2 = B.nlo[2] + g2 * RW;
        const int c0 = n2 - B.slo[2] - B.alo[2];
        const int rowoff = n1 - B.alo[1] - n1i;   // staged row of (n1, s1) is rowoff - s1
        auto stage_plane = [&](int a0, int kb) {
            const Real* src = slice + (size_t)(a0 - B.alo[0]) * planeElems + (size_t)n1i * RS;
            Real* dst = bufB + (size_t)kb * A.PB;
            const int tot = R1 * B.A[2];
            for (int e = tid; e < tot; e += nthr) {
                const int r = e / B.A[2], c = e - r * B.A[2];
                cp_async_el(dst + r * A.WS + c, src + (size_t)r * RS + c, (int)sizeof(Real));
            }
            cp_async_commit();
        };
        uint64_t acc32[RW];
        double2 acc64[RW];
        float ks[2 * RW], kc[2 * RW];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            acc32[r] = 0ull;
            acc64[r] = make_double2(0.0, 0.0);
            ks[2 * r] = ks[2 * r + 1] = 0.f;
            kc[2 * r] = kc[2 * r + 1] = 0.f;
        }
        // previous readers are done with every buffer
        __syncthreads();
        stage_plane(aHi, 0);
        // the first step needs P planes s0 = n0 - aHi for n0 in [t0, t0 + T0): only slo0 exists
        for (int s0 = max(B.slo[0], t0 - aHi); s0 <= min(shi0, t0 + T0 - 1 - aHi); ++s0) build_P(s0, -1);
        if constexpr (GS) {
            const int sN = t0 + T0 - aHi;
            if (aHi > aLo && sN <= shi0) fetch_modes(sN, 0);
        }
        cp_async_wait_all();
        __syncthreads();
        int slot = 0;
        for (int a0 = aHi; a0 >= aLo; --a0) {
            const int k = (aHi - a0) & 1;   // mode-plane slot of this step
            if (a0 > aLo) {
                stage_plane(a0 - 1, slot ^ 1);
                const int sNew = t0 + T0 - a0;   // first needed at step a0 - 1; its modes are in slot k
                if (!GS) {
                    if (sNew <= shi0) build_P(sNew, -1);
                } else if (sNew <= shi0) {
                    const int sNext = sNew + 1;
                    if (a0 - 1 > aLo && sNext <= shi0) fetch_modes(sNext, k ^ 1);
                    const bool giveup = a0 == aHi && A.giveup_first;
                    if (giveup || !nd_bar_wait(&bar[k], (phases >> k) & 1u)) {
                        // record it and wait (bounded) for the copy in flight before going on
                        if (tid == 0) atomicExch(A.err, 1);
                        nd_bar_wait(&bar[k], (phases >> k) & 1u);
                    }
                    phases ^= 1u << k;
                    build_P(sNew, k);
                }
            }
            const int s0 = n0 - a0;
            if (active && s0 >= B.slo[0] && s0 <= shi0) {
                const Real* __restrict__ plane = bufB + (size_t)slot * A.PB;
                const C* __restrict__ pplane = ring(s0);
                for (int s1 = s1a; s1 < s1b; ++s1) {
                    const Real* brow = plane + (size_t)(rowoff - s1) * A.WS;
                    const C* prow = pplane + (size_t)(s1 - B.slo[1]) * A.PS;
                    if constexpr (sizeof(Real) == 4) {
                        sweep_row_f32s<RW>(reinterpret_cast<const float*>(brow), c0,
                                           reinterpret_cast<const float2*>(prow), B.S[2], acc32);
                    }
                    else {
                        sweep_row_f64<RW>(reinterpret_cast<const double*>(brow), c0,
                                          reinterpret_cast<const double2*>(prow), B.S[2], acc64);
                    }
                }
                if constexpr (sizeof(Real) == 4) {
                    // compensated accumulation of the plane's sums
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        float lo, hi;
                        split2(acc32[r], lo, hi);
                        kahan_add_f(ks[2 * r], kc[2 * r], lo);
                        kahan_add_f(ks[2 * r + 1], kc[2 * r + 1], hi);
                        acc32[r] = 0ull;
                    }
                }
            }
            cp_async_wait_all();
            __syncthreads();   // the next slice plane and P plane are in; this plane buffer is free
            slot ^= 1;
        }
        // meet the J chunks of a task (lanes task*J .. task*J + J - 1 of one warp)
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            if constexpr (sizeof(Real) == 4) {
                float x = ks[2 * r] - kc[2 * r], y = ks[2 * r + 1] - kc[2 * r + 1];
                for (int o = 1; o < J; o <<= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                ks[2 * r] = x;
                ks[2 * r + 1] = y;
            } else {
                double x = acc64[r].x, y = acc64[r].y;
                for (int o = 1; o < J; o <<= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                acc64[r] = make_double2(x, y);
            }
        }
        if (active && jj == 0) {
            const size_t nm = (size_t)g.n[0] * g.n[1] * g.n[2];
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int nn2 = n2 + r;
                if (nn2 >= B.nlo[2] + B.L[2]) break;
                int k0 = n0 - b[0], k1 = n1 - b[1], k2 = nn2 - b[2];
                if (g.wrap) {
                    k0 = red_mod(k0, g.lo[0], g.n[0]);
                    k1 = red_mod(k1, g.lo[1], g.n[1]);
                    k2 = red_mod(k2, g.lo[2], g.n[2]);
                }
                const C gk = Gm[mode_index(g, k0, k1, k2)];
                const int on = mode_index(g, n0, n1, nn2);
                if constexpr (sizeof(Real) == 4) {
                    const float2 c = make_float2(ks[2 * r], ks[2 * r + 1]);
                    const float2 t = cmul2(gk, c);
                    float4* pp = reinterpret_cast<float4*>(A.partials) + (size_t)blockIdx.x * nm + on;
                    float4 v = *pp;
                    kahan_add_f(v.x, v.z, t.x);
                    kahan_add_f(v.y, v.w, t.y);
                    *pp = v;
                } else {
                    const double2 t = cmul2(gk, acc64[r]);
                    double2* pp = reinterpret_cast<double2*>(A.partials) + (size_t)blockIdx.x * nm + on;
                    double2 v = *pp;
                    v.x += t.x;
                    v.y += t.y;
                    *pp = v;
                }
            }
        }
    }
}

// GS: mode planes staged in shared memory (else the P planes are built from global memory).  FP32:
// up to 128 registers, 2 CTAs per SM (the staging instance is held there by its shared memory at
// N = 32 anyway; capped at 80 registers for a third CTA it ran 25 % slower).
template <typename Real, bool GS>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 2 : 1) k_triple_nd(TripleNdArgs A) {
    using C = typename CT<Real>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NdShared sm;
    C* bufG = reinterpret_cast<C*>(smem_raw);
    C* bufP = bufG + (GS ? 4 * (size_t)A.GP : 0);
    Real* bufB = reinterpret_cast<Real*>(bufP + (size_t)(A.T0max + 1) * A.PP);
    sm.G = bufG;
    sm.P = bufP;
    sm.B = bufB;
    sm.bar = reinterpret_cast<uint64_t*>(bufB + 2 * (size_t)A.PB);
    const int tid = threadIdx.x;
    if (A.stamps && tid == 0) atomicMin(A.stamps, nd_now());
    if (tid == 0) {
        nd_bar_init(&sm.bar[0]);
        nd_bar_init(&sm.bar[1]);
    }
    __syncthreads();
    uint32_t phases = 0u;   // bit i: parity of the next completion of bar[i]
    const int it0 = A.cta_off[blockIdx.x], it1 = A.cta_off[blockIdx.x + 1];
    for (int it = it0; it < it1; ++it) {
        const NdItem item = A.items[it];
        if constexpr (sizeof(Real) == 4) {
            if (item.RW == 8) triple_item<Real, 8, GS>(A, item, sm, phases);
            else triple_item<Real, 4, GS>(A, item, sm, phases);
        } else {
            triple_item<Real, 4, GS>(A, item, sm, phases);
        }
    }
    // every bulk copy issued was waited for (each fetch is consumed one step later) and every
    // element copy waited at the end of its step: nothing is in flight when the CTA exits
    __syncthreads();
    if (A.stamps && tid == 0) atomicMax(A.stamps + 1, nd_now());
}

// ------------------------------------------------------------------ quadratic and reducible sums
// CTA per t-row (t_0, t_1); TX x TX tiles of (x_2, y_2) per thread, pairs (x_0, x_1) processed
// PPC at a time (one group of threads each).  wq = beta(x,y) - beta(y,y) = sum_p (alpha_p(x) -
// alpha_p(y)) alpha'_p(y); wr = beta(x,y) - beta(t,x) - beta(x,t) = sum_p alpha_p(x) (alpha'_p(y) -
// alpha'_p(t)) - alpha_p(t) alpha'_p(x).  Products with G^_x G^_y are reduced along the
// anti-diagonals t_2 = x_2 + y_2 in a fixed order and accumulated in FP64.
struct PairNdArgs {
    NdGeo g;
    int P;
    const void* alphaI;    // [P][N^d] alpha on I_N
    const void* alphapI;
    const void* alphaE;    // [P][(2N)^d] extended-box tables (LINEAR t-rows)
    const void* alphapE;
    const void* G;         // modes (Real complex)
    double2* quad;         // N^d
    double2* S;            // t box: LINEAR (2n_x - 1) per axis, CIRCULAR I_N
    int cubic;
    int nt[3], tlo[3];     // t range per axis
    void* Wq;              // when set: write the weights wq(x, y), wr(x, y) to [x][y] tables (x, y
    void* Wr;              // flat indices in I_N) instead of forming quad and S
};

template <typename Real, int TX>
__global__ void __launch_bounds__(256) k_pair_nd(PairNdArgs A) {
    using C = typename CT<Real>::C;
    constexpr int KP = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const NdGeo& g = A.g;
    const int n2 = g.n[2];
    const int TN = (n2 + TX - 1) / TX;          // thread tiles per axis
    const int tpp = TN * TN;                    // threads per pair
    const int PPC = max(1, (int)blockDim.x / tpp);
    const int nT2 = A.nt[2];
    const int W = 2 * n2 - 1;                   // t-row entries (unwrapped x2 + y2)
    // shared: rows [PPC][4][KP][n2], trow [2][KP][W], partial [PPC*tpp][2*TX-1] (2 complex each),
    // accumulators quad/S [nT2] double2
    Real* rows = reinterpret_cast<Real*>(smem_raw);
    Real* trow = rows + (size_t)PPC * 4 * KP * n2;
    C* part = reinterpret_cast<C*>(trow + 2 * KP * W);
    double2* accQ = reinterpret_cast<double2*>(part + (size_t)PPC * tpp * (2 * TX - 1) * 2);
    double2* accS = accQ + nT2;
    const int t0 = A.tlo[0] + (int)blockIdx.x / A.nt[1], t1 = A.tlo[1] + (int)blockIdx.x % A.nt[1];
    for (int i = threadIdx.x; i < nT2; i += blockDim.x) {
        accQ[i] = make_double2(0.0, 0.0);
        accS[i] = make_double2(0.0, 0.0);
    }
    // pairs (x0, x1): LINEAR x in box_s(t) per axis; CIRCULAR all of I
    int xlo[2], xn[2];
    for (int x = 0; x < 2; ++x) {
        const int lo = g.lo[x], hi = g.lo[x] + g.n[x] - 1, t = x == 0 ? t0 : t1;
        if (g.wrap) { xlo[x] = lo; xn[x] = g.n[x]; }
        else { xlo[x] = max(lo, t - hi); xn[x] = min(hi, t - lo) - xlo[x] + 1; }
    }
    const int npairs = xn[0] * xn[1];
    const int slotp = threadIdx.x / tpp, lt = threadIdx.x % tpp;
    const int tx = lt % TN, ty = lt / TN;
    const Real* aI = reinterpret_cast<const Real*>(A.alphaI);
    const Real* apI = reinterpret_cast<const Real*>(A.alphapI);
    const Real* aE = reinterpret_cast<const Real*>(A.alphaE);
    const Real* apE = reinterpret_cast<const Real*>(A.alphapE);
    const size_t nm = (size_t)g.n[0] * g.n[1] * g.n[2];
    const size_t nE = (size_t)(g.d == 3 ? 8 : 4) * g.N * g.N * (g.d == 3 ? g.N : 1);
    for (int pb = 0; pb < npairs; pb += PPC) {
        // this thread's pair
        const int pi = pb + slotp;
        const bool pvalid = slotp < PPC && pi < npairs;
        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        if (pvalid) {
            x0 = xlo[0] + pi / xn[1];
            x1 = xlo[1] + pi % xn[1];
            y0 = t0 - x0;
            y1 = t1 - x1;
            if (g.wrap) { y0 = red_mod(y0, g.lo[0], g.n[0]); y1 = red_mod(y1, g.lo[1], g.n[1]); }
        }
        Real wq[TX][TX], wr[TX][TX];
#pragma unroll
        for (int i = 0; i < TX; ++i)
#pragma unroll
            for (int j = 0; j < TX; ++j) { wq[i][j] = 0; wr[i][j] = 0; }
        for (int p0 = 0; p0 < A.P; p0 += KP) {
            __syncthreads();
            // stage the x and y rows of the PPC pairs and the t row
            for (int e = threadIdx.x; e < PPC * 4 * KP * n2; e += blockDim.x) {
                const int c = e % n2, k = (e / n2) % KP, which = (e / (n2 * KP)) % 4, sp = e / (n2 * KP * 4);
                const int pj = pb + sp, p = p0 + k;
                Real v = 0;
                if (pj < npairs && p < A.P) {
                    const int xx0 = xlo[0] + pj / xn[1], xx1 = xlo[1] + pj % xn[1];
                    int yy0 = t0 - xx0, yy1 = t1 - xx1;
                    if (g.wrap) { yy0 = red_mod(yy0, g.lo[0], g.n[0]); yy1 = red_mod(yy1, g.lo[1], g.n[1]); }
                    const bool isx = which < 2;
                    const int m = isx ? mode_index(g, xx0, xx1, g.lo[2] + c) : mode_index(g, yy0, yy1, g.lo[2] + c);
                    v = ((which & 1) ? apI : aI)[(size_t)p * nm + m];
                }
                rows[e] = v;
            }
            for (int e = threadIdx.x; e < 2 * KP * W; e += blockDim.x) {
                const int c = e % W, k = (e / W) % KP, which = e / (W * KP);
                const int p = p0 + k;
                Real v = 0;
                if (p < A.P && A.cubic) {
                    int tt2 = 2 * g.lo[2] + c;   // unwrapped x2 + y2
                    if (g.wrap) {
                        tt2 = red_mod(tt2, g.lo[2], g.n[2]);
                        v = (which ? apI : aI)[(size_t)p * nm + mode_index(g, t0, t1, tt2)];
                    } else {
                        v = (which ? apE : aE)[(size_t)p * nE + ext_index(g, t0, t1, tt2)];
                    }
                }
                trow[e] = v;
            }
            __syncthreads();
            if (pvalid) {
                const Real* rb = rows + (size_t)slotp * 4 * KP * n2;
#pragma unroll 2
                for (int k = 0; k < KP; ++k) {
                    Real ax[TX], apx[TX], ay[TX], apy[TX], at[2 * TX - 1], apt[2 * TX - 1];
#pragma unroll
                    for (int i = 0; i < TX; ++i) {
                        const int cx = min(tx * TX + i, n2 - 1), cy = min(ty * TX + i, n2 - 1);
                        ax[i] = rb[(0 * KP + k) * n2 + cx];
                        apx[i] = rb[(1 * KP + k) * n2 + cx];
                        ay[i] = rb[(2 * KP + k) * n2 + cy];
                        apy[i] = rb[(3 * KP + k) * n2 + cy];
                    }
#pragma unroll
                    for (int i = 0; i < 2 * TX - 1; ++i) {
                        const int ct = min((tx + ty) * TX + i, W - 1);
                        at[i] = trow[(0 * KP + k) * W + ct];
                        apt[i] = trow[(1 * KP + k) * W + ct];
                    }
#pragma unroll
                    for (int i = 0; i < TX; ++i)
#pragma unroll
                        for (int j = 0; j < TX; ++j) {
                            wq[i][j] = fma(ax[i] - ay[j], apy[j], wq[i][j]);
                            wr[i][j] = fma(ax[i], apy[j] - apt[i + j], fma(-at[i + j], apx[i], wr[i][j]));
                        }
                }
            }
        }
        if (A.Wq) {
            // weight tables: every (x, y) of I_N x I_N belongs to exactly one (t-row, pair, tile)
            if (pvalid) {
                Real* wq_t = reinterpret_cast<Real*>(A.Wq);
                Real* wr_t = reinterpret_cast<Real*>(A.Wr);
#pragma unroll
                for (int i = 0; i < TX; ++i) {
                    const int x2 = g.lo[2] + tx * TX + i;
                    if (x2 >= g.lo[2] + n2) break;
                    const size_t xf = (size_t)mode_index(g, x0, x1, x2);
#pragma unroll
                    for (int j = 0; j < TX; ++j) {
                        const int y2 = g.lo[2] + ty * TX + j;
                        if (y2 >= g.lo[2] + n2) break;
                        const size_t o = xf * nm + mode_index(g, y0, y1, y2);
                        wq_t[o] = wq[i][j];
                        if (A.cubic) wr_t[o] = wr[i][j];
                    }
                }
            }
            continue;
        }
        // products with G^_x G^_y, anti-diagonal partials of this thread
        C* mypart = part + ((size_t)(slotp * tpp + lt)) * (2 * TX - 1) * 2;
        if (slotp < PPC) {
            C dq[2 * TX - 1], dr[2 * TX - 1];
#pragma unroll
            for (int i = 0; i < 2 * TX - 1; ++i) { dq[i].x = dq[i].y = 0; dr[i].x = dr[i].y = 0; }
            if (pvalid) {
                const C* Gm = reinterpret_cast<const C*>(A.G);
#pragma unroll
                for (int i = 0; i < TX; ++i) {
                    const int x2 = g.lo[2] + tx * TX + i;
                    if (x2 >= g.lo[2] + n2) break;
                    const C gx = Gm[mode_index(g, x0, x1, x2)];
#pragma unroll
                    for (int j = 0; j < TX; ++j) {
                        const int y2 = g.lo[2] + ty * TX + j;
                        if (y2 >= g.lo[2] + n2) break;
                        const C gxy = cmul2(gx, Gm[mode_index(g, y0, y1, y2)]);
                        dq[i + j].x = fma(wq[i][j], gxy.x, dq[i + j].x);
                        dq[i + j].y = fma(wq[i][j], gxy.y, dq[i + j].y);
                        dr[i + j].x = fma(wr[i][j], gxy.x, dr[i + j].x);
                        dr[i + j].y = fma(wr[i][j], gxy.y, dr[i + j].y);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 2 * TX - 1; ++i) {
                mypart[2 * i] = dq[i];
                mypart[2 * i + 1] = dr[i];
            }
        }
        __syncthreads();
        // fixed-order reduction over the unwrapped index u = x2 + y2 - 2 lo2 (0 .. 2 n2 - 2): LINEAR
        // t2 = 2 lo2 + u; CIRCULAR t2 = <2 lo2 + u>, i.e. u = (ti - lo2) mod n2 and that + n2
        for (int ti = threadIdx.x; ti < nT2; ti += blockDim.x) {
            double qx = 0, qy = 0, rx = 0, ry = 0;
            const int ubase = g.wrap ? ((ti - g.lo[2]) % n2 + n2) % n2 : ti;
            for (int sp = 0; sp < PPC; ++sp) {
                if (pb + sp >= npairs) break;
                for (int fold = 0; fold < (g.wrap ? 2 : 1); ++fold) {
                    const int u = ubase + fold * n2;
                    if (u > 2 * n2 - 2) continue;
                    for (int txx = 0; txx < TN; ++txx)
                        for (int dl = 0; dl < 2 * TX - 1; ++dl) {
                            const int rem = u - dl - txx * TX;
                            if (rem < 0 || rem % TX) continue;
                            const int tyy = rem / TX;
                            if (tyy >= TN) continue;
                            const C* pp = part + ((size_t)(sp * tpp + tyy * TN + txx)) * (2 * TX - 1) * 2;
                            qx += (double)pp[2 * dl].x;
                            qy += (double)pp[2 * dl].y;
                            rx += (double)pp[2 * dl + 1].x;
                            ry += (double)pp[2 * dl + 1].y;
                        }
                }
            }
            accQ[ti].x += qx; accQ[ti].y += qy;
            accS[ti].x += rx; accS[ti].y += ry;
        }
    }
    __syncthreads();
    // write the row: quad for t in I_N, S over the t box
    const bool qrow = g.wrap || (t0 >= g.lo[0] && t0 < g.lo[0] + g.n[0] && t1 >= g.lo[1] && t1 < g.lo[1] + g.n[1]);
    for (int ti = threadIdx.x; ti < nT2; ti += blockDim.x) {
        const int t2 = A.tlo[2] + ti;
        if (qrow && t2 >= g.lo[2] && t2 < g.lo[2] + n2) A.quad[mode_index(g, t0, t1, t2)] = accQ[ti];
        if (A.cubic) A.S[((size_t)blockIdx.x) * nT2 + ti] = accS[ti];
    }
}

// quad and S from stored weight tables: CTA per t-row (t_0, t_1); its threads form groups of
// 64, thread u of a group owns the output t_2 = tlo_2 + u and walks the pairs (x_0, x_1) of its
// group and, for each, x_2 with y_2 = t_2 - x_2 in I_N (reduced in CIRCULAR mode): the table row
// x is read along y_2, so a warp reads consecutive entries.  The group sums meet in a fixed order.
template <typename Real>
__global__ void __launch_bounds__(256) k_pairw_nd(NdGeo g, const Real* __restrict__ Wq, const Real* __restrict__ Wr,
                                                  const void* __restrict__ Gv, double2* __restrict__ quad,
                                                  double2* __restrict__ S, int cubic, int nt1, int nT2, int tlo0,
                                                  int tlo1, int tlo2) {
    using C = typename CT<Real>::C;
    __shared__ double2 red[4][2][96];
    const C* G = reinterpret_cast<const C*>(Gv);
    const int t0 = tlo0 + (int)blockIdx.x / nt1, t1 = tlo1 + (int)blockIdx.x % nt1;
    const int grp = threadIdx.x >> 6, u = threadIdx.x & 63;
    const int ngrp = blockDim.x >> 6;
    const size_t nm = (size_t)g.n[0] * g.n[1] * g.n[2];
    int xlo[2], xn[2];
    for (int x = 0; x < 2; ++x) {
        const int lo = g.lo[x], hi = g.lo[x] + g.n[x] - 1, t = x == 0 ? t0 : t1;
        if (g.wrap) { xlo[x] = lo; xn[x] = g.n[x]; }
        else { xlo[x] = max(lo, t - hi); xn[x] = min(hi, t - lo) - xlo[x] + 1; }
    }
    const int n2 = g.n[2], lo2 = g.lo[2];
    for (int half = 0; half < 2; ++half) {   // t_2 indices u and u + 64 (nT2 <= 127)
        const int ti = u + 64 * half;
        double qx = 0, qy = 0, rx = 0, ry = 0;
        if (ti < nT2) {
            const int t2 = tlo2 + ti;
            for (int pi = grp; pi < xn[0] * xn[1]; pi += ngrp) {
                const int x0 = xlo[0] + pi / xn[1], x1 = xlo[1] + pi % xn[1];
                int y0 = t0 - x0, y1 = t1 - x1;
                if (g.wrap) { y0 = red_mod(y0, g.lo[0], g.n[0]); y1 = red_mod(y1, g.lo[1], g.n[1]); }
                const size_t xrow = (size_t)mode_index(g, x0, x1, lo2);
                const size_t yrow = (size_t)mode_index(g, y0, y1, lo2);
                float sqx = 0.f, sqy = 0.f, srx = 0.f, sry = 0.f;   // FP32 pair sums (FP64 for Real = double below)
                double dqx = 0, dqy = 0, drx = 0, dry = 0;
                for (int x2 = lo2; x2 < lo2 + n2; ++x2) {
                    int y2 = t2 - x2;
                    if (g.wrap) y2 = red_mod(y2, lo2, n2);
                    else if (y2 < lo2 || y2 >= lo2 + n2) continue;
                    const size_t xi = xrow + (x2 - lo2), yi = yrow + (y2 - lo2);
                    const C gx = G[xi], gy = G[yi];
                    const C gxy = cmul2(gx, gy);
                    const size_t o = xi * nm + yi;
                    const Real wq = Wq[o];
                    if constexpr (sizeof(Real) == 4) {
                        sqx = fmaf(wq, gxy.x, sqx);
                        sqy = fmaf(wq, gxy.y, sqy);
                        if (cubic) {
                            const float wr = Wr[o];
                            srx = fmaf(wr, gxy.x, srx);
                            sry = fmaf(wr, gxy.y, sry);
                        }
                    } else {
                        dqx = fma(wq, gxy.x, dqx);
                        dqy = fma(wq, gxy.y, dqy);
                        if (cubic) {
                            const double wr = Wr[o];
                            drx = fma(wr, gxy.x, drx);
                            dry = fma(wr, gxy.y, dry);
                        }
                    }
                }
                qx += (double)sqx + dqx; qy += (double)sqy + dqy;
                rx += (double)srx + drx; ry += (double)sry + dry;
            }
        }
        if (ti < 96) {
            red[grp][0][ti] = make_double2(qx, qy);
            red[grp][1][ti] = make_double2(rx, ry);
        }
    }
    __syncthreads();
    const bool qrow = g.wrap || (t0 >= g.lo[0] && t0 < g.lo[0] + g.n[0] && t1 >= g.lo[1] && t1 < g.lo[1] + g.n[1]);
    for (int ti = threadIdx.x; ti < nT2; ti += blockDim.x) {
        double qx = 0, qy = 0, rx = 0, ry = 0;
        for (int k = 0; k < ngrp; ++k) {
            qx += red[k][0][ti].x; qy += red[k][0][ti].y;
            rx += red[k][1][ti].x; ry += red[k][1][ti].y;
        }
        const int t2 = tlo2 + ti;
        if (qrow && t2 >= g.lo[2] && t2 < g.lo[2] + n2) quad[mode_index(g, t0, t1, t2)] = make_double2(qx, qy);
        if (cubic) S[(size_t)blockIdx.x * nT2 + ti] = make_double2(rx, ry);
    }
}

// ------------------------------------------------------------------ partial sums and combination
template <typename Real>
__global__ void k_sum_partials_nd(int nm, int nPart, const void* __restrict__ partials, double2* __restrict__ q1q) {
    if constexpr (sizeof(Real) == 4) {
        sum_partials_f32_block(nm, nPart, reinterpret_cast<const float4*>(partials), q1q, blockIdx.x);
    } else {
        const double2* pp = reinterpret_cast<const double2*>(partials);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nm; i += gridDim.x * blockDim.x) {
            double x = 0, y = 0;
            for (int c = 0; c < nPart; ++c) {
                const double2 v = pp[(size_t)c * nm + i];
                x += v.x;
                y += v.y;
            }
            q1q[i] = make_double2(x, y);
        }
    }
}

// Q^(n) = quad(n) + eps (q1q(n) + red(n)), red(n) = sum_{k in I_N} G^_k S(n - k): CTA per output
// row (n0, n1); warp w takes the k rows (k0, k1) with index = w mod warps, lane the outputs n2.
__global__ void __launch_bounds__(256) k_red_combine_nd(NdGeo g, double eps, int cubic, const double2* __restrict__ G,
                                                        const double2* __restrict__ quad, const double2* __restrict__ q1q,
                                                        const double2* __restrict__ S, int nt0, int nt1, int nt2, int tlo0,
                                                        int tlo1, int tlo2, int plane_lo, int plane_hi,
                                                        double2* __restrict__ Qhat) {
    __shared__ double2 red[8][64];
    const int n0 = g.lo[0] + (int)blockIdx.x / g.n[1], n1 = g.lo[1] + (int)blockIdx.x % g.n[1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int n2c = g.n[2];
    double2 acc[2] = {make_double2(0, 0), make_double2(0, 0)};
    if (cubic) {
        const int nrows = g.n[0] * g.n[1];
        for (int kr = warp; kr < nrows; kr += nw) {
            const int k0 = g.lo[0] + kr / g.n[1], k1 = g.lo[1] + kr % g.n[1];
            int u0 = n0 - k0, u1 = n1 - k1;
            if (g.wrap) { u0 = red_mod(u0, g.lo[0], g.n[0]); u1 = red_mod(u1, g.lo[1], g.n[1]); }
            const int r0 = u0 - tlo0, r1 = u1 - tlo1;
            if (!g.wrap && (r0 < 0 || r1 < 0 || r0 >= nt0 || r1 >= nt1)) continue;
            const double2* Srow = S + ((size_t)r0 * nt1 + r1) * nt2;
            const double2* Grow = G + (size_t)mode_index(g, k0, k1, g.lo[2]);
            for (int k2i = 0; k2i < n2c; ++k2i) {
                const double2 gk = Grow[k2i];
                const int k2 = g.lo[2] + k2i;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int n2i = lane + 32 * h;
                    if (n2i >= n2c) break;
                    int u2 = g.lo[2] + n2i - k2;
                    if (g.wrap) u2 = red_mod(u2, g.lo[2], g.n[2]);
                    const int r2 = u2 - tlo2;
                    if (r2 < 0 || r2 >= nt2) continue;
                    const double2 sv = Srow[r2];
                    acc[h].x = fma(gk.x, sv.x, fma(-gk.y, sv.y, acc[h].x));
                    acc[h].y = fma(gk.x, sv.y, fma(gk.y, sv.x, acc[h].y));
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (lane + 32 * h < 64) red[warp][lane + 32 * h] = acc[h];
    __syncthreads();
    for (int n2i = threadIdx.x; n2i < n2c; n2i += blockDim.x) {
        double rx = 0, ry = 0;
        for (int w = 0; w < nw; ++w) { rx += red[w][n2i].x; ry += red[w][n2i].y; }
        const int m = mode_index(g, n0, n1, g.lo[2] + n2i);
        double2 q = quad[m];
        if (cubic) {
            q.x += eps * (q1q[m].x + rx);
            q.y += eps * (q1q[m].y + ry);
        }
        // a shard writes its own output planes n_0 only
        const bool mine = n0 - g.lo[0] >= plane_lo && n0 - g.lo[0] < plane_hi;
        Qhat[m] = mine ? q : make_double2(0.0, 0.0);
    }
}

// I_N restriction of an extended-box alpha table and FP32 copies
template <typename Real>
__global__ void k_alpha_restrict(NdGeo g, int P, const double* __restrict__ src, Real* __restrict__ dst) {
    const size_t nm = (size_t)g.n[0] * g.n[1] * g.n[2];
    const size_t nE = (size_t)(g.d == 3 ? 8 : 4) * g.N * g.N * (g.d == 3 ? g.N : 1);
    const size_t tot = (size_t)P * nm;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(i / nm), m = (int)(i % nm);
        const int a2 = m % g.n[2] + g.lo[2], r = m / g.n[2];
        const int a1 = r % g.n[1] + g.lo[1], a0 = r / g.n[1] + g.lo[0];
        dst[i] = (Real)src[(size_t)p * nE + ext_index(g, a0, a1, a2)];
    }
}
__global__ void k_to_f32(size_t n, const double* __restrict__ src, float* __restrict__ dst) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

}  // namespace

// ------------------------------------------------------------------ host plan
struct NdRound {
    size_t slice_bytes = 0;
    int ngroups = 0, nwork = 0, nitems = 0;
    NdGroup* d_groups = nullptr;
    int* d_group_b = nullptr;
    uint32_t* d_off16 = nullptr;     // per group member (same order as group_b)
    int2* d_work = nullptr;
    NdItem* d_items = nullptr;
    int* d_cta_off = nullptr;
};

struct NdPlan {
    NdGeo g{};
    int RW = 8, threads = 256, T0 = 1, nCTA = 0;
    int WS = 0, PB = 0, PS = 0, PP = 0, GP = 0, gstage = 1;
    size_t smem = 0, smem_pair = 0;
    int TXp = 4;
    int pair_threads = 256;
    int nt[3] = {1, 1, 1}, tlo[3] = {0, 0, 0};
    std::vector<NdRound> rounds;
    size_t slice_cap = 0;             // bytes of the slice buffer
    void* slices = nullptr;
    void* partials = nullptr;
    size_t partial_bytes = 0;
    double2* quad = nullptr;
    double2* S = nullptr;
    double2* q1q = nullptr;
    void* Wq = nullptr;               // pair weight tables [x][y] over I_N x I_N (when they fit)
    void* Wr = nullptr;
    size_t W_bytes = 0;
    int plane_lo = 0, plane_hi = 1 << 30;   // output planes n_0 - lo_0 of this shard
    bool resident = false;            // slices produced once and kept (single round)
    bool produced = false;
    double terms = 0;                 // Q_{1,q} terms per evaluation
    // live phase timing: per evaluation slot, events around the pair sums, each round's slice
    // production and sweep, and the tail (partial sums, reducible convolution, combination)
    static constexpr int kSlots = 4;
    std::vector<cudaEvent_t> ev;      // kSlots x (4 + 4 rounds)
    double ms[4] = {0, 0, 0, 0};      // pair, production, sweep, tail
    long long evals = 0;
    int per_slot() const { return 4 + 4 * (int)rounds.size(); }
};

namespace {

NdGeo make_geo(const bn_solver* s) {
    NdGeo g{};
    g.d = s->g.d;
    g.N = s->g.N;
    g.wrap = s->opt.wrap ? 1 : 0;
    for (int x = 0; x < 3; ++x) {
        const bool trivial = g.d == 2 && x == 0;
        g.n[x] = trivial ? 1 : g.N;
        g.lo[x] = trivial ? 0 : -g.N / 2;
        const int lo = g.lo[x], hi = lo + g.n[x] - 1;
        if (g.wrap) { g.blo[x] = lo; g.nb[x] = g.n[x]; }
        else {
            const int bl = std::max(2 * lo, lo - hi), bh = std::min(2 * hi, hi - lo);
            g.blo[x] = bl;
            g.nb[x] = bh - bl + 1;
        }
    }
    g.nbTotal = g.nb[0] * g.nb[1] * g.nb[2];
    return g;
}

// c-class of b per axis (LINEAR): boxes A(b) of equal c coincide: c = max(b + 1, -b) (b_x in the
// non-trivial axes); 0 on a trivial axis.
int cls(const NdGeo& g, int x, int b) {
    if (g.n[x] == 1) return 0;
    return std::max(b + 1, -b);
}

template <typename T>
bn_status upload(T** dst, const std::vector<T>& v, std::string* err) {
    if (v.empty()) { *dst = nullptr; return BN_OK; }
    if (cudaMalloc(dst, sizeof(T) * v.size()) != cudaSuccess ||
        cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        *err = "operator plan upload failed";
        return BN_ERR_NOMEM;
    }
    return BN_OK;
}

}  // namespace

bool use_nd(const bn_solver* s) { return s->g.d == 3 || s->opt.wrap != 0; }

size_t nd_estimate_bytes(const bn_solver* s) { return s->nd ? s->nd->slice_cap + s->nd->partial_bytes : 0; }

void free_nd(bn_solver* s) {
    NdPlan* p = s->nd;
    if (!p) return;
    for (NdRound& r : p->rounds) {
        cudaFree(r.d_groups); cudaFree(r.d_group_b); cudaFree(r.d_off16); cudaFree(r.d_work);
        cudaFree(r.d_items); cudaFree(r.d_cta_off);
    }
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    cudaFree(p->slices);
    cudaFree(p->partials);
    cudaFree(p->Wq);
    cudaFree(p->Wr);
    cudaFree(p->quad);
    cudaFree(p->S);
    cudaFree(p->q1q);
    delete p;
    s->nd = nullptr;
}

template <typename Real>
static void configure_triple_nd(size_t smem) {
    cudaFuncSetAttribute(k_triple_nd<Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_triple_nd<Real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename Real, int TX>
static void configure_pair_nd(size_t smem) {
    cudaFuncSetAttribute(k_pair_nd<Real, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Output planes n_0 (as indices 0 .. n_0 - 1) of `count` shards of one evaluation: contiguous
// ranges with nearly equal Q_{1,q} terms.  The terms of plane n_0 are w(n_0) = sum over b_0 with
// n_0 in box_n(b_0) of |box_s(b_0)| (times the same factor for every plane), i.e. the number of
// (k_0, l_0, m_0) in I^3 with k_0 + l_0 + m_0 = n_0 (LINEAR; every plane alike in CIRCULAR).
std::vector<int> shard_bounds(const NdGeo& g, int count) {
    const int n0 = g.n[0];
    std::vector<double> w(n0, 0.0);
    for (int b0 = g.blo[0]; b0 < g.blo[0] + g.nb[0]; ++b0) {
        const int bb[3] = {b0, 0, 0};
        Box3 B;
        box_of(g, bb, B);
        for (int i = 0; i < B.L[0]; ++i) w[B.nlo[0] + i - g.lo[0]] += B.S[0];
    }
    double total = 0;
    for (double x : w) total += x;
    std::vector<int> bounds(count + 1, n0);
    bounds[0] = 0;
    double acc = 0;
    int k = 1;
    for (int i = 0; i < n0 && k < count; ++i) {
        acc += w[i];
        // close shard k-1 after the plane that brings it nearest to its share
        if (acc >= total * k / count - 0.5 * w[i]) bounds[k++] = i + 1;
    }
    for (; k < count; ++k) bounds[k] = n0;
    for (int i = 1; i <= count; ++i) bounds[i] = std::max(bounds[i], bounds[i - 1]);
    return bounds;
}

std::vector<int> shard_bounds_for(int d, int N, int wrap, int count) {
    bn_solver tmp;
    tmp.g.d = d;
    tmp.g.N = N;
    tmp.opt.wrap = wrap;
    return shard_bounds(make_geo(&tmp), count);
}

// Work split of the boxes of one b (host): outputs per thread along axis 2 (RW), output planes per
// item (T0), output rows per tile (L1t) and lanes per task splitting the s_1 range (J), chosen to
// minimise a per-thread time model of the sweep: per item and tile, (T0 + S0 - 1) plane steps of
// ceil(S1 / J) rows of S2 steps of RW paired multiply-adds, plus per-row, per-plane and per-item
// overheads (instruction counts of the kernel's row setup, plane barrier and item setup).
struct ItemShape { int RW, T0, J, L1t; };
constexpr long long kRowOvh = 24, kPlaneOvh = 200, kTileOvh = 1500;
static long long shape_cost(const Box3& B, int T0, const ItemShape& sh) {
    const long long ntile = (B.L[1] + sh.L1t - 1) / sh.L1t;
    const long long rows = (B.S[1] + sh.J - 1) / sh.J;
    return ntile * ((T0 + B.S[0] - 1) * (rows * ((long long)B.S[2] * sh.RW + kRowOvh) + kPlaneOvh) + kTileOvh);
}
static ItemShape choose_shape(const Box3& B, bool fp32, int T0max, int nthr) {
    ItemShape best{fp32 ? 8 : 4, 1, 1, 1};
    long long bestc = -1;
    const int rws[2] = {8, 4};
    for (int ri = fp32 ? 0 : 1; ri < 2; ++ri) {
        const int RW = rws[ri];
        const int G2 = (B.L[2] + RW - 1) / RW;
        for (int T0 = 1; T0 <= std::min(T0max, B.L[0]); ++T0)
            for (int J = 1; J <= 8 && J <= B.S[1]; J *= 2) {
                const int maxL1 = nthr / (T0 * G2 * J);
                if (maxL1 < 1) continue;
                const int ntile = (B.L[1] + maxL1 - 1) / maxL1;
                const ItemShape sh{RW, T0, J, (B.L[1] + ntile - 1) / ntile};
                const long long c = ((B.L[0] + T0 - 1) / T0) * shape_cost(B, T0, sh);
                if (bestc < 0 || c < bestc) { bestc = c; best = sh; }
            }
    }
    return best;
}

bn_status plan_nd(bn_solver* s, std::string* err) {
    NdPlan* p = new NdPlan();
    s->nd = p;
    NdGeo& g = p->g;
    g = make_geo(s);
    const bool fp32 = s->opt.precision == BN_MIXED;
    const int elem = fp32 ? 4 : 8;
    const int N = g.N;
    if (s->opt.shard_count > 1) {
        const std::vector<int> bd = shard_bounds(g, s->opt.shard_count);
        p->plane_lo = bd[s->opt.shard_index];
        p->plane_hi = bd[s->opt.shard_index + 1];
    } else {
        p->plane_lo = 0;
        p->plane_hi = g.n[0];
    }
    // 256 threads per CTA; per box, outputs per thread along axis 2 (RW = 8 or 4 in FP32, 4 in
    // FP64), planes per item (T0 <= T0max) and s_1 split (J) are chosen on the host below
    p->RW = fp32 ? 8 : 4;                    // the widest RW (sizes the staged row slack)
    const int RW = p->RW;
    // T0max: the P-plane ring holds T0max + 1 planes; at N <= 32 four output planes share a staged
    // slice plane (sweep per N=32 evaluation: T0max 3, 4, 6 -> 1488, 1450, 1469 ms); at N = 48 a
    // second P plane would leave one CTA per SM
    p->T0 = N > 32 ? 1 : 4;
    p->threads = 256;
    // largest slice plane and P plane; staged rows at odd strides (distinct banks for the rows a
    // warp sweeps)
    int maxA1 = 1, maxA2 = 1, maxS1 = 1, maxS2 = 1;
    for (int x = 1; x < 3; ++x) {
        const int Amax = g.wrap ? 2 * g.n[x] - 1 : (g.n[x] == 1 ? 1 : 2 * N - 2);
        const int Smax = g.n[x];   // box_s(b) spans all of I_x at b = -1 (LINEAR) and always (CIRCULAR)
        if (x == 1) { maxA1 = Amax; maxS1 = Smax; }
        else { maxA2 = Amax; maxS2 = Smax; }
    }
    p->WS = (maxA2 + RW - 1) | 1;
    p->PB = maxA1 * p->WS + RW;
    p->PS = maxS2 | 1;
    p->PP = maxS1 * p->PS;
    p->GP = g.n[0] > 1 ? g.n[1] * g.n[2] : 0;
    const size_t Csz = 2 * (size_t)elem;
    // shared memory with and without the staged mode planes (two slots of two planes).  The staging
    // is dropped only when it leaves a single CTA per SM and dropping it admits a second: the P
    // planes are then built from the L2-resident modes, on the critical path of each plane step
    // (measured on the FP32 sweep: N=48, 1 -> 2 CTAs per SM, 68.5 -> 54.7 s per evaluation; N=32,
    // where both forms hold 2 CTAs per SM, 1488 ms with the staging against 1533 ms without)
    const size_t base = (size_t)(p->T0 + 1) * p->PP * Csz + 2 * (size_t)p->PB * elem;
    auto round16 = [](size_t b) { return (b + 15) / 16 * 16 + 16; };
    const size_t with_g = round16(4 * (size_t)p->GP * Csz + base), without_g = round16(base);
    if (without_g > 227 * 1024) {
        *err = "the 3-D kernel's staging does not fit in shared memory";
        return BN_ERR_UNSUPPORTED;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (sms <= 0) sms = 152;
    auto occupancy = [&](size_t smem, bool gs) {
        if (smem > 227 * 1024) return 0;
        int n = 0;
        if (fp32) {
            configure_triple_nd<float>(smem);
            if (gs) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_triple_nd<float, true>, p->threads, smem);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_triple_nd<float, false>, p->threads, smem);
        } else {
            configure_triple_nd<double>(smem);
            if (gs) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_triple_nd<double, true>, p->threads, smem);
            else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_triple_nd<double, false>, p->threads, smem);
        }
        cudaGetLastError();
        return n;
    };
    const int occ_g = p->GP > 0 ? occupancy(with_g, true) : 0, occ_ng = occupancy(without_g, false);
    p->gstage = p->GP > 0 && (occ_g >= occ_ng || occ_g >= 2) ? 1 : 0;
    p->smem = p->gstage ? with_g : without_g;
    if (fp32) configure_triple_nd<float>(p->smem);
    else configure_triple_nd<double>(p->smem);
    int per_sm = std::max(1, p->gstage ? occ_g : occ_ng);
    p->nCTA = per_sm * sms;

    // b list and groups
    std::vector<std::vector<int>> members;
    std::vector<NdGroup> groups;
    {
        std::vector<std::pair<long long, int>> keyed;
        keyed.reserve(g.nbTotal);
        const int W2 = g.d == 3 ? 8 : 16;   // c_2 band width: 2 x 2 x 2 x 8 = 64 b per group in 3-D
        for (int f = 0; f < g.nbTotal; ++f) {
            int b[3];
            b_of_flat(g, f, b);
            long long key;
            if (g.wrap) key = f / kMaxGroup;
            else key = ((long long)cls(g, 0, b[0]) * 4096 + cls(g, 1, b[1])) * 4096 + (cls(g, 2, b[2]) - 1) / W2;
            keyed.push_back({key, f});
        }
        std::stable_sort(keyed.begin(), keyed.end());
        size_t i = 0;
        while (i < keyed.size()) {
            size_t j = i;
            std::vector<int> mem;
            while (j < keyed.size() && keyed[j].first == keyed[i].first && mem.size() < (size_t)kMaxGroup) {
                mem.push_back(keyed[j].second);
                ++j;
            }
            NdGroup G{};
            int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
            for (int f : mem) {
                int b[3];
                b_of_flat(g, f, b);
                Box3 B;
                box_of(g, b, B);
                for (int x = 0; x < 3; ++x) {
                    lo[x] = std::min(lo[x], B.alo[x]);
                    hi[x] = std::max(hi[x], B.alo[x] + B.A[x] - 1);
                }
            }
            for (int x = 0; x < 3; ++x) { G.ulo[x] = lo[x]; G.uA[x] = hi[x] - lo[x] + 1; }
            G.nb = (int)mem.size();
            groups.push_back(G);
            members.push_back(mem);
            i = j;
        }
    }
    // slice bytes per b
    auto slice_bytes = [&](int f) {
        int b[3];
        b_of_flat(g, f, b);
        Box3 B;
        box_of(g, b, B);
        return (size_t)B.A[0] * B.A[1] * slice_rs(B.A[2], elem) * elem;
    };
    size_t total = 0;
    for (auto& mem : members)
        for (int f : mem) total += (slice_bytes(f) + 15) / 16 * 16;
    // pair weight tables wq, wr over I_N x I_N: formed once when they fit in 45% of the free memory
    // (8.6 GB FP32 at 3-D N = 32), else recomputed from the alpha tables at every evaluation
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    cudaGetLastError();
    {
        const size_t nmS = (size_t)g.n[0] * g.n[1] * g.n[2];
        const size_t one = nmS * nmS * (size_t)elem;
        const size_t need = one * (s->eps != 0.0 ? 2 : 1);
        if (s->opt.pair_weights == 0 && need <= (size_t)(0.45 * (double)freeb)) {
            cudaError_t e1 = cudaMalloc(&p->Wq, one);
            if (e1 == cudaSuccess && s->eps != 0.0) e1 = cudaMalloc(&p->Wr, one);
            if (e1 != cudaSuccess) {
                cudaGetLastError();
                cudaFree(p->Wq);
                cudaFree(p->Wr);
                p->Wq = p->Wr = nullptr;
            } else {
                p->W_bytes = need;
                freeb = freeb > need ? freeb - need : 0;
            }
        }
    }
    // slice buffer: everything when it fits the budget (then produced once if resident), else rounds
    size_t budget = s->opt.beta_budget_mb > 0 ? (size_t)s->opt.beta_budget_mb << 20
                                              : std::min<size_t>((size_t)(0.4 * (double)freeb), (size_t)40 << 30);
    budget = std::max<size_t>(budget, (size_t)64 << 20);
    // every group must fit on its own
    size_t maxGroup = 0;
    for (auto& mem : members) {
        size_t gb = 0;
        for (int f : mem) gb += (slice_bytes(f) + 15) / 16 * 16;
        maxGroup = std::max(maxGroup, gb);
    }
    budget = std::max(budget, maxGroup);
    // rounds: groups in order, largest groups first
    std::vector<int> gorder(groups.size());
    std::iota(gorder.begin(), gorder.end(), 0);
    {
        std::vector<size_t> gbytes(groups.size(), 0);
        for (size_t k = 0; k < groups.size(); ++k)
            for (int f : members[k]) gbytes[k] += (slice_bytes(f) + 15) / 16 * 16;
        std::stable_sort(gorder.begin(), gorder.end(), [&](int a, int c) { return gbytes[a] > gbytes[c]; });
        std::vector<std::vector<int>> rgroups(1);
        size_t used = 0;
        for (int k : gorder) {
            if (used + gbytes[k] > budget && !rgroups.back().empty()) {
                rgroups.emplace_back();
                used = 0;
            }
            rgroups.back().push_back(k);
            used += gbytes[k];
        }
        p->slice_cap = 0;
        for (auto& rg : rgroups) {
            size_t u = 0;
            for (int k : rg) u += gbytes[k];
            p->slice_cap = std::max(p->slice_cap, u);
        }
        p->resident = rgroups.size() == 1 && s->opt.beta_resident != 0;
        // per round: groups, members with offsets, producer work, items dealt to CTAs
        const int T0 = p->T0;
        for (auto& rg : rgroups) {
            NdRound R;
            std::vector<NdGroup> rgs;
            std::vector<int> gb;
            std::vector<uint32_t> off;
            std::vector<int2> work;
            struct It { long long cost; NdItem it; };
            std::vector<It> items;
            size_t cur = 0;
            for (int k : rg) {
                NdGroup G = groups[k];
                G.first = (int)gb.size();
                const int gi = (int)rgs.size();
                for (int f : members[k]) {
                    gb.push_back(f);
                    off.push_back((uint32_t)(cur / 16));
                    int b[3];
                    b_of_flat(g, f, b);
                    Box3 B;
                    box_of(g, b, B);
                    const ItemShape sh = choose_shape(B, fp32, T0, p->threads);
                    // output planes of this shard inside box_n(b) along axis 0
                    const int tb = std::max(0, p->plane_lo + g.lo[0] - B.nlo[0]);
                    const int te = std::min(B.L[0], p->plane_hi + g.lo[0] - B.nlo[0]);
                    for (int t = tb; t < te; t += sh.T0) {
                        const int tn = std::min(sh.T0, te - t);
                        NdItem it{};
                        it.bflat = (uint32_t)f;
                        it.t0i = (uint8_t)t;
                        it.T0 = (uint8_t)tn;
                        it.L1t = (uint8_t)sh.L1t;
                        it.J = (uint8_t)sh.J;
                        it.RW = (uint8_t)sh.RW;
                        it.off16 = (uint32_t)(cur / 16);
                        const long long terms = (long long)tn * B.L[1] * B.L[2] * B.S[0] * B.S[1] * B.S[2];
                        items.push_back({shape_cost(B, tn, sh), it});
                        p->terms += (double)terms;
                    }
                    cur += (slice_bytes(f) + 15) / 16 * 16;
                }
                const int uTot = G.uA[0] * G.uA[1] * G.uA[2];
                for (int t = 0; t * kPA < uTot; ++t) work.push_back(make_int2(gi, t));
                rgs.push_back(G);
            }
            // deal items: by cost descending, snake order over the CTAs
            std::stable_sort(items.begin(), items.end(), [](const It& a, const It& c) { return a.cost > c.cost; });
            std::vector<std::vector<NdItem>> per(p->nCTA);
            std::vector<long long> load(p->nCTA, 0);
            for (size_t q = 0; q < items.size(); ++q) {
                const size_t rr = q / p->nCTA, c = q % p->nCTA;
                const size_t cta = (rr & 1) ? p->nCTA - 1 - c : c;
                per[cta].push_back(items[q].it);
                load[cta] += items[q].cost;
            }
            std::vector<NdItem> flat;
            std::vector<int> ctaoff(p->nCTA + 1, 0);
            for (int c = 0; c < p->nCTA; ++c) {
                ctaoff[c] = (int)flat.size();
                flat.insert(flat.end(), per[c].begin(), per[c].end());
            }
            ctaoff[p->nCTA] = (int)flat.size();
            R.slice_bytes = cur;
            R.ngroups = (int)rgs.size();
            R.nwork = (int)work.size();
            R.nitems = (int)flat.size();
            bn_status st = upload(&R.d_groups, rgs, err);
            if (st == BN_OK) st = upload(&R.d_group_b, gb, err);
            if (st == BN_OK) st = upload(&R.d_off16, off, err);
            if (st == BN_OK) st = upload(&R.d_work, work, err);
            if (st == BN_OK) st = upload(&R.d_items, flat, err);
            if (st == BN_OK) st = upload(&R.d_cta_off, ctaoff, err);
            p->rounds.push_back(R);
            if (st != BN_OK) return st;
        }
    }
    if (s->eps == 0.0) p->terms = 0;
    // quadratic and reducible sums
    for (int x = 0; x < 3; ++x) {
        if (g.wrap) { p->nt[x] = g.n[x]; p->tlo[x] = g.lo[x]; }
        else { p->nt[x] = 2 * g.n[x] - 1; p->tlo[x] = 2 * g.lo[x]; }
    }
    p->TXp = g.n[2] > 32 && fp32 ? 6 : 4;
    {
        const int TN = (g.n[2] + p->TXp - 1) / p->TXp, tpp = TN * TN;
        if (tpp > 256) {
            *err = "operator size beyond the pair kernel's thread limit";
            return BN_ERR_UNSUPPORTED;
        }
        // pairs per CTA: enough threads to fill 256, at most 8 pairs
        const int PPC = std::max(1, std::min(256 / tpp, 8));
        p->pair_threads = PPC * tpp;
        const int W = 2 * g.n[2] - 1;
        p->smem_pair = (size_t)PPC * 4 * 8 * g.n[2] * elem + 2 * 8 * (size_t)W * elem +
                       (size_t)PPC * tpp * (2 * p->TXp - 1) * 2 * Csz + 2 * (size_t)p->nt[2] * sizeof(double2) + 64;
        if (fp32) {
            if (p->TXp == 4) configure_pair_nd<float, 4>(p->smem_pair);
            else configure_pair_nd<float, 6>(p->smem_pair);
        } else {
            configure_pair_nd<double, 4>(p->smem_pair);
        }
    }
    const size_t nm = (size_t)s->g.nModes;
    const size_t nS = (size_t)p->nt[0] * p->nt[1] * p->nt[2];
    p->partial_bytes = (size_t)p->nCTA * nm * 16;
    cudaError_t e = cudaMalloc(&p->slices, std::max<size_t>(p->slice_cap, 16) + 64);
    if (e == cudaSuccess) e = cudaMalloc(&p->partials, p->partial_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&p->quad, nm * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->S, std::max<size_t>(nS, 1) * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->q1q, nm * sizeof(double2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("3-D operator buffers: ") + cudaGetErrorString(e);
        return BN_ERR_NOMEM;
    }
    cudaMemsetAsync(p->S, 0, std::max<size_t>(nS, 1) * sizeof(double2), s->stream);
    cudaMemsetAsync(p->q1q, 0, nm * sizeof(double2), s->stream);
    return BN_OK;
}

// Build the FP32 copies and the I_N restrictions of the alpha tables (once per table set).
bn_status build_nd_tables(bn_solver* s, KernelTables* t, std::string* err) {
    NdGeo g = make_geo(s);
    g.wrap = 0;
    const size_t nE = (size_t)s->g.nExt, nm = (size_t)s->g.nModes, P = (size_t)t->P;
    cudaError_t e = cudaMalloc(&t->alpha32, sizeof(float) * P * nE);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphap32, sizeof(float) * P * nE);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphaI64, sizeof(double) * P * nm);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphapI64, sizeof(double) * P * nm);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphaI32, sizeof(float) * P * nm);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphapI32, sizeof(float) * P * nm);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("alpha table copies: ") + cudaGetErrorString(e);
        return BN_ERR_NOMEM;
    }
    t->bytes += (sizeof(float) * 2) * P * nE + (sizeof(double) + sizeof(float)) * 2 * P * nm;
    k_to_f32<<<2048, 256, 0, s->stream>>>(P * nE, t->alpha64, t->alpha32);
    k_to_f32<<<2048, 256, 0, s->stream>>>(P * nE, t->alphap64, t->alphap32);
    k_alpha_restrict<double><<<1024, 256, 0, s->stream>>>(g, (int)P, t->alpha64, t->alphaI64);
    k_alpha_restrict<double><<<1024, 256, 0, s->stream>>>(g, (int)P, t->alphap64, t->alphapI64);
    k_alpha_restrict<float><<<1024, 256, 0, s->stream>>>(g, (int)P, t->alpha64, t->alphaI32);
    k_alpha_restrict<float><<<1024, 256, 0, s->stream>>>(g, (int)P, t->alphap64, t->alphapI32);
    s->launches += 6;
    return BN_OK;
}

// The whole operator from s->Ghat (and s->Ghat32) into s->Qhat.
template <typename Real>
static void launch_nd_t(bn_solver* s, cudaStream_t st, int slot) {
    NdPlan* p = s->nd;
    unsigned long long* stamps = nullptr;
    cudaEvent_t* ev = (slot >= 0 && slot < NdPlan::kSlots && (int)p->ev.size() == NdPlan::kSlots * p->per_slot())
                          ? p->ev.data() + (size_t)slot * p->per_slot()
                          : nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (ev) cudaStreamIsCapturing(st, &cap);
    auto mark = [&](int i) {
        // inside a stream capture the record must be an external event node to be timeable
        if (ev) cudaEventRecordWithFlags(ev[i], st, cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0);
    };
    const NdGeo& g = p->g;
    const KernelTables* t = s->tabs;
    const size_t nm = (size_t)s->g.nModes;
    const bool fp32 = sizeof(Real) == 4;
    const void* G = fp32 ? (const void*)s->Ghat32 : (const void*)s->Ghat;
    const int cubic = s->eps != 0.0;
    // quadratic and reducible sums
    PairNdArgs PA;
    PA.g = g;
    PA.P = t->P;
    PA.alphaI = fp32 ? (const void*)t->alphaI32 : (const void*)t->alphaI64;
    PA.alphapI = fp32 ? (const void*)t->alphapI32 : (const void*)t->alphapI64;
    PA.alphaE = fp32 ? (const void*)t->alpha32 : (const void*)t->alpha64;
    PA.alphapE = fp32 ? (const void*)t->alphap32 : (const void*)t->alphap64;
    PA.G = G;
    PA.quad = p->quad;
    PA.S = p->S;
    PA.cubic = cubic;
    PA.Wq = PA.Wr = nullptr;
    for (int x = 0; x < 3; ++x) { PA.nt[x] = p->nt[x]; PA.tlo[x] = p->tlo[x]; }
    // LINEAR without the cubic part needs only the t rows inside I_N, but the kernel is cheap
    const int nrows = p->nt[0] * p->nt[1];
    const int pthreads = p->pair_threads;
    mark(0);
    if (p->Wq) {
        k_pairw_nd<Real><<<nrows, 256, 0, st>>>(g, (const Real*)p->Wq, (const Real*)p->Wr, G, p->quad, p->S, cubic,
                                                p->nt[1], p->nt[2], p->tlo[0], p->tlo[1], p->tlo[2]);
    } else
    if constexpr (sizeof(Real) == 4) {
        if (p->TXp == 6) k_pair_nd<Real, 6><<<nrows, pthreads, p->smem_pair, st>>>(PA);
        else k_pair_nd<Real, 4><<<nrows, pthreads, p->smem_pair, st>>>(PA);
    } else {
        k_pair_nd<Real, 4><<<nrows, pthreads, p->smem_pair, st>>>(PA);
    }
    PA.Wq = PA.Wr = nullptr;
    s->launches++;
    mark(1);
    if (cubic) {
        cudaMemsetAsync(p->partials, 0, p->partial_bytes, st);
        for (size_t r = 0; r < p->rounds.size(); ++r) {
            const NdRound& R = p->rounds[r];
            mark(4 + 4 * (int)r);
            if (!(p->resident && p->produced)) {
                k_beta_slices<Real><<<R.nwork, 256, 0, st>>>(g, t->P, fp32 ? (const Real*)t->alpha32 : (const Real*)t->alpha64,
                                                             fp32 ? (const Real*)t->alphap32 : (const Real*)t->alphap64,
                                                             R.d_groups, R.d_group_b, R.d_off16, R.d_work, (Real*)p->slices);
                s->launches++;
            }
            mark(5 + 4 * (int)r);
            mark(6 + 4 * (int)r);
            TripleNdArgs TA;
            TA.g = g;
            TA.G = G;
            TA.items = R.d_items;
            TA.cta_off = R.d_cta_off;
            TA.slices = p->slices;
            TA.partials = p->partials;
            TA.err = s->flags + 2;
            TA.giveup_first = s->opt.debug_wait_giveup;
            TA.WS = p->WS;
            TA.PB = p->PB;
            TA.PS = p->PS;
            TA.PP = p->PP;
            TA.GP = p->GP;
            TA.T0max = p->T0;
            TA.gstage = p->gstage;
            TA.stamps = stamps;
            if (p->gstage) k_triple_nd<Real, true><<<p->nCTA, p->threads, p->smem, st>>>(TA);
            else k_triple_nd<Real, false><<<p->nCTA, p->threads, p->smem, st>>>(TA);
            s->launches++;
            mark(7 + 4 * (int)r);
        }
        if (p->resident) p->produced = true;
        if (fp32) k_sum_partials_nd<float><<<(int)((nm + kPartModes - 1) / kPartModes), 256, 0, st>>>((int)nm, p->nCTA, p->partials, p->q1q);
        else k_sum_partials_nd<double><<<(int)std::min<size_t>((nm + 255) / 256, 4096), 256, 0, st>>>((int)nm, p->nCTA, p->partials, p->q1q);
        s->launches++;
    }
    mark(2);
    k_red_combine_nd<<<g.n[0] * g.n[1], 256, 0, st>>>(g, s->eps, cubic, s->Ghat, p->quad, p->q1q, p->S, p->nt[0], p->nt[1],
                                                       p->nt[2], p->tlo[0], p->tlo[1], p->tlo[2], p->plane_lo,
                                                       std::min(p->plane_hi, g.n[0]), s->Qhat);
    s->launches++;
    mark(3);
}

void launch_nd(bn_solver* s, int slot) {
    if (s->opt.precision == BN_MIXED) launch_nd_t<float>(s, s->stream, slot);
    else launch_nd_t<double>(s, s->stream, slot);
}

bn_status nd_profile_enable(bn_solver* s, bool on) {
    NdPlan* p = s->nd;
    if (!p) return BN_OK;
    if (on && p->ev.empty()) {
        p->ev.assign((size_t)NdPlan::kSlots * p->per_slot(), nullptr);
        for (cudaEvent_t& e : p->ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return BN_ERR_CUDA;
            }
    }
    for (double& m : p->ms) m = 0;
    p->evals = 0;
    return BN_OK;
}

// Add the phase times of the evaluation slots recorded since the last harvest (the stream has
// been synchronised).
void nd_profile_harvest(bn_solver* s, int slots) {
    NdPlan* p = s->nd;
    if (!p || p->ev.empty()) return;
    const int ps = p->per_slot();
    for (int k = 0; k < slots && k < NdPlan::kSlots; ++k) {
        cudaEvent_t* e = p->ev.data() + (size_t)k * ps;
        float a = 0, b = 0, c = 0, d = 0;
        if (cudaEventElapsedTime(&a, e[0], e[1]) != cudaSuccess) { cudaGetLastError(); continue; }
        for (size_t r = 0; r < p->rounds.size() && s->eps != 0.0; ++r) {
            float x = 0, y = 0;
            if (cudaEventElapsedTime(&x, e[4 + 4 * r], e[5 + 4 * r]) == cudaSuccess) b += x;
            else cudaGetLastError();
            if (cudaEventElapsedTime(&y, e[6 + 4 * r], e[7 + 4 * r]) == cudaSuccess) c += y;
            else cudaGetLastError();
        }
        if (cudaEventElapsedTime(&d, s->eps != 0.0 ? e[7 + 4 * (p->rounds.size() - 1)] : e[1], e[3]) != cudaSuccess) {
            cudaGetLastError();
            d = 0;
        }
        p->ms[0] += a; p->ms[1] += b; p->ms[2] += c; p->ms[3] += d;
        p->evals += 1;
    }
}

bn_status nd_profile_read(bn_solver* s, double* out, size_t count) {
    NdPlan* p = s->nd;
    if (!p || count < 8) return BN_ERR_ARG;
    for (int i = 0; i < 4; ++i) out[i] = p->ms[i];
    out[4] = (double)p->evals;
    out[5] = (double)p->rounds.size();
    out[6] = p->terms;
    out[7] = (double)p->nCTA;
    for (double& m : p->ms) m = 0;
    p->evals = 0;
    return BN_OK;
}

template <typename Real>
static void build_pair_weights(bn_solver* s) {
    NdPlan* p = s->nd;
    const KernelTables* t = s->tabs;
    const bool fp32 = sizeof(Real) == 4;
    PairNdArgs PA;
    PA.g = p->g;
    PA.P = t->P;
    PA.alphaI = fp32 ? (const void*)t->alphaI32 : (const void*)t->alphaI64;
    PA.alphapI = fp32 ? (const void*)t->alphapI32 : (const void*)t->alphapI64;
    PA.alphaE = fp32 ? (const void*)t->alpha32 : (const void*)t->alpha64;
    PA.alphapE = fp32 ? (const void*)t->alphap32 : (const void*)t->alphap64;
    PA.G = nullptr;
    PA.quad = p->quad;
    PA.S = p->S;
    PA.cubic = s->eps != 0.0;
    PA.Wq = p->Wq;
    PA.Wr = p->Wr;
    for (int x = 0; x < 3; ++x) { PA.nt[x] = p->nt[x]; PA.tlo[x] = p->tlo[x]; }
    const int nrows = p->nt[0] * p->nt[1];
    if constexpr (sizeof(Real) == 4) {
        if (p->TXp == 6) k_pair_nd<Real, 6><<<nrows, p->pair_threads, p->smem_pair, s->stream>>>(PA);
        else k_pair_nd<Real, 4><<<nrows, p->pair_threads, p->smem_pair, s->stream>>>(PA);
    } else {
        k_pair_nd<Real, 4><<<nrows, p->pair_threads, p->smem_pair, s->stream>>>(PA);
    }
    s->launches++;
}

// Form the pair weight tables (when allocated) and, in resident mode, the slices, once, outside
// any capture.
bn_status prepare_nd(bn_solver* s) {
    NdPlan* p = s->nd;
    if (!p) return BN_OK;
    if (p->Wq) {
        if (s->opt.precision == BN_MIXED) build_pair_weights<float>(s);
        else build_pair_weights<double>(s);
        if (cudaGetLastError() != cudaSuccess) return BN_ERR_CUDA;
    }
    if (!p->resident || p->produced || s->eps == 0.0) return BN_OK;
    const bool fp32 = s->opt.precision == BN_MIXED;
    const KernelTables* t = s->tabs;
    const NdRound& R = p->rounds[0];
    if (fp32)
        k_beta_slices<float><<<R.nwork, 256, 0, s->stream>>>(p->g, t->P, t->alpha32, t->alphap32, R.d_groups, R.d_group_b,
                                                              R.d_off16, R.d_work, (float*)p->slices);
    else
        k_beta_slices<double><<<R.nwork, 256, 0, s->stream>>>(p->g, t->P, t->alpha64, t->alphap64, R.d_groups,
                                                               R.d_group_b, R.d_off16, R.d_work, (double*)p->slices);
    s->launches++;
    p->produced = true;
    return cudaGetLastError() == cudaSuccess ? BN_OK : BN_ERR_CUDA;
}

double nd_triple_terms(const bn_solver* s) { return s->nd ? s->nd->terms : 0.0; }
int nd_rounds(const bn_solver* s) { return s->nd ? (int)s->nd->rounds.size() : 0; }
int nd_ctas(const bn_solver* s) { return s->nd ? s->nd->nCTA : 0; }
size_t nd_slice_bytes(const bn_solver* s) { return s->nd ? s->nd->slice_cap : 0; }

}  // namespace bn
