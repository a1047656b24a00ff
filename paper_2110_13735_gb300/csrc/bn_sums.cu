// bn_sums.cu -- the Fourier-Galerkin mode sums of the Boltzmann-Nordheim operator
// (Mouton & Rey, Lemma of Sec. 2.3) on CUDA cores, FP64 or FP32 (mixed precision).
//
// With the substitution a = k+m = n-l, b = l+m = n-k the dominant trilinear term is
//   Q^_{1q,n} = sum_b G^_{n-b} C_b(n),   C_b(n) = sum_s beta(n-s, b) P_b(s),   P_b(s) = G^_s G^_{b-s},
// over n, n-b, s, b-s in I_N (the same terms as the Lemma; Remark rem:computComplexity):
// for each b the inner sum is a d-dimensional Toeplitz (discrete convolution) product of
// the kernel-mode slice beta(., b) with the pair products P_b, so each term costs one
// real-by-complex multiply-add.  The reducible cubic terms Q_{2q} - Q_{3q} - Q_{4q} are
//   sum_k G^_k S(n-k),   S(t) = sum_{l+m=t} [beta(l,m) - beta(t,l) - beta(l,t)] G^_l G^_m,
// and the quadratic terms Q_{1c} - Q_{2c} are sum_{k+l=n} [beta(k,l) - beta(l,l)] G^_k G^_l.
#include <cmath>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kThreads = 256;

template <int DIM>
struct Idx {
    // flat index of a mode k in I_N (row-major, k_i + N/2)
    static __device__ __forceinline__ int modes(const int* k, int N) {
        int r = 0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) r = r * N + (k[i] + N / 2);
        return r;
    }
    // flat index of an argument a in the extended box [-N, N-1]^d
    static __device__ __forceinline__ int ext(const int* a, int N) {
        int r = 0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) r = r * (2 * N) + (a[i] + N);
        return r;
    }
};

template <typename Real>
__device__ __forceinline__ cplx<Real> ld(const cplx<Real>* p) { return *p; }

// ------------------------------------------------------------------ reducible pair sums S(t)
template <typename Real, int DIM>
__global__ void __launch_bounds__(kThreads) k_pair_S(int N, const cplx<Real>* __restrict__ G,
                                                     const Real* __restrict__ beta, double2* __restrict__ S) {
    const int E = 2 * N;
    const int nExt = DIM == 2 ? E * E : E * E * E;
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < nExt; it += gridDim.x * blockDim.x) {
        int t[DIM], lo[DIM], cnt[DIM];
        int r = it, total = 1;
#pragma unroll
        for (int i = DIM - 1; i >= 0; --i) { t[i] = r % E - N; r /= E; }
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            // l in I_N and t - l in I_N
            lo[i] = max(-N / 2, t[i] - N / 2 + 1);
            const int hi = min(N / 2 - 1, t[i] + N / 2);
            cnt[i] = max(0, hi - lo[i] + 1);
            total *= cnt[i];
        }
        Real sr = 0, si = 0;
        const int it_t = Idx<DIM>::ext(t, N);
        for (int q = 0; q < total; ++q) {
            int l[DIM], m[DIM];
            int rr = q;
#pragma unroll
            for (int i = DIM - 1; i >= 0; --i) { l[i] = lo[i] + rr % cnt[i]; rr /= cnt[i]; m[i] = t[i] - l[i]; }
            const int il = Idx<DIM>::ext(l, N), im = Idx<DIM>::ext(m, N);
            // beta(a, b) is stored at [b][a]
            const Real w = beta[(size_t)im * nExt + il] - beta[(size_t)il * nExt + it_t] - beta[(size_t)it_t * nExt + il];
            const cplx<Real> p = cmul(G[Idx<DIM>::modes(l, N)], G[Idx<DIM>::modes(m, N)]);
            sr += w * p.x;
            si += w * p.y;
        }
        S[it] = make_double2((double)sr, (double)si);
    }
}

// ------------------------------------------------------------------ quadratic and reducible cubic modes
template <typename Real, int DIM>
__global__ void __launch_bounds__(kThreads) k_quad_red(int N, const cplx<Real>* __restrict__ G,
                                                       const Real* __restrict__ beta, const double2* __restrict__ S,
                                                       double2* __restrict__ quad, double2* __restrict__ red,
                                                       int cubic) {
    const int E = 2 * N;
    const int nExt = DIM == 2 ? E * E : E * E * E;
    const int nModes = DIM == 2 ? N * N : N * N * N;
    for (int in = blockIdx.x * blockDim.x + threadIdx.x; in < nModes; in += gridDim.x * blockDim.x) {
        int n[DIM];
        int r = in;
#pragma unroll
        for (int i = DIM - 1; i >= 0; --i) { n[i] = r % N - N / 2; r /= N; }
        // quadratic: k in I_N, l = n - k in I_N
        int lo[DIM], cnt[DIM], total = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            lo[i] = max(-N / 2, n[i] - N / 2 + 1);
            const int hi = min(N / 2 - 1, n[i] + N / 2);
            cnt[i] = max(0, hi - lo[i] + 1);
            total *= cnt[i];
        }
        Real qr = 0, qi = 0;
        for (int q = 0; q < total; ++q) {
            int k[DIM], l[DIM];
            int rr = q;
#pragma unroll
            for (int i = DIM - 1; i >= 0; --i) { k[i] = lo[i] + rr % cnt[i]; rr /= cnt[i]; l[i] = n[i] - k[i]; }
            const int ik = Idx<DIM>::ext(k, N), il = Idx<DIM>::ext(l, N);
            const Real w = beta[(size_t)il * nExt + ik] - beta[(size_t)il * nExt + il];
            const cplx<Real> p = cmul(G[Idx<DIM>::modes(k, N)], G[Idx<DIM>::modes(l, N)]);
            qr += w * p.x;
            qi += w * p.y;
        }
        quad[in] = make_double2((double)qr, (double)qi);
        if (!cubic) continue;
        // reducible cubic: k in I_N, t = n - k in [-N, N-2]^d (S vanishes outside)
        double rr_ = 0, ri_ = 0;
        int klo[DIM], kcnt[DIM], ktot = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            klo[i] = max(-N / 2, n[i] - (N - 2));
            const int hi = min(N / 2 - 1, n[i] + N);
            kcnt[i] = max(0, hi - klo[i] + 1);
            ktot *= kcnt[i];
        }
        for (int q = 0; q < ktot; ++q) {
            int k[DIM], t[DIM];
            int rr = q;
#pragma unroll
            for (int i = DIM - 1; i >= 0; --i) { k[i] = klo[i] + rr % kcnt[i]; rr /= kcnt[i]; t[i] = n[i] - k[i]; }
            const cplx<Real> gk = G[Idx<DIM>::modes(k, N)];
            const double2 st = S[Idx<DIM>::ext(t, N)];
            rr_ += (double)gk.x * st.x - (double)gk.y * st.y;
            ri_ += (double)gk.x * st.y + (double)gk.y * st.x;
        }
        red[in] = make_double2(rr_, ri_);
    }
}

// ------------------------------------------------------------------ Q_{1,q} triple sum
template <typename Real>
struct TripleArgs {
    int N;
    const cplx<Real>* G;      // modes, N^d
    const Real* beta;         // [b][a]
    const int* items;         // b (flat extended index), descending work
    int count;
    double2* partials;        // [gridDim.x][N^d]
};

// One CTA walks its share of b values (static round robin over the descending-work list).
// For each b: P_b(s) into shared memory, then each thread owns RW consecutive outputs along
// the last dimension and sums over s in box_s(b) with a sliding register window of
// beta(n - s, b) along the last dimension; C_b(n) times G^_{n-b} is added to the CTA's FP64
// accumulator of Q^_{1q} in shared memory (each output has one owner per b: no atomics).
template <typename Real, int DIM, int RW>
__global__ void __launch_bounds__(kThreads) k_triple(TripleArgs<Real> A) {
    using C = cplx<Real>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = A.N, E = 2 * N;
    const int nModes = DIM == 2 ? N * N : N * N * N;
    const int nExt = DIM == 2 ? E * E : E * E * E;
    double2* Qacc = reinterpret_cast<double2*>(smem_raw);
    C* Pb = reinterpret_cast<C*>(Qacc + nModes);
    for (int i = threadIdx.x; i < nModes; i += blockDim.x) Qacc[i] = make_double2(0.0, 0.0);

    for (int item = blockIdx.x; item < A.count; item += gridDim.x) {
        const int ib = A.items[item];
        int b[DIM], nlo[DIM], L[DIM], slo[DIM], S[DIM];
        {
            int r = ib;
#pragma unroll
            for (int i = DIM - 1; i >= 0; --i) { b[i] = r % E - N; r /= E; }
        }
        int nS = 1;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            nlo[i] = max(-N / 2, b[i] - N / 2);
            L[i] = min(N / 2 - 1, b[i] + N / 2 - 1) - nlo[i] + 1;
            slo[i] = max(-N / 2, b[i] - N / 2 + 1);
            S[i] = min(N / 2 - 1, b[i] + N / 2) - slo[i] + 1;
            nS *= S[i];
        }
        __syncthreads();   // the previous item's readers of Pb are done
        for (int q = threadIdx.x; q < nS; q += blockDim.x) {
            int s[DIM], m[DIM];
            int r = q;
#pragma unroll
            for (int i = DIM - 1; i >= 0; --i) { s[i] = slo[i] + r % S[i]; r /= S[i]; m[i] = b[i] - s[i]; }
            Pb[q] = cmul(A.G[Idx<DIM>::modes(s, N)], A.G[Idx<DIM>::modes(m, N)]);
        }
        __syncthreads();
        const Real* __restrict__ bslice = A.beta + (size_t)ib * nExt;   // beta(., b)
        int rows = 1, outer = 1;
#pragma unroll
        for (int i = 0; i < DIM - 1; ++i) { rows *= L[i]; outer *= S[i]; }
        const int Ll = L[DIM - 1], Sl = S[DIM - 1];
        const int groups = (Ll + RW - 1) / RW;
        for (int task = threadIdx.x; task < rows * groups; task += blockDim.x) {
            int n[DIM];
            {
                int r = task / groups;
#pragma unroll
                for (int i = DIM - 2; i >= 0; --i) { n[i] = nlo[i] + r % L[i]; r /= L[i]; }
                n[DIM - 1] = nlo[DIM - 1] + (task % groups) * RW;
            }
            Real ar[RW], ai[RW];
#pragma unroll
            for (int r = 0; r < RW; ++r) { ar[r] = 0; ai[r] = 0; }
            for (int so = 0; so < outer; ++so) {
                // outer coordinates of s and the row of beta(a, b) with a_i = n_i - s_i (i < DIM-1)
                int rowoff = 0;
                {
                    int r = so;
                    int sc[DIM];
#pragma unroll
                    for (int i = DIM - 2; i >= 0; --i) { sc[i] = slo[i] + r % S[i]; r /= S[i]; }
#pragma unroll
                    for (int i = 0; i < DIM - 1; ++i) rowoff = rowoff * E + (n[i] - sc[i] + N);
                }
                const Real* __restrict__ brow = bslice + (size_t)rowoff * E;
                const C* __restrict__ prow = Pb + so * Sl;
                // window: w[r] = beta(a_last = n_last + r - s_last) for s_last = slo
                const int a0 = n[DIM - 1] - slo[DIM - 1] + N;   // index of a_last for r = 0 at the first s
                Real w[RW];
#pragma unroll
                for (int r = 0; r < RW; ++r) w[r] = __ldg(brow + min(a0 + r, E - 1));
                for (int sl = 0; sl < Sl; ++sl) {
                    const C p = prow[sl];
#pragma unroll
                    for (int r = 0; r < RW; ++r) {
                        ar[r] = fma(w[r], p.x, ar[r]);
                        ai[r] = fma(w[r], p.y, ai[r]);
                    }
                    // slide: s_last += 1 -> every a_last decreases by 1
#pragma unroll
                    for (int r = RW - 1; r > 0; --r) w[r] = w[r - 1];
                    w[0] = __ldg(brow + max(a0 - sl - 1, 0));
                }
            }
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                int nn[DIM], k[DIM];
#pragma unroll
                for (int i = 0; i < DIM; ++i) nn[i] = n[i];
                nn[DIM - 1] += r;
                if (nn[DIM - 1] >= nlo[DIM - 1] + Ll) break;
#pragma unroll
                for (int i = 0; i < DIM; ++i) k[i] = nn[i] - b[i];
                const C g = A.G[Idx<DIM>::modes(k, N)];
                const int on = Idx<DIM>::modes(nn, N);
                double2 q = Qacc[on];
                q.x += (double)g.x * (double)ar[r] - (double)g.y * (double)ai[r];
                q.y += (double)g.x * (double)ai[r] + (double)g.y * (double)ar[r];
                Qacc[on] = q;
            }
        }
    }
    __syncthreads();
    double2* out = A.partials + (size_t)blockIdx.x * nModes;
    for (int i = threadIdx.x; i < nModes; i += blockDim.x) out[i] = Qacc[i];
}

// Fixed-order sum of the per-CTA partials (deterministic).
__global__ void k_reduce_partials(int nModes, int nPart, const double2* __restrict__ partials, double2* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nModes; i += gridDim.x * blockDim.x) {
        double x = 0, y = 0;
        for (int c = 0; c < nPart; ++c) {
            const double2 v = partials[(size_t)c * nModes + i];
            x += v.x;
            y += v.y;
        }
        out[i] = make_double2(x, y);
    }
}

// Q^ = quad + eps (q1q + red)   (Sec. 3.3 step 2(c) with alpha = -eps)
__global__ void k_combine(int n, double eps, const double2* __restrict__ quad, const double2* __restrict__ q1q,
                          const double2* __restrict__ red, double2* __restrict__ out, int cubic) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 q = quad[i];
        if (cubic) {
            q.x += eps * (q1q[i].x + red[i].x);
            q.y += eps * (q1q[i].y + red[i].y);
        }
        out[i] = q;
    }
}

inline int blocks_for(long long n) { return (int)std::min<long long>((n + kThreads - 1) / kThreads, 65535); }

template <typename Real, int DIM>
void pair_sums_t(bn_solver* s, const cplx<Real>* G, const Real* beta) {
    const int cubic = s->eps != 0.0;
    if (cubic) {
        k_pair_S<Real, DIM><<<blocks_for(s->g.nExt), kThreads, 0, s->stream>>>(s->g.N, G, beta, s->S2);
        s->launches++;
    }
    k_quad_red<Real, DIM><<<blocks_for(s->g.nModes), kThreads, 0, s->stream>>>(s->g.N, G, beta, s->S2, s->quad,
                                                                             s->red, cubic);
    s->launches++;
}

template <typename Real, int DIM, int RW>
void triple_t(bn_solver* s, const cplx<Real>* G, const Real* beta) {
    TripleArgs<Real> A;
    A.N = s->g.N;
    A.G = G;
    A.beta = beta;
    A.items = s->work.items;
    A.count = s->work.count;
    A.partials = s->partials;
    const size_t smem = (size_t)s->g.nModes * (sizeof(double2) + sizeof(cplx<Real>));
    k_triple<Real, DIM, RW><<<s->n_partials, kThreads, smem, s->stream>>>(A);
    k_reduce_partials<<<blocks_for(s->g.nModes), kThreads, 0, s->stream>>>(s->g.nModes, s->n_partials, s->partials,
                                                                          s->q1q);
    s->launches += 2;
}

}  // namespace

template <typename Real, int DIM, int RW>
void configure_triple() {
    cudaFuncSetAttribute(k_triple<Real, DIM, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int triple_partials(const bn_solver* s) {
    // opt in to large dynamic shared memory once, outside any stream capture
    configure_triple<float, 2, 8>();
    configure_triple<double, 2, 4>();
    configure_triple<float, 3, 8>();
    configure_triple<double, 3, 4>();
    configure_fused2d();
    int dev = s->device, sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    if (s->g.d == 2) {
        // resident CTAs per SM of the fused kernel, limited by its shared memory (227 KB per SM usable)
        const size_t smem = fused2d_smem(s->g.N, s->opt.precision);
        const int per_sm = std::max(1, std::min(4, (int)((227 * 1024) / (smem + 1024))));
        return std::max(1, std::min(s->work.count, per_sm * sms));
    }
    return std::max(1, std::min(s->work.count, 2 * sms));
}

void launch_pair_sums(bn_solver* s) {
    const bool mixed = s->opt.precision == BN_MIXED;
    if (s->g.d == 2) {
        if (mixed) pair_sums_t<float, 2>(s, s->Ghat32, s->tabs->beta32);
        else pair_sums_t<double, 2>(s, s->Ghat, s->tabs->beta64);
    } else {
        if (mixed) pair_sums_t<float, 3>(s, s->Ghat32, s->tabs->beta32);
        else pair_sums_t<double, 3>(s, s->Ghat, s->tabs->beta64);
    }
}

void launch_triple_sum(bn_solver* s) {
    const bool mixed = s->opt.precision == BN_MIXED;
    if (s->g.d == 2) {
        if (mixed) triple_t<float, 2, 8>(s, s->Ghat32, s->tabs->beta32);
        else triple_t<double, 2, 4>(s, s->Ghat, s->tabs->beta64);
    } else {
        if (mixed) triple_t<float, 3, 8>(s, s->Ghat32, s->tabs->beta32);
        else triple_t<double, 3, 4>(s, s->Ghat, s->tabs->beta64);
    }
}

void launch_combine(bn_solver* s) {
    const int n = s->g.nModes;
    k_combine<<<blocks_for(n), kThreads, 0, s->stream>>>(n, s->eps, s->quad, s->q1q, s->red, s->Qhat,
                                                        s->eps != 0.0);
    s->launches++;
}

}  // namespace bn
