// bn_transform.cu -- discrete Fourier transforms of the grid values (Mouton & Rey,
// Sec. 3.3 step 2(a), with the N^-d normalisation of eq. FS), the real inverse
// transform with the classical prefactor (Sec. 3.2), Runge-Kutta stage updates,
// moments (Sec. 4, head) and the optional conservation projection. All FP64.
#include <cmath>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n) { return (int)std::min<long long>((n + kThreads - 1) / kThreads, 65535); }

// One separable pass of the DFT along the axis of stride `stride`, one warp per output:
// out[.., k, ..] = scale * sum_j in[.., j, ..] e^{sign 2 i pi k j / N}, j,k in I_N, with the
// twiddles from the table tw[m] = e^{-2 i pi m / N}; the lanes split the sum over j and a fixed
// shuffle tree combines them.  `real_in` replaces `in` with a real input; `real_out` receives
// the real part instead of `out`; `out32` (optional) receives an FP32 copy.
__global__ void k_dft_axis(const double2* __restrict__ in, const double* __restrict__ real_in,
                           double2* __restrict__ out, float2* __restrict__ out32, double* __restrict__ real_out,
                           const double2* __restrict__ tw, int N, int nTotal, int stride, int sign, double scale) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < nTotal; idx += warps) {
        const int c = (idx / stride) % N;
        const int base = idx - c * stride;
        const int k = c - N / 2;
        double sr = 0.0, si = 0.0;
        for (int jj = lane; jj < N; jj += 32) {
            const int j = jj - N / 2;
            int m = (k * j) % N;
            if (m < 0) m += N;
            double2 w = __ldg(tw + m);
            if (sign > 0) w.y = -w.y;
            if (real_in) {
                const double x = real_in[base + jj * stride];
                sr = fma(x, w.x, sr);
                si = fma(x, w.y, si);
            } else {
                const double2 x = in[base + jj * stride];
                sr = fma(x.x, w.x, fma(-x.y, w.y, sr));
                si = fma(x.x, w.y, fma(x.y, w.x, si));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
            sr *= scale;
            si *= scale;
            if (real_out) {
                real_out[idx] = sr;
            } else {
                out[idx] = make_double2(sr, si);
                if (out32) out32[idx] = make_float2((float)sr, (float)si);
            }
        }
    }
}

__global__ void k_to_fp32(const double2* __restrict__ in, float2* __restrict__ out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// acc = (first ? 0 : acc) + w_acc K ; y = f + c K
__global__ void k_rk_stage(int n, const double* __restrict__ f, const double* __restrict__ K, double* __restrict__ acc,
                           double* __restrict__ y, double w_acc, double c, int first) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double k = K[i];
        acc[i] = first ? w_acc * k : fma(w_acc, k, acc[i]);
        y[i] = fma(c, k, f[i]);
    }
}

// candidate = f + h (acc + w_last K); flags[0] |= non-finite
__global__ void k_rk_final(int n, const double* __restrict__ f, const double* __restrict__ acc,
                           const double* __restrict__ K, double* __restrict__ cand, double w_last, double h,
                           int* __restrict__ flags) {
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = fma(h, fma(w_last, K[i], acc[i]), f[i]);
        cand[i] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&flags[0], 1);
}

// Heun: candidate = (f + y + dt K)/2
__global__ void k_heun_final(int n, const double* __restrict__ f, const double* __restrict__ y,
                             const double* __restrict__ K, double* __restrict__ cand, double dt,
                             int* __restrict__ flags) {
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = 0.5 * (f[i] + fma(dt, K[i], y[i]));
        cand[i] = v;
        bad |= !isfinite(v);
    }
    if (bad) atomicOr(&flags[0], 1);
}

// f = candidate unless a non-finite value has been seen in this call; counts committed steps and
// records max f (as the bit pattern of a non-negative double, which orders like the value).
__global__ void k_commit(int n, double* __restrict__ f, const double* __restrict__ cand, int* __restrict__ flags) {
    if (flags[0] != 0) return;
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = cand[i];
        f[i] = v;
        m = fmax(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long*>(flags + 4), (unsigned long long)__double_as_longlong(m));
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[1] += 1;
}

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (threadIdx.x == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

__device__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = -INFINITY;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (threadIdx.x == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

__device__ __forceinline__ void grid_velocity(int idx, int d, int N, double h, double* v) {
    for (int i = d - 1; i >= 0; --i) {
        v[i] = h * (idx % N - N / 2);
        idx /= N;
    }
}

// out = [rho, rho u (d), e, E_c, H, max f] (Sec. 4, head); one block, fixed reduction order.
__global__ void k_moments(int d, int N, double T, double eps, const double* __restrict__ f, double* __restrict__ out) {
    __shared__ double sh[33];
    const int n = d == 2 ? N * N : N * N * N;
    const double h = 2.0 * T / N, dv = d == 2 ? h * h : h * h * h, alpha = -eps;
    double rho = 0, m0 = 0, m1 = 0, m2 = 0, ec = 0, H = 0, fm = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v[3] = {0, 0, 0};
        grid_velocity(i, d, N, h, v);
        const double fj = f[i];
        rho += fj;
        m0 += v[0] * fj;
        m1 += v[1] * fj;
        m2 += v[2] * fj;
        ec += (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * fj;
        fm = fmax(fm, fj);
        if (fj > 0) {
            double t = fj * log(fj);
            if (alpha != 0.0) {
                const double s = 1.0 - alpha * fj;
                if (s > 0) t += s / alpha * log(s);
            }
            H += t;
        }
    }
    rho = block_sum(rho, sh) * dv;
    m0 = block_sum(m0, sh) * dv;
    m1 = block_sum(m1, sh) * dv;
    m2 = block_sum(m2, sh) * dv;
    ec = block_sum(ec, sh) * dv;
    H = block_sum(H, sh) * dv;
    fm = block_max(fm, sh);
    const double u[3] = {m0 / rho, m1 / rho, d == 3 ? m2 / rho : 0.0};
    double e = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v[3] = {0, 0, 0};
        grid_velocity(i, d, N, h, v);
        const double w2 = (v[0] - u[0]) * (v[0] - u[0]) + (v[1] - u[1]) * (v[1] - u[1]) + (v[2] - u[2]) * (v[2] - u[2]);
        e += w2 * f[i];
    }
    e = block_sum(e, sh) * dv / (2.0 * rho);
    if (threadIdx.x == 0) {
        out[0] = rho;
        out[1] = m0;
        out[2] = m1;
        if (d == 3) out[3] = m2;
        out[1 + d] = e;
        out[2 + d] = ec;
        out[3 + d] = H;
        out[4 + d] = fm;
    }
}

// Q <- Q - C^T (C C^T)^{-1} C Q with rows psi = (1, v, |v|^2) on the grid: the L2 projection
// onto zero mass, momentum and energy.  ginv = (C C^T)^{-1}, (d+2)^2, row-major.
struct ConsInv { double m[25]; };
__global__ void k_conserve(int d, int N, double T, ConsInv ginv, double* __restrict__ Q) {
    __shared__ double sh[33];
    const int n = d == 2 ? N * N : N * N * N, nc = d + 2;
    const double h = 2.0 * T / N;
    double mom[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v[3] = {0, 0, 0};
        grid_velocity(i, d, N, h, v);
        const double q = Q[i];
        mom[0] += q;
        for (int c = 0; c < d; ++c) mom[1 + c] += v[c] * q;
        mom[1 + d] += (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * q;
    }
    double lam[5];
    for (int c = 0; c < nc; ++c) mom[c] = block_sum(mom[c], sh);
    for (int r = 0; r < nc; ++r) {
        lam[r] = 0;
        for (int c = 0; c < nc; ++c) lam[r] += ginv.m[r * nc + c] * mom[c];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v[3] = {0, 0, 0};
        grid_velocity(i, d, N, h, v);
        double corr = lam[0] + lam[1 + d] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int c = 0; c < d; ++c) corr += lam[1 + c] * v[c];
        Q[i] -= corr;
    }
}

}  // namespace

// warps of 32 per block; one warp per output element
inline int dft_blocks(int n) { return std::min((n + 7) / 8, 65535); }

void launch_dft_forward(bn_solver* s, const double* f, double2* out) {
    const int d = s->g.d, N = s->g.N, n = s->g.nModes;
    const double scale = 1.0 / n;
    float2* out32 = s->opt.precision == BN_MIXED ? s->Ghat32 : nullptr;
    // d passes: last axis first (reads the real input), then the others; ping-pong through work_c
    // so that the final pass lands in `out` (and its FP32 copy).
    int stride = 1;
    double2* bufs[2] = {out, s->work_c};
    int cur = (d % 2 == 1) ? 0 : 1;
    k_dft_axis<<<dft_blocks(n), kThreads, 0, s->stream>>>(nullptr, f, bufs[cur], nullptr, nullptr, s->twiddle, N, n,
                                                          stride, -1, 1.0);
    s->launches++;
    for (int ax = 1; ax < d; ++ax) {
        stride *= N;
        const int nxt = cur ^ 1;
        const bool last = ax == d - 1;
        k_dft_axis<<<dft_blocks(n), kThreads, 0, s->stream>>>(bufs[cur], nullptr, bufs[nxt], last ? out32 : nullptr,
                                                              nullptr, s->twiddle, N, n, stride, -1, last ? scale : 1.0);
        s->launches++;
        cur = nxt;
    }
}

void launch_dft_inverse_real(bn_solver* s, const double2* in, double* out, double scale) {
    const int d = s->g.d, N = s->g.N, n = s->g.nModes;
    // passes along axes 0..d-2 into work_c / Ghat-free scratch, the last pass writes Re * scale.
    int stride = n / N;  // axis 0 stride
    const double2* src = in;
    double2* bufs[2] = {s->work_c, s->red};  // `red` is consumed before the inverse transform
    int cur = 0;
    for (int ax = 0; ax < d - 1; ++ax) {
        k_dft_axis<<<dft_blocks(n), kThreads, 0, s->stream>>>(src, nullptr, bufs[cur], nullptr, nullptr, s->twiddle, N, n,
                                                              stride, +1, 1.0);
        s->launches++;
        src = bufs[cur];
        cur ^= 1;
        stride /= N;
    }
    k_dft_axis<<<dft_blocks(n), kThreads, 0, s->stream>>>(src, nullptr, nullptr, nullptr, out, s->twiddle, N, n, stride,
                                                          +1, scale);
    s->launches++;
}

// 2-D transforms into caller-chosen buffers on a given stream (used by the no-allocation entry point).
void dft2_forward_into(const bn_solver* s, cudaStream_t st, const double* f, double2* work, double2* out, float2* out32) {
    const int N = s->g.N, n = s->g.nModes;
    k_dft_axis<<<dft_blocks(n), kThreads, 0, st>>>(nullptr, f, work, nullptr, nullptr, s->twiddle, N, n, 1, -1, 1.0);
    k_dft_axis<<<dft_blocks(n), kThreads, 0, st>>>(work, nullptr, out, out32, nullptr, s->twiddle, N, n, N, -1,
                                                   1.0 / n);
}

void dft2_inverse_real_into(const bn_solver* s, cudaStream_t st, const double2* in, double2* work, double* out) {
    const int N = s->g.N, n = s->g.nModes;
    k_dft_axis<<<dft_blocks(n), kThreads, 0, st>>>(in, nullptr, work, nullptr, nullptr, s->twiddle, N, n, N, +1, 1.0);
    k_dft_axis<<<dft_blocks(n), kThreads, 0, st>>>(work, nullptr, nullptr, nullptr, out, s->twiddle, N, n, 1, +1,
                                                   s->scale);
}

void launch_to_fp32(bn_solver* s, const double2* in, float2* out, int n) {
    k_to_fp32<<<blocks_for(n), kThreads, 0, s->stream>>>(in, out, n);
    s->launches++;
}

void launch_rk_stage(bn_solver* s, const double* f, const double* K, double* acc, double* y, double w_acc,
                     double c_next, double dt, int first) {
    const int n = s->g.nModes;
    k_rk_stage<<<blocks_for(n), kThreads, 0, s->stream>>>(n, f, K, acc, y, w_acc, c_next * dt, first);
    s->launches++;
}

void launch_rk_final(bn_solver* s, double* f, const double* acc, const double* K, double w_last, double dt,
                     double* cand, int* flags) {
    const int n = s->g.nModes;
    k_rk_final<<<blocks_for(n), kThreads, 0, s->stream>>>(n, f, acc, K, cand, w_last, dt / 6.0, flags);
    k_commit<<<blocks_for(n), kThreads, 0, s->stream>>>(n, f, cand, flags);
    s->launches += 2;
}

void launch_heun_final(bn_solver* s, double* f, const double* y, const double* K, double dt, double* cand,
                       int* flags) {
    const int n = s->g.nModes;
    k_heun_final<<<blocks_for(n), kThreads, 0, s->stream>>>(n, f, y, K, cand, dt, flags);
    k_commit<<<blocks_for(n), kThreads, 0, s->stream>>>(n, f, cand, flags);
    s->launches += 2;
}

void launch_moments(bn_solver* s, const double* f, double* out) {
    k_moments<<<1, 1024, 0, s->stream>>>(s->g.d, s->g.N, s->T, s->eps, f, out);
    s->launches++;
}

void launch_conserve(bn_solver* s, double* Q) {
    const int d = s->g.d, N = s->g.N, nc = d + 2;
    const double h = 2.0 * s->T / N;
    // C C^T on the grid, then its inverse by Gauss-Jordan (host, FP64, (d+2)^2).
    double G[25] = {0}, inv[25] = {0};
    for (int idx = 0; idx < s->g.nModes; ++idx) {
        double v[3] = {0, 0, 0};
        int r = idx;
        for (int i = d - 1; i >= 0; --i) { v[i] = h * (r % N - N / 2); r /= N; }
        double psi[5];
        psi[0] = 1.0;
        for (int c = 0; c < d; ++c) psi[1 + c] = v[c];
        psi[1 + d] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) G[a * nc + b] += psi[a] * psi[b];
    }
    for (int a = 0; a < nc; ++a) inv[a * nc + a] = 1.0;
    for (int c = 0; c < nc; ++c) {
        int piv = c;
        for (int r = c + 1; r < nc; ++r)
            if (std::fabs(G[r * nc + c]) > std::fabs(G[piv * nc + c])) piv = r;
        for (int k = 0; k < nc; ++k) {
            std::swap(G[c * nc + k], G[piv * nc + k]);
            std::swap(inv[c * nc + k], inv[piv * nc + k]);
        }
        const double p = G[c * nc + c];
        for (int k = 0; k < nc; ++k) { G[c * nc + k] /= p; inv[c * nc + k] /= p; }
        for (int r = 0; r < nc; ++r) {
            if (r == c) continue;
            const double m = G[r * nc + c];
            for (int k = 0; k < nc; ++k) { G[r * nc + k] -= m * G[c * nc + k]; inv[r * nc + k] -= m * inv[c * nc + k]; }
        }
    }
    ConsInv ci;
    for (int i = 0; i < 25; ++i) ci.m[i] = inv[i];
    k_conserve<<<1, 1024, 0, s->stream>>>(d, N, s->T, ci, Q);
    s->launches++;
}


// The conservation projection on a given stream without touching the solver (no-allocation entry point).
void launch_conserve_on(const bn_solver* s, double* Q, cudaStream_t st) {
    const int d = s->g.d, N = s->g.N, nc = d + 2;
    const double h = 2.0 * s->T / N;
    // C C^T on the grid, then its inverse by Gauss-Jordan (host, FP64, (d+2)^2).
    double G[25] = {0}, inv[25] = {0};
    for (int idx = 0; idx < s->g.nModes; ++idx) {
        double v[3] = {0, 0, 0};
        int r = idx;
        for (int i = d - 1; i >= 0; --i) { v[i] = h * (r % N - N / 2); r /= N; }
        double psi[5];
        psi[0] = 1.0;
        for (int c = 0; c < d; ++c) psi[1 + c] = v[c];
        psi[1 + d] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        for (int a = 0; a < nc; ++a)
            for (int b = 0; b < nc; ++b) G[a * nc + b] += psi[a] * psi[b];
    }
    for (int a = 0; a < nc; ++a) inv[a * nc + a] = 1.0;
    for (int c = 0; c < nc; ++c) {
        int piv = c;
        for (int r = c + 1; r < nc; ++r)
            if (std::fabs(G[r * nc + c]) > std::fabs(G[piv * nc + c])) piv = r;
        for (int k = 0; k < nc; ++k) {
            std::swap(G[c * nc + k], G[piv * nc + k]);
            std::swap(inv[c * nc + k], inv[piv * nc + k]);
        }
        const double p = G[c * nc + c];
        for (int k = 0; k < nc; ++k) { G[c * nc + k] /= p; inv[c * nc + k] /= p; }
        for (int r = 0; r < nc; ++r) {
            if (r == c) continue;
            const double m = G[r * nc + c];
            for (int k = 0; k < nc; ++k) { G[r * nc + k] -= m * G[c * nc + k]; inv[r * nc + k] -= m * inv[c * nc + k]; }
        }
    }
    ConsInv ci;
    for (int i = 0; i < 25; ++i) ci.m[i] = inv[i];
    k_conserve<<<1, 1024, 0, st>>>(d, N, s->T, ci, Q);
}

}  // namespace bn
