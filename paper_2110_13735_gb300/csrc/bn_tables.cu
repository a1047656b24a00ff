// bn_tables.cu -- kernel-mode tables beta(a,b) (Mouton & Rey, Sec. 2.5, eq. betadD)
// built once per (d, N, R_xi, kernel, quadrature) in FP64 on the device and shared
// (refcounted) by every solver that uses the same operator; and the work list of the
// Q_{1,q} triple sum.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>

#include "bn_internal.cuh"

namespace bn {

namespace {

std::mutex g_tables_mutex;
std::map<std::string, KernelTables*> g_tables;

// Sinc(x) = sin(x)/x: phi_R(s) = int_{-R}^{R} e^{i rho s} d rho = 2R Sinc(Rs) (Sec. 2.5).
__device__ __forceinline__ double sinc_d(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

// 3-D radial transform for b == 1: int_{-R}^{R} |rho| e^{i rho s} d rho = 2R sin(Rs)/s - 2(1-cos Rs)/s^2.
__device__ __forceinline__ double phi3_d(double R, double s) {
    double x = R * s;
    if (fabs(x) < 1e-4) {   // series: R^2 (1 - x^2/4 + x^4/72)
        double x2 = x * x;
        return R * R * (1.0 - x2 * 0.25 + x2 * x2 / 72.0);
    }
    double h = sin(0.5 * x) / (0.5 * x);
    return R * R * (2.0 * sin(x) / x - h * h);
}

// psi(q) = int_0^pi phi3(q cos t) dt over the half great circle = 2 pi R J1(Rq)/q, psi(0) = pi R^2.
__device__ __forceinline__ double psi3_d(double R, double q) {
    double x = R * q;
    if (fabs(x) < 1e-6) return M_PI * R * R * (1.0 - x * x * 0.125);
    return 2.0 * M_PI * R * j1(x) / q;
}

// Quadrature node: direction e and weight.  2-D Maxwell: e_theta, e2 unused, w = pi/M.
// 2-D hard spheres: e_theta, e2 = rho'_j, w = (pi/M) w_j.  3-D: e on the half sphere.
struct Node { double e0, e1, e2, w; };

// alpha_p(a), alpha'_p(a) for every node p and a in the extended box.  2-D hard spheres
// (gamma = 1, not covered by the separable expansion of Sec. 2.5): the kernel modes are the
// Lemma's definition with Btilde = 2 C_Phi sqrt(rho^2 + rho'^2), z = rho e_theta,
// y = rho' e_{theta+pi/2}, Gauss-Legendre nodes `rad` (x = rho_i, y = weight) on [-R, R] in
// each radius; the sum over rho_i is taken here, leaving beta = sum over (theta, rho'_j).
__global__ void k_alpha_tables(int d, int N, int P, double Rxi, double c_phi, int kernel, int nrad,
                               const double2* __restrict__ rad, const Node* __restrict__ nodes,
                               double* __restrict__ alpha, double* __restrict__ alphap) {
    const int E = 2 * N;
    const int nExt = d == 2 ? E * E : E * E * E;
    const long long total = (long long)P * nExt;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(idx / nExt), ia = (int)(idx % nExt);
        const Node nd = nodes[p];
        if (d == 2 && kernel == 1) {
            const double a0 = ia / E - N, a1 = ia % E - N;
            const double ke = a0 * nd.e0 + a1 * nd.e1;
            const double le = -a0 * nd.e1 + a1 * nd.e0;
            const double rj2 = nd.e2 * nd.e2;
            double h = 0.0;
            for (int i = 0; i < nrad; ++i) {
                const double2 r = rad[i];
                h = fma(r.y * sqrt(fma(r.x, r.x, rj2)), cos(r.x * ke), h);
            }
            alpha[idx] = nd.w * 2.0 * c_phi * h;
            alphap[idx] = cos(nd.e2 * le);
        } else if (d == 2) {
            const double a0 = ia / E - N, a1 = ia % E - N;
            // alpha_p(k) = 2 C_Phi phi(k.e_p), alpha'_p(l) = phi(l.e_{p+pi/2}); C = pi/M folded into alpha.
            const double ke = a0 * nd.e0 + a1 * nd.e1;
            const double le = -a0 * nd.e1 + a1 * nd.e0;   // e_{theta+pi/2} = (-sin, cos)
            alpha[idx] = nd.w * 2.0 * c_phi * 2.0 * Rxi * sinc_d(Rxi * ke);
            alphap[idx] = 2.0 * Rxi * sinc_d(Rxi * le);
        } else {
            const double a0 = ia / (E * E) - N, a1 = (ia / E) % E - N, a2 = ia % E - N;
            // alpha(k) = w 4 C_Phi phi3(k.e), alpha'(l) = psi(|Pi_{e^perp} l|).
            const double ke = a0 * nd.e0 + a1 * nd.e1 + a2 * nd.e2;
            const double n2 = a0 * a0 + a1 * a1 + a2 * a2 - ke * ke;
            alpha[idx] = nd.w * 4.0 * c_phi * phi3_d(Rxi, ke);
            alphap[idx] = psi3_d(Rxi, sqrt(fmax(n2, 0.0)));
        }
    }
}

// beta[ib][ia] = sum_p alpha_p(a) alpha'_p(b) (eq. betadD), FP64, plus an FP32 copy.  A product
// of the (P x nExt) tables over p: each 256-thread CTA forms a 64 x 64 tile of (b, a) with 4 x 4
// entries per thread, staging 16 nodes of both tables per step in shared memory.  Every entry
// sums over p in increasing order with FP64 fused multiply-adds.
constexpr int kBT = 64, kBK = 16;
__global__ void __launch_bounds__(256) k_beta_table(int nExt, int P, const double* __restrict__ alpha,
                                                    const double* __restrict__ alphap, double* __restrict__ beta64,
                                                    float* __restrict__ beta32) {
    __shared__ double As[kBK][kBT];   // alpha_p(a), a in the tile
    __shared__ double Bs[kBK][kBT];   // alpha'_p(b), b in the tile
    const int a0 = blockIdx.x * kBT, b0 = blockIdx.y * kBT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int p0 = 0; p0 < P; p0 += kBK) {
        for (int t = threadIdx.x; t < kBK * kBT; t += 256) {
            const int k = t / kBT, c = t % kBT;
            const bool okp = p0 + k < P;
            As[k][c] = okp && a0 + c < nExt ? alpha[(size_t)(p0 + k) * nExt + a0 + c] : 0.0;
            Bs[k][c] = okp && b0 + c < nExt ? alphap[(size_t)(p0 + k) * nExt + b0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) av[j] = As[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i) bv[i] = Bs[k][ty + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[j], bv[i], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = b0 + ty + 16 * i, a = a0 + tx + 16 * j;
            if (a < nExt && b < nExt) {
                const size_t idx = (size_t)b * nExt + a;
                beta64[idx] = acc[i][j];
                beta32[idx] = (float)acc[i][j];
            }
        }
}

// Reducible weights W(b, s) = beta(s, b-s) - beta(b, s) - beta(s, b) for s, b-s in I_N (2-D),
// stored [b][s] so that the weights of one b are contiguous.
__global__ void k_sw_table(int N, const double* __restrict__ beta, double* __restrict__ sw64, float* __restrict__ sw32) {
    const int E = 2 * N, nExt = E * E, nm = N * N;
    const long long total = (long long)nExt * nm;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ib = (int)(idx / nm), is = (int)(idx % nm);
        const int b1 = ib / E - N, b2 = ib % E - N;
        const int s1 = is / N - N / 2, s2 = is % N - N / 2;
        const int m1 = b1 - s1, m2 = b2 - s2;
        double w = 0.0;
        if (m1 >= -N / 2 && m1 < N / 2 && m2 >= -N / 2 && m2 < N / 2) {
            const int es = (s1 + N) * E + (s2 + N), em = (m1 + N) * E + (m2 + N);
            // beta(a, b) is stored at [b][a]
            w = beta[(size_t)em * nExt + es] - beta[(size_t)es * nExt + ib] - beta[(size_t)ib * nExt + es];
        }
        sw64[idx] = w;
        sw32[idx] = (float)w;
    }
}

// Quadratic weights dq(b, a) = beta(a, b) - beta(b, b) for b in I_N (2-D), the difference taken in
// FP64 and rounded to FP32 once (the FP32 difference of two rounded weights would carry the
// rounding of beta itself, which is far larger than the difference for a near b).
// dq32lo (the rounding residual of each weight) is written beside it.
__global__ void k_dq_table(int N, const double* __restrict__ beta, float* __restrict__ dq32, float* __restrict__ dq32lo) {
    const int E = 2 * N, nExt = E * E, h = N / 2;
    const long long total = (long long)N * N * nExt;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(idx / nExt), ia = (int)(idx % nExt);
        const int b1 = q / N - h, b2 = q % N - h;
        const int ib = (b1 + N) * E + (b2 + N);
        const double v = beta[(size_t)ib * nExt + ia] - beta[(size_t)ib * nExt + ib];
        const float hi = (float)v;
        dq32[idx] = hi;
        dq32lo[idx] = (float)(v - (double)hi);
    }
}

// Rounding residuals lo = fl32(x - hi) of an FP64 table x and its FP32 rounding hi (2-D).
__global__ void k_residual_table(long long n, const double* __restrict__ x64, const float* __restrict__ hi,
                                 float* __restrict__ lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        lo[i] = (float)(x64[i] - (double)hi[i]);
}

// FP32 table with the a axes swapped: betaT[b][a2][a1] = beta[b][a1][a2] (2-D).
__global__ void k_beta_transpose(int N, const float* __restrict__ beta32, float* __restrict__ beta32T) {
    const int E = 2 * N, nExt = E * E;
    const long long total = (long long)nExt * nExt;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long ib = idx / nExt;
        const int ia = (int)(idx % nExt), a2 = ia / E, a1 = ia % E;   // destination [a2][a1]
        beta32T[idx] = beta32[ib * nExt + a1 * E + a2];
    }
}

// Gauss-Legendre rule on [-1, 1]: Newton iteration on P_n from Tricomi's initial guesses.
void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
        double dp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm1 = 1.0, pk = z;   // P_0, P_1
            for (int k = 2; k <= n; ++k) {
                double pn = ((2.0 * k - 1.0) * z * pk - (k - 1.0) * pm1) / k;
                pm1 = pk;
                pk = pn;
            }
            if (n == 1) { pk = z; pm1 = 1.0; }
            dp = n * (pm1 - z * pk) / (1.0 - z * z);
            double step = pk / dp;
            z -= step;
            if (std::fabs(step) < 4e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

std::string table_key(const bn_solver* s) {
    std::ostringstream os;
    os.precision(17);
    os << s->device << ":" << s->g.d << ":" << s->g.N << ":" << s->Rxi << ":" << s->kernel << ":";
    if (s->g.d == 2) os << s->opt.M << "r" << (s->kernel == BN_HARD_SPHERE ? s->opt.M1 : 0);
    else os << s->opt.M1 << "x" << s->opt.M2 << ":" << s->opt.quad3d;
    os << ":" << s->opt.c_phi;
    return os.str();
}

}  // namespace

bn_status acquire_tables(bn_solver* s, std::string* err) {
    std::lock_guard<std::mutex> lock(g_tables_mutex);
    const std::string key = table_key(s);
    auto it = g_tables.find(key);
    if (it != g_tables.end()) {
        it->second->refcount++;
        s->tabs = it->second;
        return BN_OK;
    }
    KernelTables* t = new KernelTables();
    t->key = key;
    t->g = s->g;
    const int d = s->g.d, nExt = s->g.nExt;
    std::vector<Node> nodes;
    std::vector<double2> rad;
    if (d == 2 && s->kernel == BN_HARD_SPHERE) {
        const int M = s->opt.M, Qr = s->opt.M1;
        std::vector<double> x, w;
        gauss_legendre_rule(Qr, x, w);
        for (int i = 0; i < Qr; ++i) rad.push_back(make_double2(s->Rxi * x[i], s->Rxi * w[i]));
        for (int p = 0; p < M; ++p) {
            double th = p * M_PI / M;
            for (int j = 0; j < Qr; ++j)
                nodes.push_back(Node{std::cos(th), std::sin(th), rad[j].x, (M_PI / M) * rad[j].y});
        }
    } else if (d == 2) {
        const int M = s->opt.M;
        for (int p = 0; p < M; ++p) {
            double th = p * M_PI / M;
            nodes.push_back(Node{std::cos(th), std::sin(th), 0.0, M_PI / M});
        }
    } else {
        const int M1 = s->opt.M1, M2 = s->opt.M2;
        std::vector<double> mu, wt;
        if (s->opt.quad3d == 0) {
            gauss_legendre_rule(M1, mu, wt);
        } else {
            mu.resize(M1);
            wt.resize(M1);
            for (int i = 0; i < M1; ++i) {
                mu[i] = std::cos(i * M_PI / M1);
                wt[i] = (M_PI / M1) * std::sin(i * M_PI / M1);
            }
        }
        for (int i = 0; i < M1; ++i)
            for (int q = 0; q < M2; ++q) {
                double st = std::sqrt(std::max(0.0, 1.0 - mu[i] * mu[i])), ph = q * M_PI / M2;
                nodes.push_back(Node{st * std::cos(ph), st * std::sin(ph), mu[i], wt[i] * (M_PI / M2)});
            }
    }
    t->P = (int)nodes.size();
    // 2-D: the full table beta(a, b) over the extended box; 3-D never forms it (the operator
    // recomputes its slices from the alpha tables)
    const size_t nAl = (size_t)t->P * nExt, nBeta = d == 2 ? (size_t)nExt * nExt : 0;
    Node* d_nodes = nullptr;
    double2* d_rad = nullptr;
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&d_nodes, sizeof(Node) * nodes.size());
    if (e == cudaSuccess && !rad.empty()) e = cudaMalloc(&d_rad, sizeof(double2) * rad.size());
    if (e == cudaSuccess) e = cudaMalloc(&t->alpha64, sizeof(double) * nAl);
    if (e == cudaSuccess) e = cudaMalloc(&t->alphap64, sizeof(double) * nAl);
    if (e == cudaSuccess && nBeta) e = cudaMalloc(&t->beta64, sizeof(double) * nBeta);
    if (e == cudaSuccess && nBeta) e = cudaMalloc(&t->beta32, sizeof(float) * nBeta);
    const size_t nSw = d == 2 ? (size_t)nExt * s->g.nModes : 0;
    if (e == cudaSuccess && nSw) e = cudaMalloc(&t->sw64, sizeof(double) * nSw);
    if (e == cudaSuccess && nSw) e = cudaMalloc(&t->sw32, sizeof(float) * nSw);
    const size_t nDq = d == 2 ? (size_t)s->g.nModes * nExt : 0;
    if (e == cudaSuccess && nDq) e = cudaMalloc(&t->dq32, sizeof(float) * nDq);
    const size_t nBT = d == 2 && s->g.N <= 32 ? nBeta : 0;
    if (e == cudaSuccess && nBT) e = cudaMalloc(&t->beta32T, sizeof(float) * nBT);
    // the rounding residuals of the four FP32 tables (kernel-mode rounding correction)
    if (e == cudaSuccess && nBeta) e = cudaMalloc(&t->beta32lo, sizeof(float) * nBeta);
    if (e == cudaSuccess && nSw) e = cudaMalloc(&t->sw32lo, sizeof(float) * nSw);
    if (e == cudaSuccess && nDq) e = cudaMalloc(&t->dq32lo, sizeof(float) * nDq);
    if (e == cudaSuccess && nBT) e = cudaMalloc(&t->beta32Tlo, sizeof(float) * nBT);
    if (e != cudaSuccess) {
        *err = std::string("kernel-mode table allocation failed: ") + cudaGetErrorString(e);
        cudaFree(d_nodes);
        cudaFree(d_rad);
        cudaFree(t->alpha64); cudaFree(t->alphap64); cudaFree(t->beta64); cudaFree(t->beta32);
        cudaFree(t->sw64); cudaFree(t->sw32); cudaFree(t->dq32); cudaFree(t->beta32T);
        cudaFree(t->beta32lo); cudaFree(t->sw32lo); cudaFree(t->dq32lo); cudaFree(t->beta32Tlo);
        delete t;
        cudaGetLastError();
        return BN_ERR_NOMEM;
    }
    t->bytes = sizeof(double) * 2 * nAl + (sizeof(double) + 2 * sizeof(float)) * (nBeta + nSw) +
               2 * sizeof(float) * (nDq + nBT);
    cudaMemcpyAsync(d_nodes, nodes.data(), sizeof(Node) * nodes.size(), cudaMemcpyHostToDevice, s->stream);
    if (d_rad) cudaMemcpyAsync(d_rad, rad.data(), sizeof(double2) * rad.size(), cudaMemcpyHostToDevice, s->stream);
    k_alpha_tables<<<1024, 256, 0, s->stream>>>(d, s->g.N, t->P, s->Rxi, s->opt.c_phi, s->kernel, (int)rad.size(),
                                               d_rad, d_nodes, t->alpha64, t->alphap64);
    s->launches++;
    if (nBeta) {
        const dim3 gb((nExt + kBT - 1) / kBT, (nExt + kBT - 1) / kBT);
        k_beta_table<<<gb, 256, 0, s->stream>>>(nExt, t->P, t->alpha64, t->alphap64, t->beta64, t->beta32);
        s->launches++;
    }
    {
        std::string e2;
        if (build_nd_tables(s, t, &e2) != BN_OK) {
            *err = e2;
            cudaStreamSynchronize(s->stream);
            cudaFree(d_nodes);
            cudaFree(d_rad);
            cudaFree(t->alpha64); cudaFree(t->alphap64); cudaFree(t->beta64); cudaFree(t->beta32);
            cudaFree(t->sw64); cudaFree(t->sw32); cudaFree(t->dq32); cudaFree(t->beta32T);
        cudaFree(t->beta32lo); cudaFree(t->sw32lo); cudaFree(t->dq32lo); cudaFree(t->beta32Tlo);
            cudaFree(t->alpha32); cudaFree(t->alphap32); cudaFree(t->alphaI64); cudaFree(t->alphapI64);
            cudaFree(t->alphaI32); cudaFree(t->alphapI32);
            delete t;
            return BN_ERR_NOMEM;
        }
    }
    if (nSw) {
        k_sw_table<<<4096, 256, 0, s->stream>>>(s->g.N, t->beta64, t->sw64, t->sw32);
        k_dq_table<<<4096, 256, 0, s->stream>>>(s->g.N, t->beta64, t->dq32, t->dq32lo);
        k_residual_table<<<4096, 256, 0, s->stream>>>((long long)nBeta, t->beta64, t->beta32, t->beta32lo);
        k_residual_table<<<4096, 256, 0, s->stream>>>((long long)nSw, t->sw64, t->sw32, t->sw32lo);
        s->launches += 3;
        if (nBT) {
            k_beta_transpose<<<4096, 256, 0, s->stream>>>(s->g.N, t->beta32, t->beta32T);
            k_beta_transpose<<<4096, 256, 0, s->stream>>>(s->g.N, t->beta32lo, t->beta32Tlo);
            s->launches += 2;
        }
        s->launches++;
    }
    e = cudaStreamSynchronize(s->stream);
    cudaFree(d_nodes);
    cudaFree(d_rad);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        *err = std::string("kernel-mode table build failed: ") + cudaGetErrorString(e);
        cudaFree(t->alpha64); cudaFree(t->alphap64); cudaFree(t->beta64); cudaFree(t->beta32);
        cudaFree(t->sw64); cudaFree(t->sw32); cudaFree(t->dq32); cudaFree(t->beta32T);
        cudaFree(t->beta32lo); cudaFree(t->sw32lo); cudaFree(t->dq32lo); cudaFree(t->beta32Tlo);
        cudaFree(t->alpha32); cudaFree(t->alphap32); cudaFree(t->alphaI64); cudaFree(t->alphapI64);
        cudaFree(t->alphaI32); cudaFree(t->alphapI32);
        delete t;
        return BN_ERR_CUDA;
    }
    t->refcount = 1;
    g_tables[key] = t;
    s->tabs = t;
    return BN_OK;
}

void release_tables(KernelTables* t) {
    if (!t) return;
    std::lock_guard<std::mutex> lock(g_tables_mutex);
    if (--t->refcount > 0) return;
    g_tables.erase(t->key);
    cudaFree(t->alpha64);
    cudaFree(t->alphap64);
    cudaFree(t->beta64);
    cudaFree(t->beta32);
    cudaFree(t->sw64);
    cudaFree(t->sw32);
    cudaFree(t->dq32);
    cudaFree(t->beta32T);
    cudaFree(t->beta32lo);
    cudaFree(t->sw32lo);
    cudaFree(t->dq32lo);
    cudaFree(t->beta32Tlo);
    cudaFree(t->alpha32);
    cudaFree(t->alphap32);
    cudaFree(t->alphaI64);
    cudaFree(t->alphapI64);
    cudaFree(t->alphaI32);
    cudaFree(t->alphapI32);
    delete t;
}

// Per dimension, for b in [-N+1, N-2]: the outputs n with n, n-b in I_N number N-|b|
// and the inner indices s with s, b-s in I_N number N-|b+1|.
static inline long long box_n(int N, int b) { return N - std::abs(b); }
static inline long long box_s(int N, int b) { return N - std::abs(b + 1); }

double count_triple_terms(int d, int N) {
    double c = 2.0 * ((double)N * N * N - N) / 3.0;   // sum_b (N-|b|)(N-|b+1|)
    return std::pow(c, d);
}
double count_pair_terms(int d, int N) { return std::pow(0.75 * N * N, d); }
double count_reducible_terms(int d, int N) {
    return std::pow((double)N * N, d) + std::pow((double)N * N - 1.0, d);
}

// Item order of the mixed kernel for a grid of nblk CTAs, which take the items k nblk + j (k = 0,
// 1, ...) in turn: the items, by estimated cost (descending), are dealt in rounds of nblk, each
// round's heaviest item to the CTA with the least load so far; the CTAs that receive an item of the
// last (partial) round are then numbered first, so that every position below the item count is
// used.  Estimated cost per item = the split cost of its sweep + kItemInstr (staging, P_b, setup).
// The order changes only which CTA adds an item's terms into its partial sums, not the terms.
constexpr long long kItemInstr = 500;
template <typename T>
static std::vector<T> balance_items(const std::vector<T>& meta, const std::vector<long long>& cost, int nblk) {
    const int n = (int)meta.size();
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<long long> load(nblk, 0);
    std::vector<std::vector<int>> mine(nblk);
    std::vector<int> ctas(nblk);
    int last = 0;   // items of the last round
    for (int k = 0; k < n; k += nblk) {
        for (int j = 0; j < nblk; ++j) ctas[j] = j;
        std::stable_sort(ctas.begin(), ctas.end(), [&](int x, int y) { return load[x] < load[y]; });
        last = std::min(nblk, n - k);
        for (int i = 0; i < last; ++i) {
            const int item = order[k + i], c = ctas[i];
            mine[c].push_back(item);
            load[c] += cost[item];
        }
    }
    const size_t rounds = n > 0 ? (size_t)((n + nblk - 1) / nblk) : 0;
    std::vector<int> id(nblk);
    int first = 0, rest = last;   // CTAs with a last-round item get ids 0 .. last-1
    for (int j = 0; j < nblk; ++j) id[j] = mine[j].size() == rounds ? first++ : rest++;
    std::vector<T> out(n);
    for (int j = 0; j < nblk; ++j)
        for (size_t k = 0; k < mine[j].size(); ++k) out[k * nblk + id[j]] = meta[mine[j][k]];
    return out;
}

// Per-item geometry and warp split of the mixed 2-D kernel (8 warps per CTA, RW outputs per
// thread, with or without the per-b orientation choice) for the items `flat` (extended indices of
// b), in the same order, with each item's estimated cost for the CTA layout.  Host only.
static void plan_mixed_items(int N, int RW, bool orientable, const std::vector<int>& flat, std::vector<ItemMeta>* meta_out,
                             std::vector<long long>* cost_out) {
    const int E = 2 * N, h = N / 2;
    std::vector<ItemMeta>& meta = *meta_out;
    std::vector<long long>& cost = *cost_out;
    meta.assign(flat.size(), ItemMeta{});
    cost.assign(flat.size(), 0);
    for (size_t i = 0; i < flat.size(); ++i) {
        const int ib = flat[i], b1 = ib / E - N, b2 = ib % E - N;
        const int bb[2] = {b1, b2};
        int nlo[2], L[2], slo[2], S[2];
        for (int dd = 0; dd < 2; ++dd) {
            nlo[dd] = std::max(-h, bb[dd] - h);
            L[dd] = std::min(h - 1, bb[dd] + h - 1) - nlo[dd] + 1;
            slo[dd] = std::max(-h, bb[dd] - h + 1);
            S[dd] = std::min(h - 1, bb[dd] + h) - slo[dd] + 1;
        }
        ItemMeta m{};
        long long best = -1;
        for (int o = 0; o < (orientable ? 2 : 1); ++o) {   // o = 0: split dim 1, window along dim 2; 1: swapped
            const int du = o == 0 ? 0 : 1, dw = 1 - du;
            const int Gg = (L[dw] + RW - 1) / RW, base = L[du] * Gg;
            SplitChoice sc;
            const long long c = choose_split_host(base, S[du], S[dw], RW, 8, &sc);
            if (best >= 0 && c >= best) continue;
            best = c;
            m.ib = ib;
            m.ginv = (65536 + Gg - 1) / Gg;
            m.linv = (65536 + L[du] - 1) / L[du];
            m.Lu = (short)L[du];
            m.orient = (short)o;
            m.b1 = (short)b1; m.b2 = (short)b2;
            m.nlo_u = (short)nlo[du]; m.nlo_w = (short)nlo[dw]; m.Lw = (short)L[dw];
            m.slo_u = (short)slo[du]; m.Su = (short)S[du]; m.slo_w = (short)slo[dw]; m.Sw = (short)S[dw];
            m.Gg = (short)Gg; m.Au = (short)(L[du] + S[du] - 1); m.Aw = (short)(RW * Gg + S[dw]);
            m.a_ulo = (short)(nlo[du] - slo[du] - S[du] + 1); m.a_wlo = (short)(nlo[dw] - slo[dw] - S[dw]);
            m.quad = (short)(b1 >= -h && b1 < h && b2 >= -h && b2 < h);
            m.J = (short)sc.J; m.tpw = (short)(32 / sc.J); m.chunk = (short)sc.chunk; m.units = (short)sc.units;
            m.base = (short)base;
            m.J2 = (short)sc.J2; m.chunk2 = (short)sc.chunk2; m.units2 = (short)sc.units2; m.tail0 = (short)sc.tail0;
        }
        meta[i] = m;
        cost[i] = best + kItemInstr;
    }
}

// The work items of the cubic part (b with non-empty boxes), heaviest first (host only).
static std::vector<int> cubic_items(int d, int N) {
    const int E = 2 * N, nb = d == 2 ? E * E : E * E * E;
    std::vector<std::pair<long long, int>> items;
    for (int ib = 0; ib < nb; ++ib) {
        int b[3];
        int r = ib;
        for (int i = d - 1; i >= 0; --i) { b[i] = r % E - N; r /= E; }
        long long w = 1;
        for (int i = 0; i < d; ++i) {
            const long long ln = box_n(N, b[i]), ls = box_s(N, b[i]);
            if (ln <= 0 || ls <= 0) { w = 0; break; }
            w *= ln * ls;
        }
        if (w > 0) items.push_back({w, ib});
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) { return x.first > y.first; });
    std::vector<int> flat(items.size());
    for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;
    return flat;
}

// The plan the mixed 2-D kernel runs for N, rw, orientation choice and nblk CTAs, as rows of
// kPlanCols ints in the order the CTAs take the items (bn_plan_mixed2d).  Host only.
std::vector<int> plan_mixed2d_rows(int N, int rw, bool oriented, int nblk) {
    std::vector<ItemMeta> meta;
    std::vector<long long> cost;
    plan_mixed_items(N, rw, oriented, cubic_items(2, N), &meta, &cost);
    meta = balance_items(meta, cost, std::max(1, std::min((int)meta.size(), nblk)));
    std::vector<int> rows;
    rows.reserve(meta.size() * kPlanCols);
    for (const ItemMeta& m : meta) {
        const int r[kPlanCols] = {m.ib, m.orient, m.J, m.chunk, m.units, m.J2, m.chunk2, m.units2, m.tail0, m.base,
                                  m.Lu, m.Lw, m.Su, m.Sw};
        rows.insert(rows.end(), r, r + kPlanCols);
    }
    return rows;
}

bn_status build_work_list(bn_solver* s, std::string* err) {
    const int d = s->g.d, N = s->g.N, E = s->g.E;
    std::vector<std::pair<long long, int>> items;
    const int nb = d == 2 ? E * E : E * E * E;
    double total = 0;
    for (int ib = 0; ib < nb; ++ib) {
        int b[3];
        int r = ib;
        for (int i = d - 1; i >= 0; --i) { b[i] = r % E - N; r /= E; }
        long long w = 1;
        for (int i = 0; i < d; ++i) {
            long long ln = box_n(N, b[i]), ls = box_s(N, b[i]);
            if (ln <= 0 || ls <= 0) { w = 0; break; }
            w *= ln * ls;
        }
        if (w > 0) { items.push_back({w, ib}); total += (double)w; }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) { return x.first > y.first; });
    std::vector<int> flat(items.size());
    for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;
    // b in I_N only (the quadratic part), ordered by output-box size
    std::vector<std::pair<long long, int>> qitems;
    for (int ib = 0; ib < nb; ++ib) {
        int b[3];
        int r = ib;
        for (int i = d - 1; i >= 0; --i) { b[i] = r % E - N; r /= E; }
        long long w = 1;
        for (int i = 0; i < d; ++i) {
            if (b[i] < -N / 2 || b[i] >= N / 2) { w = 0; break; }
            w *= box_n(N, b[i]);
        }
        if (w > 0) qitems.push_back({w, ib});
    }
    std::stable_sort(qitems.begin(), qitems.end(),
                     [](const std::pair<long long, int>& x, const std::pair<long long, int>& y) { return x.first > y.first; });
    std::vector<int> qflat(qitems.size());
    for (size_t i = 0; i < qitems.size(); ++i) qflat[i] = qitems[i].second;
    if (cudaMalloc(&s->work.items, sizeof(int) * flat.size()) != cudaSuccess ||
        cudaMalloc(&s->work_quad.items, sizeof(int) * qflat.size()) != cudaSuccess) {
        cudaGetLastError();
        *err = "work list allocation failed";
        return BN_ERR_NOMEM;
    }
    cudaMemcpy(s->work.items, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(s->work_quad.items, qflat.data(), sizeof(int) * qflat.size(), cudaMemcpyHostToDevice);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (sms <= 0) sms = 152;
    for (int v = 0; d == 2 && v < 4; ++v) {
        // per-item geometry of the mixed kernel (8 warps per CTA, RW = 8 or 16 outputs per thread,
        // with or without the per-b orientation choice)
        const int RW = v < 2 ? 8 : 16;
        const bool orientable = (v & 1) != 0;
        std::vector<ItemMeta> meta;
        std::vector<long long> cost;
        plan_mixed_items(N, RW, orientable, flat, &meta, &cost);
        configure_mixed2d();
        const int nblk = std::max(1, std::min((int)flat.size(), mixed2d_ctas_per_sm(N, RW) * sms));
        meta = balance_items(meta, cost, nblk);
        if (cudaMalloc(&s->work.meta[v], sizeof(ItemMeta) * meta.size()) != cudaSuccess) {
            cudaGetLastError();
            *err = "work list allocation failed";
            return BN_ERR_NOMEM;
        }
        cudaMemcpy(s->work.meta[v], meta.data(), sizeof(ItemMeta) * meta.size(), cudaMemcpyHostToDevice);
    }
    s->work.count = (int)flat.size();
    s->work.terms = total;
    s->work_quad.count = (int)qflat.size();
    return BN_OK;
}

// The item lists of the kernels that take items k nblk + blockIdx.x (k_fused2d: FP64, and mixed
// N > 32; k_triple in 3-D), dealt to their nblk = min(count, n_partials) CTAs as balance_items does
// for the mixed kernel, with the terms of an item (cubic list: |box_n| |box_s|; quadratic list:
// |box_n|) plus kItemTerms for its fixed work as the cost.  The mixed 2-D kernel for N <= 32 deals
// its own per-item metadata and keeps the lists as they are.
constexpr long long kItemTerms = 4000;
bn_status balance_work_lists(bn_solver* s, std::string* err) {
    const int d = s->g.d, N = s->g.N, E = s->g.E;
    if (d == 2 && s->opt.precision == BN_MIXED && N <= 32) return BN_OK;
    WorkList* lists[2] = {&s->work, &s->work_quad};
    for (int li = 0; li < 2; ++li) {
        WorkList* wl = lists[li];
        const int n = wl->count;
        if (n <= 1 || !wl->items) continue;
        const int nblk = std::max(1, std::min(n, s->n_partials));
        std::vector<int> items(n);
        if (cudaMemcpy(items.data(), wl->items, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            *err = "work list read-back failed";
            return BN_ERR_CUDA;
        }
        std::vector<long long> cost(n);
        for (int i = 0; i < n; ++i) {
            int r = items[i];
            long long w = 1;
            for (int k = d - 1; k >= 0; --k) {
                const int b = r % E - N;
                r /= E;
                w *= li == 0 ? box_n(N, b) * box_s(N, b) : box_n(N, b);
            }
            cost[i] = w + kItemTerms;
        }
        const std::vector<int> laid = balance_items(items, cost, nblk);
        if (cudaMemcpy(wl->items, laid.data(), sizeof(int) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            *err = "work list upload failed";
            return BN_ERR_CUDA;
        }
    }
    return BN_OK;
}

}  // namespace bn
