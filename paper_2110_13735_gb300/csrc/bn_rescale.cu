// bn_rescale.cu -- the velocity-rescaling method (Mouton & Rey, Sec. 3), 2-D and 3-D: the kernels of one
// forward Euler step of Sec. 3.3 around the operator evaluation (and the stage average of the RK2 form
// that bn_api.cu builds from them), and the host-side temperature solve.
//
// The state is G on the grid xi_j = 2 pi j / N of [-pi, pi]^d (the solver's box T = pi), with
// f(v) = (pi w / L)^d G((pi w / L)(v - u)).  Per step (bn_step_rescaled in bn_api.cu):
//   Q^n = Q_{eps (pi w / L)^d}(G^n)                         (the solver's operator, eps rescaled)
//   S0, S1, S2 = sum_j Q^n_j (1, xi_j, |xi_j|^2)           (k_resc_moments, fixed order, FP64)
//   rho, u, e advanced with them; T, z solved; w = sqrt(T) (quantum) or sqrt(T + |u|^2/d)
//   div = sum_c d/dxi_c ((a xi_c - b_c) G^n): per component the flux (k_resc_flux), its modes, times
//         i k_c (k_resc_deriv; the k_c = -N/2 mode gets 0), summed, transformed back
//   G^{n+1} = G^n + dt (-div + (pi w / L)^{-gamma} Q^n)   (k_resc_update)
// The temperature solve (step 3(b) of Sec. 3.3; Sec. 1.2): T = 2e/d classically; for eps != 0,
// x = |eps| rho (d / (4 pi e))^{d/2} must lie in I_eq, then z solves x = K_1(z)^2 / K_2(z) by Brent's
// method (on mu = ln z for Fermi-Dirac particles) and T = |eps| rho / (2 pi K_1(z)); K_1 and K_2 are
// the Fermi-Dirac (eps < 0) or Bose-Einstein (eps > 0) integrals of orders 1 and 2: ln(1 + z) or
// -ln(1 - z), and -Li_2(-z) or Li_2(z).  In 3-D the orders are 3/2 and 5/2 (nu = d/2 in eq_fugacity),
// x = |eps| rho (3 / (4 pi e))^{3/2} = K_{3/2}^{5/2} / K_{5/2}^{3/2} and T = (|eps| rho / K_{3/2})^{2/3} / (2 pi);
// those integrals are taken by double-exponential quadrature of their definition.
#include <cmath>
#include <string>

#include "bn_internal.cuh"

namespace bn {

namespace {

constexpr int kResThreads = 256;

// coordinate c of grid index j in d dimensions (axis 0 slowest), shifted to I_N
__device__ __forceinline__ int coord(int j, int c, int d, int N) {
    for (int a = d - 1; a > c; --a) j /= N;
    return j % N - N / 2;
}

// sums over the grid of Q, xi_c Q (c < d), |xi|^2 Q into out[0], out[1..d], out[d+1] (one block,
// fixed order: deterministic)
__global__ void __launch_bounds__(kResThreads) k_resc_moments(int d, int N, const double* __restrict__ Q,
                                                              double* __restrict__ out) {
    __shared__ double sh[5][kResThreads];
    const int n = d == 2 ? N * N : N * N * N, tid = threadIdx.x;
    const double h = 2.0 * M_PI / N;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int j = tid; j < n; j += kResThreads) {
        const double q = Q[j];
        double r2 = 0.0;
        acc[0] += q;
        for (int c = 0; c < d; ++c) {
            const double x = h * coord(j, c, d, N);
            acc[1 + c] = fma(x, q, acc[1 + c]);
            r2 = fma(x, x, r2);
        }
        acc[1 + d] = fma(r2, q, acc[1 + d]);
    }
    for (int c = 0; c < 5; ++c) sh[c][tid] = acc[c];
    __syncthreads();
    for (int st = kResThreads / 2; st >= 1; st >>= 1) {
        if (tid < st)
            for (int c = 0; c < 5; ++c) sh[c][tid] += sh[c][tid + st];
        __syncthreads();
    }
    if (tid < d + 2) out[tid] = sh[tid][0];
}

// H = (a xi_c - b) G, component c of the rescaling flux
__global__ void k_resc_flux(int d, int N, int n, const double* __restrict__ G, double a, double b, int c,
                            double* __restrict__ H) {
    const double h = 2.0 * M_PI / N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        H[j] = (a * (h * coord(j, c, d, N)) - b) * G[j];
}

// acc (+)= i k_c M: the modes of the derivative along axis c (k in I_N; the k_c = -N/2 mode gets 0)
__global__ void k_resc_deriv(int d, int N, int n, const double2* __restrict__ M, double2* __restrict__ acc, int c,
                             int first) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int k = coord(j, c, d, N);
        const double kk = k == -N / 2 ? 0.0 : (double)k;
        const double2 m = M[j];
        const double2 v = make_double2(-kk * m.y, kk * m.x);
        if (first) {
            acc[j] = v;
        } else {
            double2 t = acc[j];
            t.x += v.x;
            t.y += v.y;
            acc[j] = t;
        }
    }
}

// G += dt (-div + qc Q)
__global__ void k_resc_update(int n, double* __restrict__ G, const double* __restrict__ div, const double* __restrict__ Q,
                              double dt, double qc) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        G[j] = fma(dt, fma(qc, Q[j], -div[j]), G[j]);
}

// G = (G0 + G) / 2
__global__ void k_resc_average(int n, double* __restrict__ G, const double* __restrict__ G0) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) G[j] = 0.5 * (G0[j] + G[j]);
}

inline int blocks_for(int n) { return (n + kResThreads - 1) / kResThreads; }

// ------------------------------------------------------------------ host: dilogarithm, K, Brent
// Li_2(x) for x <= 1: the series sum x^k / k^2 for |x| <= 1/2; Euler's reflection
// Li_2(x) = pi^2/6 - ln(x) ln(1 - x) - Li_2(1 - x) on (1/2, 1]; Landen's identity
// Li_2(x) = -Li_2(x / (x - 1)) - ln(1 - x)^2 / 2 on [-1, -1/2); the inversion
// Li_2(x) = -pi^2/6 - ln(-x)^2 / 2 - Li_2(1 / x) below -1.
double li2_series(double x) {
    double total = 0.0, term = x;
    for (int k = 1; k < 200; ++k) {
        const double add = term / ((double)k * k);
        total += add;
        if (std::fabs(add) <= 1e-18 * std::fabs(total)) break;
        term *= x;
    }
    return total;
}

double li2(double x) {
    const double pi2_6 = M_PI * M_PI / 6.0;
    if (x == 1.0) return pi2_6;
    if (std::fabs(x) <= 0.5) return li2_series(x);
    if (x > 0.5) return pi2_6 - std::log(x) * std::log1p(-x) - li2_series(1.0 - x);
    if (x >= -1.0) {
        const double l = std::log1p(-x);
        return -li2_series(x / (x - 1.0)) - 0.5 * l * l;
    }
    const double l = std::log(-x);
    return -pi2_6 - 0.5 * l * l - li2(1.0 / x);
}

// K_nu(z), nu = 1, 2: Fermi-Dirac (eps < 0) or Bose-Einstein (eps > 0, 0 < z < 1)
double k_nu(int nu, double z, double eps) {
    if (eps < 0) return nu == 1 ? std::log1p(z) : -li2(-z);
    return nu == 1 ? -std::log1p(-z) : li2(z);
}

// int_a^b f(t) dt by the tanh-sinh rule t = a + (b - a) / (1 + e^{-2 phi}), phi = (pi/2) sinh(u),
// halving the step u from 1/2 until two levels agree to 1e-15 (Takahasi and Mori's double-exponential
// quadrature).  The nodes crowd both ends, where the integrands below have their only sharp features.
template <typename F>
double tanh_sinh(F f, double a, double b) {
    const double half = 0.5 * (b - a);
    auto term = [&](double u) {
        const double phi = 0.5 * M_PI * std::sinh(u);
        const double c = std::cosh(phi);
        const double w = half * 0.5 * M_PI * std::cosh(u) / (c * c);
        if (!(w > 0.0)) return 0.0;
        // distance to the nearer end without cancellation: (b - a) / (1 + e^{2|phi|})
        const double near = (b - a) / (1.0 + std::exp(2.0 * std::fabs(phi)));
        return w * f(phi < 0 ? a + near : b - near);
    };
    const double umax = 4.0;   // weights there are below 1e-35 of the central one
    double h = 0.5;
    double sum = term(0.0);
    for (double u = h; u <= umax; u += h) sum += term(u) + term(-u);
    double prev = h * sum;
    for (int level = 0; level < 9; ++level) {
        h *= 0.5;
        for (double u = h; u <= umax; u += 2.0 * h) sum += term(u) + term(-u);
        const double cur = h * sum;
        if (level >= 2 && std::fabs(cur - prev) <= 1e-15 * std::fabs(cur)) return cur;
        prev = cur;
    }
    return prev;
}

// K_nu(e^mu) for nu = n2 / 2 in {3/2, 5/2}: Gamma(nu)^{-1} int_0^inf x^{nu-1} / (e^{x - mu} + s) dx,
// s = +1 Fermi-Dirac (eps < 0), s = -1 Bose-Einstein (eps > 0, mu < 0).  In t = sqrt(x) the
// integrand 2 t^{n2-1} / (e^{t^2 - mu} + s) is smooth; for mu > 0 the range is split at t = sqrt(mu),
// where the Fermi step sits, and it ends where e^{t^2 - mu} > e^{49}.
double k_half(int n2, double mu, double eps) {
    const bool fd = eps < 0;
    auto f = [&](double t) {
        const double t2 = t * t, p = n2 == 3 ? t2 : t2 * t2;
        const double den = fd ? std::exp(t2 - mu) + 1.0 : std::expm1(t2 - mu);
        return 2.0 * p / den;
    };
    const double t0 = std::sqrt(std::max(mu, 0.0));
    double v = tanh_sinh(f, t0, t0 + 7.0);
    if (t0 > 0.0) v += tanh_sinh(f, 0.0, t0);
    return v / std::tgamma(0.5 * n2);
}

// Brent's root finder on [a, b] with f(a) f(b) < 0: inverse quadratic interpolation or the secant
// step when it stays inside the bracket and shrinks it fast enough, bisection otherwise.
template <typename F>
bool brent(F f, double a, double b, double tol, double* root) {
    double fa = f(a), fb = f(b);
    if (!(fa * fb <= 0.0) || !std::isfinite(fa) || !std::isfinite(fb)) return false;
    if (std::fabs(fa) < std::fabs(fb)) {
        std::swap(a, b);
        std::swap(fa, fb);
    }
    double c = a, fc = fa, d = b - a, e = d;
    for (int it = 0; it < 300; ++it) {
        if (fb == 0.0) break;
        if ((fb > 0) == (fc > 0)) {   // keep the root between b and c
            c = a;
            fc = fa;
            d = e = b - a;
        }
        if (std::fabs(fc) < std::fabs(fb)) {
            a = b; b = c; c = a;
            fa = fb; fb = fc; fc = fa;
        }
        const double m = 0.5 * (c - b);
        const double t = 2.0 * 2.2e-16 * std::fabs(b) + 0.5 * tol;
        if (std::fabs(m) <= t) break;
        if (std::fabs(e) >= t && std::fabs(fa) > std::fabs(fb)) {
            double p, q;
            const double s = fb / fa;
            if (a == c) {   // secant
                p = 2.0 * m * s;
                q = 1.0 - s;
            } else {        // inverse quadratic interpolation through a, b, c
                const double qa = fa / fc, r = fb / fc;
                p = s * (2.0 * m * qa * (qa - r) - (b - a) * (r - 1.0));
                q = (qa - 1.0) * (r - 1.0) * (s - 1.0);
            }
            if (p > 0) q = -q;
            else p = -p;
            if (2.0 * p < std::min(3.0 * m * q - std::fabs(t * q), std::fabs(e * q))) {
                e = d;
                d = p / q;
            } else {
                d = m;
                e = m;
            }
        } else {
            d = m;
            e = m;
        }
        a = b;
        fa = fb;
        b += std::fabs(d) > t ? d : (m > 0 ? t : -t);
        fb = f(b);
    }
    *root = b;
    return std::isfinite(b);
}

}  // namespace

bn_status rescale_temperature(int d, double eps, double rho, double e, double* T, double* z, std::string* err) {
    if (!(rho > 0) || !(e > 0) || !std::isfinite(rho) || !std::isfinite(e)) {
        *err = "rescaling: non-positive or non-finite mass or internal energy";
        return BN_ERR_STATE;
    }
    if (eps == 0.0) {
        *T = 2.0 * e / d;
        *z = 0.0;
        return BN_OK;
    }
    if (d == 3) {
        // nu = 3/2: x = K_{3/2}(z)^{5/2} / K_{5/2}(z)^{3/2} (eq_fugacity), compared in logarithms so that
        // integrals of size e^{-600} do not underflow; Fermi-Dirac on mu = ln z in [-600, 700], I_eq =
        // (0, (5/3) sqrt(10/pi)); Bose-Einstein on lambda = ln(-mu) in [-690, ln 600] (z = e^{-e^lambda},
        // which resolves z -> 1), I_eq = (0, zeta(3/2)^{5/2} / zeta(5/2)^{3/2})
        const double x = std::fabs(eps) * rho * std::pow(3.0 / (4.0 * M_PI * e), 1.5);
        const double lx = std::log(x);
        auto lF = [&](double mu) {
            return 2.5 * std::log(k_half(3, mu, eps)) - 1.5 * std::log(k_half(5, mu, eps)) - lx;
        };
        double mu = 0.0;
        bool ok;
        if (eps < 0) {
            const double xmax = 5.0 / 3.0 * std::sqrt(10.0 / M_PI);
            if (!(x > 0.0 && x < xmax)) {
                *err = "rescaling: Fermi-Dirac moments outside I_eq (degenerate state)";
                return BN_ERR_STATE;
            }
            ok = brent(lF, -600.0, 700.0, 1e-14, &mu);
        } else {
            const double zeta32 = 2.612375348685488, zeta52 = 1.341487257250917;
            const double xmax = std::pow(zeta32, 2.5) / std::pow(zeta52, 1.5);
            if (!(x > 0.0 && x < xmax)) {
                *err = "rescaling: Bose-Einstein moments outside I_eq (condensed state)";
                return BN_ERR_STATE;
            }
            double lam = 0.0;
            ok = brent([&](double l) { return lF(-std::exp(l)); }, -690.0, std::log(600.0), 1e-14, &lam);
            mu = -std::exp(lam);
        }
        if (!ok) {
            *err = "rescaling: the fugacity equation has no root in its bracket";
            return BN_ERR_STATE;
        }
        *z = std::exp(mu);
        *T = std::pow(std::fabs(eps) * rho / k_half(3, mu, eps), 2.0 / 3.0) / (2.0 * M_PI);
        return BN_OK;
    }
    const double x = std::fabs(eps) * rho * (d / (4.0 * M_PI * e));
    double zz = 0.0;
    bool ok;
    if (eps < 0) {
        if (!(x > 0.0 && x < 2.0)) {
            *err = "rescaling: Fermi-Dirac moments outside I_eq (degenerate state)";
            return BN_ERR_STATE;
        }
        auto g = [&](double mu) {
            const double zz1 = std::exp(mu);
            const double k1 = k_nu(1, zz1, eps);
            return k1 * k1 / k_nu(2, zz1, eps) - x;
        };
        double mu = 0.0;
        ok = brent(g, -60.0, 60.0, 1e-15, &mu);
        zz = std::exp(mu);
    } else {
        auto g = [&](double zz1) {
            const double k1 = k_nu(1, zz1, eps);
            return k1 * k1 / k_nu(2, zz1, eps) - x;
        };
        ok = brent(g, 1e-300, 1.0 - 1e-16, 1e-300, &zz);
    }
    if (!ok || !(zz > 0)) {
        *err = "rescaling: the fugacity equation has no root in its bracket";
        return BN_ERR_STATE;
    }
    *z = zz;
    *T = std::fabs(eps) * rho / k_nu(1, zz, eps) / (2.0 * M_PI);
    return BN_OK;
}

void launch_resc_moments(bn_solver* s, const double* Q, double* out_dev) {
    k_resc_moments<<<1, kResThreads, 0, s->stream>>>(s->g.d, s->g.N, Q, out_dev);
    s->launches++;
}

// div = sum_c d/dxi_c ((a xi_c - b_c) G) into `div`, then G += dt (-div + qc Q).
void launch_resc_advance(bn_solver* s, double* G, const double* Q, double a, const double* b, double dt, double qc,
                         double* H, double2* M, double2* acc, double* div) {
    const int d = s->g.d, N = s->g.N, n = s->g.nModes;
    for (int c = 0; c < d; ++c) {
        k_resc_flux<<<blocks_for(n), kResThreads, 0, s->stream>>>(d, N, n, G, a, b[c], c, H);
        launch_dft_forward(s, H, M);
        k_resc_deriv<<<blocks_for(n), kResThreads, 0, s->stream>>>(d, N, n, M, acc, c, c == 0);
        s->launches += 2;
    }
    launch_dft_inverse_real(s, acc, div, 1.0);
    k_resc_update<<<blocks_for(n), kResThreads, 0, s->stream>>>(n, G, div, Q, dt, qc);
    s->launches++;
}

void launch_resc_average(bn_solver* s, double* G, const double* G0) {
    const int n = s->g.nModes;
    k_resc_average<<<blocks_for(n), kResThreads, 0, s->stream>>>(n, G, G0);
    s->launches++;
}

}  // namespace bn
