/*
 * bn.h -- C ABI of the GB300 (sm_103a) Fourier-Galerkin Boltzmann-Nordheim
 * collision-operator library (libbn.so).
 *
 * The library evaluates the Fourier-Galerkin (Filbet-Hu-Jin) approximation of
 * the space-homogeneous Boltzmann-Nordheim collision operator Q_eps(f) on the
 * periodised velocity box [-T,T]^d, d = 2 or 3 (Mouton & Rey,
 * arXiv:2110.13735), and advances d f/dt = Q_eps(f) in time:
 *
 *   grid        v_j = 2 T j / N, j in I_N = {-N/2, ..., N/2-1}^d        (Sec. 3.3)
 *   transform   G^_k = N^-d sum_j f_j exp(-2 i pi k.j/N)                   (Sec. 3.3, step 2(a))
 *   operator    Q^_n = sum_{k+l=n} [beta(k,l) - beta(l,l)] G^_k G^_l
 *                      - alpha sum_{k+l+m=n} [beta(k+m,l+m) + beta(l,m)
 *                                             - beta(l+m,l) - beta(l,l+m)] G^_k G^_l G^_m
 *               with alpha = -eps, k,l,m,n in I_N, no wrap-around       (Lemma, Sec. 2.3; step 2(c))
 *   kernel      beta(a,b) = C sum_p alpha_p(a) alpha'_p(b)                (Sec. 2.5, eq. betadD;
 *               2-D hard spheres: the Lemma's definition of beta^R by quadrature)
 *   scaling     Q_eps(f)(v_j) = (T/pi)^{d+gamma} Re sum_n Q^_n exp(2 i pi n.j/N)   (Sec. 3.2)
 *
 * eps = +1 bosons, -1 fermions, 0 classical particles (any real eps is
 * accepted, e.g. eps = -hbar^d).  Kernels: 2-D Maxwell molecules (gamma = 0),
 * 2-D and 3-D hard spheres (gamma = 1), b == 1, truncation radius R in velocity
 * units with R_xi = pi R / T satisfying R_xi (3 + sqrt 2) <= 2 pi (Sec. 4.1).
 *
 * Conventions (all entry points):
 *  - Every call returns a bn_status; no call aborts, throws or exits.  After a
 *    failure bn_last_error() returns a message for the calling thread.
 *  - Host arrays are owned by the caller; the library copies in and out and
 *    keeps no host pointer.  Device arrays passed in ("_device" calls) must be
 *    on the solver's device; the library reads/writes them on the solver's
 *    stream and keeps no pointer after the call returns.
 *  - Arrays of grid values are row-major over I_N^d (index j_i + N/2, last
 *    dimension fastest), FP64, count = N^d.
 *  - A solver owns all of its device memory and one CUDA stream (the one given
 *    to bn_create_solver, or the legacy default stream if NULL).  A solver is
 *    not thread-safe; distinct solvers may be used from distinct threads.
 *  - Calls that return host data synchronise the solver's stream; the others
 *    are asynchronous with respect to the host unless stated.
 */
#ifndef BN_H
#define BN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bn_solver bn_solver;

typedef enum {
    BN_OK = 0,
    BN_ERR_ARG = -1,         /* invalid argument (sizes, d, N, kernel, null pointer) */
    BN_ERR_ALIAS = -2,       /* R_xi (3 + sqrt 2) > 2 pi: anti-aliasing condition violated (Sec. 4.1) */
    BN_ERR_NOMEM = -3,       /* device or host allocation failed */
    BN_ERR_CUDA = -4,        /* a CUDA runtime call failed */
    BN_ERR_NONFINITE = -5,   /* the state became NaN/Inf during step_rk (state rolled back) */
    BN_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    BN_ERR_STATE = -7,       /* call out of order (e.g. no state set), or moments that admit no
                                equilibrium temperature (velocity rescaling: outside I_eq) */
    BN_ERR_UNSUPPORTED = -8  /* combination not implemented (e.g. 3-D Maxwell molecules) */
} bn_status;

typedef enum { BN_MAXWELL = 0, BN_HARD_SPHERE = 1 } bn_kernel;

typedef enum { BN_FP64 = 0, BN_MIXED = 1 } bn_precision;

typedef struct {
    int M;            /* 2-D angular points of eq. beta2D; 0 = default 2N */
    int M1, M2;       /* 3-D (theta, phi) points of eq. beta3D; 0 = default N/2 each.
                         2-D hard spheres: M1 = Gauss-Legendre points per radius of the
                         kernel-mode quadrature (default N + 8); M2 unused */
    int precision;    /* BN_FP64, or BN_MIXED: FP32 bulk pair/triple sums with
                         compensated accumulation, FP64 kernel modes, transforms,
                         combination, moments, conservation correction and state */
    int conserve;     /* 1: project Q onto zero mass, momentum and energy (FP64) */
    double c_phi;     /* C_Phi; 0 = default 1/(2 pi) (2-D), 1/(4 pi) (3-D) */
    int integrator;   /* 0 = classical RK4, 1 = SSP-RK2 (Heun) */
    int quad3d;       /* 3-D theta rule: 0 = Gauss-Legendre in cos(theta),
                         1 = the printed sin(theta_p)-weighted rectangle rule */
    double escalate_at; /* mixed precision only: when |eps| max f >= escalate_at after a
                         bn_step_rk / bn_step_rk_batch call (near Fermi saturation or
                         condensation onset), the solver switches to FP64 for the rest of its
                         life; 0 = never.  Sizes with no FP64 kernel (3-D N > 32) stay in
                         mixed precision and clear escalate_at */
    int mixed_rw;     /* mixed precision, d = 2, N <= 32: outputs per thread of the fused
                         kernel's sweep, 8 or 16; 0 = chosen by the autotuner (the variants
                         timed on the solver's stream at creation, cached per device and N;
                         the per-b orientation choice is tuned in either case) */
    int mixed_variant; /* mixed 2-D N <= 32: 0 = as mixed_rw says; 1..4 forces the kernel
                         variant (8, 8 oriented, 16, 16 oriented outputs per thread) */
    int wrap;         /* 0 = LINEAR truncation (the Lemma: k, l, m, n in I_N, sums exact; the
                         default); 1 = CIRCULAR: every index sum reduced into I_N modulo N and
                         beta taken at the reduced representatives, the index arithmetic of the
                         Appendix's discrete-transform evaluation */
    int beta_resident; /* 3-D and CIRCULAR: 1 = produce the kernel-mode slices beta(., b) once and
                         keep them on the device when they fit the slice budget (else they are
                         recomputed from the quadrature factors at every evaluation, the default) */
    long long beta_budget_mb; /* 3-D and CIRCULAR: device memory (MiB) for the slices of one round
                         (0 = 40% of the free memory, at most 40 GiB); slices that do not fit are
                         produced and consumed in several rounds per evaluation */
    int pair_weights; /* 3-D and CIRCULAR: 0 = form the weights of the quadratic and reducible pair
                         sums over I_N x I_N once, when they fit in 45% of the free memory (the
                         default); 1 = recompute them from the quadrature factors at every
                         evaluation */
    int shard_index, shard_count; /* 3-D and CIRCULAR, one evaluation split over shard_count
                         solvers (one per GPU): with shard_count > 1, bn_eval_collision_modes returns
                         the modes Q^_n of the output planes n_0 of shard shard_index of
                         bn_plan_shards and zero elsewhere, so that the sum of the shard_count
                         results (one all-reduce of N^d complex values) is Q^; bn_eval_collision and
                         the stepping calls of such a solver return BN_ERR_UNSUPPORTED.  0 = none */
    int debug_wait_giveup; /* testing only: 1 = the first bounded wait for a bulk copy in the
                         operator kernels gives up at once, so that the call reports BN_ERR_TIMEOUT
                         (the kernel records it and still waits, bounded, for its copy before going
                         on or returning; the next call starts clean); 0 = normal waits */
    int beta_split;   /* mixed precision, d = 2, LINEAR: 1 = kernel-mode rounding correction.  The
                         FP32 tables hold beta (and the weights formed from it) rounded to FP32; a
                         second pass of the same FP32 kernels over tables of the residuals
                         x - fl32(x) gives the part of Q^ that the rounding leaves out (Q^ is
                         linear in beta), so that the two passes carry the weights to about 48
                         bits.  The rounding of beta is one fixed perturbation of the operator:
                         its error does not average out over time steps and, without the
                         correction, it dominates the drift of a mixed run from the FP64 one.  In
                         the stepping calls the correction is formed at the first stage of each
                         step and reused by the later stages of that step; a standalone
                         evaluation forms it every call.  0 = off (ignored in FP64) */
} bn_options;

/* Fill *opt with the defaults (all zero: FP64, RK4, no correction). */
bn_status bn_default_options(bn_options* opt);

/* sizeof(bn_options) and sizeof(bn_request) as this library was compiled, for bindings that
 * declare the structures themselves to check their layout against.  No error case. */
size_t bn_options_bytes(void);
size_t bn_request_bytes(void);

/*
 * Create a solver for the operator (d, N, T, R, kernel, eps).  d in {2,3};
 * N even, 4 <= N <= 64 (2-D) or <= 48 (3-D; FP64 up to 32, CIRCULAR FP64 2-D up
 * to 62); T > 0 the box half-width; R > 0
 * the truncation radius (velocity units); kernel BN_MAXWELL (d = 2) or
 * BN_HARD_SPHERE (d = 2 or 3); opt may be NULL; cuda_stream is a cudaStream_t or
 * NULL.  Builds the kernel-mode tables in FP64 on the device (once per
 * solver; solvers with equal (d, N, R_xi, kernel, M, precision) share them).
 * On success *out owns the solver; release it with bn_destroy_solver.
 */
bn_status bn_create_solver(int d, int N, double T, double R, int kernel, double eps,
                           const bn_options* opt, void* cuda_stream, bn_solver** out);

/* Release the solver and its device memory (shared tables are refcounted). */
void bn_destroy_solver(bn_solver* s);

/* State f_j = f(v_j) from host memory (count = N^d); resets t to 0. */
bn_status bn_set_state(bn_solver* s, const double* f, size_t count);
/* Same from device memory on the solver's device. */
bn_status bn_set_state_device(bn_solver* s, const double* f_dev, size_t count);
/* Copy the current state to host memory (synchronises). */
bn_status bn_get_state(bn_solver* s, double* f, size_t count);
/* Copy the current state to device memory (asynchronous on the solver's stream). */
bn_status bn_get_state_device(bn_solver* s, double* f_dev, size_t count);

/* Q_eps(f)(v_j) of the current state, in velocity units, to host memory (synchronises). */
bn_status bn_eval_collision(bn_solver* s, double* Q, size_t count);
/* Q_eps(f) of the device array f_dev into the device array Q_dev (both N^d FP64);
 * the solver's state is not touched.  Asynchronous on the solver's stream. */
bn_status bn_eval_collision_device(bn_solver* s, const double* f_dev, double* Q_dev, size_t count);

/* Fourier modes Q^_n, n in I_N^d (row-major at n_i + N/2), of the current
 * state (Lemma, Sec. 2.3; before the inverse transform and the (T/pi)^{d+gamma}
 * prefactor), as interleaved (re, im) FP64 pairs: count = 2 N^d.  Synchronises. */
bn_status bn_eval_collision_modes(bn_solver* s, double* Qhat, size_t count);

/*
 * Q_eps(f) of the device array f_dev into the device array Q_dev (both N^d FP64,
 * on the solver's device), like bn_eval_collision_device but without allocating
 * any device memory.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate while they evaluate -- cudaMalloc/cudaFree
 * synchronise the whole device and fail when another allocator in the process
 * (for instance a framework's caching allocator) has already reserved the
 * memory -- and it also leaves the solver's own buffers untouched.
 *
 * Its working memory is one file-scope device array of 12 MiB that every
 * device loading the library holds until the process exits; every 2-D solver
 * (N <= 64) fits, larger needs are rejected with BN_ERR_ARG.  All calls in the
 * process share that array and it keeps the last call's contents; each call
 * clears what must start at zero.  Calls whose GPU work overlaps in time (other
 * threads, other streams) race on it: serialise them.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), which is
 * also when the CUDA driver loads the array onto that device.  Every call reads an
 * error flag back and synchronises cuda_stream, so no call can be made while a stream is
 * being captured.  The current device must be the solver's device (BN_ERR_ARG
 * otherwise).  The solver's read-only kernel-mode
 * tables, work lists and twiddles are used; the solver itself is not modified.
 * With opt.beta_split the residual-table pass runs first in the same scratch and its
 * modes are added, as in bn_eval_collision_device.
 * 2-D solvers only (BN_ERR_UNSUPPORTED otherwise).  Runs on cuda_stream (NULL =
 * legacy default stream) and returns when Q_dev holds the result.
 */
bn_status bn_eval_collision_noalloc(const bn_solver* s, const double* f_dev, double* Q_dev, size_t count,
                                    void* cuda_stream);

/* Advance the state by nsteps steps of size dt with the chosen integrator
 * (c = 1 in eq. Boltzmann_homo).  The steps run as one captured CUDA graph per
 * step.  If the state turns non-finite the call returns BN_ERR_NONFINITE and
 * the state is that of the last finite step (bn_moments reports its time).
 * Synchronises the solver's stream. */
bn_status bn_step_rk(bn_solver* s, double dt, int nsteps);

/*
 * Moments of the current state (Sec. 4, head), FP64, count >= d + 6:
 * out = [rho, rho u_1 .. rho u_d, e, E_c, H, max f, t] with
 * rho = dv sum f, rho u = dv sum v f, e = dv sum |v-u|^2 f / (2 rho),
 * E_c = dv sum |v|^2 f, H = dv sum [f ln f + (1 + eps f)/(-eps) ln(1 + eps f)]
 * (eps != 0; dv sum f ln f for eps = 0; non-positive arguments skipped),
 * dv = (2T/N)^d.  Synchronises.
 */
bn_status bn_moments(bn_solver* s, double* out, size_t count);

/* Work counts of one evaluation: out[0] = quadratic terms (C2), out[1] =
 * terms of the reducible cubic sums, out[2] = terms of the Q_{1,q} triple sum
 * (C3, 0 when eps = 0), out[3] = N^d.  count >= 4. */
bn_status bn_work_counts(const bn_solver* s, double* out, size_t count);

/* Device kernel launches issued by this solver since creation (all kernels). */
long long bn_kernel_launches(const bn_solver* s);

/*
 * Live timing of the dominant kernel (the Q_{1,q} triple sum): when enabled,
 * CUDA events are recorded on the solver's stream around every launch of that
 * kernel (also inside the captured step graph).  bn_profile_read returns
 * out[0] = summed event duration in ms and out[1] = number of launches timed
 * since the last read; with count >= 4 also out[2] = summed kernel span in ms
 * from the kernel's own %globaltimer stamps (first CTA start to last CTA end)
 * and out[3] = launches stamped; then resets all.  Within one bn_step_rk call only the last
 * step's launches can be timed (earlier replays reuse the same events); call
 * it with nsteps = 1 to time every launch.  Enabling or disabling recaptures
 * the step graph.  count >= 2.
 */
bn_status bn_profile_enable(bn_solver* s, int enable);
bn_status bn_profile_read(bn_solver* s, double* out, size_t count);

/*
 * Phase timing of the 3-D / CIRCULAR operator (bn_profile_enable must be on; the times of one
 * bn_step_rk call cover its last step, so call it with nsteps = 1 to time every step).
 * out[0..3] = summed ms of the quadratic and reducible pair sums, of the production of the
 * kernel-mode slices (the sum of eq. betadD), of the Toeplitz sweeps of Q_{1,q}, and of the tail
 * (partial sums, reducible convolution, combination); out[4] = evaluations timed; out[5] = rounds
 * per evaluation; out[6] = Q_{1,q} terms per evaluation; out[7] = CTAs of the sweep launch; then
 * resets.  count >= 8.  BN_ERR_UNSUPPORTED for a 2-D LINEAR solver.
 */
bn_status bn_profile_nd(bn_solver* s, double* out, size_t count);

/* Precision state: *precision = BN_FP64 or BN_MIXED now in use; *t_escalated = the
 * time at which a mixed-precision solver switched to FP64 (-1 if it has not);
 * *max_f = the largest max_j f_j at the end of any step of the last stepping call
 * (|eps| max_f is what escalate_at tests after that call).  Any pointer may be NULL. */
bn_status bn_precision_state(const bn_solver* s, int* precision, double* t_escalated, double* max_f);

/* Velocity rescaling (Sec. 3 of the paper; the velocity rescaling method of Sec. 3.2 with
 * lambda = mu = 1), LINEAR solvers, 2-D and 3-D.  The solver must have been created with T = pi: its state (bn_set_state / bn_get_state) is
 * then G on the grid xi_j = 2 pi j / N of [-pi, pi]^d (row-major, j in I_N), with
 * f(t, v) = (pi w / L)^d G(t, (pi w / L)(v - u)), i.e. f_j = (pi w / L)^d G_j at the velocities
 * v_j = u + 2 L j / (N w); R is the kernel truncation in xi.
 * bn_rescale_set: L > 0 the half-width of the velocity box at w = 1, omega > 0 the scale w, u the mean
 * velocity (du = d values), rho, e > 0 the mass and internal energy of the state; also solves the
 * temperature (and the fugacity).  Allocates the step's scratch (4 arrays of N^d) once.
 * BN_ERR_ARG for bad values or T != pi, BN_ERR_UNSUPPORTED for CIRCULAR or sharded solvers,
 * BN_ERR_STATE when the moments admit no temperature (x = |eps| rho (d / (4 pi e))^{d/2} outside
 * I_eq: x >= 2 for 2-D Fermi-Dirac, x >= (5/3) sqrt(10/pi) for 3-D Fermi-Dirac, x >=
 * zeta(3/2)^{5/2} / zeta(5/2)^{3/2} for 3-D Bose-Einstein, whose equilibrium then carries a
 * condensate that the grid cannot hold). */
bn_status bn_rescale_set(bn_solver* s, double L, double omega, const double* u, size_t du, double rho, double e);

/* nsteps forward Euler steps of the procedure of Sec. 3.3: Q of G with the quantum parameter
 * eps (pi w / L)^d; rho, u, e advanced with the moments of Q (Delta xi = (2 pi / N)^d, the
 * collision frequency of d_t f = Q(f)); T (and z: Brent's method on the equilibrium relations,
 * mu = ln z for fermions) and w = sqrt(T) (quantum) or sqrt(T + |u|^2 / d) (classical); the
 * divergence term div(((w' - w) / (dt w) xi - (pi w / L)(u' - u) / dt) G) by spectral
 * differentiation (the k_c = -N/2 mode of each derivative set to 0); G += dt (-div +
 * (pi w / L)^{-gamma} Q).  One host synchronisation per step (the moments of Q).  BN_ERR_STATE when
 * the moments of a step admit no temperature, BN_ERR_NONFINITE for non-finite moments (both leave the
 * state of the start of that step), BN_ERR_TIMEOUT as for bn_eval_collision. */
bn_status bn_step_rescaled(bn_solver* s, double dt, int nsteps);

/* nsteps steps of an SSP-RK2 (Heun) form of the same procedure, second order in dt for G, w, u, e:
 * the predictor is the forward Euler step of bn_step_rescaled (G^(1), rho^(1), u^(1), e^(1), w^(1));
 * rho, rho u, rho e are the average of their values at the start and after a second Euler moment
 * update from the predictor with the moments of Q(G^(1)) (at the scale of G^(1)); T, z and w^{n+1}
 * follow from them; G^{n+1} = G^n + dt/2 [F(G^n) + F(G^(1))], F(G) = -div((a xi - b) G) +
 * (pi w / L)^{-gamma} Q(G) at each stage's scale w, with the midpoint rates a = ln(w^{n+1} / w^n) / dt
 * and b = (pi w / L)(u^{n+1} - u^n) / dt.  Two operator evaluations per step.  Allocates one more
 * array of N^d on its first call.  Errors as for bn_step_rescaled; on an error the state of the start
 * of the failed step is restored. */
bn_status bn_step_rescaled_rk2(bn_solver* s, double dt, int nsteps);

/* The temperature (and fugacity) of the equilibrium with mass rho and internal energy e, as the
 * rescaled step solves it (Sec. 3.3 step 3(b), Sec. 1.2): T = 2e/d for eps = 0 (*z = 0); for
 * eps != 0 z from x = |eps| rho (d / (4 pi e))^{d/2} = K_nu(z)^{nu+1} / K_{nu+1}(z)^nu, nu = d/2
 * (eq_fugacity), by Brent's method (on mu = ln z for Fermi-Dirac, on ln(-ln z) for 3-D
 * Bose-Einstein), and T = (|eps| rho / K_nu(z))^{1/nu} / (2 pi) (mom0_qmaxwell); K_nu is the complete
 * Fermi-Dirac (eps < 0) or Bose-Einstein (eps > 0) integral, in closed form for nu = 1, 2 and by
 * double-exponential quadrature for nu = 3/2, 5/2.  Host only, no GPU needed.  BN_ERR_ARG for null
 * pointers or d not 2 or 3, BN_ERR_STATE outside I_eq (as for bn_rescale_set), when the root lies
 * beyond the bracket (3-D Fermi-Dirac: ln z > 700) or for non-positive rho or e. */
bn_status bn_equilibrium_temperature(int d, double eps, double rho, double e, double* T, double* z);

/* out[0..8] = [w, u_0, u_1, u_2, rho, e, T, z, t] of the rescaled solve (u_2 = 0 in 2-D, z = 0
 * classically); count >= 9.  BN_ERR_STATE before bn_rescale_set. */
bn_status bn_rescale_get(const bn_solver* s, double* out, size_t count);

/* Kernel configuration of the operator: out[0] = outputs per thread of the fused
 * sweep (mixed 2-D N <= 32: 8 or 16; else 0), out[1] = CTAs (partial sums) per
 * launch, out[2] = 1 if the sweep orientation is chosen per b (else the register
 * window always runs along n_2), out[3..6] = the autotuner's time per launch in ms
 * of the variants (8, 8 oriented, 16, 16 oriented; 0 when not timed: cached, excluded
 * by opt.mixed_rw, or not applicable).  count >= 7. */
bn_status bn_kernel_config(const bn_solver* s, double* out, size_t count);

/* Host-side plan of the mixed 2-D operator kernel (N <= 32), computed on the CPU
 * exactly as a solver computes it, no GPU needed.  The work items are the b of the
 * Lemma's factorised sum with non-empty boxes (Sec. 3.3 step 2(c)); for RW = rw
 * outputs per thread (8 or 16), the per-b orientation choice on (oriented = 1) or
 * off, and a grid of nblk CTAs, one row of 14 ints per item is written to out, in
 * the order the kernel's CTAs take them (row k nblk + j is CTA j's k-th item):
 *   [ib, orient, J, chunk, units, J2, chunk2, units2, tail0, base, Lu, Lw, Su, Sw]
 * ib = (b1 + N) 2N + (b2 + N); the sweep splits dimension u (orient 0: u = 1,
 * w = 2; 1: swapped) into units of 32/J tasks x J chunks of `chunk` s_u rows
 * (`units` units), the last partial round re-split into units2 units of 32/J2 tasks
 * x J2 chunks of chunk2 rows covering the tasks [tail0, base); base = Lu x ceil(Lw
 * / rw) tasks; Lu, Lw, Su, Sw are the output and inner box sizes along u and w.
 * *n_items receives the item count; with out = NULL only the count is returned.
 * BN_ERR_ARG if N is odd or outside [2, 32], rw is not 8 or 16, nblk < 1,
 * n_items is NULL, or count < 14 x items. */
bn_status bn_plan_mixed2d(int N, int rw, int oriented, int nblk, int* out, size_t count, int* n_items);

/*
 * Measured CUDA-core FMA rate of the current device, the roofline denominator of the operator
 * kernels (not part of the paper).  kind 0 = FP32 FMA (fmaf), 1 = paired FP32 FMA
 * (fma.rn.f32x2, two multiply-adds per instruction), 2 = FP64 FMA.  Runs 4 CTAs of 256 threads
 * per SM, each thread 8 independent chains of dependent multiply-adds, on cuda_stream (NULL =
 * legacy default stream); the fastest of three timed launches (CUDA events) after an untimed
 * one.  out[0] = TFLOP/s (2 flops per multiply-add), out[1] = ms of that launch, out[2] = its
 * flops; count >= 3.  Allocates and frees a small device buffer; synchronises cuda_stream.
 * The rate is that of the SM clock during the run: sample the clock alongside.
 */
bn_status bn_measure_fma_peak(int kind, void* cuda_stream, double* out, size_t count);

/*
 * Partition of one 3-D evaluation over `count` GPUs (no GPU needed): the output planes n_0 of I_N
 * (as indices n_0 + N/2) in contiguous ranges [bounds[r], bounds[r+1]), r < count, with nearly
 * equal terms of the Q_{1,q} sum (the number of (k_0, l_0, m_0) in I_N^3 with k_0 + l_0 + m_0 = n_0
 * per plane in the LINEAR truncation, equal planes in the CIRCULAR one).  The shards of a solver's
 * shard_index / shard_count options.  bounds[0] = 0, bounds[count] = N.  BN_ERR_ARG unless d = 3,
 * N even in [4, 48], wrap 0 or 1, 1 <= count <= N and nbounds >= count + 1.
 */
bn_status bn_plan_shards(int d, int N, int wrap, int count, int* bounds, size_t nbounds);

/* Message of the last failed call on this thread ("" if none). */
const char* bn_last_error(void);

/*
 * Batched stepping: advance n solvers by nsteps RK steps of their own dt
 * (dts[i]) in shared launches.  The solvers may differ in d, N, eps, kernel
 * and precision; each must have a state.  All run on the stream of solvers[0].
 * Stops at the first non-finite solver (status BN_ERR_NONFINITE, *failed set
 * to its index, its state rolled back); others keep their progress.
 * When two or more 2-D solvers share an integrator, one captured graph advances
 * all of them and each operator evaluation is one launch of the fused kernel
 * per precision group.  If profiling is enabled on solvers[0], the kernel span
 * of those launches (first CTA start to last CTA end over every request of the
 * evaluation, %globaltimer) is added to solvers[0]'s bn_profile_read out[2..3],
 * one entry per evaluation, for every step of the call.
 */
bn_status bn_step_rk_batch(bn_solver** solvers, int n, const double* dts, int nsteps, int* failed);

/*
 * ---------------------------------------------------------------------------
 * Continuous-batching solve server.
 *
 * A request is one homogeneous solve: the operator (as in bn_create_solver),
 * the initial state f0 (N^d FP64 values on the grid, row-major), the step dt
 * and the final time t_end (steps = round(t_end / dt) of the chosen
 * integrator, from t = 0).  bn_server_submit copies f0 and returns at once; a
 * worker thread owned by the server admits queued requests, the one with the
 * least estimated work (steps x terms per evaluation) first and, past 60 s in
 * the queue, the oldest first, as long as max_active and the device-memory
 * budget allow (the kernel-mode tables of one operator are shared and counted
 * once), advances all running requests
 * together in shared launches (a few RK steps per tick; 2-D requests in one
 * captured graph per set of running requests), and retires finished requests
 * with their final state copied to host memory.  A request's result does not
 * depend on the other requests in the batch.  Server calls are thread-safe.
 * Errors of server calls are reported by bn_server_last_error().
 * ---------------------------------------------------------------------------
 */
typedef struct bn_server bn_server;

typedef struct {
    int d, N;           /* as in bn_create_solver */
    double T, R;
    int kernel;
    double eps;
    bn_options opt;     /* zero-filled = defaults */
    double dt, t_end;   /* step and final time (> 0) */
} bn_request;

/* Create a server on the current device.  device_bytes: budget for admission
 * (0 = 80% of the free device memory); max_active: most requests running at
 * once; cuda_stream: stream for all work (NULL = a new stream). */
bn_status bn_server_create(size_t device_bytes, int max_active, void* cuda_stream, bn_server** out);

/* Queue a request; *id receives its identifier (> 0).  f0 is copied. */
bn_status bn_server_submit(bn_server* srv, const bn_request* req, const double* f0, size_t count, long long* id);

/* State of a request: *state = 0 queued, 1 running, 2 done, 3 failed.  When
 * done and f_out != NULL, the final state (count = N^d) is copied to f_out.
 * times (ntimes >= 3, may be NULL) receives [submit, admit, done] in seconds
 * since the server was created, and with ntimes >= 4 also the solve time t at which
 * a done request switched to FP64 (escalate_at; -1 if it never did).  Returns
 * BN_ERR_STATE for a failed request. */
bn_status bn_server_poll(bn_server* srv, long long id, int* state, double* f_out, size_t count, double* times,
                         size_t ntimes);

/* Block until nothing is queued or running, or timeout_s elapses (BN_ERR_TIMEOUT). */
bn_status bn_server_wait_idle(bn_server* srv, double timeout_s);

/* out (count >= 8): [submitted, admitted, done, failed, ticks, most running at once,
 * budgeted bytes in use, budget]. */
bn_status bn_server_stats(bn_server* srv, double* out, size_t count);

/* Message of the last failed server call on this thread. */
const char* bn_server_last_error(void);

/* Stop the worker (queued and running requests are abandoned) and free everything. */
void bn_server_destroy(bn_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* BN_H */
