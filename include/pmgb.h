/*
 * pmgb.h -- C ABI of the GB300 particle-mesh (PM) library.
 *
 * The library implements the hot path of the differentiable cosmological
 * particle-mesh method of pmwd (arXiv:2211.09958): a PM force evaluation per
 * time step inside growth-factor kick-drift-kick (KDK) integration (paper,
 * Summary), and the adjoint method that integrates backward in time by
 * reversing the trajectory instead of storing it (Summary; Statement of Need:
 * adjoint method, reverse time integration, discretize-then-optimize).  The
 * paper prints no equations; the operations below are its prose written in
 * the standard comoving PM form:
 *
 *   units      box L [Mpc/h], H0 = 1, flat LCDM, E(a)^2 = Om a^-3 + 1 - Om
 *   lattice    q_i = i L / n_p + h / 2 (half a mesh cell h = L / n_m off the
 *              mesh nodes), lattice order: i = (ix n_p + iy) n_p + iz
 *   state      displacement s = x - q [Mpc/h], momentum p = a^3 E dx/da
 *   density    delta(c) = alpha sum_i W(x_i - c) - 1, CIC weights W,
 *              alpha = (n_m / n_p)^3, periodic
 *   force      F_j(k) = i D_j(k) (3/2) Om delta(k) / k^2 with the 4-point
 *              difference D_j = (8 sin k_j h - sin 2 k_j h) / (6 h) (k_j with
 *              PM_SOLVER_SPECTRAL_GRADIENT), zero at k = 0 and at the Nyquist
 *              index of axis j; F_i = sum_c W(x_i - c) F(c)
 *   step n     p += K_a[n] F(s); s += Dr[n] p; p += K_b[n] F(s), with
 *              growth-matched factors K(a->b; c) = (g_p(b) - g_p(a)) / g_f(c),
 *              Dr(a->b; c) = (D1(b) - D1(a)) / g_p(c), g_p = a^3 E D1',
 *              g_f = 3/2 Om D1, steps uniform in a from a_init to a_final
 *   ICs        unit white noise -> delta_L(k) = noise(k) sqrt(P(k) / V_c),
 *              BBKS P(k) normalised to sigma8, 2LPT at a_init
 *
 * Memory: every particle or mesh pointer is caller-owned DEVICE memory,
 * contiguous, 4-byte aligned float32 unless stated, on the device that was
 * current at pm_create.  Particle arrays are [n_batch][n_p^3][3] (xyz
 * innermost).  Meshes handed across the boundary are [n_batch][n_m^3]
 * (z fastest).  Host outputs are marked "host".  The library owns its
 * scratch meshes, cuFFT plans and coefficient tables and frees them in
 * pm_destroy.
 *
 * Streams: every call enqueues its work on the context stream (pm_set_stream,
 * default: the legacy default stream) and returns without waiting, except
 * calls that fill host outputs, which synchronise that stream before
 * returning.
 *
 * Errors: calls return PM_OK (0) or a negative PM_E* code and never abort or
 * trap; pm_last_error gives a message.  After an error the outputs of that
 * call are unspecified and the context stays usable.
 */
#ifndef PMGB_H
#define PMGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_OK 0
#define PM_EINVAL (-1)    /* bad size, NULL pointer or argument            */
#define PM_ENOMEM (-2)    /* device or host allocation failed              */
#define PM_ECUDA (-3)     /* a CUDA runtime call or launch failed          */
#define PM_ECUFFT (-4)    /* a cuFFT call failed                           */
#define PM_ERANGE (-5)    /* sizes overflow the supported index range      */
#define PM_ESTATE (-6)    /* call not valid in the context's state         */

/* pm_adjoint_integrate flag: the caller guarantees mu (the cotangent of the
 * final momentum) is zero, so the VJP of the last half kick is skipped. */
#define PM_ADJ_MU_ZERO 1u

typedef struct pm_ctx pm_ctx;

typedef struct pm_config {
    int32_t n_p;        /* particles per side of each simulation; even, >= 2  */
    int32_t n_m;        /* mesh cells per side; even, >= 4, <= 4096           */
    int32_t n_batch;    /* independent simulations sharing the geometry, >= 1 */
    int32_t n_steps;    /* KDK steps from a_init to a_final, >= 1             */
    double box;         /* L [Mpc/h], > 0                                     */
    double a_init;      /* start scale factor (2LPT), 0 < a_init < a_final    */
    double a_final;     /* end scale factor                                   */
    double h;           /* dimensionless Hubble parameter (BBKS shape Om h)   */
    double n_s;         /* primordial spectral index                          */
    const double *omega_m; /* host [n_batch]: matter density, (0, 1]         */
    const double *sigma8;  /* host [n_batch]: amplitude at a = 1, > 0         */
    int32_t solver;        /* bit mask of PM_SOLVER_* variants, 0 = defaults  */
} pm_config;

/* Solver variants (readings the paper leaves open; the defaults are the
 * 4-point difference gradient, no window correction, steps uniform in a):
 *   PM_SOLVER_SPECTRAL_GRADIENT  gradient i k_j (zero at the Nyquist index)
 *                                instead of i (8 sin k_j h - sin 2 k_j h)/6h;
 *                                on meshes finer than the particle lattice it
 *                                overestimates the linear force by O(k)
 *   PM_SOLVER_DECONVOLVE         Green's function divided by the paint and
 *                                read CIC windows, prod_j sinc^4(k_j h / 2)
 *                                (sharper force at n_m = n_p; amplifies
 *                                lattice aliasing at n_m > n_p)
 *   PM_SOLVER_LOG_A              KDK steps uniform in ln a, half steps at the
 *                                geometric midpoint
 *   PM_SOLVER_TSC                triangular-shaped-cloud paint and read (the
 *                                quadratic B-spline over 3 nodes per axis,
 *                                nodes j - 1, j, j + 1 of the nearest node j)
 *                                instead of cloud-in-cell; with
 *                                PM_SOLVER_DECONVOLVE the window is
 *                                prod_j sinc^6(k_j h / 2)
 *   PM_SOLVER_GROWTH_EMULATOR    the growth quantities behind the KDK, 2LPT
 *                                and d/dOm tables come from the growth
 *                                emulator (pm_growth_emulate) instead of one
 *                                ODE solve per cosmology; needs Omega_m in
 *                                [0.1, 0.6] and a_init, a_final in [1e-3, 1]
 *                                (PM_ERANGE otherwise) */
#define PM_SOLVER_SPECTRAL_GRADIENT 1
#define PM_SOLVER_DECONVOLVE 2
#define PM_SOLVER_LOG_A 4
#define PM_SOLVER_TSC 8
#define PM_SOLVER_GROWTH_EMULATOR 16

/* Create a context: validates cfg, computes the FP64 growth and coefficient
 * tables on the host, allocates the scratch meshes and creates the cuFFT
 * plans.  *out receives the context (NULL on error). */
int pm_create(const pm_config *cfg, pm_ctx **out);

/* Free everything the context owns.  NULL is accepted. */
int pm_destroy(pm_ctx *ctx);

/* Message of the last error on ctx (or of the last failed pm_create when
 * ctx is NULL).  The string is owned by the library. */
const char *pm_last_error(const pm_ctx *ctx);

/* Set the CUDA stream (a cudaStream_t passed as void*) used by later calls. */
int pm_set_stream(pm_ctx *ctx, void *stream);

/* Replace the cosmology of every simulation (host [n_batch] arrays) and
 * recompute the host tables. */
int pm_set_cosmology(pm_ctx *ctx, const double *omega_m, const double *sigma8);

/* Host copy of the KDK factors: out[b][n][0..2] = K_a, Dr, K_b of step n,
 * and (if dout != NULL) their derivatives with respect to Om. */
int pm_get_coefficients(pm_ctx *ctx, double *out, double *dout);

/* init_lpt -- 2LPT initial conditions at a_init (paper: initial conditions
 * of the Universe as optimisation variables, Statement of Need).
 *   noise  device [n_batch][n_p^3] unit white noise, or NULL to draw it on
 *          the device with Philox4x32-10 (key = seed + b, counter = site)
 *          and Box-Muller.
 *   s, p   device [n_batch][n_p^3][3] outputs (displacement, momentum). */
int pm_init_lpt(pm_ctx *ctx, const float *noise, uint64_t seed, float *s, float *p);

/* Adjoint of pm_init_lpt: cotangents (lam, mu) of (s, p) -> cotangent of the
 * noise and of (Om, sigma8).
 *   noise  as in pm_init_lpt (NULL: regenerate from seed)
 *   lam,mu device [n_batch][n_p^3][3] inputs
 *   dnoise device [n_batch][n_p^3] output (may be NULL)
 *   dcosmo host [n_batch][2] output: dL/dOm, dL/dsigma8 of this stage. */
int pm_init_lpt_adjoint(pm_ctx *ctx, const float *noise, uint64_t seed,
                        const float *lam, const float *mu,
                        float *dnoise, double *dcosmo);

/* pm_force -- PM gravity on each particle: CIC paint, real FFT, Green's
 * function times gradient, inverse FFTs, CIC read (paper: PM force).
 *   s  device [n_batch][n_p^3][3] input; f same shape output. */
int pm_force(pm_ctx *ctx, const float *s, float *f);

/* kdk_step -- one KDK step n (0 <= n < n_steps) in place:
 * (s_n, p_n, f = F(s_n)) -> (s_{n+1}, p_{n+1}, F(s_{n+1})):
 * p += K_a F(s_n), s += Dr p, p += K_b F(s_{n+1}), the growth-matched
 * kick and drift factors of pm_host_coefficients.  This is the discrete time
 * step whose trajectory the adjoint differentiates and reverses (paper,
 * Statement of Need: gradients along the same discrete trajectory as the
 * forward integrator; Summary: reverse time integration).
 *   s, p, f  device [n_batch][n_p^3][3], read and overwritten.
 * Returns PM_EINVAL for a step outside 0 .. n_steps - 1 or a NULL array. */
int pm_kdk_step(pm_ctx *ctx, int32_t step, float *s, float *p, float *f);

/* integrate -- steps [step_begin, step_end) in place: (s, p) at
 * a[step_begin] -> (s, p) at a[step_end]; f receives F(s) at a[step_end].
 * Kicks of adjacent steps are merged; step_end - step_begin + 1 force
 * evaluations. */
int pm_integrate(pm_ctx *ctx, int32_t step_begin, int32_t step_end,
                 float *s, float *p, float *f);

/* adjoint_integrate -- reverse-time adjoint of pm_integrate over the same
 * steps (paper: adjoint method with reverse time integration,
 * discretize-then-optimize).  In: the state (s, p) at a[step_end] with
 * f = F(s), the cotangents lam = dL/ds, mu = dL/dp there.  Out, in place:
 * (s, p) reconstructed at a[step_begin], (lam, mu) = dL/d(s, p) there.
 * f is read only.  domega (host [n_batch], may be NULL) receives dL/dOm of
 * the dynamics (through the KDK factors and the force prefactor).
 * flags: PM_ADJ_MU_ZERO or 0. */
int pm_adjoint_integrate(pm_ctx *ctx, int32_t step_begin, int32_t step_end,
                         float *s, float *p, const float *f,
                         float *lam, float *mu, double *domega, uint32_t flags);

/* Sparse checkpoints against FP32 reversal drift (a solver variant).  The
 * adjoint reconstructs the trajectory by reverse time integration (paper:
 * adjoint method with reverse time integration); in FP32 the reconstructed
 * states drift from the forward ones by rounding, step after step.  With
 * every > 0, pm_integrate stores, for each step m = every, 2 every, ...
 * (0 < m < n_steps) that it runs, the displacement s_m at the start of step m
 * and the half-step momentum p_{m+1/2} after that step's kick.
 * pm_adjoint_integrate restores both when it enters step m, so a
 * reconstructed state drifts over at most `every` steps.  The stored states
 * are those of the latest pm_integrate: a caller that runs the adjoint of
 * another trajectory turns checkpoints off first.  pm_kdk_step neither
 * stores nor restores.
 *   every  0 = off; values >= n_steps leave no slot and also turn them off
 *   ckpt   caller-owned device buffer of pm_checkpoint_floats(ctx, every)
 *          floats, 4-byte aligned, layout [slot][s | p][n_batch][n_p^3][3]
 *          with slot = m / every - 1; it must outlive its use; NULL allowed
 *          when there is no slot.
 * pm_checkpoint_floats returns that size (0 when there is no slot; -1 for
 * a NULL ctx or every < 0).  pm_set_checkpoints returns PM_EINVAL for
 * every < 0 or a NULL / misaligned buffer that has slots; it drops the
 * cached CUDA graphs of the integration loops (they hold the copies). */
int64_t pm_checkpoint_floats(const pm_ctx *ctx, int32_t every);
int pm_set_checkpoints(pm_ctx *ctx, int32_t every, float *ckpt);

/* pm_density -- CIC density contrast alpha sum_i W(x_i - c) - 1 of the
 * particles at s, the mesh the PM force starts from (paper, Summary: a
 * particle-mesh simulation) and the field that density losses and the power
 * spectrum (paper, Statement of Need: fields and summary statistics as
 * outputs) are computed on.  W is the CIC (or, with solver flag 8, TSC)
 * assignment; alpha = (n_m / n_p)^3.
 *   s      device [n_batch][n_p^3][3] input
 *   delta  device [n_batch][n_m^3] output (x slowest, z fastest). */
int pm_density(pm_ctx *ctx, const float *s, float *delta);

/* Adjoint of pm_density: ds = sum_c ddelta(c) d delta(c)/ds, the first step
 * of the adjoint of any loss on the final density (paper, Summary: gradients
 * by the adjoint method).  Uses the one-sided CIC weight slopes -1/h, +1/h.
 *   ddelta device [n_batch][n_m^3] input; ds [n_batch][n_p^3][3] output. */
int pm_density_adjoint(pm_ctx *ctx, const float *s, const float *ddelta, float *ds);

/* MSE of the final CIC density against a target field (the loss of the
 * gradient workload) and its adjoint seed:
 *   L_b = n_m^-3 sum_c (delta_b(c) - target_b(c))^2,
 *   dlds = dL/ds = sum_c 2 (delta - target)(c) / n_m^3 d delta(c)/ds.
 *   target device [n_batch][n_m^3]; loss host [n_batch];
 *   dlds device [n_batch][n_p^3][3] output or NULL. */
int pm_mse_loss(pm_ctx *ctx, const float *s, const float *target, double *loss, float *dlds);

/* Allocation-free variant of pm_mse_loss, for callers that cannot call
 * cudaMalloc: code whose device memory is all reserved up front by another
 * allocator (a framework's caching pool, a serving process's fixed arena)
 * and latency-critical loops that cannot take the implicit device-wide
 * synchronisation of cudaMalloc / cudaFree.  The paper has no counterpart;
 * this is an interface convenience.
 *
 * Needs no context.  Computes the same loss and adjoint seed as
 * pm_mse_loss of a context with cloud-in-cell assignment (this entry point
 * has no solver flags: it never paints with TSC) for the geometry (n_p, n_m,
 * n_batch, box) on the given CUDA stream (void* cudaStream_t, NULL = legacy
 * default stream), asynchronously.  n_p and n_m follow pm_create's rules
 * (even, n_p 2..4096, n_m 4..4096).
 *   s       device [n_batch][n_p^3][3] displacements
 *   target  device [n_batch][n_m^3]
 *   loss    device [n_batch] doubles (8-byte aligned) output
 *   dlds    device [n_batch][n_p^3][3] output, or NULL
 * Scratch: one file-scope __device__ array (8 MiB + 512 B) that every GPU
 * loading the library holds until exit; it limits n_batch * n_m^3 to 2^21
 * cells (a single 128^3 mesh) and n_batch to 64 -- larger sizes return
 * PM_ERANGE before any device work.  Nothing is allocated or freed.  All
 * calls share that array: each call clears what it needs, and calls that
 * overlap on the GPU (on different streams, or concurrently from several
 * host threads) race on it and give wrong results.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, with that device current); make that first call before any stream
 * capture.  The looked-up address is cached for the life of the process: a
 * cudaDeviceReset makes it stale, so do not call this entry point on a
 * device after resetting it.
 * Returns PM_OK, PM_EINVAL (bad size, NULL or misaligned pointer),
 * PM_ERANGE or PM_ECUDA; there is no error message for this entry point. */
int pm_mse_loss_noalloc(int32_t n_p, int32_t n_m, int32_t n_batch, double box, const float *s,
                        const float *target, double *loss, float *dlds, void *stream);

/* The library's unnormalised 3D real FFT of n_m^3 meshes (the transform of
 * the force pipeline), forward X(k) = sum_c x(c) e^{-i k.c h} and inverse
 * without the 1/n_m^3 factor.
 *   real  device [n_batch][n_m^3] floats
 *   spec  device [n_batch][n_m][n_m][n_m/2 + 1] complex (re, im float pairs)
 * pm_mesh_irfft reads only the Hermitian half spectrum and treats the
 * imaginary parts of the kz = 0 and kz = n_m/2 entries as zero. */
int pm_mesh_rfft(pm_ctx *ctx, const float *real, float *spec);
int pm_mesh_irfft(pm_ctx *ctx, const float *spec, float *real);

/* power_spectrum -- binned power of the CIC density contrast (paper:
 * summary statistics such as the power spectrum, Statement of Need).
 * Bins b = 0 .. n_m/2 - 1 have edges (b + 1/2) k_F .. (b + 3/2) k_F,
 * k_F = 2 pi / L, over the full k space; k = 0 excluded; no shot-noise or
 * window correction.  P_b = L^3 / n_m^6 <|delta_k|^2>.
 *   k_mean, power, n_modes  host [n_batch][n_m/2] outputs. */
int pm_power_spectrum(pm_ctx *ctx, const float *s, double *k_mean,
                      double *power, double *n_modes);

/* Host-only growth-function emulator (needs no GPU).  The paper names a
 * growth-function emulator as separate work adjacent to pmwd (Statement of
 * Need) and does not describe it; this one is a two-dimensional Chebyshev
 * series in (ln a, Omega_m), 48 x 16 terms of each of D1/a, dD1/da, D2/a^2
 * and (dD2/da)/a, fitted once per process to the library's own growth ODE
 * solve (the one pm_create uses; D1(1) = 1, D2 with the same factor
 * squared).  It reproduces that solve to ~1e-10 over the domain.
 *   omega_m  in [0.1, 0.6]
 *   a        host [n] scale factors, each in [1e-3, 1]
 *   out      host [n][8]: D1, D2, dD1/da, dD2/da, dD1/dOm, dD2/dOm,
 *            d(dD1/da)/dOm, d(dD2/da)/dOm
 * Returns PM_OK, PM_EINVAL (n < 0, NULL arrays with n > 0) or PM_ERANGE
 * (a value outside the domain; nothing is written). */
int pm_growth_emulate(double omega_m, int32_t n, const double *a, double *out);

/* Host-only (needs no GPU): the FP64 tables pm_create would compute.
 *   kdk   [n_batch][n_steps][3]  K_a, Dr, K_b per step       (may be NULL)
 *   dkdk  same shape, d/dOm                                    (may be NULL)
 *   lpt   [n_batch][4]  D1, D2, g1 = a^3 E D1', g2 = a^3 E D2' at a_init
 *   amp   [n_batch][2]  P(k) amplitude A and d ln A / dOm      (may be NULL) */
int pm_host_coefficients(const pm_config *cfg, double *kdk, double *dkdk, double *lpt, double *amp);

/* Learned force correction (requires a power-of-two n_m).  The paper names
 * a learned optimisation of the PM gravity solver as ongoing work (Statement
 * of Need) without describing it; this library's network is a per-cell MLP
 * on the coarse CIC density: features asinh(delta) at the cell and its 26
 * periodic neighbours plus the scale factor a (32 inputs), layers
 * 32 -> 128 -> 128 -> 3 with ReLU, BF16 weights and activations on tensor
 * cores with FP32 accumulation; the output times 3/2 Om h (h = cell size) is
 * added to the force meshes before the CIC read.  Parameters are one flat
 * FP32 vector [W1 32x128, b1 128, W2 128x128, b2 128, W3 128x3, b3 3]
 * (row-major, inputs first) of pm_nn_param_count() values.
 *
 * pm_nn_set_params   upload theta (host), reset the Adam moments
 * pm_nn_get_params   download theta and/or the last gradient (host; NULL skips)
 * pm_nn_enable       apply the correction in pm_integrate and pm_kdk_step at
 *                    each evaluation's scale factor (pm_force stays the plain
 *                    PM force); pm_adjoint_integrate then differentiates the
 *                    corrected dynamics (the correction's VJPs at every
 *                    reconstructed state) and leaves the gradient of its
 *                    objective with respect to the network parameters in the
 *                    context (pm_nn_get_params); its dOm output ignores the
 *                    Om dependence of the correction's output scale.
 *                    Synchronises the stream and returns PM_ECUDA if a
 *                    tensor-core wait of an earlier correction timed out
 * pm_nn_adam_step    one Adam step (lr, beta 0.9 / 0.999, eps 1e-8, bias
 *                    correction for step >= 1) with the gradient in the
 *                    context (from pm_adjoint_integrate or pm_nn_train_step)
 * pm_nn_predict      dF device [n_batch][n_p^3][3]: the correction read at
 *                    the particles s for scale factor a
 * pm_nn_train_step   force matching at particles s: loss = mean over
 *                    particles of |pm_nn_predict - target|^2 (target device,
 *                    same layout), gradient of weight * loss into the context
 *                    (weight > 0 balances samples of different force scale),
 *                    then one Adam step (lr, beta 0.9 / 0.999, eps 1e-8, bias
 *                    correction for step >= 1) when apply != 0; loss (host,
 *                    unweighted) may be NULL. */
int pm_nn_param_count(void);
int pm_nn_set_params(pm_ctx *ctx, const float *theta);
int pm_nn_get_params(pm_ctx *ctx, float *theta, float *grad);
int pm_nn_enable(pm_ctx *ctx, int enable);
int pm_nn_adam_step(pm_ctx *ctx, double lr, int64_t step);
int pm_nn_predict(pm_ctx *ctx, const float *s, double a, float *dF);
int pm_nn_train_step(pm_ctx *ctx, const float *s, const float *target, double a, double weight, double lr,
                     int64_t step, int apply, double *loss);

/* Launch-shape autotuner.  Four kernel families have a tunable block size
 * (128, 256 or 512 threads): [0] CIC paint, [1] CIC read, [2] spectral
 * force / adjoint multiply, [3] z-pass FFT (own transform, n_m >= 256; other
 * meshes keep 256); defaults 256.  [4] is the x-pass FFT pencil width in
 * complex columns, 8 or 16 (16: two adjacent y rows of 8 kz, 128 contiguous
 * bytes per x row; own transform only); default 8.  [5] is how the z-pass
 * inverse reads the spectrum (own transform, n_m >= 256): 1 per-thread
 * loads, 2 one TMA tensor copy per field into shared memory (default where
 * the driver provides the tensor-map encoder; a copy that does not complete
 * within a bounded wait is reported as PM_ECUDA by the next call that
 * synchronises for a host output: pm_adjoint_integrate with domega,
 * pm_init_lpt_adjoint, pm_mse_loss, pm_power_spectrum, pm_nn_get_params,
 * pm_profile_read).  [6] is how the z-pass forward of 4 interleaved fields reads its
 * rows (own transform): 1 per-thread strided loads, 2 coalesced 16-byte
 * loads staged through shared memory; default 1.  [7] is how a force
 * evaluation crosses the x axis of the spectrum (own transform): 1 three
 * launches (forward x pass, Green's function times gradient, inverse x
 * pass), 2 one fused kernel that takes each x line through all three
 * without writing the spectrum back in between, 3 the fused kernel for the
 * force and the three launches for the adjoint; default 2 (3 for n_m >= 512).
 * [8] is the force pipeline (own transform, 4-point difference gradient):
 * 1 the three force components (and the adjoint's psi) as inverse
 * transforms of i D_j g delta, the form [7] chooses among; 2 one inverse
 * transform of the potential phi = IFFT(g delta) (and psi), then
 * F_j = S_j phi on the real mesh, S_j the periodic 4-point difference
 * [8 (phi(c + e_j) - phi(c - e_j)) - (phi(c + 2 e_j) - phi(c - 2 e_j))] / 12h,
 * whose Fourier symbol is i D_j: the same linear map with two fewer inverse
 * transforms per evaluation; default 2 (1 with the spectral-gradient flag,
 * which has no stencil form).  [9] is the mass assignment into the own
 * transform's meshes: 1 zero the mesh, then one thread per particle adds
 * its weights with global float atomics; 2 bin the particles by the
 * 16^3-cell tile of their base cell (counting sort), then one block per
 * 16 x 16 column of tiles sums its particles in shared memory and writes
 * every cell of the column once, with the faces shared between columns
 * added by a second pass.  2 applies with the own transform, CIC, n_m a
 * multiple of 16 and n_batch n_p^3 < 2^31 (elsewhere it runs as 1); its
 * buffers (16 B per particle, about 1/8 of a 4-field mesh) are allocated
 * when it is first selected, PM_ENOMEM if they cannot be.  Default 1: on
 * the benchmark's workloads the atomic scatter measured faster.
 *
 * pm_autotune     times every candidate of each family in turn (the others
 *                 held at their current best) on this context's scratch
 *                 meshes, filled by a force evaluation of the particles s
 *                 (device [n_batch][n_p^3][3], not modified), 3 launches
 *                 after a warm-up, CUDA events on the context stream; keeps
 *                 the fastest.  ms (host, may be NULL) receives the mean
 *                 time in ms of each candidate, [family][3] in the order
 *                 above (0 where not timed).  Synchronises the stream.
 * pm_set_tuning   set all of them explicitly (PM_EINVAL for other values)
 * pm_get_tuning   read them (host int[PM_TUNE_KINDS])
 * Results do not depend on the choice beyond the order of FP32 sums (atomics,
 * [9]) and, for [7] and [8], the FP32 rounding order of the transforms. */
#define PM_TUNE_KINDS 10
int pm_autotune(pm_ctx *ctx, const float *s, float *ms);
int pm_set_tuning(pm_ctx *ctx, const int *threads);
int pm_get_tuning(pm_ctx *ctx, int *threads);

/* Test hook for the failure path of the bounded device waits.  Sets, on the
 * context stream, the error flag a kernel sets when its wait runs out,
 * without making any kernel wait:
 *   which = 0  the z-pass inverse's TMA copy of the spectrum; reported by
 *              the calls listed under tuning family [5]
 *   which = 1  the learned correction's MMA completion; reported by
 *              pm_nn_predict and pm_nn_enable
 * The reporting call returns PM_ECUDA and clears the flag; the context stays
 * usable.  Returns PM_EINVAL for another `which`.  Returns PM_ESTATE when the
 * context has no such wait: no library FFT (0), or no network parameters
 * set (1). */
int pm_inject_wait_timeout(pm_ctx *ctx, int which);

/* Device-kernel launch counter since pm_create (for benchmarking). */
int64_t pm_launch_count(const pm_ctx *ctx);

/* pm_integrate and pm_adjoint_integrate capture their launch sequence in a
 * CUDA graph on first use and replay it when called again with the same
 * steps and buffers (up to 8 graphs per context; the default).  enable = 0
 * runs every call as individual launches. */
int pm_use_graphs(pm_ctx *ctx, int enable);

/* Kernel timing.  pm_profile(ctx, 1) makes every later library kernel, cuFFT
 * call and scratch memset record a CUDA event pair on the context stream,
 * tagged with a kind name; pm_profile_read synchronises that stream and
 * returns per kind (index 0 .. pm_profile_kinds() - 1, named by
 * pm_profile_name) the number of launches and the summed device time in ms
 * (host arrays of n entries), then clears the records. */
int pm_profile(pm_ctx *ctx, int enable);
int pm_profile_kinds(const pm_ctx *ctx);
const char *pm_profile_name(const pm_ctx *ctx, int kind);
int pm_profile_read(pm_ctx *ctx, int64_t *counts, double *ms, int n);

#ifdef __cplusplus
}
#endif

#endif /* PMGB_H */
