/*
 * se.h -- C ABI of libse, the Spectral Ewald (SE) k-space library for
 * NVIDIA GB300 (sm_103a).
 *
 * Method: D. Saffar Shamshirgar, B. Hess, A.-K. Tornberg, "A comparison of
 * the Spectral Ewald and Smooth Particle Mesh Ewald methods in GROMACS",
 * arXiv:1712.04718.  Section numbers below refer to that paper.
 *
 * Problem (Sec. 1, Eq. 1.1-1.3): N charges q_n at x_n in the periodic box
 * [0, L)^3.  The library computes the Fourier-space (long-range) part of the
 * Ewald sum (superscript L in Eq. 1.5-1.7) with the SE method of Sec. 3,
 * i.e. the five steps of Algorithm 1 with the SE formulas of Table 2:
 *   spread (Eq. 3.5) -> 3-D FFT -> scale (Eq. 3.6) -> inverse FFT ->
 *   gather of potential (Eq. 3.9) and force (Sec. 3.1, Eq. 3.13).
 * Results: phi^L_m, E^L = 1/2 sum q_m phi^L_m and F^L_m = -dE^L/dx_m.  The
 * real-space and self terms of the Ewald sum are not included.  Units are
 * the paper's Gaussian units (phi = sum q / r) times the prefactor set with
 * se_plan_set_prefactor (default 1; 138.935458 gives kJ mol^-1 with nm and e).
 *
 * Parameters (Sec. 3 and Eq. 4.2): grid M^3, spacing h = L/M, support of P
 * grid points per dimension (P even, 2..32, P <= M), half width w = P h / 2,
 * shape m = c sqrt(pi P) with c = 0.95 by default, eta = (2 w xi / m)^2 =
 * P L^2 xi^2 / (c^2 pi M^2), Gaussian exponent alpha = 2 xi^2 / eta.  For
 * even P a particle in cell i = floor(x/h) (per dimension) covers grid
 * points i - P/2 + 1 .. i + P/2 (the tensor-product box).
 *
 * Conventions for every call:
 *  - Positions xyz are [N][3] (x, y, z interleaved), charges q are [N],
 *    forces F are [N][3] and potentials phi are [N], all in the plan's
 *    floating type (double for SE_FP64, float for SE_FP32).  Unless a
 *    function says "host", pointers are DEVICE pointers on the plan's device.
 *  - The caller owns every array it passes; outputs are overwritten, not
 *    accumulated.  The plan owns its grids, tables, sort buffers and FFT
 *    plans.
 *  - Positions outside [0, L) are wrapped periodically.
 *  - Calls are asynchronous on the plan's stream unless they return a host
 *    value.  A plan must not be used by two host threads at once.
 *  - Return value: SE_OK (0), a positive warning, or a negative error.  An
 *    error leaves the outputs unspecified and the plan usable.
 */
#ifndef SE_H
#define SE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SE_OK 0
#define SE_WARN_NONNEUTRAL 1   /* |sum q| > 1e-10 sum |q|; the k = 0 mode is still dropped,
                                  which equals a uniform neutralising background */
#define SE_ERR_ARG (-1)        /* invalid argument (see each call) */
#define SE_ERR_CUDA (-2)       /* a CUDA runtime call or kernel launch failed */
#define SE_ERR_NOMEM (-3)      /* device or host allocation failed */
#define SE_ERR_UNSUPPORTED (-4)/* valid but not supported: odd P, P > 32 */
#define SE_ERR_CUFFT (-5)      /* a cuFFT call failed */
#define SE_ERR_NONFINITE (-6)  /* a position or charge was NaN or infinite */

/* precision modes */
#define SE_FP64 0   /* every step in double precision */
#define SE_FP32 1   /* single precision with compensated (two-sum) grid
                       accumulation; Green's function table, grid energy and
                       the final energy reduction in double precision */
#define SE_FP32_PLAIN 2  /* as SE_FP32 without the compensation of the grid sums */

typedef struct se_plan se_plan;

/* Create a plan for N particles in the box [0, L)^3 with Ewald parameter xi,
 * grid M^3 and support P (Sec. 3; Eq. 4.2 fixes eta from c = 0.95).
 * N >= 0 (N = 0 gives zero results), L > 0, xi > 0, 2 <= P <= min(M, 32),
 * P even; otherwise SE_ERR_ARG (SE_ERR_UNSUPPORTED for odd P or P > 32).
 * Device memory is allocated on the current CUDA device at the first
 * computing call.  *out is set to NULL on failure. */
int se_plan_create(se_plan **out, int64_t N, double L, double xi, int M, int P);

/* Release every resource of the plan (NULL is accepted). */
int se_plan_destroy(se_plan *plan);

/* SE_FP64 (default), SE_FP32 or SE_FP32_PLAIN. */
int se_plan_set_precision(se_plan *plan, int prec);

/* Shape of the Gaussian (Eq. 4.2): is_eta = 0 sets c (default 0.95), 1 sets
 * eta directly; 0 < eta < 1 and c > 0 required. */
int se_plan_set_shape(se_plan *plan, double value, int is_eta);

/* Multiply phi, E and F by kc (default 1, Gaussian units; Sec. 4 remark:
 * 1/(4 pi eps0) = 138.935458 kJ mol^-1 nm e^-2). */
int se_plan_set_prefactor(se_plan *plan, double kc);

/* CUDA stream (cudaStream_t) for every later call; NULL = legacy default. */
int se_plan_set_stream(se_plan *plan, void *stream);

/* Kernel tuning: spread_variant 0 = automatic, 1 = shared-memory tiles and
 * cuFFT, 2 = direct global accumulation and cuFFT (not with SE_FP32),
 * 3 = the single-precision pipeline without cuFFT (SE_FP32 or SE_FP32_PLAIN,
 * M <= 128; the default there): exact 64-bit fixed-point spreading, line DFTs
 * with the scaling fused into the x pass, kernels chained by programmatic
 * dependent launch; 4 = the same pipeline with the particles left unsorted:
 * one kernel adds every weight into a float grid with global reductions
 * (the last bits of the grid then depend on the order of the additions);
 * 5 = the pipeline of 3 with the inverse transform fused with the gather:
 * each x-slab's real plane stays in shared memory, every particle takes its
 * share of each plane of its support there, and a last kernel adds the P
 * shares in a fixed order (the real grid is written only when se_copy_grid
 * asks for it); SE_ERR_UNSUPPORTED where its shared memory (about
 * 15 M^2 bytes) does not fit one CTA of the device (M = 128 on GB300).
 * tile = edge of a spreading tile in grid cells (0 = automatic, else
 * 2..32; for P <= 16 edges above 16 are reduced to 16, the largest the
 * staged tile regions' fixed row stride holds).  For benchmarking and
 * tests. */
int se_plan_set_tuning(se_plan *plan, int spread_variant, int tile);

/* Derived parameters: out[0..9] = h, w, eta, alpha, c_g, m, tile edge,
 * spread variant in use (1 to 4), precision, prefactor.
 * c_g = (2 xi^2 / (pi eta))^{3/2} is the Gaussian's normalisation (Eq. 3.5). */
int se_plan_get_params(const se_plan *plan, double *out);

/* How the gather obtains the force (Sec. 2.3 lists three ways; the paper's
 * SE uses the first below):
 *   SE_FORCE_ANALYTIC (default): the derivative of the window (Sec. 3.1),
 *     F = -dE/dx of the discrete SE energy exactly; one inverse FFT.
 *   SE_FORCE_IK: differentiation by i k in Fourier space.  The scaling step
 *     also forms D_d = i k_d G(k)/M^3 Hhat (d = x, y, z; k_d = 2 pi n_d / L
 *     with n_d the signed index, 0 at the Nyquist index of an even M), three
 *     more inverse FFTs give the gradient grids, and the gather applies the
 *     plain window: F_m,d = -kc q_m h^3 sum_j D_d,j W(x_j - x_m).  These
 *     forces conserve momentum (sum_m F_m = 0 to rounding) but are not the
 *     exact derivative of the energy.  They are evaluated by the cuFFT
 *     pipeline (spread variant 1 or 2; a tuning of 3 or 4 is overridden),
 *     with 3 M^3 more real and 3 M^2 (M/2+1) more complex values of grid
 *     memory.  Potentials, energies and se_adjoint are the same in both modes.
 * Returns SE_ERR_ARG for another mode.  Takes effect at the next call. */
#define SE_FORCE_ANALYTIC 0
#define SE_FORCE_IK 1
int se_plan_set_force_mode(se_plan *plan, int mode);

/* Step (a) of Algorithm 1 with the SE window (Eq. 3.5): sort particles into
 * grid tiles and spread H_j = sum_n q_n c_g exp(-alpha |x_j - x_n|^2) onto
 * the plan's real grid (M^3, z fastest).  xyz, q: device. */
int se_spread(se_plan *plan, const void *xyz, const void *q);

/* Steps 3-5 of Algorithm 1: forward FFT of the spread grid, scaling by
 * G(k)/M^3 with G(k) = 4 pi exp(-(1-eta) k^2 / (4 xi^2)) / k^2, G(0) = 0
 * (Eq. 3.6 and the 4 pi of Eq. 3.7), inverse FFT into the gather grid.
 * E_grid (device pointer to one double, or NULL) receives the grid energy
 * kc h^3 / (2 M^3) sum_k G(k) |H^_k|^2, which equals E^L of the gather step
 * to rounding.  Requires a preceding se_spread on this plan. */
int se_scale(se_plan *plan, double *E_grid);

/* Step 6 of Algorithm 1 (Eq. 3.9 and the analytic force of Sec. 3.1):
 *   phi_m = kc h^3 sum_j Ht_j c_g exp(-alpha |x_j - x_m|^2)
 *   F_m   = -kc 2 alpha h^3 q_m sum_j (x_j - x_m) Ht_j c_g exp(-alpha |x_j - x_m|^2)
 * F_m is -dE/dx_m of the discrete SE energy.  Requires se_spread (with the
 * same xyz, q) and se_scale.  phi, F and E (device pointer to one double,
 * E = 1/2 sum q phi) may each be NULL.  With F NULL the gather runs with the
 * plain window alone (potential-only mode: about half the arithmetic of the
 * gather with forces).  With SE_FORCE_IK, F is the ik force (see
 * se_plan_set_force_mode). */
int se_gather(se_plan *plan, const void *xyz, const void *q, void *phi, void *F,
              double *E);

/* Adjoint of the energy (the backward step of E^L as a differentiable
 * function of positions and charges): with the upstream gradient
 * g = dl/dE^L (DEVICE pointer to one double), writes
 *   grad_x = dl/dx = -g F     (F = -dE/dx, Sec. 1 Eq. 1.3)
 *   grad_q = dl/dq = g phi    (E is quadratic in q and 1/2 sum q phi, Eq. 1.2)
 * into DEVICE arrays of the plan's type ([N][3] and [N]; each may be NULL).
 * Reuses the grid of the last se_scale (same xyz, q); no host sync. */
int se_adjoint(se_plan *plan, const void *xyz, const void *q, const double *gE,
               void *grad_x, void *grad_q);

/* The whole k-space evaluation: se_spread, se_scale, se_gather.  E is a HOST
 * pointer (the call waits for the stream); F and phi are device pointers and
 * may be NULL.  With both NULL (energy-only mode) the gather is skipped and E
 * is the grid energy of se_scale, equal to 1/2 sum q phi to rounding.  Returns SE_WARN_NONNEUTRAL for a non-neutral system and
 * SE_ERR_NONFINITE for NaN/Inf input. */
int se_energy_force(se_plan *plan, const void *xyz, const void *q, double *E,
                    void *F, void *phi);

/* The whole evaluation with every result on the device and no host
 * synchronisation: F, phi and E (one double, E = 1/2 sum q phi) are device
 * pointers and may each be NULL; F and phi both NULL is the energy-only mode
 * of se_energy_force.  Status checks (non-neutral, non-finite)
 * are kept on the device; read them with se_plan_get_status. */
int se_evaluate(se_plan *plan, const void *xyz, const void *q, void *F, void *phi,
                double *E);

/* Status of the last evaluation's input checks (SE_OK, SE_WARN_NONNEUTRAL or
 * SE_ERR_NONFINITE) into *status; waits for the plan's stream. */
int se_plan_get_status(se_plan *plan, int *status);

/* enable = 1 (default): se_evaluate, se_energy_force and se_energy_force_host
 * replay one CUDA graph of the whole evaluation, captured at the first call
 * and again whenever an argument pointer or the prefactor changes.  The
 * graph is not used while the plan's stream is itself being captured, nor
 * while stage timing is on.  enable = 0 launches every kernel directly. */
int se_plan_set_graph(se_plan *plan, int enable);

/* As se_energy_force but every array is in HOST memory: the call copies xyz
 * and q to the device, evaluates, and copies F, phi and E back before it
 * returns.  When every host array is page-locked and mapped into the
 * device's address space (cudaMallocHost, cudaHostAlloc, or cudaHostRegister
 * with cudaHostRegisterMapped) and graphs are enabled (se_plan_set_graph),
 * the kernels read xyz and q and write F and phi in host memory directly
 * (over the host link, no staging copies), and the evaluation is one CUDA
 * graph, captured at the first call and again whenever a host pointer or the
 * prefactor changes, then replayed; otherwise the arrays are copied through
 * device staging buffers one by one.  The results are the same either way. */
int se_energy_force_host(se_plan *plan, const void *xyz, const void *q,
                         double *E, void *F, void *phi);

/* Copy one of the plan's grids into dst (device, M^3 values of the plan's
 * type, z fastest): which = 0 spread grid H (after se_spread), 1 scaled and
 * back-transformed grid Ht (after se_scale).  With the single-precision
 * pipeline (spread variants 3 and 4) the spread grid is cleared by se_scale:
 * which = 0 after se_scale returns SE_ERR_ARG.  For tests and inspection. */
int se_copy_grid(se_plan *plan, int which, void *dst);

/* Self-energy term of Eq. 1.6, -kc xi / sqrt(pi) sum q^2, from HOST charges
 * (double). Not part of the k-space result; provided for completeness. */
int se_self_energy(const se_plan *plan, const double *q_host, int64_t n, double *E_self);

/* ---- Ensembles: many independent systems in one launch sequence ----
 * S systems, system s with N[s] charges in its own box [0, L[s])^3 and grid
 * M[s]^3 (2 <= P <= M[s] <= 128), common xi and support P (c = 0.95, Eq. 4.2
 * per system), evaluated by the single-precision pipeline (exact fixed-point
 * spreading; SE_FP32 semantics) with one kernel launch per stage for all
 * systems, replayed as one CUDA graph.  Positions, charges, forces and
 * potentials are the systems' arrays concatenated in order: xyz [sum N][3],
 * q [sum N], F [sum N][3], phi [sum N] (float, DEVICE).  E: DEVICE array of S
 * doubles (E^L of each system, 1/2 sum q phi).  Limits: S <= 1024,
 * sum N < 2^31, at most 8192 spreading tiles per system. */
typedef struct se_batch se_batch;
int se_batch_create(se_batch **out, int S, const int64_t *N, const double *L, const int *M,
                    double xi, int P);
int se_batch_destroy(se_batch *batch);
int se_batch_set_stream(se_batch *batch, void *stream);
/* Multiply phi, E and F by kc (default 1). */
int se_batch_set_prefactor(se_batch *batch, double kc);
/* Edge of the spreading tiles in grid cells (2..32, default 8; for P <= 16
 * edges above 16 are reduced to 16). */
int se_batch_set_tile(se_batch *batch, int tile);
/* enable = 0: launch every kernel directly instead of replaying a graph. */
int se_batch_set_graph(se_batch *batch, int enable);
/* One evaluation of every system (F, phi, E may each be NULL). */
int se_batch_evaluate(se_batch *batch, const void *xyz, const void *q, void *F, void *phi,
                      double *E);
/* Grid energies of the last evaluation (DEVICE array of S doubles), equal to
 * E to rounding. */
int se_batch_grid_energy(se_batch *batch, double *E_grid);
/* Worst input check over the systems of the last evaluation (SE_OK,
 * SE_WARN_NONNEUTRAL or SE_ERR_NONFINITE); waits for the stream. */
int se_batch_get_status(se_batch *batch, int *status);
/* Stage timing of se_batch_evaluate: enable = 1 launches every kernel
 * directly (no graph) with a CUDA event after each of the 8 stages (bin,
 * scatter, spread, forward transform, scaling pass, inverse transform,
 * gather, energy finish) and waits for them; se_batch_get_timing writes the
 * summed milliseconds of each stage (nstages >= 8) and the number of timed
 * evaluations, and clears them if reset. */
int se_batch_set_timing(se_batch *batch, int enable);
int se_batch_get_timing(se_batch *batch, double *ms, int nstages, int64_t *count, int reset);
/* Autotuner: times `reps` evaluations with each tile edge in candidates[0..
 * ncand) (CUDA events, after warm-up) and keeps the fastest; reports it in
 * *best_tile and its time per evaluation in *best_ms. */
int se_batch_autotune(se_batch *batch, const void *xyz, const void *q, void *F, void *phi,
                      double *E, const int *candidates, int ncand, int reps, int *best_tile,
                      float *best_ms);

/* se_spread_noalloc -- the spreading step without any device allocation.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc (a program that reserves all device memory at start-up and
 * forbids allocation in its inner loop, or a component whose device memory
 * belongs to another framework's allocator).
 * Writes the spread grid of se_spread, H_j = sum_n q_n c_g
 * exp(-alpha |x_j - x_n|^2) in FP64 with the parameters of se_plan_create
 * (c = 0.95), into the caller's DEVICE grid H (M^3 doubles, z fastest;
 * cleared by the call), from DEVICE xyz [N][3] and q [N], asynchronously on
 * `stream` (cudaStream_t, NULL = default).
 * All intermediate buffers live in one static device array of about 1.5 MB,
 * reserved on every GPU that loads the library until the process exits.
 * Limits: N <= 32768 and M <= 128; larger sizes return SE_ERR_ARG, as do a
 * NULL H, P < 2 or P > M; odd P returns SE_ERR_UNSUPPORTED.  All of these are
 * decided on the host before any CUDA call.
 * Non-finite positions or charges are not detected here (there is no status
 * to read back without a host synchronisation): a NaN charge gives a NaN
 * grid; the plan path reports them through se_plan_get_status.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process: make that first call before any stream capture, and do not
 * call this entry point again on a device after cudaDeviceReset (the kept
 * address is then stale).
 * Calls share the array: calls that overlap on the GPU race; issue them on
 * one stream.  Allocates nothing (no cudaMalloc, cudaFree or allocating
 * library call). */
int se_spread_noalloc(const double *xyz, const double *q, int64_t N, double L, double xi,
                      int M, int P, double *H, void *stream);

/* ---- Real-space part of the Ewald sum (the complement of the k-space path) ----
 * Sec. 1, Eq. 1.5-1.7: for charges in [0, L)^3 with splitting parameter xi
 * and cut-off rc (0 < rc <= L/3):
 *   phi_m = kc [ sum over particles n and periodic images with 0 < r < rc of
 *                q_n erfc(xi r)/r  -  2 xi/sqrt(pi) q_m ]
 *   F_m   = kc q_m sum_{r < rc} q_n (2 xi/sqrt(pi) e^{-xi^2 r^2} + erfc(xi r)/r)
 *           (x_m - x_n)/r^2            (the image of x_n at distance r)
 *   E     = 1/2 sum q_m phi_m  (real-space energy plus the self energy)
 * Added to se_evaluate's k-space results they give the whole Ewald potential,
 * force and energy.  Cells of edge >= rc/K hold the particles (K L/rc per
 * dimension, at most 40; K = 2, or 3 when K = 2 gives fewer than 512 cells;
 * se_real_get_cells reports the count, se_real_set_reach overrides K);
 * se_real_create returns SE_ERR_ARG for N < 0 or N >= 2^31, or a
 * non-positive or non-finite L, xi or rc, and SE_ERR_UNSUPPORTED for
 * rc > L/3.
 * se_real_evaluate: xyz [N][3], q [N], F [N][3], phi [N] DEVICE arrays of the
 * precision's type (SE_FP64 double, SE_FP32 float), E a DEVICE double; F,
 * phi and E may be NULL.  accumulate = 0 overwrites the outputs, 1 adds to
 * them (F += ..., phi += ..., *E += ...).  Asynchronous on the stream.  The
 * order of the additions inside a cell follows atomic slot claims, so results
 * are reproducible to rounding, not bitwise. */
typedef struct se_real se_real;
int se_real_create(se_real **out, int64_t N, double L, double xi, double rc);
int se_real_destroy(se_real *real);
int se_real_set_precision(se_real *real, int prec);   /* SE_FP64 (default) or SE_FP32 */
int se_real_set_prefactor(se_real *real, double kc);
int se_real_set_stream(se_real *real, void *stream);
int se_real_get_cells(const se_real *real, int *cells_per_dim);
/* Stencil reach K (cells of edge >= rc/K, a (2K+1)^3 stencil): 1, 2 or 3, or
 * 0 for the automatic choice; SE_ERR_UNSUPPORTED if 2K+1 cells do not fit in
 * L (at most 40 cells per dimension). */
int se_real_set_reach(se_real *real, int K);
int se_real_evaluate(se_real *real, const void *xyz, const void *q, void *F, void *phi,
                     double *E, int accumulate);

/* ---- Parameter selection (host only; no device is touched) ----
 * For an absolute rms error tolerance tol of the potential, the energy or
 * the force (quantity), a real-space cut-off rc, the box L and
 * Q = sum_n q_n^2, following the paper's estimates:
 *   xi     from the real-space truncation estimate (Eq. 2.3: through W0
 *          for the potential and energy, a logarithm for the force);
 *   k_inf  from the Fourier-space truncation estimate (Eq. 2.4) and
 *          M = 2 ceil(k_inf) (Sec. 3);
 *   P      the smallest even P with A e^{-pi P c^2/2} <= tol (Sec. 4:
 *          A = sqrt(Q xi L)/L, Q sqrt(xi L)/L, 4 pi Q sqrt(xi^3/L) for the
 *          potential, energy and force); M is raised where needed so that
 *          eta of Eq. 4.2 stays at most 1/2 (the bounds fail near eta = 1),
 *          and to P, and rounded up to even.
 * c: the shape constant of Eq. 4.2 (0 selects 0.95).  Writes *xi, *M, *P
 * and, if k_inf is not NULL, the unrounded k_inf.  Returns SE_ERR_ARG for a
 * non-positive or non-finite tol, rc, L or Q, a negative c, a NULL xi, M or
 * P, or an unknown quantity; SE_ERR_UNSUPPORTED, with nothing written, when
 * the tolerance is met without a Fourier part or needs k_inf above 1e6, and
 * SE_ERR_UNSUPPORTED with the outputs written when the selected P exceeds 32. */
#define SE_QUANTITY_POTENTIAL 0
#define SE_QUANTITY_ENERGY 1
#define SE_QUANTITY_FORCE 2
int se_select_params(int quantity, double tol, double rc, double L, double Q, double c,
                     double *xi, int *M, int *P, double *k_inf);

/* The even support P >= 2 with e^{-pi P c^2/2} <= scaled_tol, the error
 * relative to the bound's constant A (Sec. 4; c = 0 selects 0.95), or
 * SE_ERR_ARG for a non-positive scaled_tol or negative c. */
int se_select_support(double scaled_tol, double c);

/* The principal branch W0 of the Lambert function (w e^w = z) for z >= 0,
 * NaN otherwise: the inverse the estimates of Eq. 2.3-2.4 need. */
double se_lambert_w0(double z);

/* Static message for a status code. */
const char *se_strerror(int status);

/* Stage timing (tracing).  enable = 1 records a CUDA event before and after
 * every stage of each later evaluation on the plan's stream: 0 bin, 1
 * scatter, 2 spread, 3 forward FFT, 4 scale, 5 inverse FFT, 6 gather.
 * Events are recycled from a ring of 64 evaluations; completed ones are
 * folded into running sums.  enable = 0 stops recording (sums are kept). */
int se_plan_set_timing(se_plan *plan, int enable);

/* Wait for recorded evaluations, then write the summed milliseconds of each
 * stage to ms[0..6] (nstages >= 7) and the number of evaluations summed to
 * *count; reset = 1 clears the sums afterwards. */
int se_plan_get_timing(se_plan *plan, double *ms, int nstages, int64_t *count, int reset);

/* Throughput probe of the current GPU (measurement helper; the paper has no
 * counterpart): runs a short timed kernel on a private stream, waits for it,
 * and writes to *out the rate of one unit that bounds the spread, gather and
 * transform kernels: SE_PROBE_FP32_FMA and SE_PROBE_FP64_FMA in flop/s (an
 * FMA counts 2), SE_PROBE_SMEM_ATOMIC_U32 and SE_PROBE_SMEM_ATOMIC_F32 in
 * shared-memory atomic adds per second (non-returning, no bank conflicts).
 * About a millisecond of GPU time; allocates a small device buffer.
 * SE_ERR_ARG for an unknown kind or a null out. */
#define SE_PROBE_FP32_FMA 0
#define SE_PROBE_FP64_FMA 1
#define SE_PROBE_SMEM_ATOMIC_U32 2
#define SE_PROBE_SMEM_ATOMIC_F32 3
int se_probe_peak(int kind, double *out);

/* Library version as major*10000 + minor*100 + patch. */
int se_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SE_H */
