/*
 * gb300dft.h -- C ABI of the GB300 (sm_103a) FFT/Picard classical-DFT library.
 *
 * The library evaluates, on one GPU, the hot path of the 3D density functional
 * solver for charged hard spheres of Knepley, Karpeev, Davidovits, Eisenberg
 * and Gillespie (arXiv:0910.1531): the FFT convolutions of one Picard
 * residual evaluation (Sec. "Hard Sphere Interaction", Sec. "Electrostatics",
 * App. B) and the Picard iteration with line search around them
 * (Sec. "Discretization and Solution in Equilibrium").
 *
 * Conventions for every entry point below:
 *  - Units: lengths nm, energies kT, number densities nm^-3, concentrations
 *    mol/L.  V (the external potential beta*mu_ext, which defines the
 *    geometry, Sec. "Theory") is in kT; +inf marks hard exclusion.
 *  - Fields are caller-owned DEVICE memory, contiguous, x fastest:
 *    a species field set is [S][nz][ny][nx]; the ten weighted densities are
 *    [10][nz][ny][nx] in the order n0, n1, n2, n3, nV1x, nV1y, nV1z, nV2x,
 *    nV2y, nV2z.  The element type is float for DFT_FP32_STAB plans and
 *    double for DFT_FP64 plans.  Pointers must be 16-byte aligned.
 *  - All work is issued on the plan's CUDA stream, in stream order.  Calls
 *    that return host scalars (resid_out, alpha_out, iters_out, omega_out,
 *    ...) synchronise that stream before returning; the others return as soon
 *    as the work is queued.
 *  - The plan owns its scratch memory (allocated at create, freed at
 *    destroy) and never frees caller memory.  A plan is not thread-safe; use
 *    one plan per host thread.
 *  - Every call returns a dft_status and never aborts or throws.  On error
 *    dft_last_error() gives a one-line description.
 */
#ifndef GB300DFT_H
#define GB300DFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dft_plan dft_plan;

typedef enum {
    DFT_OK = 0,
    DFT_EINVAL = -1,       /* bad argument (sizes, radii, NULL pointer, ...) */
    DFT_ENONNEUTRAL = -2,  /* bath is not electroneutral */
    DFT_ENOMEM = -3,       /* device allocation failed */
    DFT_ECUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    DFT_EN3BOUND = -5,     /* local packing fraction n3 >= 1 somewhere (log(1-n3) undefined) */
    DFT_ENONFINITE = -6,   /* NaN or Inf appeared in a density */
    DFT_ENOCONV = -7,      /* dft_solve reached max_it without reaching tol */
    DFT_ETIMEOUT = -8      /* a bounded device-side wait on an asynchronous (TMA) copy gave up */
} dft_status;

enum { DFT_FP32_STAB = 0, DFT_FP64 = 1 };
enum { DFT_MAX_SPECIES = 5 };
/* Hard-sphere free-energy density Phi_HS (dft_params.functional).  The paper uses the
 * antisymmetrised Rosenfeld form, eq. Phi (DFT_PHI_RSLT, the default, with the |nV2| <= n2
 * bound of Sec. "Numerical Stability"), and notes that the other Phi_HS it cites leave the
 * numerical scheme unchanged: DFT_PHI_ROSENFELD (original 1989 form, last term
 * (n2^3 - 3 n2 nV2.nV2) / (24 pi (1 - n3)^2)) and DFT_PHI_WHITE_BEAR (2002 form, last term
 * (n2^3 - 3 n2 nV2.nV2) (n3 + (1 - n3)^2 ln(1 - n3)) / (36 pi n3^2 (1 - n3)^2)).  The bath
 * mu^HS and P are App. A's Percus-Yevick values for the first two and the uniform limit of the
 * White Bear form (Carnahan-Starling / BMCSL) for the third. */
enum { DFT_PHI_RSLT = 0, DFT_PHI_ROSENFELD = 1, DFT_PHI_WHITE_BEAR = 2 };

typedef struct {
    int nx, ny, nz;                 /* grid points per axis, 4 <= n <= 512, prime factors <= 31 */
    double hx, hy, hz;              /* spacing (nm); periodic box L_d = n_d h_d */
    int nspecies;                   /* 1 .. DFT_MAX_SPECIES */
    const double* radius_nm;        /* [nspecies] hard-sphere radii R_i > 0 */
    const double* valence;          /* [nspecies] z_i */
    const double* bulk_molar;       /* [nspecies] bath concentrations (mol/L) >= 0 */
    double temperature_K;           /* T > 0 */
    double eps_r;                   /* relative permittivity > 0 */
    int precision;                  /* DFT_FP32_STAB or DFT_FP64 */
    /* [nspecies] or NULL: n_fixed[i] > 0 makes species i a fixed-number (canonical)
     * species of n_fixed[i] particles in the box (normally with bulk_molar[i] = 0, i.e.
     * absent from the bath): G_i = n_fixed[i] e_i / (h^3 sum_x e_i), e_i its Boltzmann
     * factor exp(-V_i - beta mu_ex_i(x)) (the paper has no such species; canonical reading
     * of eq. rhoEquation); its residual weight is its mean density n_fixed[i] / (N h^3).
     * dft_grad rejects plans with such species (DFT_EINVAL). */
    const double* n_fixed;
    int functional;                 /* DFT_PHI_RSLT (0, eq. Phi), DFT_PHI_ROSENFELD or DFT_PHI_WHITE_BEAR */
} dft_params;

/*
 * Create a plan: checks the parameters, computes the bath thermodynamics of
 * App. A (Percus-Yevick mu^HS and P -- or the White Bear uniform limit, see
 * DFT_PHI_WHITE_BEAR --, MSA Gamma, eta, Omega and mu^ES; Gamma by Newton's
 * method as in App. A), builds the FFT plans of each axis and allocates scratch
 * on the current CUDA device.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream).
 * Rejects (DFT_EINVAL) sizes outside the supported set, R <= 0, negative
 * concentrations, a bath packing fraction >= 0.9, an unknown functional; rejects a bath with
 * |sum z_i c_i| > 1e-12 sum |z_i| c_i (DFT_ENONNEUTRAL).
 * On success *out owns device memory until dft_plan_destroy.
 */
dft_status dft_plan_create(const dft_params* params, void* cuda_stream, dft_plan** out);

/* Free the plan and its scratch (synchronises the plan's stream). NULL is a no-op. */
dft_status dft_plan_destroy(dft_plan* plan);

/* One-line description of the last error on this plan (or of the last failed create if plan is NULL). */
const char* dft_last_error(const dft_plan* plan);

/*
 * Bath values computed at create (App. A), all host arrays of length nspecies
 * except the scalars; any pointer may be NULL.  rho_bulk in nm^-3, mu_* in kT,
 * gamma in nm^-1, beta_p in nm^-3, lambda_b the Bjerrum length in nm.
 */
dft_status dft_plan_bulk(const dft_plan* plan, double* rho_bulk, double* mu_hs, double* mu_es,
                         double* gamma, double* beta_p, double* lambda_b);

/*
 * Weighted densities n_alpha(x) = sum_i int rho_i(x') w_i^alpha(x' - x) d^3x'
 * (eq. nDef) by the convolution theorem (eq. conv) with the analytic weight
 * transforms of App. B.  rho: [S][N] device, n_out: [10][N] device.
 */
dft_status dft_weighted_densities(dft_plan* plan, const void* rho, void* n_out);

/*
 * Hard-sphere one-body direct correlation c1_hs_i(x) = -beta mu^HS_i(x):
 * the back-convolution of the ten dPhi/dn_alpha of eq. Phi with the weights
 * (eq. muHS), with the |nV2| <= n2 bound of Sec. "Numerical Stability".
 * rho: [S][N], c1_out: [S][N] device.
 */
dft_status dft_c1_hs(dft_plan* plan, const void* rho, void* c1_out);

/*
 * Electrostatic part c1_es_i(x) = -(beta mu^SC_i(x) + z_i psi(x)) with the
 * bulk-fluid screening term of eq. muESexpansion (kernel eq. CplusPsiFunc,
 * transform eq. CplusPsiHat with the prefactor read as 2 pi lambda_B z_i z_j / k)
 * and the mean-field potential psi = e phi / kT of eq. potentialSolution
 * (psi_hat(0) = 0, eq. potentialConstraint).
 * rho: [S][N]; c1_out: [S][N]; psi_out: [N] or NULL.
 */
dft_status dft_c1_es(dft_plan* plan, const void* rho, void* c1_out, void* psi_out);

/*
 * The Picard map G of eq. rhoEquation:
 * G_i(x) = rho_bath_i exp(beta mu^ex,bath_i - V_i(x) - beta mu^ex_i(x)), 0 where V_i = +inf.
 * rho, V: [S][N]; g_out: [S][N] device.  resid_out (may be NULL) receives
 * r = sqrt(sum_i sum_x ((rho_i - G_i)/rho_bath_i)^2 / (S N)).
 */
dft_status dft_picard_map(dft_plan* plan, const void* rho, const void* V, void* g_out, double* resid_out);

/*
 * One Picard iteration (eq. picard) with the line search of Sec. "Nonlinear
 * solver": rho <- (1 - alpha) rho + alpha G(rho).  alpha_or_neg >= 0 gives
 * fixed mixing alpha = min(alpha_or_neg, alpha_max); a negative value selects
 * the quadratic line search on r^2 sampled at alpha_s/2 and alpha_s, with
 * alpha_s = min(alpha_max, 2 alpha_prev) (alpha_prev: the previous step's alpha
 * within dft_solve / dft_iter_step; alpha_s = alpha_max on a first step).
 * alpha_max = min(1, (0.9 - max n3(rho)) / (max n3(G) - max n3(rho))) when
 * max n3(G) > max n3(rho), else 1.  rho_inout: [S][N] device, updated in place.
 * resid_out receives r(rho) before the update, alpha_out the alpha used (either may be NULL).
 */
dft_status dft_picard_step(dft_plan* plan, void* rho_inout, const void* V, double alpha_or_neg,
                           double* resid_out, double* alpha_out);

/*
 * Iterate dft_picard_step until r(rho) < tol or max_it iterations.  Returns
 * DFT_ENOCONV (with rho holding the last iterate) if tol was not reached.
 * iters_out: iterations taken; resid_out: r of the returned rho.
 */
dft_status dft_solve(dft_plan* plan, void* rho_inout, const void* V, double alpha_or_neg, double tol,
                     int max_it, int* iters_out, double* resid_out);

/*
 * Newton-Krylov alternative to dft_solve (the paper reports trying Newton-GMRES; Sec.
 * "Nonlinear solver"): Newton on F(u) = u - log G(e^u) over the accessible voxels
 * (u = log rho), each Newton step solving J d = -F by restarted-free GMRES with at most
 * krylov_dim (1..200) Jacobian-vector products J v = (F(u + eps v) - F(u)) / eps (one G
 * evaluation each; eps = sqrt(machine epsilon) sqrt(S N) for unit v) to relative residual
 * 0.1, then a backtracking line search (u + lam d, lam = 1, 1/2, ... 1/128) requiring
 * |F| to decrease; a trial whose G meets n3 >= 1 or a non-finite value is shortened.
 * Stops when the Picard residual r(rho) of dft_picard_step is below tol (DFT_OK) or after
 * max_newton steps / a line search that finds no decrease (DFT_ENOCONV, rho = the last
 * accepted iterate).  rho_inout: [S][N] device, positive on accessible voxels.  Work
 * vectors ((krylov_dim + 7) S N reals) are allocated for the call.  newton_out,
 * gevals_out (G evaluations), resid_out may be NULL.
 */
dft_status dft_solve_newton(dft_plan* plan, void* rho_inout, const void* V, double tol, int max_newton,
                            int krylov_dim, int* newton_out, int* gevals_out, double* resid_out);

/*
 * Stateful iteration for callers that drive the loop themselves (and for
 * timing): dft_iter_begin evaluates G(rho) and keeps it, with the weighted
 * densities of rho, inside the plan; each dft_iter_step then performs one
 * Picard iteration on rho_inout exactly as dft_picard_step does, reusing the
 * kept state (no re-evaluation of G(rho)).  rho_inout and V must be the same
 * buffers, unmodified by the caller, between begin and the steps.
 * resid_out/alpha_out: as dft_picard_step; NULL skips the synchronisation.
 * DFT_FP32_STAB plans carry the iterate in extended precision: rho_inout holds
 * its float value and the plan a float low part (its rounding error, zero at
 * dft_iter_begin), the mixing rho0 + alpha (G - rho0) adds into the pair
 * without rounding steps below half an ulp away, and the residual is that of
 * the pair.  rho_inout alone is the pair rounded to float.  The same holds within dft_solve,
 * dft_iter_run, dft_picard_step and dft_picard_step_host (each call starts
 * from a zero low part).
 */
dft_status dft_iter_begin(dft_plan* plan, void* rho_inout, const void* V);
dft_status dft_iter_step(dft_plan* plan, void* rho_inout, const void* V, double alpha_or_neg,
                         double* resid_out, double* alpha_out);

/*
 * `iters` consecutive dft_iter_step iterations (same arithmetic, same order) queued as ONE
 * launch of a CUDA graph whose body -- one iteration, captured on the first call for these
 * (rho_inout, V, alpha_or_neg) -- repeats on the device `iters` times (a conditional WHILE
 * graph node counting down a device-side counter), so the host takes no part between
 * iterations; a runtime without conditional graph nodes gets `iters` replays of a graph of
 * one iteration instead.  The graph is kept in the plan until those arguments change,
 * dft_iter_begin or dft_autotune is called or the plan is destroyed.  Requires a preceding
 * dft_iter_begin on the same buffers.  resid_out (may be NULL; NULL skips the
 * synchronisation) receives r of rho after the last iteration.  While kernel profiling is
 * enabled the iterations are launched one by one instead (the per-kernel events are not
 * captured).
 */
dft_status dft_iter_run(dft_plan* plan, void* rho_inout, const void* V, int iters, double alpha_or_neg,
                        double* resid_out);

/*
 * Autotuner (no counterpart in the paper): on the plan's own data (rho, V: [S][N] device,
 * read only; `reps` timed launches per candidate, < 1 selects 5) it times and keeps the fastest
 *  - rows per block of the x passes that run every iteration (forward x transform of the
 *    densities; the Phi' pass and its paired-sample form; the update pass and its paired form,
 *    over candidates 1..16; the n3-maximum pass of the line search over 8..64);
 *  - the Phi' x passes: one CTA per row block, or persistent CTAs whose row blocks arrive by
 *    bulk copies two blocks ahead, or by per-thread cp.async copies one block ahead (each with
 *    its own rows per block);
 *  - the x transform: the compile-time kernels (where the length has them) against the
 *    run-time ones under each candidate radix order (the default plan -- 3s, other odd primes,
 *    16s, then 2/4/8 --, its reverse, and for powers of two a plan of 8s and one of 4s);
 *  - the y transform: the persistent TMA pass against the run-time column kernel;
 *  - the z passes: the persistent TMA passes against the grouped one-tile-per-CTA kernels;
 *    then the first half's z stage as one pass against three (z transform, products, z
 *    transform).
 * Results are cached per (grid, species count, precision) for the life of the process, so
 * later plans of the same shape reuse them without timing.  Invalidates a preceding
 * dft_iter_begin (call it again).  lines_out (may be NULL) receives the first three row
 * choices; dft_plan_tuning describes all of them.  Runs on the plan's stream and synchronises it.
 */
dft_status dft_autotune(dft_plan* plan, const void* rho, const void* V, int reps, int lines_out[3]);

/* One line describing the plan's transform variants, radix orders and rows per block (the
 * defaults until dft_autotune chooses); owned by the plan, valid until its next call.  "" for NULL. */
const char* dft_plan_tuning(const dft_plan* plan);

/* Pin the transform variants instead of letting dft_autotune choose them (and for tests):
 * x_variant 0 = the compile-time x kernels (only for lengths that have them), k >= 1 = the
 * run-time ones under candidate radix order k (in dft_autotune's order; DFT_EINVAL past the
 * last); x_persistent 1 = with the compile-time kernels, the Phi' passes as the persistent
 * kernel whose row blocks arrive by bulk copies two blocks ahead, 2 = by per-thread cp.async
 * copies one block ahead (0 = one CTA per row block);
 * y_variant 0 = persistent TMA pass (run-time kernel for lengths without one), 1 = run-time
 * column kernel; z_variant bit 0: 0 = persistent TMA passes, 1 = grouped one-tile-per-CTA
 * kernels; bit 1: the first half's z stage as three passes (persistent TMA z transform of the
 * species, a k-space products pass, z transform of the nine weighted densities) instead of one
 * (lengths without compile-time kernels run the run-time ones either way).  Invalidates a
 * preceding dft_iter_begin. */
dft_status dft_set_variants(dft_plan* plan, int x_variant, int x_persistent, int y_variant, int z_variant);

/*
 * Grand potential and its gradients (differentiated form).  The paper asserts
 * the functional (Sec. "Introduction") and its bulk-fluid expansion (eq.
 * muESexpansion2); the discrete functional whose stationarity condition is
 * eq. rhoEquation is, in kT units,
 *   Omega = h^3 sum_x sum_i [rho_i (ln(rho_i/rho_bath_i) - 1) + rho_i (V_i - mu_ex_bath_i)]
 *         + h^3 sum_x Phi(n(x))                                   (eq. Phi)
 *         + h^3 sum_i mu_ES_bath_i sum_x drho_i
 *         - (h^3/2) sum_i sum_x drho_i (DC_ij (*) drho_j - z_i psi)(x)
 * with drho = rho - rho_bath over all voxels and an electroneutral bath.
 * Outputs (any may be NULL):
 *   omega_out     Omega (host double)
 *   dOmega_drho   [S][N] device: h^3 [ln(rho_i/rho_bath_i) + V_i - mu_ex_bath_i + mu_ex_i(x)]
 *                 = h^3 ln(rho_i / G_i), zero where V_i = +inf or rho_i = 0
 *   dOmega_dV     [S][N] device: h^3 rho_i (the explicit partial; at a solution of
 *                 eq. rhoEquation it is the total derivative, by stationarity)
 *   dOmega_dbulk  [S] host: dOmega/drho_bath_k at fixed rho and V, kT nm^3 (bath
 *                 derivatives of mu_ex, mu_ES and Gamma by extrapolated central
 *                 differences of the App. A solver; the Gamma dependence of DC by
 *                 its analytic derivative).
 * Weighted densities are recomputed, not stored.  Synchronous.
 */
dft_status dft_grad(dft_plan* plan, const void* rho, const void* V, double* omega_out, void* dOmega_drho,
                    void* dOmega_dV, double* dOmega_dbulk);

/*
 * End-to-end convenience for host buffers: copies rho (and V) from HOST
 * memory to the plan's device scratch, performs one dft_picard_step, and
 * copies the updated rho back to HOST memory.  rho_host: [S][N], V_host:
 * [S][N], element type as the plan's precision.  Synchronous.
 */
dft_status dft_picard_step_host(dft_plan* plan, void* rho_host, const void* V_host, double alpha_or_neg,
                                double* resid_out, double* alpha_out);

/*
 * Batched state points.  A batch holds `count` independent state points (each
 * with its own grid -- ragged sizes allowed --, species, bath and precision, as
 * in dft_plan_create; each owns a plan and a CUDA stream).  dft_batch_begin
 * takes per-state DEVICE pointers rho[i] ([S_i][N_i], updated in place) and V[i]
 * and evaluates G for every state.  dft_batch_iterate then advances every state
 * by `iters` Picard iterations (alpha_or_neg as in dft_picard_step); one
 * iteration of all states is captured once into the body of an on-device loop (a
 * CUDA graph with a conditional WHILE node; fork/join across the state streams
 * inside the body), so one graph launch runs all `iters` iterations of all states,
 * the states concurrently (a runtime without conditional graph nodes gets one
 * graph launch per iteration instead).  resid_out ([count], may be NULL)
 * receives each state's r after the last iteration (synchronises).
 * cuda_stream: stream the batch orders its work after (NULL: an internal one).
 * The rho and V pointers must stay valid and unmoved between begin and iterate.
 */
typedef struct dft_batch dft_batch;
dft_status dft_batch_create(const dft_params* params, int count, void* cuda_stream, dft_batch** out);
dft_status dft_batch_destroy(dft_batch* batch);
const char* dft_batch_last_error(const dft_batch* batch);
dft_status dft_batch_begin(dft_batch* batch, void* const* rho, const void* const* V);
/* Autotune every state's plan (dft_autotune on rho[i], V[i], reps repetitions), one state at a
 * time; states with the same grid, species count and precision share the cached choice.
 * Synchronises the states' streams; a following dft_batch_begin is needed before iterating. */
dft_status dft_batch_autotune(dft_batch* batch, void* const* rho, const void* const* V, int reps);
dft_status dft_batch_iterate(dft_batch* batch, int iters, double alpha_or_neg, double* resid_out);

/*
 * Bound of the bounded device-side waits (failure detection; no counterpart in the paper).
 * The y passes move their column tiles by TMA and wait for each tile on an mbarrier; a wait
 * gives up after `polls` polls (default DFT_WAIT_POLLS_DEFAULT), the CTA then drains the copies
 * it still has in flight (those waits keep the default bound, so no copy outlives the CTA),
 * records the timeout in the plan's device status word and stops, and the call that queued the
 * work returns DFT_ETIMEOUT (the context stays usable; results of that call are undefined).
 * polls = 0 makes every such wait give up at once, which is how the timeout path is exercised
 * without a fault or a hang.  Applies to the plan's later calls (a cached iteration graph is
 * dropped and recaptured).  polls < 0: DFT_EINVAL.
 */
#define DFT_WAIT_POLLS_DEFAULT (1LL << 24)
dft_status dft_set_wait_polls(dft_plan* plan, long long polls);

/*
 * Programmatic dependent launch of the plan's passes (no counterpart in the paper; a GPU
 * scheduling option).  Enabled by default: each pass is launched with CUDA's programmatic
 * stream serialization attribute, so that its launch overlaps the completion of the previous
 * kernel in the stream; every pass waits (griddepcontrol.wait) for the kernels before it to
 * complete before it reads or writes data they touch, so results are the same either way
 * (bitwise).  enable = 0 launches
 * the passes in plain stream order.  Per-kernel profiling (dft_profile_enable) launches in
 * stream order while it is on.  A runtime that cannot capture such launches into the iteration
 * graph of dft_iter_run / dft_batch_iterate gets the graph in stream order instead.  Applies to
 * later calls (a cached iteration graph is dropped and recaptured).
 */
dft_status dft_set_dependent_launch(dft_plan* plan, int enable);

/*
 * Per-kernel timing with CUDA events recorded on the plan's stream around
 * each launch.  enable != 0 starts collection (and clears totals).
 * dft_profile_read returns, for the kernel kind named by `name`, the number
 * of launches, their total duration (ms) and their total algorithmic global
 * memory traffic (bytes: every input element read once and every output
 * element written once by each launch) since the last enable; it
 * synchronises the stream.  Names: "xfwd", "yfft", "zconv_fwd", "xphi",
 * "zconv_bwd", "xupdate", "xinv", "finalize".  Any out pointer may be NULL.
 */
dft_status dft_profile_enable(dft_plan* plan, int enable);
dft_status dft_profile_read(dft_plan* plan, const char* name, int* launches, double* total_ms,
                            double* total_bytes);

/*
 * Allocation-free weighted densities.  The paper has no counterpart: this is a
 * deployment variant of dft_weighted_densities for callers that cannot allocate
 * device memory -- code running inside a memory pool whose owner has reserved the
 * GPU's memory and forbids cudaMalloc, code that must not trigger the implicit
 * device synchronisation an allocation can cause, and users who must know their
 * whole device footprint when the library loads.  It computes exactly what
 * dft_weighted_densities computes, with the same kernels, but needs no plan: all
 * of its scratch (twiddles, spectra, weighted densities) lives in one file-scope
 * device array of DFT_NOALLOC_SCRATCH_BYTES that every GPU loading this part of
 * the library holds until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.  Under lazy module loading (CUDA_MODULE_LOADING=LAZY)
 * the first call on a device loads the module and so reserves the array there; a
 * caller that needs a fixed footprint makes that first call at initialisation.
 *
 * params: as for dft_plan_create; precision must be DFT_FP32_STAB; only the
 *   grid and the radii are used (the weighted densities need no bath).
 * cuda_stream: cudaStream_t for all work (NULL = legacy default stream).
 * rho: [S][N] float device input; n_out: [10][N] float device output.
 * errbuf/errbuf_len: optional buffer for a one-line error text (may be NULL).
 * Limits: a grid and species count whose scratch exceeds
 *   DFT_NOALLOC_SCRATCH_BYTES is rejected with DFT_EINVAL and a message naming the
 *   bytes needed (64^3 fits with up to 5 species; 96^3 does not).
 * Set-up: the first call on each device looks up the device address of the
 *   scratch array (and sets the kernels' shared-memory limits) with that device
 *   current and keeps it for the life of the process; make that first call before
 *   any CUDA stream capture.  A cudaDeviceReset invalidates it: do not use this entry
 *   point on a device after resetting it in the same process.
 * Completion: the call clears the scratch's status word (where a bounded wait of the
 *   TMA passes records that it gave up), queues the work and reads the status word
 *   back, so it returns only when n_out is complete (it synchronises cuda_stream);
 *   DFT_ETIMEOUT if a wait gave up (n_out is then incomplete).
 * Sharing: every call on a device uses the same array and leaves its contents
 *   behind; each call clears the status word and writes every other scratch element
 *   before reading it, but calls whose work overlaps on the GPU (different streams,
 *   or host threads without ordering) race on the array and corrupt each other.
 *   Order the calls (one stream, or events) to keep them apart.
 */
#define DFT_NOALLOC_SCRATCH_BYTES (24u << 20)
dft_status dft_weighted_densities_noalloc(const dft_params* params, void* cuda_stream, const void* rho,
                                          void* n_out, char* errbuf, size_t errbuf_len);

/* Library version string. */
const char* dft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300DFT_H */
