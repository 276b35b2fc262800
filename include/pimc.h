/*
 * pimc.h -- C ABI of the GB300 (sm_103a) path-integral Monte Carlo sampler
 * for data assimilation (Quinn & Abarbanel, "Data Assimilation using a GPU
 * Accelerated Path Integral Monte Carlo Approach").
 *
 * The sampler draws paths X = {x_0..x_M} (x_n in R^D, SoA layout
 * X[a*(M+1)+n]) and parameters p (N_p of them) from P(X|Y) ~ exp(-A):
 *
 *   A = 1/2 Rm sum_{n=1}^{M} (x_{n,0} - y_n)^2                       (A_o)
 *     + beta/2 sum_{n=0}^{M-1} sum_a Rf_a (x_{n+1,a} - f_a(x_n,p;I_n))^2  (A_f)
 *
 * -- Eq. (action) under the Gaussian measurement/model-error assumptions of
 * Sec. 2.1 (Eq. (obsError), Eq. (modelError)), with the model-error residual
 * taken against an explicit one-step RK4 map f of the model vector field and
 * beta the annealing multiplier of Sec. 4.2.  The observation function is
 * h(x) = x_0 (L = 1, Sec. 5.1).  A uniform prior box on p (Sec. 2.1, last
 * assumption; Sec. 4.2, "boundaries on parameters") rejects out-of-box moves.
 *
 * Conventions
 *   * Every function returns PIMC_OK (0) or a negative pimc_status.  The text
 *     of the last error of a handle is pimc_last_error(h).
 *   * A handle owns all of its device buffers.  Host arrays passed in are
 *     caller-owned and copied; host arrays passed out are caller-allocated
 *     and filled.  Functions taking *_dev pointers use caller-owned device
 *     memory and never free it.
 *   * Work is enqueued on the handle's stream (pimc_set_stream; default: a
 *     stream the handle creates).  pimc_sweep returns once its kernels are
 *     enqueued; functions that return host data synchronise the stream and
 *     report any error flagged by a kernel (e.g. PIMC_ERR_TIMEOUT).
 *   * A handle is not thread-safe; separate handles are independent.
 *   * Sizes: M >= 1; D and N_p are fixed by the model (HH and HH_PAPER: D = 4,
 *     N_p = 7; LINGAUSS: D = 2, N_p = 1; TOY1D: D = 1, N_p = 1).
 */
#ifndef PIMC_H
#define PIMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pimc_handle_s* pimc_t;

typedef enum {
    PIMC_OK = 0,
    PIMC_ERR_ARG = -1,      /* invalid argument (size, pointer, non-finite value) */
    PIMC_ERR_STATE = -2,    /* call out of order (e.g. sweep before set_data) */
    PIMC_ERR_CUDA = -3,     /* a CUDA runtime call failed */
    PIMC_ERR_OOM = -4,      /* device allocation failed */
    PIMC_ERR_TIMEOUT = -5,  /* a bounded device-side wait expired; the launch returned early */
    PIMC_ERR_NUMERIC = -6,  /* non-finite value where a finite one is required */
    PIMC_ERR_IO = -7        /* checkpoint file missing, short or corrupt */
} pimc_status;

typedef enum {
    PIMC_MODEL_HH = 0,       /* Hodgkin-Huxley, x = (V, m, h, n),
                                p = (gNa, gK, gL, ENa, EK, EL, C) (Sec. 5.1) */
    PIMC_MODEL_LINGAUSS = 1, /* dx/dt = K x + (p0, I), K = [[-0.5,-2],[2,-0.5]] (test model) */
    PIMC_MODEL_TOY1D = 2,    /* dx/dt = p0 sin(x) - x/2 + I (test model) */
    PIMC_MODEL_HH_PAPER = 3  /* the paper's HH form (Sec. 5.1, Eq. (dVdt), Eq. (dadt)):
                                dV/dt = p1 I + p2 m^3 h (p3 - V) + p4 n^4 (p5 - V) + p6 (p7 - V),
                                tanh gate kinetics with the Table 1 constants */
} pimc_model;

typedef enum {
    PIMC_SCHEME_RK4 = 0,       /* eps_{n+1} = x_{n+1} - f(x_n), f one RK4 step (default) */
    PIMC_SCHEME_TRAPEZOID = 1  /* eps_{n+1} = x_{n+1} - x_n - dt/2 [F(x_{n+1}) + F(x_n)],
                                  Eq. (modelError); F cached per site (Sec. 4.3) */
} pimc_scheme;

typedef enum {
    PIMC_PROPOSAL_GAUSS = 0,   /* x' = x + sigma . N(0, 1) (default) */
    PIMC_PROPOSAL_UNIFORM = 1  /* x' = x + sigma . U(-1, 1), Fig. 1 step (a) */
} pimc_proposal;

typedef enum {
    PIMC_FP64 = 0,           /* every step in FP64 */
    PIMC_FP32_MIXED = 1      /* path, cache and per-site arithmetic in FP32; the
                                parameter-move reduction, its accept test, the
                                global action and the moment sums in FP64 */
} pimc_precision;

/* ---- lifetime ----------------------------------------------------------- */

/* Create a sampler for `model` over sites n = 0..M with time step dt.
 * L must be 1 and D must equal the model's dimension.  Rm points to one
 * double (the measurement precision R_o of Eq. (obsError), > 0); Rf to D
 * doubles (the diagonal model-error precision R_d of Eq. (modelError), >= 0).
 * The device is the CUDA device current on the calling thread.
 * Errors: PIMC_ERR_ARG (bad sizes/values), PIMC_ERR_OOM, PIMC_ERR_CUDA. */
int pimc_create(pimc_t* out, int model, int64_t M, int D, int L, double dt,
                const double* Rm, const double* Rf);
int pimc_destroy(pimc_t h);
const char* pimc_last_error(pimc_t h);
/* Use `stream` (a cudaStream_t, may be NULL for the legacy default stream)
 * for all further work of this handle.  The caller keeps ownership. */
int pimc_set_stream(pimc_t h, void* stream);
/* Select the arithmetic (pimc_precision).  Re-initialises the path from its
 * current FP64 value; call before pimc_sweep. */
int pimc_set_precision(pimc_t h, int precision);

/* Model-error discretisation (pimc_scheme).  With the trapezoid rule the
 * vector field is evaluated at grid points; the drive there is I_inj[n] for
 * n < M and I_inj[M-1] at t_M.  Refreshes the cache. */
int pimc_set_scheme(pimc_t h, int scheme);
/* Proposal increments of site and parameter moves (pimc_proposal). */
int pimc_set_proposal(pimc_t h, int kind);

/* ---- problem data (Sec. 4.1, "the current path, the observation time series,
 *      the external drive signal ... are allocated in GPU memory") ---------- */

/* y: M+1 observations (y_0 only seeds the initial path); I_inj: M drive values,
 * held over [t_n, t_{n+1}).  Both must be finite.  Re-initialises the path to
 * the default initial guess: x_{n,0} = y_n, other components at the model's
 * steady state for that voltage (HH gates a_inf = alpha/(alpha+beta)). */
int pimc_set_data(pimc_t h, const double* y, const double* I_inj);
/* Replace y and I_inj without re-initialising the path (new data for a running
 * chain, e.g. the next observation window); refreshes the f cache.  Enqueued
 * on the handle's stream: with pinned host arrays the copies are asynchronous
 * and the arrays must stay unchanged until the next synchronising call. */
int pimc_load_data(pimc_t h, const double* y, const double* I_inj);
/* p, lo, hi: Np doubles; free_mask: Np bytes (1 = sampled, 0 = fixed).
 * lo <= p <= hi is required for free parameters. */
int pimc_set_params(pimc_t h, const double* p, const double* lo, const double* hi,
                    const uint8_t* free_mask, int Np);
/* Optional explicit path, D*(M+1) doubles in SoA layout. */
int pimc_set_path(pimc_t h, const double* X);
/* Proposal scales: sigma_x has D doubles (same for every site) when
 * per_site == 0, or D*(M+1) doubles when per_site == 1; sigma_p has Np doubles. */
int pimc_set_steps(pimc_t h, const double* sigma_x, int per_site, const double* sigma_p);
/* Burn-in and recording schedule (Sec. 4.1-4.2): statistics are recorded at
 * sweeps s >= n_init with (s - n_init) % n_skip == 0; during s < n_init the
 * proposal scales are adapted every n_skip sweeps by
 * sigma <- sigma [1 + alpha (N_acc/n_skip - f_acc)]; beta starts at beta0 and
 * is multiplied by f_beta = (1/beta0)^(1/n_cool) after each sweep until
 * sweep n_cool, then stays 1 (Eq. (fbeta)).  Requires n_skip >= 1,
 * 0 < beta0 <= 1.  Resets the sweep counter to 0 and clears the statistics. */
int pimc_set_schedule(pimc_t h, int64_t n_init, int64_t n_skip, double beta0, int64_t n_cool,
                      double f_acc, double alpha);
/* Chain index (fourth Philox counter word); distinct chains on the same data
 * and seed draw independent streams. */
int pimc_set_chain(pimc_t h, uint32_t chain);

/* ---- the hot path ---------------------------------------------------------- */

/* Run n_sweeps checkerboard sweeps (Fig. 1, Sec. 4.1): even sites, then odd
 * sites, then each free parameter in order, then (when due) the statistics,
 * the step adaptation and the annealing step.  Random numbers are
 * Philox-4x32-10 keyed by `seed` with counters (n or l, sweep, kind, chain),
 * so a run resumes exactly at the handle's sweep counter.  Asynchronous. */
int pimc_sweep(pimc_t h, int64_t n_sweeps, uint64_t seed);
/* Whole-path Hybrid Monte Carlo: n_traj trajectories, each moving X and the
 * free parameters together by n_leap leapfrog steps of the Hamiltonian
 * H = A + 1/2 P^T diag(inv_mass) P (beta = 1), with the step jittered
 * uniformly in [0.8, 1.2] eps per trajectory and the usual accept test
 * (Eq. (Paccept) on Delta H).  The gradient is the reverse-mode adjoint of
 * the action through the RK4 map (pimc_grad).  inv_mass: D*(M+1)+Np host
 * doubles (NULL: all ones; entries of fixed parameters are ignored).  A
 * trajectory that takes a parameter out of its box is rejected.  Momenta and
 * uniforms are Philox draws keyed by (component pair | 0, trajectory, kind 2 |
 * 3, chain) with the trajectory counter = the sweep counter, which advances by
 * one per trajectory; statistics follow the schedule of pimc_set_schedule.
 * The launch sequence of one trajectory is captured once as a CUDA graph on
 * the handle's stream and replayed.  The call first waits for the handle's
 * stream (inv_mass is uploaded), then enqueues the trajectories.
 * *n_accepted (may be NULL) receives the accepted count of this call and makes
 * the call wait for them; with NULL it returns once they are enqueued, so
 * handles on different streams, driven from different host threads, run
 * their trajectories concurrently. */
int pimc_hmc(pimc_t h, int64_t n_traj, int n_leap, double eps, const double* inv_mass, uint64_t seed,
             int64_t* n_accepted);

/* Synchronise and return the sticky device status (PIMC_ERR_TIMEOUT if a
 * bounded wait expired in any launch since the last call; the flag is cleared). */
int pimc_sync(pimc_t h);

/* Full action of the current state at beta = 1: A = A_o + A_f (Sec. 2.1). */
int pimc_action(pimc_t h, double* A_out, double* Ao_out, double* Af_out);
/* Gradient of A_o + beta A_f with respect to X (D*(M+1) doubles, SoA) and p
 * (Np doubles; entries of fixed parameters are still filled). */
int pimc_grad(pimc_t h, double beta, double* gX, double* gp);

/* Action and gradient of caller-owned device arrays against this handle's
 * data and settings (for autograd / HMC drivers).  X_dev: D*(M+1) doubles,
 * p_dev: Np doubles, out_dev: 3 doubles (A, A_o, A_f at beta = 1);
 * gX_dev: D*(M+1), gp_dev: Np doubles.  Enqueued on `stream`; no sync. */
int pimc_action_dev(pimc_t h, const double* X_dev, const double* p_dev, double* out_dev,
                    void* stream);
int pimc_grad_dev(pimc_t h, const double* X_dev, const double* p_dev, double beta,
                  double* gX_dev, double* gp_dev, void* stream);

/* Allocation-free action.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they call --
 * code held to a fixed memory budget or a caller-owned pool, plugin hosts
 * that forbid cudaMalloc/cudaFree on their threads, and real-time loops in
 * which an allocation (which may synchronise the device) is not allowed.
 * It computes the FP64 action (A, A_o, A_f at beta = 1) with the explicit
 * RK4 model error, without a handle: the value pimc_action_dev gives for an
 * FP64 handle with the RK4 scheme.  Supported models: PIMC_MODEL_HH,
 * PIMC_MODEL_LINGAUSS and PIMC_MODEL_TOY1D; PIMC_MODEL_HH_PAPER (and the
 * trapezoid scheme, which has no argument here) are not, and that model
 * returns PIMC_ERR_ARG.  X_dev (D*(M+1) doubles, SoA), p_dev (Np), y_dev
 * (M+1), I_dev (M) and out_dev (3 doubles) are caller-owned device arrays;
 * Rf is host memory holding exactly D doubles (the model's dimension); work
 * is enqueued on `stream`.
 * Its scratch (per-CTA partial sums and a last-block counter, 33,024 bytes)
 * is one fixed array in device memory that every GPU loading this library
 * holds until the process exits, so M is limited to 1 <= M <= 262,143;
 * larger M (and bad pointers or sizes) return PIMC_ERR_ARG with a message in
 * pimc_last_error(NULL).  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  Every call looks up the array's device address in
 * the current context (cudaGetSymbolAddress, which allocates nothing); the
 * first call on a device may also load the library's device code there, so
 * make that first call before any stream capture.  Every call shares the array: calls that overlap on the GPU
 * (different streams, devices excepted) race and must be serialised by the
 * caller. */
int pimc_action_static(int model, int64_t M, double dt, double Rm, const double* Rf,
                       const double* X_dev, const double* p_dev, const double* y_dev,
                       const double* I_dev, double* out_dev, void* stream);

/* ---- diagnostics of the hot path (parity tests) ------------------------------ */

/* Local change of action Delta A_n for replacing x_n by Xp[:,n], each site
 * against the current path (Fig. 1 steps (b)-(g)), for all n = 0..M. */
int pimc_site_delta(pimc_t h, const double* Xp, double beta, double* dA_out);
/* Change of action for moving parameter l to pl_new over the whole path. */
int pimc_param_delta(pimc_t h, int l, double pl_new, double beta, double* dA_out);

/* ---- statistics (Sec. 4.1, "path statistics ... on the GPU") --------------- */

/* mean, var: D*(M+1)+Np doubles each (path components in SoA order, then p);
 * var is the unbiased sample variance.  n_samples may be NULL. */
int pimc_moments(pimc_t h, double* mean, double* var, int64_t* n_samples);
/* Moments of the residuals of the recorded paths (Sec. 6: for a correct model
 * their means vanish and their variances match 1/Rf and 1/Rm): mean and var
 * hold (D+1)*M doubles, eps_{n+1,a} = x_{n+1,a} - f_a(x_n) at [a*M + n]
 * (n = 0..M-1) and delta_n = x_{n,0} - y_n at [D*M + n - 1] (n = 1..M). */
int pimc_residual_moments(pimc_t h, double* mean, double* var, int64_t* n_samples);
/* Ensemble forecast from the current state (Sec. 6; explicit RK4 scheme only): n_ens members integrate
 * x_{k+1} = f(x_k, p; I_future[k]) + xi_k from x_M for n_steps steps, with
 * model noise xi_{k,a} ~ N(0, 1/Rf_a) when noise != 0 (none where Rf_a = 0);
 * normals are Philox draws keyed by (member, step, kind 4 | pair, chain).
 * out (host): n_ens * D * (n_steps+1) doubles, [member][component][step].
 * Synchronous. */
int pimc_forecast(pimc_t h, int64_t n_steps, const double* I_future, int n_ens, int noise, uint64_t seed,
                  double* out);
/* Histograms of n_sel components (index c < D*(M+1) selects X[c], otherwise
 * p[c - D*(M+1)]): n_bins equal bins on [lo, hi) plus under/overflow slots.
 * 1 <= n_sel <= 64, 1 <= n_bins <= 4096.  Clears the counts. */
int pimc_set_histograms(pimc_t h, int n_sel, const int64_t* comp_index, const double* lo,
                        const double* hi, int n_bins);
/* counts: n_sel*(n_bins+2) uint64, per component [under, bins..., over]. */
int pimc_histograms(pimc_t h, uint64_t* counts);
/* Current histogram configuration (0, 0 when none is set). */
int pimc_histogram_shape(pimc_t h, int* n_sel, int* n_bins);

/* Parameter trace: after every sweep the kernel writes p into a device ring
 * of `cap` vectors (0 disables).  Resets the trace.  For effective-sample-
 * size diagnostics of the parameter chain. */
int pimc_set_param_trace(pimc_t h, int64_t cap);
/* The last min(n, ring capacity, cap) parameter vectors in chronological
 * order, Np doubles each; *n_written receives that count (out may be NULL to
 * query it). */
int pimc_param_trace(pimc_t h, double* out, int64_t cap, int64_t* n_written);

/* ---- state ----------------------------------------------------------------- */
int pimc_get_state(pimc_t h, double* X, double* p);
/* The parameter vector p (Np doubles) as it stands after the work enqueued so
 * far, copied into caller-owned host memory p_host by a copy enqueued on the
 * handle's stream, without waiting: the values are there once the stream has
 * reached the copy (pimc_sync, or any synchronisation of that stream).  For
 * streaming use (data in, sweeps, result out, step after step) with no host
 * stall per step; p_host should be page-locked, else the copy is not
 * asynchronous.  PIMC_ERR_ARG for NULL arguments. */
int pimc_params_async(pimc_t h, double* p_host);
int pimc_get_steps(pimc_t h, double* sigma_x /*D*(M+1)*/, double* sigma_p /*Np*/);
/* Current sweep counter and beta. */
int pimc_get_sweep(pimc_t h, int64_t* sweep, double* beta);
/* Totals since the last pimc_set_schedule: accepted and proposed site moves
 * (index 0 even, 1 odd), accepted and proposed parameter moves (Np each). */
int pimc_accept_stats(pimc_t h, uint64_t* site_acc, uint64_t* site_prop, uint64_t* par_acc,
                      uint64_t* par_prop);
/* Launch geometry chosen for the sweep kernel (grid CTAs, threads per CTA). */
int pimc_launch_info(pimc_t h, int* grid, int* block);
/* Form the sweep takes at the current size, precision and grid: *resident = 1
 * when every site lives in one thread for the whole launch (FP32-mixed, at
 * most 224 sites per CTA; the site phases then order on flags between
 * neighbouring CTAs), 0 for the general form (threads stride over the tile).
 * Both forms give the same bits for the same tiles. */
int pimc_sweep_form(pimc_t h, int* resident);
/* Which forms the sweep may take: PIMC_FORM_AUTO (default; the resident form
 * where it fits) or PIMC_FORM_GENERAL (always the general form, e.g. to
 * compare the two).  PIMC_ERR_ARG for other values. */
typedef enum { PIMC_FORM_AUTO = 0, PIMC_FORM_GENERAL = 1 } pimc_form;
int pimc_set_sweep_form(pimc_t h, int form);

/* ---- batched launch: many chains and data sets of uneven M ----------------- */

typedef struct pimc_batch_s* pimc_batch_t;

/* Group n handles (same model, precision and device; data and parameters set)
 * into one launch.  Every CTA runs whole chains one after another with
 * CTA-local synchronisation, or tiles of long chains shared with other CTAs
 * (pimc_batch_set_tuning); chains are assigned to CTAs longest-first onto the
 * least loaded CTA(s), with a chain's cost (M + 1)(1 + free parameters).  Each chain keeps its own handle: state,
 * schedule, statistics, trace and checkpoints are read and set through it.
 * Handles must have no work in flight and must not be used while a batch
 * sweep runs (call pimc_batch_sync first).  A chain runs exactly the sweeps it
 * would run alone with pimc_set_grid(h, 1) (bit-identical).  The handles must
 * outlive the batch. */
int pimc_batch_create(pimc_batch_t* out, const pimc_t* handles, int n);
int pimc_batch_destroy(pimc_batch_t b);
const char* pimc_batch_last_error(pimc_batch_t b);
/* n_sweeps sweeps of every chain (Philox key `seed`; counters continue each
 * chain's own sweep counter).  Enqueued on the first handle's stream as a
 * CUDA graph of launches of at most 256 sweeps each (re-captured when n_sweeps
 * or seed change). */
int pimc_batch_sweep(pimc_batch_t b, int64_t n_sweeps, uint64_t seed);
int pimc_batch_sync(pimc_batch_t b);
/* Tile shape (the block decomposition of Sec. 4.3 for many chains): threads
 * per CTA (128 or 256), resident CTAs per SM (0 = as many as fit), i.e. how
 * many chains share a CTA, and ctas_per_chain (1..64): a chain costing more
 * than a CTA's mean load is cut into up to that many tiles of even length (at
 * least 2 * threads_per_cta sites each), run together by as many CTAs of the
 * launch, which synchronise on the chain's own barrier word and exact-sum
 * slots with bounded waits (the launch is then cooperative); 1 keeps every
 * chain whole.  A chain's results do not depend on the tile shape.
 * PIMC_ERR_ARG for values out of range. */
int pimc_batch_set_tuning(pimc_batch_t b, int threads_per_cta, int ctas_per_sm, int ctas_per_chain);
/* The current plan: CTAs of a launch, threads per CTA, chains split over
 * several CTAs (any output may be NULL). */
int pimc_batch_info(pimc_batch_t b, int* n_ctas, int* threads_per_cta, int* n_split);
/* Time trial_sweeps real sweeps (they advance every chain: run this during
 * burn-in) for each tile shape -- threads per CTA x CTAs per SM x CTAs per
 * long chain (1, 2, 4) -- and keep the fastest; the choice is cached per
 * process for batches of the same model, precision, size and chain count. */
int pimc_batch_autotune(pimc_batch_t b, int64_t trial_sweeps, uint64_t seed, int* threads_per_cta, int* ctas_per_sm,
                        int* ctas_per_chain);

/* ---- checkpoint / resume ------------------------------------------------------ */
/* Binary file with a version and a CRC: sizes, settings, path, p, steps,
 * schedule position, statistics and counters.  Resuming and continuing gives
 * bit-identical results to an uninterrupted run (counter-based RNG). */
int pimc_checkpoint_save(pimc_t h, const char* path);
int pimc_checkpoint_load(pimc_t h, const char* path);

/* ---- test hooks ---------------------------------------------------------------- */
/* Bounded-wait limit of the grid barrier in nanoseconds (default 2e9). */
int pimc_set_wait_limit(pimc_t h, int64_t ns);
/* Checked builds only (libpimc_check.so: the same sources compiled with
 * PIMC_CHECK, in which the sweep kernels count site visits and check site
 * indices; the race and bounds check of the checkerboard, Sec. 4.1 and
 * Sec. 4.3).  Since the last reset: even[n], odd[n] (M+1 each, host,
 * caller-owned): visits of site n in the even and the odd site phases;
 * param[n] (M+1): the parameter moves' cache writes of site n; *moves: the
 * parameter moves executed (in-box proposals); *status: the handle's sticky
 * status, bit 2 set when a site index outside [0, M] was met (that access
 * skipped, nothing trapped).  Any output may be NULL; reset != 0 clears the
 * counts and bit 2 afterwards.  Synchronous.  PIMC_ERR_STATE in an unchecked
 * build. */
int pimc_debug_check_counts(pimc_t h, uint32_t* even, uint32_t* odd, uint32_t* param, uint64_t* moves,
                            int* status, int reset);
/* Make CTA `cta` skip its barrier arrivals in later sweeps (-1: off), so the
 * other CTAs' bounded waits expire and pimc_sync reports PIMC_ERR_TIMEOUT. */
int pimc_debug_skip_arrive(pimc_t h, int cta);
/* The exact sum that parameter moves use for their change of action, applied
 * to n caller terms (host array, copied): *out = the sum of terms[0..n), each
 * first rounded to FP32 when as_float != 0, computed on the current device in
 * 42-bit integer chunks of 2^-64 and rounded once to FP64; terms of magnitude
 * >= 2^62 count as infinite, NaN gives NaN.  as_float == 2 adds the FP32
 * terms through the per-thread 128-bit accumulator the parameter moves of the
 * general sweep form use (same result).  No handle; synchronous.
 * PIMC_ERR_ARG for n < 0 or n > 2^20, PIMC_ERR_CUDA on a device error. */
int pimc_debug_fix_sum(const double* terms, int64_t n, int as_float, double* out);
/* Throughput probe of the model map f (the RK4 map of Eq. (action)'s
 * model-error term): ctas_per_sm (1, 2 or 4) CTAs of 256 threads on every SM,
 * each thread iterating f from registers `iters` times (1 <= iters <= 2^24):
 * packed = 0, the FP32 form, one state a thread; 1, two states as the lanes
 * of the packed f32x2 form; 2, the FP64 form, one state a thread.
 * *maps_per_s (host) receives the rate.  No memory traffic and no
 * synchronisation: the ceiling a sweep's map arithmetic can reach on this
 * device.  Synchronous, on the current device; PIMC_ERR_ARG for arguments out
 * of range, PIMC_ERR_CUDA on a device error. */
int pimc_debug_map_rate(int packed, int ctas_per_sm, int64_t iters, double* maps_per_s);
/* The FP32 form of the model map f (one classical RK4 step of the HH field of
 * Sec. 5.1 with the textbook rates, drive held over the step; the map of the
 * model-error term of Eq. (action)) at n sites, for tests of its two lane
 * forms: X (4*n doubles, component-major [a][n]), I_inj (n), p (7: gNa, gK,
 * gL, ENa, EK, EL, C) and dt are host inputs, rounded to FP32 on the device;
 * f_out (4*n doubles, host, caller-owned) receives the single-site map, and
 * *n_mismatch the number of components of the sites (2i, 2i + 1), evaluated
 * as the two lanes of one packed f32x2 map, whose bits differ from it.  No
 * handle; synchronous; allocates and frees its device buffers.
 * PIMC_ERR_ARG for n outside [1, 2^22], dt <= 0 or a NULL array,
 * PIMC_ERR_CUDA on a device error. */
int pimc_debug_lane_maps(const double* X, const double* I_inj, const double* p, double dt, int64_t n,
                         double* f_out, int64_t* n_mismatch);
/* Force the sweep grid size (0: automatic). */
int pimc_set_grid(pimc_t h, int grid);

#ifdef __cplusplus
}
#endif
#endif /* PIMC_H */
