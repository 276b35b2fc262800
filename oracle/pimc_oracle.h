/*
 * Plain serial FP64 CPU oracle for path-integral Monte Carlo data assimilation
 * (Quinn & Abarbanel, "Data Assimilation using a GPU Accelerated Path Integral
 * Monte Carlo Approach").
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, obviously-correct
 * statement of what the sampler computes. Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Notation follows the paper: sites n = 0..M, state x_n in R^D (SoA layout
 * X[a*(M+1)+n]), observations y_n (n = 1..M; y_0 only seeds the initial path),
 * parameters p (N_p of them), drive current I_n (zero-order hold over
 * [t_n, t_{n+1}), n = 0..M-1).  The model map f(x, p; I_n) is one classical
 * RK4 step of size dt of the model vector field F.
 *
 * Action (Eq. (action) with the Gaussian assumptions of Sec. 2.1):
 *   A = 1/2 Rm sum_{n=1}^{M} (x_{n,0} - y_n)^2
 *     + beta/2 sum_{n=0}^{M-1} sum_a Rf_a (x_{n+1,a} - f_a(x_n, p; I_n))^2
 * with beta the annealing multiplier on the dynamics term (Sec. 4.2).
 *
 * Parity status of each function is stated beside it; see the test suite for
 * the pins (closed-form linear-Gaussian posterior, brute-force quadrature,
 * exact detailed balance, Random123 known-answer vectors, finite differences).
 */
#ifndef PIMC_ORACLE_H
#define PIMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_MODEL_HH = 0, ORC_MODEL_LINGAUSS = 1, ORC_MODEL_TOY1D = 2, ORC_MODEL_HH_PAPER = 3 };
/* Model-error discretisation: explicit one-step RK4 map, or the trapezoid
 * rule of Eq. (modelError) with the vector field cached per site. */
enum { ORC_SCHEME_RK4 = 0, ORC_SCHEME_TRAPEZOID = 1 };
/* Site/parameter proposal increments: N(0, 1) or U(-1, 1) (Fig. 1) times the step. */
enum { ORC_PROPOSAL_GAUSS = 0, ORC_PROPOSAL_UNIFORM = 1 };

typedef struct orc_state orc_state;

/* ---- counter-based RNG (Philox-4x32-10, Salmon et al. SC'11) ---------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Open-interval uniform from two 32-bit words: ((hi>>6)*2^26 + (lo>>6) + 0.5) * 2^-52 */
double orc_u01(uint32_t hi, uint32_t lo);
/* Draw kinds used in the counter's third word (kind << 24 | block). */
enum { ORC_KIND_SITE = 0, ORC_KIND_PARAM = 1, ORC_KIND_HMC_MOM = 2, ORC_KIND_HMC_ACC = 3, ORC_KIND_FORECAST = 4 };
/* Site draw: D normals (Box-Muller, cos then sin per pair) and one uniform. */
void orc_site_draws(uint64_t seed, uint32_t chain, uint64_t sweep, int64_t n, int D,
                    double* z, double* u);
/* Accept-test uniforms of sites n0..n0+nn-1 over sweeps sweep0..sweep0+ns-1 (row per site). */
void orc_fill_site_uniforms(uint64_t seed, uint32_t chain, int64_t n0, int64_t nn,
                            uint64_t sweep0, int64_t ns, double* out);
/* Parameter draw: one normal and one uniform. */
void orc_param_draws(uint64_t seed, uint32_t chain, uint64_t sweep, int l, double* z, double* u);

/* ---- model: vector field, RK4 map and their vector-Jacobian products ---- */
int  orc_model_dims(int model, int* D, int* Np);
void orc_model_rhs(int model, const double* x, const double* p, double I, double* F);
void orc_model_map(int model, double dt, const double* x, const double* p, double I, double* fx);
/* w^T df/dx and w^T df/dp accumulated into gx[D], gp[Np] (reverse mode, stages recomputed). */
void orc_model_map_vjp(int model, double dt, const double* x, const double* p, double I,
                       const double* w, double* gx, double* gp);
/* HH rate functions alpha/beta for gate g (0:m 1:h 2:n) at voltage V. */
void orc_hh_rates(double V, double* alpha, double* beta);
/* The paper's gate kinetics (Table 1): a_inf(V) and tau(V) for m, h, n. */
void orc_paper_gates(double V, double* ainf, double* tau);

/* ---- sampler state ---------------------------------------------------- */
orc_state* orc_create(int model, int64_t M, double dt, double Rm, const double* Rf);
void orc_destroy(orc_state* s);
int  orc_set_data(orc_state* s, const double* y, const double* I);
int  orc_set_params(orc_state* s, const double* p, const double* lo, const double* hi,
                    const uint8_t* free_mask);
int  orc_set_path(orc_state* s, const double* X);          /* NULL => default initial path */
int  orc_set_steps(orc_state* s, const double* sig_x, int per_site, const double* sig_p);
int  orc_set_schedule(orc_state* s, int64_t n_init, int64_t n_skip, double beta0,
                      int64_t n_cool, double f_acc, double alpha);
int  orc_set_chain(orc_state* s, uint32_t chain);
int  orc_set_state_box(orc_state* s, const double* lo, const double* hi);
int  orc_set_scheme(orc_state* s, int scheme);
int  orc_set_proposal(orc_state* s, int kind);
/* Single moves with explicit draws (the sweep calls these with Philox draws). */
int  orc_site_update(orc_state* s, int64_t n, const double* z, double u);
int  orc_param_update(orc_state* s, int l, double z, double u);
int  orc_set_sweep_counter(orc_state* s, int64_t sweep, double beta);

int  orc_sweep(orc_state* s, int64_t n_sweeps, uint64_t seed);
/* Full action at beta = 1: A = Ao + Af. */
void orc_action(const orc_state* s, double* A, double* Ao, double* Af);
/* Per-site change of action for proposals Xp (all sites, each against the
 * current path), with the condition scale sum of 1/2 R (d'^2 + d^2). */
void orc_site_delta_all(const orc_state* s, const double* Xp, double beta, double* dA, double* scale);
/* Change of action for moving parameter l to pl_new (full-path reduction). */
double orc_param_delta(const orc_state* s, int l, double pl_new, double beta, double* scale);
/* Gradient of Ao + beta*Af with respect to X (D*(M+1)) and p (Np). */
void orc_grad(const orc_state* s, double beta, double* gX, double* gp);

void orc_get_state(const orc_state* s, double* X, double* p);
void orc_get_cache(const orc_state* s, double* f);
void orc_get_steps(const orc_state* s, double* sig_x, double* sig_p);
int64_t orc_get_sweep(const orc_state* s, double* beta);
/* Decision margins |log u + dA| of the last sweep (sites M+1, params Np; +inf where no test). */
void orc_last_margins(const orc_state* s, double* site_margin, double* param_margin);
void orc_accept_stats(const orc_state* s, uint64_t* site_acc /*2: even, odd*/,
                      uint64_t* site_prop /*2*/, uint64_t* par_acc, uint64_t* par_prop);

/* Running moments of every path component and parameter (Sec. 4.1): returns J. */
int64_t orc_moments(const orc_state* s, double* mean, double* var);
/* Moments of the residuals eps_{n+1,a} ([a*M+n]) and delta_n ([D*M+n-1]) of the recorded paths. */
int64_t orc_residual_moments(const orc_state* s, double* mean, double* var);
/* Ensemble forecast from the current state; out[e][a][k], k = 0..n_steps. */
void orc_forecast(const orc_state* s, int64_t n_steps, const double* I, int n_ens, int noise, uint64_t seed,
                  double* out);
int  orc_set_histograms(orc_state* s, int n_sel, const int64_t* comp, const double* lo,
                        const double* hi, int n_bins);
void orc_histograms(const orc_state* s, uint64_t* counts);

/* Threads of an OpenMP build (liboracle_omp: timing only, its parameter sums
 * add in another order); 1 for the serial test build. */
int  orc_threads(void);

/* Whole-path Hybrid Monte Carlo trajectory (X and free p move together). */
int  orc_hmc(orc_state* s, int64_t n_traj, int n_leap, double eps, const double* inv_mass,
             uint64_t seed, int64_t* n_acc);

#ifdef __cplusplus
}
#endif
#endif
