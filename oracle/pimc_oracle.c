/*
 * Plain serial FP64 CPU oracle for path-integral Monte Carlo data assimilation
 * (Quinn & Abarbanel).  TEST INFRASTRUCTURE ONLY: loaded by the test suite, the
 * smoke check and the benchmark's CPU-baseline leg; never by the CUDA library.
 *
 * Every loop runs in the paper's order and notation, one site at a time, with
 * no blocking, fusion or reordering.  Compile with -ffp-contract=off so that
 * the result is the same on every host architecture.
 *
 * Parity status by function:
 *   orc_philox4x32_10        pinned: Random123 known-answer vectors
 *   orc_model_map (RK4)      pinned: linear model vs the 4th-order Taylor
 *                            polynomial of exp(h K) (RK4 stability polynomial)
 *   orc_model_rhs (HH)       pinned: textbook HH properties (resting potential,
 *                            steady-state gates, repetitive firing at 10 uA/cm^2)
 *   orc_site_delta_all,      pinned: equal to A(X') - A(X) of the full action;
 *   orc_param_delta          the full action pinned by the closed-form
 *                            quadratic form of the linear-Gaussian model
 *   orc_sweep                pinned: closed-form linear-Gaussian posterior,
 *                            brute-force quadrature (M = 2, D = 1), exact
 *                            detailed balance on a lattice
 *   orc_moments, histograms  pinned: numpy mean/var/histogram of recorded samples
 *   orc_grad, map_vjp        pinned: central finite differences of the action
 *   orc_hmc                  pinned: closed-form linear-Gaussian posterior
 *   trapezoid scheme,        pinned: closed-form linear-Gaussian posterior of
 *   uniform proposals        the trapezoid system (T-LG), both proposal laws
 *   orc_paper_gates, the     pinned: a_inf(V_a) = 1/2 and tau(V_a) = tau0 +
 *   paper's HH variant       tau1 for each gate (Table 1), a resting state near
 *                            0 mV, repeated spikes under a 10 uA/cm^2 drive;
 *                            its map VJP by central differences
 *   orc_residual_moments,    pinned: numpy over the recorded residuals;
 *   orc_forecast             deterministic forecast = iterated map, noise law
 *   HH drive hold, initial   parity unpinned against the paper (the paper's own
 *   path, HH constants       example uses tanh rates and a trapezoid rule)
 */
#include "pimc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 4
#define ORC_MAXP 8

/* ======================================================================== */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 5): ten rounds of  */
/* two 32x32->64 multiplies whose high halves are xored with the other words */
/* and the round key; the key is bumped by the Weyl constants between rounds.*/
/* ======================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        uint32_t n3 = lo_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform on the open interval (0, 1): a 52-bit integer k from the top 26 bits
 * of each word, u = (k + 1/2) 2^-52, so 2^-53 <= u <= 1 - 2^-53 exactly. */
double orc_u01(uint32_t hi, uint32_t lo)
{
    uint64_t k = ((uint64_t)(hi >> 6) << 26) | (uint64_t)(lo >> 6);
    return ((double)k + 0.5) * (1.0 / 4503599627370496.0); /* 2^-52 */
}

static void orc_block(uint64_t seed, uint32_t chain, uint64_t sweep, uint32_t idx,
                      uint32_t kind, uint32_t blk, uint32_t w[4])
{
    uint32_t ctr[4] = { idx, (uint32_t)sweep, (kind << 24) | blk, chain };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, w);
}

void orc_fill_site_uniforms(uint64_t seed, uint32_t chain, int64_t n0, int64_t nn,
                            uint64_t sweep0, int64_t ns, double* out)
{
    uint32_t w[4];
    for (int64_t i = 0; i < nn; ++i)
        for (int64_t k = 0; k < ns; ++k) {
            orc_block(seed, chain, sweep0 + (uint64_t)k, (uint32_t)(n0 + i), ORC_KIND_SITE, 2u, w);
            out[i * ns + k] = orc_u01(w[0], w[1]);
        }
}

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

/* Box-Muller on two open uniforms: r cos(2 pi u2), r sin(2 pi u2). */
static void orc_box_muller(double u1, double u2, double* z0, double* z1)
{
    double r = sqrt(-2.0 * log(u1));
    double t = ORC_TWO_PI * u2;
    *z0 = r * cos(t);
    *z1 = r * sin(t);
}

void orc_site_draws(uint64_t seed, uint32_t chain, uint64_t sweep, int64_t n, int D,
                    double* z, double* u)
{
    uint32_t w[4];
    for (int pair = 0; 2 * pair < D; ++pair) {
        double z0, z1;
        orc_block(seed, chain, sweep, (uint32_t)n, ORC_KIND_SITE, (uint32_t)pair, w);
        orc_box_muller(orc_u01(w[0], w[1]), orc_u01(w[2], w[3]), &z0, &z1);
        z[2 * pair] = z0;
        if (2 * pair + 1 < D) z[2 * pair + 1] = z1;
    }
    orc_block(seed, chain, sweep, (uint32_t)n, ORC_KIND_SITE, 2u, w);
    *u = orc_u01(w[0], w[1]);
}

void orc_param_draws(uint64_t seed, uint32_t chain, uint64_t sweep, int l, double* z, double* u)
{
    uint32_t w[4];
    double z1;
    orc_block(seed, chain, sweep, (uint32_t)l, ORC_KIND_PARAM, 0u, w);
    orc_box_muller(orc_u01(w[0], w[1]), orc_u01(w[2], w[3]), z, &z1);
    orc_block(seed, chain, sweep, (uint32_t)l, ORC_KIND_PARAM, 1u, w);
    *u = orc_u01(w[0], w[1]);
}

/* ======================================================================== */
/* Models                                                                    */
/* ======================================================================== */
int orc_model_dims(int model, int* D, int* Np)
{
    switch (model) {
    case ORC_MODEL_HH:       *D = 4; *Np = 7; return 0;
    case ORC_MODEL_LINGAUSS: *D = 2; *Np = 1; return 0;
    case ORC_MODEL_TOY1D:    *D = 1; *Np = 1; return 0;
    case ORC_MODEL_HH_PAPER: *D = 4; *Np = 7; return 0;
    default: return -1;
    }
}

/* psi(u) = u / (1 - e^{-u}), the form of alpha_m and alpha_n; removable
 * singularity at u = 0 replaced by its series 1 + u/2 + u^2/12. */
static double orc_psi(double u)
{
    if (fabs(u) < 1e-6) return 1.0 + u * (0.5 + u / 12.0);
    return -u / expm1(-u);
}

/* d psi / du = (1 - e^{-u} - u e^{-u}) / (1 - e^{-u})^2, series near 0. */
static double orc_dpsi(double u)
{
    if (fabs(u) < 1e-3) return 0.5 + u / 6.0 - u * u * u / 180.0;
    double em = -expm1(-u);          /* 1 - e^{-u} */
    double e = exp(-u);
    return (em - u * e) / (em * em);
}

/* Hodgkin & Huxley (1952) rate functions, modern convention (rest near -65 mV),
 * in 1/ms; V in mV.  Gate order m, h, n. */
void orc_hh_rates(double V, double* alpha, double* beta)
{
    alpha[0] = orc_psi((V + 40.0) / 10.0);                 /* 0.1 (V+40)/(1-exp(-(V+40)/10)) */
    beta[0]  = 4.0 * exp(-(V + 65.0) / 18.0);
    alpha[1] = 0.07 * exp(-(V + 65.0) / 20.0);
    beta[1]  = 1.0 / (1.0 + exp(-(V + 35.0) / 10.0));
    alpha[2] = 0.1 * orc_psi((V + 55.0) / 10.0);           /* 0.01 (V+55)/(1-exp(-(V+55)/10)) */
    beta[2]  = 0.125 * exp(-(V + 65.0) / 80.0);
}

static void orc_hh_rate_derivs(double V, double* dalpha, double* dbeta)
{
    double a[3], b[3];
    orc_hh_rates(V, a, b);
    dalpha[0] = orc_dpsi((V + 40.0) / 10.0) / 10.0;
    dbeta[0]  = -b[0] / 18.0;
    dalpha[1] = -a[1] / 20.0;
    dbeta[1]  = b[1] * (1.0 - b[1]) / 10.0;
    dalpha[2] = 0.1 * orc_dpsi((V + 55.0) / 10.0) / 10.0;
    dbeta[2]  = -b[2] / 80.0;
}

/* The paper's HH form (Sec. 5.1, Eq. (dVdt), Eq. (dadt)): gates relax to
 * a_inf(V) = 1/2 + 1/2 tanh((V - V_a)/dV_a) with time constant
 * tau_a(V) = tau_a0 + tau_a1 (1 - tanh^2((V - V_a)/dV_a)); constants of
 * Table 1, here in the gate order m, h, n. */
static const double ORC_TAB1[3][4] = {
    /* V_a, dV_a, tau_a0, tau_a1 */
    { 25.0, 15.0, 0.1, 0.4 },   /* m, Na activation */
    { 5.0, -15.0, 1.0, 7.0 },   /* h, Na inactivation */
    { 10.0, 30.0, 1.0, 5.0 },   /* n, K activation */
};

void orc_paper_gates(double V, double* ainf, double* tau)
{
    for (int g = 0; g < 3; ++g) {
        double t = tanh((V - ORC_TAB1[g][0]) / ORC_TAB1[g][1]);
        ainf[g] = 0.5 + 0.5 * t;
        tau[g] = ORC_TAB1[g][2] + ORC_TAB1[g][3] * (1.0 - t * t);
    }
}

/* Linear test model: dx/dt = K x + (p0, I), K a damped rotation. */
static const double ORC_LG_K[2][2] = { { -0.5, -2.0 }, { 2.0, -0.5 } };

/* Model vector field F(x; p, I).
 * HH (Sec. 5.1, Eq. (dVdt)/(dadt) structure, conductance form):
 *   C dV/dt = I - gNa m^3 h (V - ENa) - gK n^4 (V - EK) - gL (V - EL)
 *   da/dt   = alpha_a(V) (1 - a) - beta_a(V) a,   a in {m, h, n}
 * p = (gNa, gK, gL, ENa, EK, EL, C). */
void orc_model_rhs(int model, const double* x, const double* p, double I, double* F)
{
    if (model == ORC_MODEL_HH) {
        double V = x[0], m = x[1], h = x[2], n = x[3];
        double a[3], b[3];
        orc_hh_rates(V, a, b);
        double iNa = p[0] * m * m * m * h * (V - p[3]);
        double iK  = p[1] * n * n * n * n * (V - p[4]);
        double iL  = p[2] * (V - p[5]);
        F[0] = (I - iNa - iK - iL) / p[6];
        F[1] = a[0] * (1.0 - m) - b[0] * m;
        F[2] = a[1] * (1.0 - h) - b[1] * h;
        F[3] = a[2] * (1.0 - n) - b[2] * n;
    } else if (model == ORC_MODEL_HH_PAPER) {
        /* dV/dt = p1 I + p2 m^3 h (p3 - V) + p4 n^4 (p5 - V) + p6 (p7 - V) */
        double V = x[0], m = x[1], h = x[2], n = x[3];
        double ainf[3], tau[3];
        orc_paper_gates(V, ainf, tau);
        F[0] = p[0] * I + p[1] * m * m * m * h * (p[2] - V) + p[3] * n * n * n * n * (p[4] - V)
             + p[5] * (p[6] - V);
        for (int g = 0; g < 3; ++g) F[1 + g] = (ainf[g] - x[1 + g]) / tau[g];
    } else if (model == ORC_MODEL_LINGAUSS) {
        F[0] = ORC_LG_K[0][0] * x[0] + ORC_LG_K[0][1] * x[1] + p[0];
        F[1] = ORC_LG_K[1][0] * x[0] + ORC_LG_K[1][1] * x[1] + I;
    } else { /* TOY1D: dx/dt = p0 sin(x) - x/2 + I */
        F[0] = p[0] * sin(x[0]) - 0.5 * x[0] + I;
    }
}

/* Transposed Jacobian products of F: gx += J_x^T w, gp += J_p^T w. */
static void orc_model_rhs_vjp(int model, const double* x, const double* p, double I,
                              const double* w, double* gx, double* gp)
{
    if (model == ORC_MODEL_HH) {
        double V = x[0], m = x[1], h = x[2], n = x[3];
        double gNa = p[0], gK = p[1], gL = p[2], ENa = p[3], EK = p[4], EL = p[5], C = p[6];
        double a[3], b[3], da[3], db[3];
        orc_hh_rates(V, a, b);
        orc_hh_rate_derivs(V, da, db);
        double m3h = m * m * m * h, n4 = n * n * n * n;
        double num = I - gNa * m3h * (V - ENa) - gK * n4 * (V - EK) - gL * (V - EL);
        double wv = w[0] / C;
        /* voltage equation */
        gx[0] += wv * (-gNa * m3h - gK * n4 - gL);
        gx[1] += wv * (-3.0 * gNa * m * m * h * (V - ENa));
        gx[2] += wv * (-gNa * m * m * m * (V - ENa));
        gx[3] += wv * (-4.0 * gK * n * n * n * (V - EK));
        gp[0] += wv * (-m3h * (V - ENa));
        gp[1] += wv * (-n4 * (V - EK));
        gp[2] += wv * (-(V - EL));
        gp[3] += wv * (gNa * m3h);
        gp[4] += wv * (gK * n4);
        gp[5] += wv * gL;
        gp[6] += w[0] * (-num / (C * C));
        /* gate equations */
        for (int g = 0; g < 3; ++g) {
            double s = x[1 + g];
            gx[1 + g] += w[1 + g] * (-(a[g] + b[g]));
            gx[0] += w[1 + g] * (da[g] * (1.0 - s) - db[g] * s);
        }
    } else if (model == ORC_MODEL_HH_PAPER) {
        double V = x[0], m = x[1], h = x[2], n = x[3];
        double m3h = m * m * m * h, n4 = n * n * n * n;
        gx[0] += w[0] * (-p[1] * m3h - p[3] * n4 - p[5]);
        gx[1] += w[0] * (3.0 * p[1] * m * m * h * (p[2] - V));
        gx[2] += w[0] * (p[1] * m * m * m * (p[2] - V));
        gx[3] += w[0] * (4.0 * p[3] * n * n * n * (p[4] - V));
        gp[0] += w[0] * I;
        gp[1] += w[0] * (m3h * (p[2] - V));
        gp[2] += w[0] * (p[1] * m3h);
        gp[3] += w[0] * (n4 * (p[4] - V));
        gp[4] += w[0] * (p[3] * n4);
        gp[5] += w[0] * (p[6] - V);
        gp[6] += w[0] * p[5];
        for (int g = 0; g < 3; ++g) {
            double t = tanh((V - ORC_TAB1[g][0]) / ORC_TAB1[g][1]);
            double sech2 = 1.0 - t * t;
            double ainf = 0.5 + 0.5 * t, tau = ORC_TAB1[g][2] + ORC_TAB1[g][3] * sech2;
            double dainf = 0.5 * sech2 / ORC_TAB1[g][1];
            double dtau = -2.0 * ORC_TAB1[g][3] * t * sech2 / ORC_TAB1[g][1];
            double a = x[1 + g];
            gx[1 + g] += w[1 + g] * (-1.0 / tau);
            gx[0] += w[1 + g] * ((dainf * tau - (ainf - a) * dtau) / (tau * tau));
        }
    } else if (model == ORC_MODEL_LINGAUSS) {
        gx[0] += ORC_LG_K[0][0] * w[0] + ORC_LG_K[1][0] * w[1];
        gx[1] += ORC_LG_K[0][1] * w[0] + ORC_LG_K[1][1] * w[1];
        gp[0] += w[0];
    } else {
        gx[0] += w[0] * (p[0] * cos(x[0]) - 0.5);
        gp[0] += w[0] * sin(x[0]);
    }
}

/* One classical fourth-order Runge-Kutta step of size dt, drive held at I. */
void orc_model_map(int model, double dt, const double* x, const double* p, double I, double* fx)
{
    int D, Np;
    orc_model_dims(model, &D, &Np);
    double k1[ORC_MAXD], k2[ORC_MAXD], k3[ORC_MAXD], k4[ORC_MAXD], xs[ORC_MAXD];
    orc_model_rhs(model, x, p, I, k1);
    for (int a = 0; a < D; ++a) xs[a] = x[a] + 0.5 * dt * k1[a];
    orc_model_rhs(model, xs, p, I, k2);
    for (int a = 0; a < D; ++a) xs[a] = x[a] + 0.5 * dt * k2[a];
    orc_model_rhs(model, xs, p, I, k3);
    for (int a = 0; a < D; ++a) xs[a] = x[a] + dt * k3[a];
    orc_model_rhs(model, xs, p, I, k4);
    for (int a = 0; a < D; ++a)
        fx[a] = x[a] + dt / 6.0 * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
}

/* Reverse mode through the RK4 step, stages recomputed from x (none stored):
 * f = x + dt/6 (k1 + 2 k2 + 2 k3 + k4), k1 = F(x), k2 = F(x + dt/2 k1),
 * k3 = F(x + dt/2 k2), k4 = F(x + dt k3). */
void orc_model_map_vjp(int model, double dt, const double* x, const double* p, double I,
                       const double* w, double* gx, double* gp)
{
    int D, Np;
    orc_model_dims(model, &D, &Np);
    double k1[ORC_MAXD], k2[ORC_MAXD], k3[ORC_MAXD], k4[ORC_MAXD];
    double x2[ORC_MAXD], x3[ORC_MAXD], x4[ORC_MAXD];
    orc_model_rhs(model, x, p, I, k1);
    for (int a = 0; a < D; ++a) x2[a] = x[a] + 0.5 * dt * k1[a];
    orc_model_rhs(model, x2, p, I, k2);
    for (int a = 0; a < D; ++a) x3[a] = x[a] + 0.5 * dt * k2[a];
    orc_model_rhs(model, x3, p, I, k3);
    for (int a = 0; a < D; ++a) x4[a] = x[a] + dt * k3[a];
    (void)k4;

    double bk1[ORC_MAXD], bk2[ORC_MAXD], bk3[ORC_MAXD], bk4[ORC_MAXD], u[ORC_MAXD];
    for (int a = 0; a < D; ++a) {
        gx[a] += w[a];
        bk1[a] = dt / 6.0 * w[a];
        bk2[a] = dt / 3.0 * w[a];
        bk3[a] = dt / 3.0 * w[a];
        bk4[a] = dt / 6.0 * w[a];
    }
    /* stage 4: x4 = x + dt k3 */
    memset(u, 0, sizeof u);
    orc_model_rhs_vjp(model, x4, p, I, bk4, u, gp);
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; bk3[a] += dt * u[a]; }
    /* stage 3: x3 = x + dt/2 k2 */
    memset(u, 0, sizeof u);
    orc_model_rhs_vjp(model, x3, p, I, bk3, u, gp);
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; bk2[a] += 0.5 * dt * u[a]; }
    /* stage 2: x2 = x + dt/2 k1 */
    memset(u, 0, sizeof u);
    orc_model_rhs_vjp(model, x2, p, I, bk2, u, gp);
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; bk1[a] += 0.5 * dt * u[a]; }
    /* stage 1 */
    memset(u, 0, sizeof u);
    orc_model_rhs_vjp(model, x, p, I, bk1, u, gp);
    for (int a = 0; a < D; ++a) gx[a] += u[a];
}

/* ======================================================================== */
/* Sampler state                                                             */
/* ======================================================================== */
struct orc_state {
    int model, D, Np;
    int64_t M;
    double dt, Rm, Rf[ORC_MAXD];
    double *y, *I;             /* y[M+1], I[M] */
    double *X;                 /* D*(M+1) */
    double *f;                 /* D*(M+1) cache g_n: RK4 map f(x_n) (n < M) or field F(x_n) (trapezoid, n <= M) */
    int scheme;                /* ORC_SCHEME_RK4 or ORC_SCHEME_TRAPEZOID */
    int proposal;              /* ORC_PROPOSAL_GAUSS or ORC_PROPOSAL_UNIFORM */
    double p[ORC_MAXP], lo[ORC_MAXP], hi[ORC_MAXP];
    uint8_t free_[ORC_MAXP];
    double xlo[ORC_MAXD], xhi[ORC_MAXD]; /* optional state box (default unbounded) */
    double *sig;               /* D*(M+1) */
    double sigp[ORC_MAXP];
    int64_t n_init, n_skip, n_cool;
    double beta0, fbeta, f_acc, alpha, beta;
    int64_t sweep;
    uint32_t chain;
    int have_data, have_params;
    uint32_t* acc_win;         /* M+1 */
    uint32_t accp_win[ORC_MAXP];
    uint64_t site_acc[2], site_prop[2], par_acc[ORC_MAXP], par_prop[ORC_MAXP];
    double *site_margin, par_margin[ORC_MAXP];
    /* statistics */
    int64_t J;
    double *S1, *S2, *shift;   /* D*(M+1)+Np each */
    double *E1, *E2;           /* residual sums: eps_{n+1,a} at [a*M+n], delta_n at [D*M+n-1] */
    int n_sel, n_bins;
    int64_t* h_comp;
    double *h_lo, *h_hi;
    uint64_t* h_counts;
};

#define XI(s, a, n) ((s)->X[(int64_t)(a) * ((s)->M + 1) + (n)])
#define FI(s, a, n) ((s)->f[(int64_t)(a) * ((s)->M + 1) + (n)])

static void orc_load_site(const orc_state* s, int64_t n, double* x)
{
    for (int a = 0; a < s->D; ++a) x[a] = XI(s, a, n);
}

/* Number of cached sites: f(x_n) for n < M (RK4) or F(x_n) for n <= M (trapezoid). */
static int64_t orc_cache_len(const orc_state* s) { return s->scheme == ORC_SCHEME_RK4 ? s->M : s->M + 1; }

/* Drive at grid point n for the trapezoid rule: the held value of [t_n, t_{n+1}),
 * and at t_M the last one. */
static double orc_drive_at(const orc_state* s, int64_t n) { return n < s->M ? s->I[n] : s->I[s->M - 1]; }

/* Cached value g_n of state x at site n for parameters p. */
static void orc_cache_value(const orc_state* s, const double* x, const double* p, int64_t n, double* g)
{
    if (s->scheme == ORC_SCHEME_RK4) orc_model_map(s->model, s->dt, x, p, s->I[n], g);
    else orc_model_rhs(s->model, x, p, orc_drive_at(s, n), g);
}

/* Model-error residual eps_{n+1} from x_n, x_{n+1} and their cached values:
 * RK4: x_{n+1} - f(x_n); trapezoid (Eq. (modelError)):
 * x_{n+1} - x_n - dt/2 [F(x_{n+1}) + F(x_n)]. */
static double orc_eps(const orc_state* s, double xn, double xn1, double gn, double gn1)
{
    if (s->scheme == ORC_SCHEME_RK4) return xn1 - gn;
    return xn1 - xn - 0.5 * s->dt * (gn1 + gn);
}

static void orc_refresh_cache(orc_state* s)
{
    double x[ORC_MAXD], g[ORC_MAXD];
    for (int64_t n = 0; n < orc_cache_len(s); ++n) {
        orc_load_site(s, n, x);
        orc_cache_value(s, x, s->p, n, g);
        for (int a = 0; a < s->D; ++a) FI(s, a, n) = g[a];
    }
}

int orc_set_scheme(orc_state* s, int scheme)
{
    if (scheme != ORC_SCHEME_RK4 && scheme != ORC_SCHEME_TRAPEZOID) return -1;
    s->scheme = scheme;
    if (s->have_data && s->have_params) orc_refresh_cache(s);
    return 0;
}

int orc_set_proposal(orc_state* s, int kind)
{
    if (kind != ORC_PROPOSAL_GAUSS && kind != ORC_PROPOSAL_UNIFORM) return -1;
    s->proposal = kind;
    return 0;
}

orc_state* orc_create(int model, int64_t M, double dt, double Rm, const double* Rf)
{
    int D, Np;
    if (orc_model_dims(model, &D, &Np) != 0 || M < 1 || !(dt > 0.0) || !(Rm > 0.0)) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->model = model; s->D = D; s->Np = Np; s->M = M; s->dt = dt; s->Rm = Rm;
    for (int a = 0; a < D; ++a) s->Rf[a] = Rf[a];
    int64_t nc = (int64_t)D * (M + 1);
    s->y = (double*)calloc((size_t)(M + 1), sizeof(double));
    s->I = (double*)calloc((size_t)M, sizeof(double));
    s->X = (double*)calloc((size_t)nc, sizeof(double));
    s->f = (double*)calloc((size_t)nc, sizeof(double));
    s->sig = (double*)calloc((size_t)nc, sizeof(double));
    s->acc_win = (uint32_t*)calloc((size_t)(M + 1), sizeof(uint32_t));
    s->site_margin = (double*)calloc((size_t)(M + 1), sizeof(double));
    s->S1 = (double*)calloc((size_t)(nc + Np), sizeof(double));
    s->S2 = (double*)calloc((size_t)(nc + Np), sizeof(double));
    s->shift = (double*)calloc((size_t)(nc + Np), sizeof(double));
    s->E1 = (double*)calloc((size_t)((D + 1) * M), sizeof(double));
    s->E2 = (double*)calloc((size_t)((D + 1) * M), sizeof(double));
    s->n_skip = 1; s->n_init = 0; s->n_cool = 0;
    s->beta0 = 1.0; s->fbeta = 1.0; s->beta = 1.0; s->f_acc = 0.4; s->alpha = 0.0;
    for (int l = 0; l < ORC_MAXP; ++l) { s->lo[l] = -INFINITY; s->hi[l] = INFINITY; }
    for (int a = 0; a < ORC_MAXD; ++a) { s->xlo[a] = -INFINITY; s->xhi[a] = INFINITY; }
    return s;
}

void orc_destroy(orc_state* s)
{
    if (!s) return;
    free(s->y); free(s->I); free(s->X); free(s->f); free(s->sig); free(s->acc_win);
    free(s->site_margin); free(s->S1); free(s->S2); free(s->shift); free(s->E1); free(s->E2);
    free(s->h_comp); free(s->h_lo); free(s->h_hi); free(s->h_counts);
    free(s);
}

/* Default initial path: V (component 0) from the observations, the other
 * components at their steady state for that V (HH gates a_inf = alpha/(alpha+beta);
 * zero for the test models). */
static void orc_default_path(orc_state* s)
{
    for (int64_t n = 0; n <= s->M; ++n) {
        XI(s, 0, n) = s->y[n];
        if (s->model == ORC_MODEL_HH) {
            double a[3], b[3];
            orc_hh_rates(s->y[n], a, b);
            for (int g = 0; g < 3; ++g) XI(s, 1 + g, n) = a[g] / (a[g] + b[g]);
        } else if (s->model == ORC_MODEL_HH_PAPER) {
            double ainf[3], tau[3];
            orc_paper_gates(s->y[n], ainf, tau);
            for (int g = 0; g < 3; ++g) XI(s, 1 + g, n) = ainf[g];
        } else {
            for (int a = 1; a < s->D; ++a) XI(s, a, n) = 0.0;
        }
    }
}

int orc_set_data(orc_state* s, const double* y, const double* I)
{
    memcpy(s->y, y, sizeof(double) * (size_t)(s->M + 1));
    memcpy(s->I, I, sizeof(double) * (size_t)s->M);
    s->have_data = 1;
    orc_default_path(s);
    if (s->have_params) orc_refresh_cache(s);
    return 0;
}

int orc_set_params(orc_state* s, const double* p, const double* lo, const double* hi,
                   const uint8_t* free_mask)
{
    for (int l = 0; l < s->Np; ++l) {
        s->p[l] = p[l];
        s->lo[l] = lo ? lo[l] : -INFINITY;
        s->hi[l] = hi ? hi[l] : INFINITY;
        s->free_[l] = free_mask ? free_mask[l] : 0;
    }
    s->have_params = 1;
    if (s->have_data) orc_refresh_cache(s);
    return 0;
}

int orc_set_path(orc_state* s, const double* X)
{
    if (X) memcpy(s->X, X, sizeof(double) * (size_t)(s->D * (s->M + 1)));
    else orc_default_path(s);
    if (s->have_params) orc_refresh_cache(s);
    return 0;
}

int orc_set_steps(orc_state* s, const double* sig_x, int per_site, const double* sig_p)
{
    for (int a = 0; a < s->D; ++a)
        for (int64_t n = 0; n <= s->M; ++n)
            s->sig[(int64_t)a * (s->M + 1) + n] = per_site ? sig_x[(int64_t)a * (s->M + 1) + n] : sig_x[a];
    for (int l = 0; l < s->Np; ++l) s->sigp[l] = sig_p ? sig_p[l] : 0.0;
    return 0;
}

/* Annealing factor f_beta = (1/beta0)^(1/N_cool), Eq. (fbeta). */
int orc_set_schedule(orc_state* s, int64_t n_init, int64_t n_skip, double beta0,
                     int64_t n_cool, double f_acc, double alpha)
{
    if (n_skip < 1 || n_init < 0 || n_cool < 0 || !(beta0 > 0.0) || beta0 > 1.0) return -1;
    s->n_init = n_init; s->n_skip = n_skip; s->n_cool = n_cool;
    s->beta0 = beta0; s->f_acc = f_acc; s->alpha = alpha;
    s->fbeta = n_cool > 0 ? pow(1.0 / beta0, 1.0 / (double)n_cool) : 1.0;
    s->beta = (n_cool > 0 && s->sweep < n_cool) ? beta0 : 1.0;
    return 0;
}

int orc_set_chain(orc_state* s, uint32_t chain) { s->chain = chain; return 0; }

/* Uniform prior box on every state component (Sec. 2.1 "uniform inside the
 * boundaries"); a proposal outside it is rejected like an out-of-box parameter. */
int orc_set_state_box(orc_state* s, const double* lo, const double* hi)
{
    for (int a = 0; a < s->D; ++a) { s->xlo[a] = lo[a]; s->xhi[a] = hi[a]; }
    return 0;
}

int orc_set_sweep_counter(orc_state* s, int64_t sweep, double beta)
{
    s->sweep = sweep; s->beta = beta; return 0;
}

/* Threads an OpenMP build uses (1 for the serial build). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- action ------------------------------------------------------------ */
/* A_o = 1/2 sum_{n=1}^M Rm (x_{n,0} - y_n)^2;  A_f = 1/2 sum_{n=0}^{M-1} sum_a Rf_a eps_{n+1,a}^2
 * (Sec. 2.1), eps from the explicit RK4 map or the trapezoid rule. */
void orc_action(const orc_state* s, double* A, double* Ao, double* Af)
{
    double ao = 0.0, af = 0.0, x[ORC_MAXD], x1[ORC_MAXD], g[ORC_MAXD], g1[ORC_MAXD];
    for (int64_t n = 1; n <= s->M; ++n) {
        double d = XI(s, 0, n) - s->y[n];
        ao += 0.5 * s->Rm * d * d;
    }
    for (int64_t n = 0; n < s->M; ++n) {
        orc_load_site(s, n, x);
        orc_load_site(s, n + 1, x1);
        orc_cache_value(s, x, s->p, n, g);
        if (s->scheme == ORC_SCHEME_TRAPEZOID) orc_cache_value(s, x1, s->p, n + 1, g1);
        for (int a = 0; a < s->D; ++a) {
            double e = orc_eps(s, x[a], x1[a], g[a], g1[a]);
            af += 0.5 * s->Rf[a] * e * e;
        }
    }
    *Ao = ao; *Af = af; *A = ao + af;
}

/* Contribution 1/2 R (d'^2 - d^2) written as 1/2 R (d' - d)(d' + d). */
static double orc_sqdiff(double R, double dp, double d, double* scale)
{
    *scale += 0.5 * R * (dp * dp + d * d);
    return 0.5 * R * (dp - d) * (dp + d);
}

/* Local change of action for replacing x_n by xp with cached value gp
 * (Fig. 1 steps (c)-(g)): measurement term at n (n >= 1), model-error terms
 * eps_n (n >= 1) and eps_{n+1} (n <= M-1) against the cached neighbours. */
static double orc_site_delta(const orc_state* s, int64_t n, const double* xp, const double* gp,
                             double beta, double* scale)
{
    double dA = 0.0, sc = 0.0;
    if (n >= 1) {
        double d = XI(s, 0, n) - s->y[n], dp = xp[0] - s->y[n];
        dA += orc_sqdiff(s->Rm, dp, d, &sc);
        double dAf = 0.0;
        for (int a = 0; a < s->D; ++a) {
            double gn = s->scheme == ORC_SCHEME_RK4 ? 0.0 : FI(s, a, n);
            double e = orc_eps(s, XI(s, a, n - 1), XI(s, a, n), FI(s, a, n - 1), gn);
            double ep = orc_eps(s, XI(s, a, n - 1), xp[a], FI(s, a, n - 1), s->scheme == ORC_SCHEME_RK4 ? 0.0 : gp[a]);
            double t = 0.0;
            dAf += orc_sqdiff(s->Rf[a], ep, e, &t);
            sc += beta * t;
        }
        dA += beta * dAf;
    }
    if (n <= s->M - 1) {
        double dAf = 0.0;
        for (int a = 0; a < s->D; ++a) {
            double g1 = s->scheme == ORC_SCHEME_RK4 ? 0.0 : FI(s, a, n + 1);
            double e = orc_eps(s, XI(s, a, n), XI(s, a, n + 1), FI(s, a, n), g1);
            double ep = orc_eps(s, xp[a], XI(s, a, n + 1), gp[a], g1);
            double t = 0.0;
            dAf += orc_sqdiff(s->Rf[a], ep, e, &t);
            sc += beta * t;
        }
        dA += beta * dAf;
    }
    if (scale) *scale = sc;
    return dA;
}

void orc_site_delta_all(const orc_state* s, const double* Xp, double beta, double* dA, double* scale)
{
    double xp[ORC_MAXD], gp[ORC_MAXD] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t n = 0; n <= s->M; ++n) {
        for (int a = 0; a < s->D; ++a) xp[a] = Xp[(int64_t)a * (s->M + 1) + n];
        if (n < orc_cache_len(s)) orc_cache_value(s, xp, s->p, n, gp);
        dA[n] = orc_site_delta(s, n, xp, gp, beta, scale ? &scale[n] : NULL);
    }
}

/* Parameter move: the change of the model-error sum over the whole path when
 * p -> pn (Sec. 4.1, "Perturb parameter p_l" of Fig. 1): new cached values
 * for every site, then the sum over n = 0..M-1 of the residual changes. */
static double orc_param_delta_cache(const orc_state* s, const double* pn, double beta,
                                    double* gnew, double* scale)
{
    int64_t nc = orc_cache_len(s);
    double* g = gnew ? gnew : (double*)malloc(sizeof(double) * (size_t)(s->D * (s->M + 1)));
    double dA = 0.0, sc = 0.0;
    /* (the OpenMP build, timing only, splits both loops over threads; its sum
     * order then differs from this serial order) */
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < nc; ++n) {
        double x[ORC_MAXD], gv[ORC_MAXD];
        orc_load_site(s, n, x);
        orc_cache_value(s, x, pn, n, gv);
        for (int a = 0; a < s->D; ++a) g[(int64_t)a * (s->M + 1) + n] = gv[a];
    }
#pragma omp parallel for schedule(static) reduction(+ : dA, sc)
    for (int64_t n = 0; n < s->M; ++n) {
        for (int a = 0; a < s->D; ++a) {
            double g1o = s->scheme == ORC_SCHEME_RK4 ? 0.0 : FI(s, a, n + 1);
            double g1n = s->scheme == ORC_SCHEME_RK4 ? 0.0 : g[(int64_t)a * (s->M + 1) + n + 1];
            double e = orc_eps(s, XI(s, a, n), XI(s, a, n + 1), FI(s, a, n), g1o);
            double ep = orc_eps(s, XI(s, a, n), XI(s, a, n + 1), g[(int64_t)a * (s->M + 1) + n], g1n);
            double t = 0.0;
            dA += beta * orc_sqdiff(s->Rf[a], ep, e, &t);
            sc += beta * t;
        }
    }
    if (!gnew) free(g);
    if (scale) *scale = sc;
    return dA;
}

double orc_param_delta(const orc_state* s, int l, double pl_new, double beta, double* scale)
{
    double pn[ORC_MAXP];
    memcpy(pn, s->p, sizeof pn);
    pn[l] = pl_new;
    return orc_param_delta_cache(s, pn, beta, NULL, scale);
}

/* Metropolis rule, Eq. (Paccept): accept iff dA <= 0 or u < exp(-dA); a
 * non-finite dA is a rejection. */
static int orc_accept(double dA, double u, double* margin)
{
    if (!isfinite(dA)) { *margin = INFINITY; return 0; }
    *margin = fabs(log(u) + dA);
    if (dA <= 0.0) return 1;
    return u < exp(-dA);
}

/* ---- statistics -------------------------------------------------------- */
static double orc_component(const orc_state* s, int64_t c)
{
    int64_t nx = (int64_t)s->D * (s->M + 1);
    return c < nx ? s->X[c] : s->p[c - nx];
}

/* Running shifted sums (Sec. 4.1): S1 += x - r, S2 += (x - r)^2 with r the
 * first recorded value; bin counts for the selected components. */
static void orc_record(orc_state* s)
{
    int64_t nc = (int64_t)s->D * (s->M + 1) + s->Np;
    for (int64_t c = 0; c < nc; ++c) {
        double v = orc_component(s, c);
        if (s->J == 0) s->shift[c] = v;
        double d = v - s->shift[c];
        s->S1[c] += d;
        s->S2[c] += d * d;
    }
    s->J += 1;
    /* residuals of the recorded path (Sec. 6: their means should vanish and
     * their variances match the assumed noise): eps_{n+1} = x_{n+1} - f(x_n),
     * delta_n = x_{n,0} - y_n */
    for (int64_t n = 0; n < s->M; ++n)
        for (int a = 0; a < s->D; ++a) {
            double e = orc_eps(s, XI(s, a, n), XI(s, a, n + 1), FI(s, a, n),
                               s->scheme == ORC_SCHEME_RK4 ? 0.0 : FI(s, a, n + 1));
            s->E1[(int64_t)a * s->M + n] += e;
            s->E2[(int64_t)a * s->M + n] += e * e;
        }
    for (int64_t n = 1; n <= s->M; ++n) {
        double d = XI(s, 0, n) - s->y[n];
        s->E1[(int64_t)s->D * s->M + n - 1] += d;
        s->E2[(int64_t)s->D * s->M + n - 1] += d * d;
    }
    for (int k = 0; k < s->n_sel; ++k) {
        double v = orc_component(s, s->h_comp[k]);
        int64_t slot;
        if (!(v >= s->h_lo[k])) slot = 0;
        else if (v >= s->h_hi[k]) slot = s->n_bins + 1;
        else {
            double t = (v - s->h_lo[k]) / (s->h_hi[k] - s->h_lo[k]);
            int64_t b = (int64_t)floor(t * (double)s->n_bins);
            if (b > s->n_bins - 1) b = s->n_bins - 1;
            slot = 1 + b;
        }
        s->h_counts[(int64_t)k * (s->n_bins + 2) + slot] += 1;
    }
}

int64_t orc_moments(const orc_state* s, double* mean, double* var)
{
    int64_t nc = (int64_t)s->D * (s->M + 1) + s->Np;
    double J = (double)s->J;
    for (int64_t c = 0; c < nc; ++c) {
        mean[c] = s->J > 0 ? s->shift[c] + s->S1[c] / J : NAN;
        var[c] = s->J > 1 ? (s->S2[c] - s->S1[c] * s->S1[c] / J) / (J - 1.0) : NAN;
    }
    return s->J;
}

int64_t orc_residual_moments(const orc_state* s, double* mean, double* var)
{
    int64_t nr = (int64_t)(s->D + 1) * s->M;
    double J = (double)s->J;
    for (int64_t i = 0; i < nr; ++i) {
        mean[i] = s->J > 0 ? s->E1[i] / J : NAN;
        var[i] = s->J > 1 ? (s->E2[i] - s->E1[i] * s->E1[i] / J) / (J - 1.0) : NAN;
    }
    return s->J;
}

/* Ensemble forecast from the current state (Sec. 6): member e integrates
 * x_{k+1} = f(x_k, p; I_k) + xi_k with xi_{k,a} ~ N(0, 1/Rf_a) (none where
 * Rf_a = 0, or for every member when noise == 0), starting at x_M; normals are
 * Philox draws keyed by (member, step, kind 4 | pair, chain).
 * out[e][a][k], k = 0..n_steps. */
void orc_forecast(const orc_state* s, int64_t n_steps, const double* I, int n_ens, int noise, uint64_t seed,
                  double* out)
{
    double x[ORC_MAXD], fx[ORC_MAXD];
    for (int e = 0; e < n_ens; ++e) {
        double* o = out + (int64_t)e * s->D * (n_steps + 1);
        for (int a = 0; a < s->D; ++a) { x[a] = XI(s, a, s->M); o[(int64_t)a * (n_steps + 1)] = x[a]; }
        for (int64_t k = 0; k < n_steps; ++k) {
            orc_model_map(s->model, s->dt, x, s->p, I[k], fx);
            for (int pair = 0; 2 * pair < s->D; ++pair) {
                uint32_t w[4];
                double z0 = 0.0, z1 = 0.0;
                if (noise) {
                    orc_block(seed, s->chain, (uint64_t)k, (uint32_t)e, ORC_KIND_FORECAST, (uint32_t)pair, w);
                    orc_box_muller(orc_u01(w[0], w[1]), orc_u01(w[2], w[3]), &z0, &z1);
                }
                for (int q = 0; q < 2 && 2 * pair + q < s->D; ++q) {
                    int a = 2 * pair + q;
                    double z = q == 0 ? z0 : z1;
                    fx[a] += (noise && s->Rf[a] > 0.0) ? z / sqrt(s->Rf[a]) : 0.0;
                }
            }
            for (int a = 0; a < s->D; ++a) { x[a] = fx[a]; o[(int64_t)a * (n_steps + 1) + k + 1] = x[a]; }
        }
    }
}

int orc_set_histograms(orc_state* s, int n_sel, const int64_t* comp, const double* lo,
                       const double* hi, int n_bins)
{
    free(s->h_comp); free(s->h_lo); free(s->h_hi); free(s->h_counts);
    s->n_sel = n_sel; s->n_bins = n_bins;
    s->h_comp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_sel > 0 ? n_sel : 1));
    s->h_lo = (double*)malloc(sizeof(double) * (size_t)(n_sel > 0 ? n_sel : 1));
    s->h_hi = (double*)malloc(sizeof(double) * (size_t)(n_sel > 0 ? n_sel : 1));
    s->h_counts = (uint64_t*)calloc((size_t)(n_sel > 0 ? n_sel : 1) * (size_t)(n_bins + 2), sizeof(uint64_t));
    for (int k = 0; k < n_sel; ++k) { s->h_comp[k] = comp[k]; s->h_lo[k] = lo[k]; s->h_hi[k] = hi[k]; }
    return 0;
}

void orc_histograms(const orc_state* s, uint64_t* counts)
{
    memcpy(counts, s->h_counts, sizeof(uint64_t) * (size_t)s->n_sel * (size_t)(s->n_bins + 2));
}

/* ---- one checkerboard sweep (Fig. 1; even sites first, Sec. 4.1) ------- */
/* One site move of Fig. 1 with given draws: x' = x_n + sigma_n . z, then
 * f(x'), the local change of action, the Metropolis decision and, on accept,
 * the store of x_n and its cached f_n. Returns 1 on accept. */
int orc_site_update(orc_state* s, int64_t n, const double* z, double u)
{
    double x[ORC_MAXD], xp[ORC_MAXD], fp[ORC_MAXD] = {0.0, 0.0, 0.0, 0.0}, margin;
    int parity = (int)(n & 1);
    orc_load_site(s, n, x);
    int inside = 1;
    for (int a = 0; a < s->D; ++a) {
        xp[a] = x[a] + s->sig[(int64_t)a * (s->M + 1) + n] * z[a];
        if (!(xp[a] >= s->xlo[a] && xp[a] <= s->xhi[a])) inside = 0;
    }
#pragma omp atomic
    s->site_prop[parity] += 1;
    s->site_margin[n] = INFINITY;
    if (!inside) return 0;
    const int cached = n < orc_cache_len(s);
    if (cached) orc_cache_value(s, xp, s->p, n, fp);
    double dA = orc_site_delta(s, n, xp, fp, s->beta, NULL);
    int acc = orc_accept(dA, u, &margin);
    s->site_margin[n] = margin;
    if (acc) {
        for (int a = 0; a < s->D; ++a) XI(s, a, n) = xp[a];
        if (cached) for (int a = 0; a < s->D; ++a) FI(s, a, n) = fp[a];
        s->acc_win[n] += 1;
#pragma omp atomic
        s->site_acc[parity] += 1;
    }
    return acc;
}

/* Uniform proposal increments of Fig. 1, U(-1, 1) per component, from the same
 * Philox words as the Gaussian ones: 2 u - 1 with u the open uniform of each
 * word pair. */
static void orc_site_uniform_draws(uint64_t seed, uint32_t chain, uint64_t sweep, int64_t n, int D, double* z,
                                   double* u)
{
    uint32_t w[4];
    for (int pair = 0; 2 * pair < D; ++pair) {
        orc_block(seed, chain, sweep, (uint32_t)n, ORC_KIND_SITE, (uint32_t)pair, w);
        z[2 * pair] = 2.0 * orc_u01(w[0], w[1]) - 1.0;
        if (2 * pair + 1 < D) z[2 * pair + 1] = 2.0 * orc_u01(w[2], w[3]) - 1.0;
    }
    orc_block(seed, chain, sweep, (uint32_t)n, ORC_KIND_SITE, 2u, w);
    *u = orc_u01(w[0], w[1]);
}

/* The sites of one parity are independent given the other parity, so the
 * OpenMP build (timing only; the test build is serial) may move them in
 * parallel. */
static void orc_site_phase(orc_state* s, int parity, uint64_t seed)
{
#pragma omp parallel for schedule(static)
    for (int64_t n = parity; n <= s->M; n += 2) {
        double z[ORC_MAXD], u;
        if (s->proposal == ORC_PROPOSAL_UNIFORM) orc_site_uniform_draws(seed, s->chain, (uint64_t)s->sweep, n, s->D, z, &u);
        else orc_site_draws(seed, s->chain, (uint64_t)s->sweep, n, s->D, z, &u);
        orc_site_update(s, n, z, u);
    }
}

/* Sequential parameter moves l = 1..N_p (Sec. 4.1): one full-path change of
 * action, one decision; an out-of-box proposal is rejected without compute
 * (uniform prior inside the bounds, Sec. 4.2). */
/* One parameter move with given draws: p'_l = p_l + sigma_l z; returns 1 on accept. */
int orc_param_update(orc_state* s, int l, double z, double u)
{
    double margin;
    s->par_margin[l] = INFINITY;
    if (!s->free_[l]) return 0;
    double pl = s->p[l] + s->sigp[l] * z;
    s->par_prop[l] += 1;
    if (!(pl >= s->lo[l] && pl <= s->hi[l])) return 0;
    double pn[ORC_MAXP];
    memcpy(pn, s->p, sizeof pn);
    pn[l] = pl;
    double* fnew = (double*)calloc((size_t)(s->D * (s->M + 1)), sizeof(double));
    double dA = orc_param_delta_cache(s, pn, s->beta, fnew, NULL);
    int acc = orc_accept(dA, u, &margin);
    s->par_margin[l] = margin;
    if (acc) {
        s->p[l] = pl;
        memcpy(s->f, fnew, sizeof(double) * (size_t)(s->D * (s->M + 1)));
        s->accp_win[l] += 1;
        s->par_acc[l] += 1;
    }
    free(fnew);
    return acc;
}

static void orc_param_phase(orc_state* s, uint64_t seed)
{
    for (int l = 0; l < s->Np; ++l) {
        double z, u;
        s->par_margin[l] = INFINITY;
        if (!s->free_[l]) continue;
        orc_param_draws(seed, s->chain, (uint64_t)s->sweep, l, &z, &u);
        if (s->proposal == ORC_PROPOSAL_UNIFORM) {
            uint32_t w[4];
            orc_block(seed, s->chain, (uint64_t)s->sweep, (uint32_t)l, ORC_KIND_PARAM, 0u, w);
            z = 2.0 * orc_u01(w[0], w[1]) - 1.0;
        }
        orc_param_update(s, l, z, u);
    }
}

/* Step-size rule of Sec. 4.2, every N_skip sweeps during the first N_init:
 * Delta_i <- Delta_i [1 + alpha (N_acc,i / N_skip - f_acc)].  A site's joint
 * D-vector move shares one acceptance count, so all its components scale together. */
static void orc_adapt(orc_state* s)
{
    for (int64_t n = 0; n <= s->M; ++n) {
        double fac = 1.0 + s->alpha * ((double)s->acc_win[n] / (double)s->n_skip - s->f_acc);
        for (int a = 0; a < s->D; ++a) s->sig[(int64_t)a * (s->M + 1) + n] *= fac;
        s->acc_win[n] = 0;
    }
    for (int l = 0; l < s->Np; ++l) {
        if (s->free_[l]) {
            double fac = 1.0 + s->alpha * ((double)s->accp_win[l] / (double)s->n_skip - s->f_acc);
            s->sigp[l] *= fac;
        }
        s->accp_win[l] = 0;
    }
}

int orc_sweep(orc_state* s, int64_t n_sweeps, uint64_t seed)
{
    if (!s->have_data || !s->have_params) return -2;
    for (int64_t k = 0; k < n_sweeps; ++k) {
        orc_site_phase(s, 0, seed);
        orc_site_phase(s, 1, seed);
        orc_param_phase(s, seed);
        int64_t sw = s->sweep;
        if (sw >= s->n_init && (sw - s->n_init) % s->n_skip == 0) orc_record(s);
        if (sw < s->n_init && (sw + 1) % s->n_skip == 0) orc_adapt(s);
        /* beta_{s+1} = beta_s f_beta during the first N_cool sweeps, then 1 (Sec. 4.2) */
        s->beta = (sw + 1 < s->n_cool) ? s->beta * s->fbeta : 1.0;
        s->sweep = sw + 1;
    }
    return 0;
}

/* ---- gradient of the action ---------------------------------------------- */
/* dA/dx_n = Rm (x_{n,0} - y_n) e_0 [n>=1] + beta Rf . eps_n [n>=1]
 *         - beta J_x f(x_n)^T (Rf . eps_{n+1}) [n<=M-1]
 * dA/dp   = -beta sum_n J_p f(x_n)^T (Rf . eps_{n+1}). */
void orc_grad(const orc_state* s, double beta, double* gX, double* gp)
{
    int D = s->D;
    double x[ORC_MAXD], fx[ORC_MAXD], w[ORC_MAXD], gx[ORC_MAXD], gpl[ORC_MAXP];
    memset(gX, 0, sizeof(double) * (size_t)(D * (s->M + 1)));
    for (int l = 0; l < s->Np; ++l) gp[l] = 0.0;
    for (int64_t n = 1; n <= s->M; ++n)
        gX[n] += s->Rm * (XI(s, 0, n) - s->y[n]);
    if (s->scheme == ORC_SCHEME_TRAPEZOID) {
        /* eps_{n+1} = x_{n+1} - x_n - dt/2 [F(x_{n+1}) + F(x_n)], w = beta Rf . eps_{n+1}:
         * dA/dx_{n+1} += w - dt/2 J(x_{n+1})^T w, dA/dx_n += -w - dt/2 J(x_n)^T w,
         * dA/dp -= dt/2 [J_p(x_{n+1}) + J_p(x_n)]^T w */
        double x1[ORC_MAXD], F0[ORC_MAXD], F1[ORC_MAXD], g0[ORC_MAXD], g1[ORC_MAXD];
        for (int64_t n = 0; n < s->M; ++n) {
            orc_load_site(s, n, x);
            orc_load_site(s, n + 1, x1);
            orc_model_rhs(s->model, x, s->p, orc_drive_at(s, n), F0);
            orc_model_rhs(s->model, x1, s->p, orc_drive_at(s, n + 1), F1);
            for (int a = 0; a < D; ++a) {
                double e = x1[a] - x[a] - 0.5 * s->dt * (F1[a] + F0[a]);
                w[a] = beta * s->Rf[a] * e;
                g0[a] = 0.0;
                g1[a] = 0.0;
            }
            for (int l = 0; l < s->Np; ++l) gpl[l] = 0.0;
            orc_model_rhs_vjp(s->model, x, s->p, orc_drive_at(s, n), w, g0, gpl);
            orc_model_rhs_vjp(s->model, x1, s->p, orc_drive_at(s, n + 1), w, g1, gpl);
            for (int a = 0; a < D; ++a) {
                gX[(int64_t)a * (s->M + 1) + n + 1] += w[a] - 0.5 * s->dt * g1[a];
                gX[(int64_t)a * (s->M + 1) + n] += -w[a] - 0.5 * s->dt * g0[a];
            }
            for (int l = 0; l < s->Np; ++l) gp[l] -= 0.5 * s->dt * gpl[l];
        }
        return;
    }
    for (int64_t n = 0; n < s->M; ++n) {
        orc_load_site(s, n, x);
        orc_model_map(s->model, s->dt, x, s->p, s->I[n], fx);
        for (int a = 0; a < D; ++a) {
            double e = XI(s, a, n + 1) - fx[a];
            w[a] = beta * s->Rf[a] * e;
            gX[(int64_t)a * (s->M + 1) + n + 1] += w[a];
            gx[a] = 0.0;
        }
        for (int l = 0; l < s->Np; ++l) gpl[l] = 0.0;
        orc_model_map_vjp(s->model, s->dt, x, s->p, s->I[n], w, gx, gpl);
        for (int a = 0; a < D; ++a) gX[(int64_t)a * (s->M + 1) + n] -= gx[a];
        for (int l = 0; l < s->Np; ++l) gp[l] -= gpl[l];
    }
}

/* ---- Hybrid Monte Carlo over (X, free p) ---------------------------------- */
/* Leapfrog with diagonal inverse mass; a trajectory that leaves the parameter
 * box at any step is rejected (the potential is infinite outside).  Momenta are
 * Philox normals keyed by (component pair, trajectory, kind HMC_MOM, chain). */
int orc_hmc(orc_state* s, int64_t n_traj, int n_leap, double eps, const double* inv_mass,
            uint64_t seed, int64_t* n_acc)
{
    if (!s->have_data || !s->have_params) return -2;
    int64_t nx = (int64_t)s->D * (s->M + 1), nq = nx + s->Np;
    double* q0 = (double*)malloc(sizeof(double) * (size_t)nq);
    double* mom = (double*)malloc(sizeof(double) * (size_t)nq);
    double* g = (double*)malloc(sizeof(double) * (size_t)nq);
    double A0, A1, tmp1, tmp2;
    int64_t acc_count = 0;
    for (int64_t t = 0; t < n_traj; ++t) {
        uint64_t traj = (uint64_t)s->sweep;
        /* step jittered uniformly in [0.8, 1.2] eps per trajectory, drawn
         * independently of the state, so a fixed trajectory length cannot
         * resonate with a mode of the target (Neal 2011, Sec. 5.4.2.2) */
        uint32_t wj[4];
        orc_block(seed, s->chain, traj, 0u, ORC_KIND_HMC_ACC, 0u, wj);
        double eps_t = eps * (0.8 + 0.4 * orc_u01(wj[2], wj[3]));
        /* momenta */
        for (int64_t j = 0; j < nq; j += 2) {
            uint32_t w[4];
            double z0, z1;
            orc_block(seed, s->chain, traj, (uint32_t)(j >> 1), ORC_KIND_HMC_MOM, 0u, w);
            orc_box_muller(orc_u01(w[0], w[1]), orc_u01(w[2], w[3]), &z0, &z1);
            mom[j] = z0 / sqrt(inv_mass[j]);
            if (j + 1 < nq) mom[j + 1] = z1 / sqrt(inv_mass[j + 1]);
        }
        for (int l = 0; l < s->Np; ++l) if (!s->free_[l]) mom[nx + l] = 0.0;
        memcpy(q0, s->X, sizeof(double) * (size_t)nx);
        memcpy(q0 + nx, s->p, sizeof(double) * (size_t)s->Np);
        orc_action(s, &A0, &tmp1, &tmp2);
        double K0 = 0.0;
        for (int64_t j = 0; j < nq; ++j) K0 += 0.5 * mom[j] * mom[j] * inv_mass[j];
        int out_of_box = 0;
        orc_grad(s, 1.0, g, g + nx);
        for (int l = 0; l < s->Np; ++l) if (!s->free_[l]) g[nx + l] = 0.0;
        for (int64_t j = 0; j < nq; ++j) mom[j] -= 0.5 * eps_t * g[j];
        for (int i = 1; i <= n_leap; ++i) {
            for (int64_t j = 0; j < nx; ++j) s->X[j] += eps_t * inv_mass[j] * mom[j];
            for (int l = 0; l < s->Np; ++l) {
                if (!s->free_[l]) continue;
                s->p[l] += eps_t * inv_mass[nx + l] * mom[nx + l];
                if (!(s->p[l] >= s->lo[l] && s->p[l] <= s->hi[l])) out_of_box = 1;
            }
            if (out_of_box) break;
            orc_grad(s, 1.0, g, g + nx);
            for (int l = 0; l < s->Np; ++l) if (!s->free_[l]) g[nx + l] = 0.0;
            double c = (i < n_leap) ? eps_t : 0.5 * eps_t;
            for (int64_t j = 0; j < nq; ++j) mom[j] -= c * g[j];
        }
        int acc = 0;
        if (!out_of_box) {
            orc_action(s, &A1, &tmp1, &tmp2);
            double K1 = 0.0;
            for (int64_t j = 0; j < nq; ++j) K1 += 0.5 * mom[j] * mom[j] * inv_mass[j];
            double dH = (A1 + K1) - (A0 + K0);
            uint32_t w[4];
            orc_block(seed, s->chain, traj, 0u, ORC_KIND_HMC_ACC, 0u, w);
            double u = orc_u01(w[0], w[1]), margin;
            acc = orc_accept(dH, u, &margin);
        }
        if (!acc) {
            memcpy(s->X, q0, sizeof(double) * (size_t)nx);
            memcpy(s->p, q0 + nx, sizeof(double) * (size_t)s->Np);
        } else {
            acc_count += 1;
        }
        orc_refresh_cache(s);
        int64_t sw = s->sweep;
        if (sw >= s->n_init && (sw - s->n_init) % s->n_skip == 0) orc_record(s);
        s->sweep = sw + 1;
    }
    free(q0); free(mom); free(g);
    if (n_acc) *n_acc = acc_count;
    return 0;
}

/* ---- accessors ------------------------------------------------------------ */
void orc_get_state(const orc_state* s, double* X, double* p)
{
    if (X) memcpy(X, s->X, sizeof(double) * (size_t)(s->D * (s->M + 1)));
    if (p) for (int l = 0; l < s->Np; ++l) p[l] = s->p[l];
}

void orc_get_cache(const orc_state* s, double* f)
{
    memcpy(f, s->f, sizeof(double) * (size_t)(s->D * (s->M + 1)));
}

void orc_get_steps(const orc_state* s, double* sig_x, double* sig_p)
{
    if (sig_x) memcpy(sig_x, s->sig, sizeof(double) * (size_t)(s->D * (s->M + 1)));
    if (sig_p) for (int l = 0; l < s->Np; ++l) sig_p[l] = s->sigp[l];
}

int64_t orc_get_sweep(const orc_state* s, double* beta)
{
    if (beta) *beta = s->beta;
    return s->sweep;
}

void orc_last_margins(const orc_state* s, double* site_margin, double* param_margin)
{
    if (site_margin) memcpy(site_margin, s->site_margin, sizeof(double) * (size_t)(s->M + 1));
    if (param_margin) for (int l = 0; l < s->Np; ++l) param_margin[l] = s->par_margin[l];
}

void orc_accept_stats(const orc_state* s, uint64_t* site_acc, uint64_t* site_prop,
                      uint64_t* par_acc, uint64_t* par_prop)
{
    for (int k = 0; k < 2; ++k) { site_acc[k] = s->site_acc[k]; site_prop[k] = s->site_prop[k]; }
    for (int l = 0; l < s->Np; ++l) { par_acc[l] = s->par_acc[l]; par_prop[l] = s->par_prop[l]; }
}
