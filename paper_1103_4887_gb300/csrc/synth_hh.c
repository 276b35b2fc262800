/*
 * Synthetic "physical system" for the seeded input recipe: a Hodgkin-Huxley
 * membrane driven by a given injected current, integrated finely (classical
 * RK4 with `substeps` substeps per sample interval, current held over each
 * interval).  It produces the true path from which the noisy voltage
 * observations are drawn, the way the paper simulated its neuron data
 * (Sec. 5.1).  It is an input generator only: neither the sampler library nor
 * the test oracle calls it for their own arithmetic.
 *
 * Parameters q = (gNa, gK, gL, ENa, EK, EL, C); rates are the textbook 1952
 * forms with rest near -65 mV.
 */
#include <math.h>
#include <stdint.h>

static double lin_rate(double k, double v0, double V)
{
    /* k (V + v0) / (1 - exp(-(V + v0)/10)) with its limit 10 k at V = -v0 */
    double w = (V + v0) / 10.0;
    if (fabs(w) < 1e-7) return 10.0 * k * (1.0 + 0.5 * w);
    return 10.0 * k * w / (1.0 - exp(-w));
}

static void field(const double* s, const double* q, double I, double* ds)
{
    double V = s[0], m = s[1], h = s[2], n = s[3];
    double am = lin_rate(0.1, 40.0, V), bm = 4.0 * exp(-(V + 65.0) / 18.0);
    double ah = 0.07 * exp(-(V + 65.0) / 20.0), bh = 1.0 / (1.0 + exp(-(V + 35.0) / 10.0));
    double an = lin_rate(0.01, 55.0, V), bn = 0.125 * exp(-(V + 65.0) / 80.0);
    double cur = I - q[0] * m * m * m * h * (V - q[3]) - q[1] * n * n * n * n * (V - q[4])
               - q[2] * (V - q[5]);
    ds[0] = cur / q[6];
    ds[1] = am * (1.0 - m) - bm * m;
    ds[2] = ah * (1.0 - h) - bh * h;
    ds[3] = an * (1.0 - n) - bn * n;
}

static void advance(double* s, const double* q, double I, double h)
{
    double k1[4], k2[4], k3[4], k4[4], t[4];
    field(s, q, I, k1);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + 0.5 * h * k1[i];
    field(t, q, I, k2);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + 0.5 * h * k2[i];
    field(t, q, I, k3);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + h * k3[i];
    field(t, q, I, k4);
    for (int i = 0; i < 4; ++i) s[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Relax from V = -65 with gates at their steady state for `relax_ms` with no
 * current, then integrate across M intervals of length dt with current I[n]
 * on [t_n, t_{n+1}).  X is SoA: X[a*(M+1)+n]. */
int synth_hh_truth(int64_t M, double dt, int substeps, const double* q, const double* I,
                   double relax_ms, double* X)
{
    if (M < 1 || substeps < 1 || !(dt > 0.0)) return -1;
    double s[4];
    double V0 = -65.0;
    double am = lin_rate(0.1, 40.0, V0), bm = 4.0 * exp(-(V0 + 65.0) / 18.0);
    double ah = 0.07 * exp(-(V0 + 65.0) / 20.0), bh = 1.0 / (1.0 + exp(-(V0 + 35.0) / 10.0));
    double an = lin_rate(0.01, 55.0, V0), bn = 0.125 * exp(-(V0 + 65.0) / 80.0);
    s[0] = V0; s[1] = am / (am + bm); s[2] = ah / (ah + bh); s[3] = an / (an + bn);
    double h = dt / (double)substeps;
    int64_t nrelax = (int64_t)(relax_ms / h);
    for (int64_t k = 0; k < nrelax; ++k) advance(s, q, 0.0, h);
    for (int a = 0; a < 4; ++a) X[(int64_t)a * (M + 1)] = s[a];
    for (int64_t n = 0; n < M; ++n) {
        for (int k = 0; k < substeps; ++k) advance(s, q, I[n], h);
        for (int a = 0; a < 4; ++a) X[(int64_t)a * (M + 1) + n + 1] = s[a];
    }
    return 0;
}
