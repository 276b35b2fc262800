// Path statistics (Sec. 4.1): running shifted sums S1 += x - r, S2 += (x - r)^2
// in FP64 (r = first recorded value) and equal-width bin counts with
// under/overflow slots, for the sites [n0, n1) a caller owns and, when
// `params_here`, the parameters.  Shared by the sweep and HMC kernels.
#pragma once

#include "device.cuh"
#include "internal.h"
#include "scheme.cuh"

namespace pimc {

__device__ __forceinline__ int64_t hist_slot(double v, double lo, double hi, int nb)
{
    if (!(v >= lo)) return 0;
    if (v >= hi) return nb + 1;
    const double t = (v - lo) / (hi - lo);
    int64_t b = (int64_t)floor(t * (double)nb);
    if (b > nb - 1) b = nb - 1;
    return 1 + b;
}

__device__ __forceinline__ void accumulate(const Ctx& c, int64_t ci, double v, bool first_rec)
{
    if (first_rec) c.shift[ci] = v;
    const double d = v - c.shift[ci];
    c.S1[ci] += d;
    c.S2[ci] += d * d;
}

// Thread t of nt records its share; p is the current parameter vector and Fc
// the current cache (f(x_n) or F(x_n)), which gives the model-error residuals
// eps_{n+1} without another map evaluation; the
// measurement residuals are delta_n = x_{n,0} - y_n (their statistics are the
// model check of Sec. 6).  Per site, every operand is loaded before any sum
// is stored: the compiler cannot tell the arrays apart, and interleaved
// read-modify-writes would cost one memory round trip per array.
template <class Model, class R>
__device__ void record_sample(const Ctx& c, int64_t n0, int64_t n1, bool params_here, const double* p,
                              bool first_rec, int t, int nt, const R* Fc)
{
    constexpr int D = Model::D, NP = Model::NP;
    const int64_t M = c.M, nx = (int64_t)D * (M + 1);
    const R* X = (const R*)c.X;
    const bool trap = c.scheme != kSchemeRK4;
    for (int64_t n = n0 + t; n < n1; n += nt) {
        const bool has_eps = n < M, has_d = n >= 1;
        double xv[D], sv[D], s1[D], s2[D], e[D + 1], r1[D + 1], r2[D + 1];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int64_t ci = (int64_t)a * (M + 1) + n;
            xv[a] = (double)X[a * c.ldx + n];
            sv[a] = first_rec ? xv[a] : c.shift[ci];
            s1[a] = c.S1[ci];
            s2[a] = c.S2[ci];
            e[a] = r1[a] = r2[a] = 0.0;
            if (has_eps) {
                const double xn1 = (double)X[a * c.ldx + n + 1];
                const double gn = (double)Fc[a * c.ldf + n];
                e[a] = trap ? xn1 - xv[a] - 0.5 * c.dt * ((double)Fc[a * c.ldf + n + 1] + gn) : xn1 - gn;
                r1[a] = c.R1[(int64_t)a * M + n];
                r2[a] = c.R2[(int64_t)a * M + n];
            }
        }
        e[D] = r1[D] = r2[D] = 0.0;
        if (has_d) {
            e[D] = xv[0] - (double)((const R*)c.y)[n];
            r1[D] = c.R1[(int64_t)D * M + n - 1];
            r2[D] = c.R2[(int64_t)D * M + n - 1];
        }
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const int64_t ci = (int64_t)a * (M + 1) + n;
            const double d = xv[a] - sv[a];
            if (first_rec) c.shift[ci] = sv[a];
            c.S1[ci] = s1[a] + d;
            c.S2[ci] = s2[a] + d * d;
            if (has_eps) {
                c.R1[(int64_t)a * M + n] = r1[a] + e[a];
                c.R2[(int64_t)a * M + n] = r2[a] + e[a] * e[a];
            }
        }
        if (has_d) {
            c.R1[(int64_t)D * M + n - 1] = r1[D] + e[D];
            c.R2[(int64_t)D * M + n - 1] = r2[D] + e[D] * e[D];
        }
    }
    if (params_here && t < NP) accumulate(c, nx + t, p[t], first_rec);
    for (int kk = t; kk < c.n_sel; kk += nt) {
        const int64_t ci = c.h_comp[kk];
        double v;
        bool mine;
        if (ci < nx) {
            const int64_t a = ci / (M + 1), n = ci - a * (M + 1);
            mine = (n >= n0 && n < n1);
            v = mine ? (double)X[a * c.ldx + n] : 0.0;
        } else {
            mine = params_here;
            v = p[ci - nx];
        }
        if (mine) c.hist[(int64_t)kk * (c.n_bins + 2) + hist_slot(v, c.h_lo[kk], c.h_hi[kk], c.n_bins)] += 1ull;
    }
}

}  // namespace pimc
