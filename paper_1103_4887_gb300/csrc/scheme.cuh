// Scheme-generic pieces shared by the sweep, whole-path and statistics
// kernels: scalar constants in the arithmetic type, the per-site cached value,
// the model-error residual of the two discretisations and the reverse mode of
// one model term (gradient and HMC kernels).
#pragma once

#include "device.cuh"
#include "internal.h"

namespace pimc {

// Scalar constants of the action in the arithmetic type, formed once per
// kernel so the per-site code does no FP64 -> FP32 conversions.
template <class R> struct Coef {
    R dt, Rm, Rf[kMaxD];
    __device__ __forceinline__ explicit Coef(const Ctx& c)
    {
        dt = R(c.dt);
        Rm = R(c.Rm);
#pragma unroll
        for (int a = 0; a < kMaxD; ++a) Rf[a] = R(c.Rf[a]);
    }
};

// ---- scheme-generic pieces --------------------------------------------------
// Cached value g_n of a site: the RK4 map f(x_n) (RK4 scheme, n < M) or the
// vector field F(x_n) (trapezoid rule, n <= M; the drive at t_M is I_{M-1}).
__device__ __forceinline__ int64_t cache_len(const Ctx& c) { return c.scheme == kSchemeRK4 ? c.M : c.M + 1; }

__device__ __forceinline__ int64_t drive_index(const Ctx& c, int64_t n)
{
    return (c.scheme == kSchemeRK4 || n < c.M) ? n : c.M - 1;
}

// Cached value from a drive value already loaded.
template <class Model, class R>
__device__ __forceinline__ void cache_value_at(const Ctx& c, const Coef<R>& k, const R* x, const R* q, R drive, R* g)
{
    if (c.scheme == kSchemeRK4) rk4_map<Model, R>(x, q, drive, k.dt, g);
    else Model::rhs(x, q, drive, g);
}

template <class Model, class R>
__device__ __forceinline__ void cache_value(const Ctx& c, const Coef<R>& k, const R* x, const R* q, int64_t n, R* g)
{
    cache_value_at<Model, R>(c, k, x, q, ((const R*)c.I)[drive_index(c, n)], g);
}

// Model-error residual eps_{n+1} from x_n, x_{n+1} and their cached values:
// x_{n+1} - f(x_n) (RK4), or x_{n+1} - x_n - dt/2 (F_{n+1} + F_n) (trapezoid).
template <class R>
__device__ __forceinline__ R eps_of(const Ctx& c, const Coef<R>& k, R xn, R xn1, R gn, R gn1)
{
    if (c.scheme == kSchemeRK4) return xn1 - gn;
    return xn1 - xn - R(0.5) * k.dt * (gn1 + gn);
}

// Reverse mode of model term k of the action, wr/2 |e|^2 with wr = beta Rf
// (x_k -> x_{k+1}): its residual e, the cotangent it sends to x_k (own) and
// to x_{k+1} (nxt), and its dA/dp (gp).  RK4: e = x_{k+1} - f(x_k),
// w = wr . e, own = -J_x f^T w, nxt = w, gp = -J_p f^T w.  Trapezoid:
// e = x_{k+1} - x_k - dt/2 (F_{k+1} + F_k), w = wr . e,
// own = -w - dt/2 J_k^T w, nxt = w - dt/2 J_{k+1}^T w,
// gp = -dt/2 (J_p F_k + J_p F_{k+1})^T w.  In, In1: the drive at t_k and at
// t_{k+1} (the trapezoid's second vector field).
template <class Model, class R>
__device__ __forceinline__ void term_adjoint(const Ctx& c, const Coef<R>& kc, const R* wr, const R* x, const R* x1,
                                             const R* pr, R In, R In1, R* e, R* own, R* nxt, R* gp)
{
    constexpr int D = Model::D;
    R jp[kMaxP];
#pragma unroll
    for (int l = 0; l < kMaxP; ++l) jp[l] = R(0);
    if (c.scheme == kSchemeRK4) {
        R gx[D];
#pragma unroll
        for (int a = 0; a < D; ++a) gx[a] = R(0);
        rk4_vjp<Model, R>(x, pr, In, kc.dt,
                          [&](const R* f, R* w) {
#pragma unroll
                              for (int a = 0; a < D; ++a) {
                                  e[a] = x1[a] - f[a];
                                  w[a] = wr[a] * e[a];
                              }
                          },
                          nxt, gx, jp);
#pragma unroll
        for (int a = 0; a < D; ++a) own[a] = -gx[a];
#pragma unroll
        for (int l = 0; l < kMaxP; ++l) gp[l] = -jp[l];
    } else {
        R F0[D], F1[D], w[D], g0[D], g1[D];
        Model::rhs(x, pr, In, F0);
        Model::rhs(x1, pr, In1, F1);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            e[a] = x1[a] - x[a] - R(0.5) * kc.dt * (F1[a] + F0[a]);
            w[a] = wr[a] * e[a];
            g0[a] = R(0);
            g1[a] = R(0);
        }
        Model::rhs_vjp(x, pr, In, w, g0, jp);
        Model::rhs_vjp(x1, pr, In1, w, g1, jp);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            own[a] = -w[a] - R(0.5) * kc.dt * g0[a];
            nxt[a] = w[a] - R(0.5) * kc.dt * g1[a];
        }
#pragma unroll
        for (int l = 0; l < kMaxP; ++l) gp[l] = -(R(0.5) * kc.dt) * jp[l];
    }
}

}  // namespace pimc
