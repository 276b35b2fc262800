// Scheme-generic pieces shared by the sweep, whole-path and statistics
// kernels: scalar constants in the arithmetic type, the per-site cached value
// and the model-error residual of the two discretisations.
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

}  // namespace pimc
