// Device building blocks of the sampler: counter-based RNG, model vector
// fields with their transposed Jacobian products, the RK4 map and its reverse
// mode, and the per-site / per-parameter changes of action.  Templated on the
// arithmetic type R (double for PIMC_FP64, float for PIMC_FP32_MIXED).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace pimc {

constexpr int kMaxD = 4;
constexpr int kMaxP = 8;

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products whose high words are xored with the other counter
// words and the round key; the key advances by the Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t ha = __umulhi(0xD2511F53u, c.x), la = 0xD2511F53u * c.x;
        const uint32_t hb = __umulhi(0xCD9E8D57u, c.z), lb = 0xCD9E8D57u * c.z;
        c = make_uint4(hb ^ c.y ^ k0, lb, ha ^ c.w ^ k1, la);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

enum : uint32_t { kKindSite = 0, kKindParam = 1, kKindHmcMom = 2, kKindHmcAcc = 3 };

__device__ __forceinline__ uint4 draw_block(uint64_t seed, uint32_t chain, uint64_t sweep,
                                            uint32_t idx, uint32_t kind, uint32_t blk)
{
    return philox(make_uint4(idx, (uint32_t)sweep, (kind << 24) | blk, chain),
                  (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Open-interval uniforms.  FP64: 52-bit integer from the top 26 bits of two
// words, (k + 1/2) 2^-52.  FP32: top 24 bits of one word, (k + 1/2) 2^-24
// (the same high bits as the FP64 form, so both precisions see nearly the
// same number).
__device__ __forceinline__ double u01d(uint32_t hi, uint32_t lo)
{
    const uint64_t k = ((uint64_t)(hi >> 6) << 26) | (uint64_t)(lo >> 6);
    return ((double)k + 0.5) * 0x1.0p-52;
}
__device__ __forceinline__ float u01f(uint32_t hi) { return ((float)(hi >> 8) + 0.5f) * 0x1.0p-24f; }

template <class R> struct Num;

template <> struct Num<double> {
    static __device__ __forceinline__ double th(double x) { return tanh(x); }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double exm1(double x) { return expm1(x); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double uni(uint32_t hi, uint32_t lo) { return u01d(hi, lo); }
    // Box-Muller: r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 log u1)
    static __device__ __forceinline__ void box_muller(uint4 w, double& z0, double& z1)
    {
        const double r = sqrt(-2.0 * log(u01d(w.x, w.y)));
        double s, c;
        sincospi(2.0 * u01d(w.z, w.w), &s, &c);
        z0 = r * c;
        z1 = r * s;
    }
    static constexpr double psi_cut = 1e-6;
    static constexpr double dpsi_cut = 1e-3;
};

template <> struct Num<float> {
    // SFU hyperbolic tangent (one MUFU.TANH instruction)
    static __device__ __forceinline__ float th(float x)
    {
        float y;
        asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // SFU exponential (ex2.approx) and reciprocal for the per-site arithmetic
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float exm1(float x) { return __expf(x) - 1.0f; }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    static __device__ __forceinline__ float uni(uint32_t hi, uint32_t) { return u01f(hi); }
    static __device__ __forceinline__ void box_muller(uint4 w, float& z0, float& z1)
    {
        const float r = sqrtf(-2.0f * __logf(u01f(w.x)));
        float s, c;
        __sincosf(6.283185307179586f * u01f(w.z), &s, &c);
        z0 = r * c;
        z1 = r * s;
    }
    static constexpr float psi_cut = 1e-2f;
    static constexpr float dpsi_cut = 1e-1f;
};

// ---------------------------------------------------------------------------
// Models.  Parameters arrive as R p[kMaxP].
// ---------------------------------------------------------------------------

// u / (1 - e^{-u}): the alpha_m / alpha_n form; its removable singularity at
// u = 0 is replaced by the series 1 + u/2 + u^2/12 below the cut.
template <class R> __device__ __forceinline__ R psi(R u)
{
    if (fabs(u) < Num<R>::psi_cut) return R(1) + u * (R(0.5) + u * R(1.0 / 12.0));
    return Num<R>::div(-u, Num<R>::exm1(-u));
}
// psi(u) as a quotient num/den: (u, 1 - e^{-u}), or (series, 1) below the cut.
template <class R> __device__ __forceinline__ void psi_frac(R u, R& num, R& den)
{
    if (fabs(u) < Num<R>::psi_cut) {
        num = R(1) + u * (R(0.5) + u * R(1.0 / 12.0));
        den = R(1);
    } else {
        num = u;
        den = -Num<R>::exm1(-u);
    }
}
// The numerator psi_frac gives: u, or the series below the cut.
template <class R> __device__ __forceinline__ R psi_num(R u)
{
    return fabs(u) < Num<R>::psi_cut ? R(1) + u * (R(0.5) + u * R(1.0 / 12.0)) : u;
}
// d psi/du = (1 - e^{-u} - u e^{-u}) / (1 - e^{-u})^2, series
// 1/2 + u/6 - u^3/180 + u^5/5040 below the cut.  Formed from em = 1 - e^{-u},
// the denominator psi_frac already computed (|u| >= dpsi_cut > psi_cut, so
// psi_frac took that branch), and its reciprocal inv_em: e^{-u} = 1 - em, no
// second exponential and no division.
template <class R> __device__ __forceinline__ R dpsi_em(R u, R em, R inv_em)
{
    if (fabs(u) < Num<R>::dpsi_cut) {
        const R u2 = u * u;
        return R(0.5) + u * (R(1.0 / 6.0) + u2 * (R(-1.0 / 180.0) + u2 * R(1.0 / 5040.0)));
    }
    return (em - u * (R(1) - em)) * (inv_em * inv_em);
}

// ---------------------------------------------------------------------------
// FP32 lanes.  The FP32 HH field and RK4 map are written once over a lane type
// T: float (one site) or float2 (two sites, on the packed f32x2 add, mul and
// fma of sm_100 and later, one issue slot for both lanes).  Every operation is
// an explicitly rounded IEEE operation, and no product feeds an addition:
// the code generator may fuse a packed multiply into a following packed add
// (it never fuses the scalar __fmul_rn), so every such pair is written as an
// fma on both sides.  A site's bits are then the same evaluated alone or as
// one lane of a pair.  The SFU operations (ex2, rcp) run per lane.
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }

__device__ __forceinline__ float ladd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 ladd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float lsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 lsub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float lmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 lmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float lfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 lfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// c - a b, rounded once
__device__ __forceinline__ float lfnma(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ float2 lfnma(float2 a, float2 b, float2 c)
{
    return __ffma2_rn(make_float2(-a.x, -a.y), b, c);
}
// 2^x and 1/x on the SFU (ex2.approx, rcp.approx), per lane
__device__ __forceinline__ float lex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 lex2(float2 x) { return make_float2(lex2(x.x), lex2(x.y)); }
__device__ __forceinline__ float lrcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 lrcp(float2 x) { return make_float2(lrcp(x.x), lrcp(x.y)); }
// |u| < cut ? s : v, per lane
__device__ __forceinline__ float lsel_small(float u, float cut, float s, float v) { return fabsf(u) < cut ? s : v; }
__device__ __forceinline__ float2 lsel_small(float2 u, float cut, float2 s, float2 v)
{
    return make_float2(lsel_small(u.x, cut, s.x, v.x), lsel_small(u.y, cut, s.y, v.y));
}

// The transcendental part of the HH rates at V (see HH below): E = e^{-(V+65)/80},
// e^{-(V+65)/18}, the psi denominators dm, dn and the reciprocal r = 1/(dm dn dh).
template <class T> struct HHCache {
    T E, e18, dm, dn, r;
};

// HH rates and field over FP32 lanes.  e^y is formed as 2^(y log2 e) on the
// SFU, with log2 e folded into each argument's constant; psi(u) = u/(1 - e^{-u})
// takes the series 1 + u/2 + u^2/12 below |u| < 1e-2 (a per-lane select).
template <class T> struct HHLanes {
    static constexpr double kLog2e = 1.4426950408889634;
    static constexpr float kCut = 1e-2f;
    static __device__ __forceinline__ T psi_series(T u)
    {
        return lfma(u, lfma(u, splat<T>(float(1.0 / 12.0)), splat<T>(0.5f)), splat<T>(1.0f));
    }
    // arguments of alpha_m and alpha_n: (V + 40)/10 and (V + 55)/10
    static __device__ __forceinline__ T um_of(T V) { return lfma(V, splat<T>(0.1f), splat<T>(4.0f)); }
    static __device__ __forceinline__ T un_of(T V) { return lfma(V, splat<T>(0.1f), splat<T>(5.5f)); }
    // dh = 1 + E^8 e^3 (= 1 + e^{-(V+35)/10})
    static __device__ __forceinline__ T dh_of(T E)
    {
        const T E2 = lmul(E, E), E4 = lmul(E2, E2), E8 = lmul(E4, E4);
        return lfma(E8, splat<T>(20.085536923187668f), splat<T>(1.0f));
    }
    static __device__ __forceinline__ void cache_at(T V, HHCache<T>& k)
    {
        const T t = ladd(V, splat<T>(65.0f));
        k.E = lex2(lmul(t, splat<T>(float(-kLog2e / 80.0))));
        k.e18 = lex2(lmul(t, splat<T>(float(-kLog2e / 18.0))));
        const T um = um_of(V), un = un_of(V);
        const T one = splat<T>(1.0f);
        k.dm = lsel_small(um, kCut, one, lsub(one, lex2(lmul(um, splat<T>(float(-kLog2e))))));
        k.dn = lsel_small(un, kCut, one, lsub(one, lex2(lmul(un, splat<T>(float(-kLog2e))))));
        k.r = lrcp(lmul(lmul(k.dm, k.dn), dh_of(k.E)));
    }
    // alpha (a) and beta (b) of the gates m, h, n from the cache
    static __device__ __forceinline__ void rates_from(T V, const HHCache<T>& k, T a[3], T b[3])
    {
        const T um = um_of(V), un = un_of(V);
        const T nm = lsel_small(um, kCut, psi_series(um), um);
        const T nn = lsel_small(un, kCut, psi_series(un), un);
        const T dh = dh_of(k.E);
        const T E2 = lmul(k.E, k.E), E4 = lmul(E2, E2);
        b[2] = lmul(splat<T>(0.125f), k.E);
        a[1] = lmul(splat<T>(0.07f), E4);
        b[0] = lmul(splat<T>(4.0f), k.e18);
        a[0] = lmul(nm, lmul(lmul(k.dn, dh), k.r));
        a[2] = lmul(lmul(splat<T>(0.1f), nn), lmul(lmul(k.dm, dh), k.r));
        b[1] = lmul(lmul(k.dm, k.dn), k.r);
    }
    // F = (dV/dt, dm/dt, dh/dt, dn/dt); q = (gNa, gK, gL, ENa, EK, EL, C, 1/C).
    // The same rates as rates_from, with each alpha + beta formed by an fma
    // and the currents scaled by 1/C term by term, so that every value that
    // reaches an addition is an fma result (see the lane rules above).
    static __device__ __forceinline__ void rhs(const T* x, const T* q, T I, T* F, HHCache<T>& k)
    {
        const T V = x[0], m = x[1], h = x[2], n = x[3];
        cache_at(V, k);
        const T um = um_of(V), un = un_of(V);
        const T nm = lsel_small(um, kCut, psi_series(um), um);
        const T nn = lsel_small(un, kCut, psi_series(un), un);
        const T dh = dh_of(k.E);
        const T E2 = lmul(k.E, k.E), E4 = lmul(E2, E2);
        const T a0 = lmul(nm, lmul(lmul(k.dn, dh), k.r));
        const T a1 = lmul(splat<T>(0.07f), E4);
        const T a2 = lmul(lmul(splat<T>(0.1f), nn), lmul(lmul(k.dm, dh), k.r));
        // alpha (1 - s) - beta s = alpha - (alpha + beta) s; beta_m = 4 e18,
        // beta_h = dm dn r, beta_n = E / 8
        F[1] = lfnma(lfma(splat<T>(4.0f), k.e18, a0), m, a0);
        F[2] = lfnma(lfma(lmul(k.dm, k.dn), k.r, a1), h, a1);
        F[3] = lfnma(lfma(splat<T>(0.125f), k.E, a2), n, a2);
        const T iC = q[7];
        const T m3h = lmul(lmul(lmul(m, m), m), h);
        const T n2 = lmul(n, n), n4 = lmul(n2, n2);
        T acc = lfnma(lmul(lmul(q[0], iC), m3h), lsub(V, q[3]), lmul(I, iC));
        acc = lfnma(lmul(lmul(q[1], iC), n4), lsub(V, q[4]), acc);
        F[0] = lfnma(lmul(q[2], iC), lsub(V, q[5]), acc);
    }
};

// One classical RK4 step of the HH field over FP32 lanes (drive held at I):
// f = x + dt/6 (k1 + 2 k2 + 2 k3 + k4); hdt = dt/2 and sdt = dt/6 as formed
// by the caller.
template <class T>
__device__ __forceinline__ void hh_rk4_lanes(const T* x, const T* q, T I, T dt, T hdt, T sdt, T* f)
{
    T k[4], xs[4], acc[4];
    HHCache<T> c;
    HHLanes<T>::rhs(x, q, I, k, c);
#pragma unroll
    for (int a = 0; a < 4; ++a) { acc[a] = k[a]; xs[a] = lfma(hdt, k[a], x[a]); }
    HHLanes<T>::rhs(xs, q, I, k, c);
#pragma unroll
    for (int a = 0; a < 4; ++a) { acc[a] = lfma(splat<T>(2.0f), k[a], acc[a]); xs[a] = lfma(hdt, k[a], x[a]); }
    HHLanes<T>::rhs(xs, q, I, k, c);
#pragma unroll
    for (int a = 0; a < 4; ++a) { acc[a] = lfma(splat<T>(2.0f), k[a], acc[a]); xs[a] = lfma(dt, k[a], x[a]); }
    HHLanes<T>::rhs(xs, q, I, k, c);
#pragma unroll
    for (int a = 0; a < 4; ++a) f[a] = lfma(sdt, ladd(acc[a], k[a]), x[a]);
}

// RK4 change of the model-error term of one site over FP32 lanes:
// beta sum_a 1/2 Rf_a (d'_a - d_a)(d'_a + d_a), d' = x_{n+1} - f', d = x_{n+1} - f.
template <class T, int D>
__device__ __forceinline__ T rk4_term_lanes(T beta, const float* Rf, const T* xn1, const T* fnew, const T* fold)
{
    T t = splat<T>(0.0f);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T dp = lsub(xn1[a], fnew[a]), d = lsub(xn1[a], fold[a]);
        const T w = lmul(lmul(splat<T>(0.5f * Rf[a]), lsub(dp, d)), ladd(dp, d));
        t = lfma(beta, w, t);
    }
    return t;
}

// Hodgkin-Huxley (1952) in the modern convention, conductance form:
//   C dV/dt = I - gNa m^3 h (V - ENa) - gK n^4 (V - EK) - gL (V - EL)
//   da/dt = alpha_a(V)(1 - a) - beta_a(V) a          (Sec. 5.1, Eq. (dadt) structure)
// p = (gNa, gK, gL, ENa, EK, EL, C).
template <class R> struct HH {
    static constexpr int D = 4, NP = 7;
    // q = (gNa, gK, gL, ENa, EK, EL, C, 1/C): the reciprocal capacitance is
    // formed once per parameter value instead of once per vector-field call.
    static __device__ __forceinline__ void prep(const double* p, R* q)
    {
#pragma unroll
        for (int l = 0; l < NP; ++l) q[l] = R(p[l]);
        q[7] = R(1.0 / p[6]);
    }
    // Rates in 1/ms, V in mV.  With t = V + 65 and E = e^{-t/80}:
    // beta_n = 0.125 E, alpha_h = 0.07 E^4 (= 0.07 e^{-t/20}),
    // beta_h = 1/(1 + E^8 e^3) (= 1/(1 + e^{-(V+35)/10})), beta_m = 4 e^{-t/18};
    // alpha_m = psi((V+40)/10), alpha_n = 0.1 psi((V+55)/10).  The three
    // quotients share one reciprocal.  Divisions by constants are products.
    static __device__ __forceinline__ void rates(R V, R a[3], R b[3])
    {
        Cache k;
        cache_at(V, k);
        rates_from(V, k, a, b);
    }
    // The transcendental part of the rates at V: E, e^{-t/18}, the psi
    // denominators dm, dn (1 - e^{-u} of alpha_m, alpha_n) and the shared
    // reciprocal r = 1/(dm dn dh), dh = 1 + E^8 e^3.  The reverse pass of an
    // RK4 step reuses the forward pass's (kReuseRates): in FP64 each
    // exponential and division is a long FP64 instruction sequence, in FP32
    // the reuse shortens the latency-bound adjoint's chain.
    // FP32 (the FP32-mixed form): the same rates, evaluated by HHLanes<float>.
    using Cache = HHCache<R>;
    static constexpr bool kReuseRates = true;
    static constexpr bool kLanes = std::is_same<R, float>::value;
    static __device__ __forceinline__ R dh_of(R E)
    {
        if constexpr (kLanes) {
            return HHLanes<float>::dh_of(E);
        } else {
            const R E2 = E * E, E4 = E2 * E2, E8 = E4 * E4;
            return R(1) + E8 * R(20.085536923187668);  // e^3
        }
    }
    static __device__ __forceinline__ void cache_at(R V, Cache& k)
    {
        if constexpr (kLanes) {
            HHLanes<float>::cache_at(V, k);
            return;
        }
        const R t = V + R(65);
        k.E = Num<R>::ex(t * R(-0.0125));
        k.e18 = Num<R>::ex(t * R(-1.0 / 18.0));
        R nm, nn;
        psi_frac<R>((V + R(40)) * R(0.1), nm, k.dm);
        psi_frac<R>((V + R(55)) * R(0.1), nn, k.dn);
        k.r = Num<R>::div(R(1), k.dm * k.dn * dh_of(k.E));
    }
    static __device__ __forceinline__ void rates_from(R V, const Cache& k, R a[3], R b[3])
    {
        if constexpr (kLanes) {
            HHLanes<float>::rates_from(V, k, a, b);
            return;
        }
        const R E2 = k.E * k.E, E4 = E2 * E2;
        b[2] = R(0.125) * k.E;
        a[1] = R(0.07) * E4;
        b[0] = R(4) * k.e18;
        const R nm = psi_num<R>((V + R(40)) * R(0.1)), nn = psi_num<R>((V + R(55)) * R(0.1));
        const R dh = dh_of(k.E);
        a[0] = nm * (k.dn * dh * k.r);
        a[2] = R(0.1) * nn * (k.dm * dh * k.r);
        b[1] = k.dm * k.dn * k.r;
    }
    static __device__ __forceinline__ void rhs(const R* x, const R* q, R I, R* F)
    {
        Cache k;
        rhs_c(x, q, I, F, k);
    }
    // rhs, keeping the rates' transcendental part in k
    static __device__ __forceinline__ void rhs_c(const R* x, const R* q, R I, R* F, Cache& k)
    {
        if constexpr (kLanes) {
            HHLanes<float>::rhs(x, q, I, F, k);
            return;
        }
        R a[3], b[3];
        cache_at(x[0], k);
        rates_from(x[0], k, a, b);
        const R V = x[0], m = x[1], h = x[2], n = x[3];
        const R iNa = q[0] * m * m * m * h * (V - q[3]);
        const R iK = q[1] * n * n * n * n * (V - q[4]);
        const R iL = q[2] * (V - q[5]);
        F[0] = (I - iNa - iK - iL) * q[7];
        F[1] = a[0] * (R(1) - m) - b[0] * m;
        F[2] = a[1] * (R(1) - h) - b[1] * h;
        F[3] = a[2] * (R(1) - n) - b[2] * n;
    }
    // gx += J_x^T w, gp += J_p^T w (gp indexed like p: 7 entries)
    static __device__ __forceinline__ void rhs_vjp(const R* x, const R* q, R I, const R* w, R* gx, R* gp)
    {
        Cache k;
        cache_at(x[0], k);
        rhs_vjp_c(x, q, I, w, gx, gp, k);
    }
    // rhs_vjp from the rates' transcendental part at x[0] (no exponential, no
    // division: 1/dm = r dn dh and 1/dn = r dm dh)
    static __device__ __forceinline__ void rhs_vjp_c(const R* x, const R* q, R I, const R* w, R* gx, R* gp,
                                                     const Cache& k)
    {
        R a[3], b[3];
        rates_from(x[0], k, a, b);
        const R V = x[0], m = x[1], h = x[2], n = x[3];
        const R dh = dh_of(k.E);
        R da[3], db[3];
        da[0] = dpsi_em<R>((V + R(40)) * R(0.1), k.dm, k.r * k.dn * dh) * R(0.1);
        db[0] = b[0] * R(-1.0 / 18.0);
        da[1] = a[1] * R(-0.05);
        db[1] = b[1] * (R(1) - b[1]) * R(0.1);
        da[2] = dpsi_em<R>((V + R(55)) * R(0.1), k.dn, k.r * k.dm * dh) * R(0.01);
        db[2] = b[2] * R(-0.0125);
        const R gNa = q[0], gK = q[1], gL = q[2], ENa = q[3], EK = q[4], EL = q[5], iC = q[7];
        const R m3h = m * m * m * h, n4 = n * n * n * n;
        const R num = I - gNa * m3h * (V - ENa) - gK * n4 * (V - EK) - gL * (V - EL);
        const R wv = w[0] * iC;
        gx[0] += wv * (-gNa * m3h - gK * n4 - gL);
        gx[1] += wv * (R(-3) * gNa * m * m * h * (V - ENa));
        gx[2] += wv * (-gNa * m * m * m * (V - ENa));
        gx[3] += wv * (R(-4) * gK * n * n * n * (V - EK));
        gp[0] += wv * (-m3h * (V - ENa));
        gp[1] += wv * (-n4 * (V - EK));
        gp[2] += wv * (-(V - EL));
        gp[3] += wv * (gNa * m3h);
        gp[4] += wv * (gK * n4);
        gp[5] += wv * gL;
        gp[6] += w[0] * (-num * iC * iC);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            const R s = x[1 + g];
            gx[1 + g] += w[1 + g] * (-(a[g] + b[g]));
            gx[0] += w[1 + g] * (da[g] * (R(1) - s) - db[g] * s);
        }
    }
    // default initial path: V from the observation, gates at a_inf(V)
    static __device__ __forceinline__ void init_site(R V, R* x)
    {
        R a[3], b[3];
        rates(V, a, b);
        x[0] = V;
        for (int g = 0; g < 3; ++g) x[1 + g] = a[g] / (a[g] + b[g]);
    }
};

// The paper's HH form (Sec. 5.1, Eq. (dVdt) and Eq. (dadt)), shifted voltage
// convention: dV/dt = p1 I + p2 m^3 h (p3 - V) + p4 n^4 (p5 - V) + p6 (p7 - V);
// da/dt = (a_inf(V) - a)/tau_a(V), a_inf = 1/2 + 1/2 tanh((V - V_a)/dV_a),
// tau_a = tau_a0 + tau_a1 (1 - tanh^2); Table 1 constants (gates m, h, n).
template <class R> struct HHPaper {
    static constexpr int D = 4, NP = 7;
    static __device__ __forceinline__ void prep(const double* p, R* q)
    {
#pragma unroll
        for (int l = 0; l < NP; ++l) q[l] = R(p[l]);
        q[7] = R(0);
    }
    // V_a, 1/dV_a, tau_a0, tau_a1 of gate g (m, h, n)
    static __device__ __forceinline__ void gate_const(int g, R& Va, R& idV, R& t0, R& t1)
    {
        if (g == 0) { Va = R(25); idV = R(1.0 / 15.0); t0 = R(0.1); t1 = R(0.4); }
        else if (g == 1) { Va = R(5); idV = R(-1.0 / 15.0); t0 = R(1.0); t1 = R(7.0); }
        else { Va = R(10); idV = R(1.0 / 30.0); t0 = R(1.0); t1 = R(5.0); }
    }
    static __device__ __forceinline__ void rhs(const R* x, const R* q, R I, R* F)
    {
        const R V = x[0], m = x[1], h = x[2], n = x[3];
        F[0] = q[0] * I + q[1] * m * m * m * h * (q[2] - V) + q[3] * n * n * n * n * (q[4] - V) + q[5] * (q[6] - V);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            R Va, idV, t0, t1;
            gate_const(g, Va, idV, t0, t1);
            const R t = Num<R>::th((V - Va) * idV);
            const R ainf = R(0.5) + R(0.5) * t;
            const R tau = t0 + t1 * (R(1) - t * t);
            F[1 + g] = Num<R>::div(ainf - x[1 + g], tau);
        }
    }
    static __device__ __forceinline__ void rhs_vjp(const R* x, const R* q, R I, const R* w, R* gx, R* gp)
    {
        const R V = x[0], m = x[1], h = x[2], n = x[3];
        const R m3h = m * m * m * h, n4 = n * n * n * n;
        gx[0] += w[0] * (-q[1] * m3h - q[3] * n4 - q[5]);
        gx[1] += w[0] * (R(3) * q[1] * m * m * h * (q[2] - V));
        gx[2] += w[0] * (q[1] * m * m * m * (q[2] - V));
        gx[3] += w[0] * (R(4) * q[3] * n * n * n * (q[4] - V));
        gp[0] += w[0] * I;
        gp[1] += w[0] * (m3h * (q[2] - V));
        gp[2] += w[0] * (q[1] * m3h);
        gp[3] += w[0] * (n4 * (q[4] - V));
        gp[4] += w[0] * (q[3] * n4);
        gp[5] += w[0] * (q[6] - V);
        gp[6] += w[0] * q[5];
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            R Va, idV, t0, t1;
            gate_const(g, Va, idV, t0, t1);
            const R t = Num<R>::th((V - Va) * idV);
            const R sech2 = R(1) - t * t;
            const R ainf = R(0.5) + R(0.5) * t, tau = t0 + t1 * sech2;
            const R dainf = R(0.5) * sech2 * idV;
            const R dtau = R(-2) * t1 * t * sech2 * idV;
            const R a = x[1 + g];
            gx[1 + g] += w[1 + g] * (-R(1) / tau);
            gx[0] += w[1 + g] * ((dainf * tau - (ainf - a) * dtau) / (tau * tau));
        }
    }
    static __device__ __forceinline__ void init_site(R V, R* x)
    {
        x[0] = V;
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            R Va, idV, t0, t1;
            gate_const(g, Va, idV, t0, t1);
            x[1 + g] = R(0.5) + R(0.5) * Num<R>::th((V - Va) * idV);
        }
    }
};

// Linear test model: dx/dt = K x + (p0, I), K = [[-0.5, -2], [2, -0.5]].
template <class R> struct LinGauss {
    static constexpr int D = 2, NP = 1;
    static __device__ __forceinline__ void prep(const double* p, R* q) { q[0] = R(p[0]); }
    static __device__ __forceinline__ void rhs(const R* x, const R* p, R I, R* F)
    {
        F[0] = R(-0.5) * x[0] + R(-2.0) * x[1] + p[0];
        F[1] = R(2.0) * x[0] + R(-0.5) * x[1] + I;
    }
    static __device__ __forceinline__ void rhs_vjp(const R* x, const R* p, R I, const R* w, R* gx, R* gp)
    {
        gx[0] += R(-0.5) * w[0] + R(2.0) * w[1];
        gx[1] += R(-2.0) * w[0] + R(-0.5) * w[1];
        gp[0] += w[0];
    }
    static __device__ __forceinline__ void init_site(R V, R* x) { x[0] = V; x[1] = R(0); }
};

// Scalar test model: dx/dt = p0 sin(x) - x/2 + I.
template <class R> struct Toy1D {
    static constexpr int D = 1, NP = 1;
    static __device__ __forceinline__ void prep(const double* p, R* q) { q[0] = R(p[0]); }
    static __device__ __forceinline__ void rhs(const R* x, const R* p, R I, R* F)
    {
        F[0] = p[0] * sin(x[0]) - R(0.5) * x[0] + I;
    }
    static __device__ __forceinline__ void rhs_vjp(const R* x, const R* p, R I, const R* w, R* gx, R* gp)
    {
        gx[0] += w[0] * (p[0] * cos(x[0]) - R(0.5));
        gp[0] += w[0] * sin(x[0]);
    }
    static __device__ __forceinline__ void init_site(R V, R* x) { x[0] = V; }
};

// pimc_model value of each model type.
template <class Model> struct ModelId;
template <class R> struct ModelId<HH<R>> { static constexpr int value = 0; };
template <class R> struct ModelId<LinGauss<R>> { static constexpr int value = 1; };
template <class R> struct ModelId<Toy1D<R>> { static constexpr int value = 2; };
template <class R> struct ModelId<HHPaper<R>> { static constexpr int value = 3; };

// Model-error discretisations: the explicit one-step RK4 map, or the
// trapezoid rule of Eq. (modelError) with the vector field cached per site.
enum : int { kSchemeRK4 = 0, kSchemeTrapezoid = 1 };
enum : int { kProposalGauss = 0, kProposalUniform = 1 };

// Host-side dispatch of a template FN<Model, R> on (model, prec).
#define PIMC_DISPATCH(FN, ...)                                                            \
    do {                                                                                  \
        if (prec == 0) {                                                                  \
            if (model == 0) return FN<HH<double>, double>(__VA_ARGS__);                   \
            if (model == 1) return FN<LinGauss<double>, double>(__VA_ARGS__);             \
            if (model == 3) return FN<HHPaper<double>, double>(__VA_ARGS__);              \
            return FN<Toy1D<double>, double>(__VA_ARGS__);                                \
        }                                                                                 \
        if (model == 0) return FN<HH<float>, float>(__VA_ARGS__);                         \
        if (model == 1) return FN<LinGauss<float>, float>(__VA_ARGS__);                   \
        if (model == 3) return FN<HHPaper<float>, float>(__VA_ARGS__);                    \
        return FN<Toy1D<float>, float>(__VA_ARGS__);                                      \
    } while (0)

// Forward stage evaluations that keep what the reverse pass can reuse: for a
// model with kReuseRates, rhs_c / rhs_vjp_c and its Cache; otherwise an empty
// record and the plain rhs / rhs_vjp.
template <class Model, class = void> struct ModelCache {
    struct type {};
    template <class R>
    static __device__ __forceinline__ void rhs(const R* x, const R* q, R I, R* F, type&) { Model::rhs(x, q, I, F); }
    template <class R>
    static __device__ __forceinline__ void vjp(const R* x, const R* q, R I, const R* w, R* gx, R* gp, const type&)
    {
        Model::rhs_vjp(x, q, I, w, gx, gp);
    }
};
template <class Model> struct ModelCache<Model, typename std::enable_if<Model::kReuseRates>::type> {
    using type = typename Model::Cache;
    template <class R>
    static __device__ __forceinline__ void rhs(const R* x, const R* q, R I, R* F, type& k) { Model::rhs_c(x, q, I, F, k); }
    template <class R>
    static __device__ __forceinline__ void vjp(const R* x, const R* q, R I, const R* w, R* gx, R* gp, const type& k)
    {
        Model::rhs_vjp_c(x, q, I, w, gx, gp, k);
    }
};

// One classical RK4 step of size dt with the drive held at I:
// f = x + dt/6 (k1 + 2 k2 + 2 k3 + k4).
template <class Model, class R>
__device__ __forceinline__ void rk4_map(const R* x, const R* p, R I, R dt, R* f)
{
    if constexpr (std::is_same<Model, HH<float>>::value) {
        // FP32 HH: the lane form, bit for bit what a paired evaluation gives
        hh_rk4_lanes<float>(x, p, I, dt, __fmul_rn(0.5f, dt), __fdiv_rn(dt, 6.0f), f);
        return;
    }
    constexpr int D = Model::D;
    R k[D], xs[D], acc[D];
    Model::rhs(x, p, I, k);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = k[a]; xs[a] = x[a] + R(0.5) * dt * k[a]; }
    Model::rhs(xs, p, I, k);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = acc[a] + R(2) * k[a]; xs[a] = x[a] + R(0.5) * dt * k[a]; }
    Model::rhs(xs, p, I, k);
#pragma unroll
    for (int a = 0; a < D; ++a) { acc[a] = acc[a] + R(2) * k[a]; xs[a] = x[a] + dt * k[a]; }
    Model::rhs(xs, p, I, k);
#pragma unroll
    for (int a = 0; a < D; ++a) f[a] = x[a] + dt / R(6) * (acc[a] + k[a]);
}

// Reverse mode through the RK4 step: the stage states are recomputed from x
// (nothing stored); once f = f(x) is formed, cot(f, w) fills the cotangent w
// of f (e.g. from the residual x_{n+1} - f), which is then pulled back stage
// by stage -- one forward pass serves both the residual and the adjoint.
// gx, gp are accumulated into; w is left holding the cotangent.
template <class Model, class R, class Cot>
__device__ __forceinline__ void rk4_vjp(const R* x, const R* p, R I, R dt, Cot cot, R* w, R* gx, R* gp)
{
    constexpr int D = Model::D;
    R k1[D], k2[D], k3[D], k4[D], x2[D], x3[D], x4[D];
    typename ModelCache<Model>::type c1, c2, c3, c4;
    ModelCache<Model>::rhs(x, p, I, k1, c1);
#pragma unroll
    for (int a = 0; a < D; ++a) x2[a] = x[a] + R(0.5) * dt * k1[a];
    ModelCache<Model>::rhs(x2, p, I, k2, c2);
#pragma unroll
    for (int a = 0; a < D; ++a) x3[a] = x[a] + R(0.5) * dt * k2[a];
    ModelCache<Model>::rhs(x3, p, I, k3, c3);
#pragma unroll
    for (int a = 0; a < D; ++a) x4[a] = x[a] + dt * k3[a];
    ModelCache<Model>::rhs(x4, p, I, k4, c4);
    R f[D];
#pragma unroll
    for (int a = 0; a < D; ++a)
        f[a] = x[a] + dt / R(6) * (((k1[a] + R(2) * k2[a]) + R(2) * k3[a]) + k4[a]);
    cot(f, w);

    R b1[D], b2[D], b3[D], b4[D], u[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        gx[a] += w[a];
        b1[a] = dt / R(6) * w[a];
        b2[a] = dt / R(3) * w[a];
        b3[a] = dt / R(3) * w[a];
        b4[a] = dt / R(6) * w[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) u[a] = R(0);
    ModelCache<Model>::vjp(x4, p, I, b4, u, gp, c4);
#pragma unroll
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; b3[a] += dt * u[a]; u[a] = R(0); }
    ModelCache<Model>::vjp(x3, p, I, b3, u, gp, c3);
#pragma unroll
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; b2[a] += R(0.5) * dt * u[a]; u[a] = R(0); }
    ModelCache<Model>::vjp(x2, p, I, b2, u, gp, c2);
#pragma unroll
    for (int a = 0; a < D; ++a) { gx[a] += u[a]; b1[a] += R(0.5) * dt * u[a]; u[a] = R(0); }
    ModelCache<Model>::vjp(x, p, I, b1, u, gp, c1);
#pragma unroll
    for (int a = 0; a < D; ++a) gx[a] += u[a];
}

// 1/2 R (d'^2 - d^2) evaluated as 1/2 R (d' - d)(d' + d): no cancellation of
// two large squares (the local change of action of Fig. 1, steps (e)-(f)).
template <class R> __device__ __forceinline__ R sqdiff(R Rw, R dp, R d)
{
    return R(0.5) * Rw * (dp - d) * (dp + d);
}

// Metropolis rule written with E = -log(u), which can be formed before dA is
// known: u < exp(-dA) <=> dA < E (and dA <= 0 < E); NaN compares false.
template <class R> __device__ __forceinline__ R neglog(R u);
template <> __device__ __forceinline__ double neglog<double>(double u) { return -log(u); }
template <> __device__ __forceinline__ float neglog<float>(float u) { return -__logf(u); }

// Metropolis rule, Eq. (Paccept): accept iff dA <= 0 or u < exp(-dA);
// a non-finite dA is a rejection.
template <class R> __device__ __forceinline__ bool metropolis(R dA, R u)
{
    if (!isfinite(dA)) return false;
    if (dA <= R(0)) return true;
    return u < Num<R>::ex(-dA);
}

}  // namespace pimc
