// Whole-path operations outside the sweep: the default initial path, the f
// cache refresh, the global action (FP64 sums), its gradient by reverse mode
// through the RK4 map (stages recomputed) or the trapezoid rule, and path
// layout conversion.
#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "scheme.cuh"

namespace pimc {

template <class Model, class R>
__global__ void init_path_kernel(Ctx c)
{
    constexpr int D = Model::D;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n > c.M) return;
    R x[D];
    Model::init_site(((const R*)c.y)[n], x);
    for (int a = 0; a < D; ++a) ((R*)c.X)[a * c.ldx + n] = x[a];
}

// g_n = f(x_n, p; I_n) (RK4) or F(x_n, p; I_n) (trapezoid) into the current cache.
template <class Model, class R>
__global__ void refresh_cache_kernel(Ctx c)
{
    constexpr int D = Model::D;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= cache_len(c)) return;
    R pr[kMaxP], x[D], f[D];
    Model::prep(c.st->p, pr);
    const Coef<R> kc(c);
    const R* X = (const R*)c.X;
    for (int a = 0; a < D; ++a) x[a] = X[a * c.ldx + n];
    cache_value<Model, R>(c, kc, x, pr, n, f);
    R* F = (R*)c.F[c.st->fidx];
    for (int a = 0; a < D; ++a) F[a * c.ldf + n] = f[a];
}

// Streaming data in one pass (pimc_load_data): the FP64 device copies of y
// and I into the storage precision and, with parameters set, every cached
// value refreshed from the new drive -- site n converts its own drive (the
// trapezoid rule's last site converts I_{M-1} itself: the same value), so no
// thread waits for another's conversion.  The same bits as the conversion
// kernels followed by refresh_cache_kernel.
template <class Model, class R>
__global__ void load_refresh_kernel(Ctx c, const double* y64, const double* I64, int refresh)
{
    constexpr int D = Model::D;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n > c.M) return;
    ((R*)c.y)[n] = R(y64[n]);
    if (n < c.M) ((R*)c.I)[n] = R(I64[n]);
    if (!refresh || n >= cache_len(c)) return;
    R pr[kMaxP], x[D], f[D];
    Model::prep(c.st->p, pr);
    const Coef<R> kc(c);
    const R* X = (const R*)c.X;
    for (int a = 0; a < D; ++a) x[a] = X[a * c.ldx + n];
    cache_value_at<Model, R>(c, kc, x, pr, R(I64[drive_index(c, n)]), f);
    R* F = (R*)c.F[c.st->fidx];
    for (int a = 0; a < D; ++a) F[a * c.ldf + n] = f[a];
}

// Path element (a, n) from either the handle's storage or a dense FP64 array.
template <class R>
__device__ __forceinline__ R path_at(const Ctx& c, const double* Xe, int a, int64_t n)
{
    return Xe ? R(Xe[a * (c.M + 1) + n]) : ((const R*)c.X)[a * c.ldx + n];
}

// A = A_o + A_f (beta = 1): out = (A, A_o, A_f).  Per-site residuals in R,
// squares accumulated in FP64.
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) action_kernel(Ctx c, const double* Xe, const double* pe, double* out)
{
    constexpr int D = Model::D;
    __shared__ double wsum[2][kBlock / 32];
    __shared__ int last;
    __shared__ double res[2];
    R pr[kMaxP];
    Model::prep(pe ? pe : c.st->p, pr);
    const Coef<R> kc(c);
    double v[2] = {0.0, 0.0};
    const R* y = (const R*)c.y;
    for (int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x; n <= c.M; n += (int64_t)gridDim.x * kBlock) {
        R x[D];
        for (int a = 0; a < D; ++a) x[a] = path_at<R>(c, Xe, a, n);
        if (n >= 1) {
            const R d = x[0] - y[n];
            v[0] += 0.5 * c.Rm * (double)d * (double)d;
        }
        if (n < c.M) {
            R g[D], g1[D], x1[D];
            for (int a = 0; a < D; ++a) { x1[a] = path_at<R>(c, Xe, a, n + 1); g1[a] = R(0); }
            cache_value<Model, R>(c, kc, x, pr, n, g);
            if (c.scheme != kSchemeRK4) cache_value<Model, R>(c, kc, x1, pr, n + 1, g1);
            for (int a = 0; a < D; ++a) {
                const R e = eps_of<R>(c, kc, x[a], x1[a], g[a], g1[a]);
                v[1] += 0.5 * c.Rf[a] * (double)e * (double)e;
            }
        }
    }
    grid_sums_last_block<2>(c, v, res, wsum, &last);
    if (last && threadIdx.x == 0) {
        out[0] = res[0] + res[1];
        out[1] = res[0];
        out[2] = res[1];
    }
}

// Gradient of A_o + beta A_f, in gather form: a CTA owns T <= kBlock - 1
// sites n0..n0+T-1 a tile and thread i <= T takes model term n0 - 1 + i
// (term_adjoint; thread 0 recomputes the term of the tile before, whose
// cotangent reaches x_{n0}).  The owner of site n writes
// g_n = Rm (x_{n,0} - y_n) e_0 + own_n + nxt_{n-1}, the per-term pieces in R
// added in FP64 -- every element written once, no atomics, no zeroing pass.
// dA/dp = sum over terms of their gp, FP64 sums (fixed order).
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) grad_kernel(Ctx c, const double* Xe, const double* pe, double beta,
                                                      double* gX, double* gp, int T)
{
    constexpr int D = Model::D, NP = Model::NP;
    __shared__ R xs[D][kBlock + 1];
    __shared__ R nxs[D][kBlock];
    __shared__ double wsum[NP][kBlock / 32];
    __shared__ int last;
    __shared__ double res[NP];
    R pr[kMaxP], wr[kMaxD];
    Model::prep(pe ? pe : c.st->p, pr);
    const Coef<R> kc(c);
#pragma unroll
    for (int a = 0; a < kMaxD; ++a) wr[a] = R(beta * c.Rf[a]);
    const R* y = (const R*)c.y;
    const R* I = (const R*)c.I;
    const int i = threadIdx.x;
    const int64_t ld = c.M + 1, ntile = (ld + T - 1) / T;
    double vp[NP];
    for (int l = 0; l < NP; ++l) vp[l] = 0.0;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t n0 = tile * T, k = n0 - 1 + i;
        const bool has_x = i <= T && k >= 0 && k <= c.M, term = i <= T && k >= 0 && k < c.M;
        const bool owner = i >= 1 && i <= T && k <= c.M;
        if (has_x)
            for (int a = 0; a < D; ++a) xs[a][i] = path_at<R>(c, Xe, a, k);
        if (i == 0 && n0 + T <= c.M)
            for (int a = 0; a < D; ++a) xs[a][T + 1] = path_at<R>(c, Xe, a, n0 + T);
        __syncthreads();
        R own[D];
        for (int a = 0; a < D; ++a) own[a] = R(0);
        if (term) {
            R x[D], x1[D], e[D], nxt[D], gpl[kMaxP];
            for (int a = 0; a < D; ++a) {
                x[a] = xs[a][i];
                x1[a] = xs[a][i + 1];
            }
            const R In = I[k];
            const R In1 = c.scheme == kSchemeRK4 ? R(0) : I[k + 1 < c.M ? k + 1 : c.M - 1];
            term_adjoint<Model, R>(c, kc, wr, x, x1, pr, In, In1, e, own, nxt, gpl);
            for (int a = 0; a < D; ++a) nxs[a][i] = nxt[a];
            if (i >= 1)
                for (int l = 0; l < NP; ++l) vp[l] += (double)gpl[l];
        }
        __syncthreads();
        if (owner) {
            double g[D];
            for (int a = 0; a < D; ++a) g[a] = (double)own[a];
            if (k >= 1) {
                g[0] = c.Rm * (double)(xs[0][i] - y[k]) + g[0];
                for (int a = 0; a < D; ++a) g[a] += (double)nxs[a][i - 1];
            }
            for (int a = 0; a < D; ++a) gX[a * ld + k] = g[a];
        }
        if (tile + gridDim.x < ntile) __syncthreads();  // xs and nxs are reused by the next tile
    }
    grid_sums_last_block<NP>(c, vp, res, wsum, &last);
    if (last && threadIdx.x == 0)
        for (int l = 0; l < NP; ++l) gp[l] = res[l];
}

// Ensemble forecast (Sec. 6): member e (one thread) integrates
// x_{k+1} = f(x_k, p; I_k) + xi_k, xi_{k,a} ~ N(0, 1/Rf_a) (none where Rf_a = 0 or
// when noise == 0) from the current x_M; normals are Philox draws keyed by
// (member, step, kind 4 | pair, chain).
template <class Model, class R>
__global__ void forecast_kernel(Ctx c, int64_t n_steps, const double* I, int n_ens, int noise, uint64_t seed,
                                double* out)
{
    constexpr int D = Model::D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ens) return;
    R q[kMaxP], x[D], fx[D];
    Model::prep(c.st->p, q);
    const R* X = (const R*)c.X;
    double* o = out + (int64_t)e * D * (n_steps + 1);
    for (int a = 0; a < D; ++a) {
        x[a] = X[a * c.ldx + c.M];
        o[(int64_t)a * (n_steps + 1)] = (double)x[a];
    }
    for (int64_t k = 0; k < n_steps; ++k) {
        rk4_map<Model, R>(x, q, R(I[k]), R(c.dt), fx);
        if (noise) {
            for (int pair = 0; 2 * pair < D; ++pair) {
                double z0, z1;
                Num<double>::box_muller(draw_block(seed, c.chain, (uint64_t)k, (uint32_t)e, 4u, (uint32_t)pair), z0, z1);
                if (c.Rf[2 * pair] > 0.0) fx[2 * pair] += R(z0 / sqrt(c.Rf[2 * pair]));
                if (2 * pair + 1 < D && c.Rf[2 * pair + 1] > 0.0) fx[2 * pair + 1] += R(z1 / sqrt(c.Rf[2 * pair + 1]));
            }
        }
        for (int a = 0; a < D; ++a) {
            x[a] = fx[a];
            o[(int64_t)a * (n_steps + 1) + k + 1] = (double)x[a];
        }
    }
}

template <class Model, class R>
static cudaError_t forecast_t(const Ctx& c, int64_t n_steps, const double* I, int n_ens, int noise, uint64_t seed,
                              double* out, cudaStream_t s)
{
    forecast_kernel<Model, R><<<(n_ens + 127) / 128, 128, 0, s>>>(c, n_steps, I, n_ens, noise, seed, out);
    return cudaGetLastError();
}

template <class R>
__global__ void convert_kernel(const double* src, R* dst, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = R(src[i]);
}

// Handle storage <-> dense FP64 [D][M+1].
template <class R>
__global__ void path_io_kernel(Ctx c, int D, double* dense, int to_state)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)D * (c.M + 1);
    if (i >= tot) return;
    const int64_t a = i / (c.M + 1), n = i - a * (c.M + 1);
    R* X = (R*)c.X;
    if (to_state) X[a * c.ldx + n] = R(dense[i]);
    else dense[i] = (double)X[a * c.ldx + n];
}

// ---------------------------------------------------------------------------

template <class Model, class R> static cudaError_t init_t(const Ctx& c, cudaStream_t s)
{
    init_path_kernel<Model, R><<<(unsigned)((c.M + 1 + 255) / 256), 256, 0, s>>>(c);
    return cudaGetLastError();
}
template <class Model, class R>
static cudaError_t load_refresh_t(const Ctx& c, const double* y64, const double* I64, int refresh, cudaStream_t s)
{
    load_refresh_kernel<Model, R><<<(unsigned)((c.M + 1 + 255) / 256), 256, 0, s>>>(c, y64, I64, refresh);
    return cudaGetLastError();
}
template <class Model, class R> static cudaError_t refresh_t(const Ctx& c, cudaStream_t s)
{
    // every cached value: M + 1 of them under the trapezoid rule
    refresh_cache_kernel<Model, R><<<(unsigned)((c.M + 1 + 255) / 256), 256, 0, s>>>(c);
    return cudaGetLastError();
}
static int reduce_grid(int64_t M)
{
    int64_t g = (M + 1 + kBlock - 1) / kBlock;
    if (g > kMaxGrid) g = kMaxGrid;
    return (int)(g < 1 ? 1 : g);
}
template <class Model, class R>
static cudaError_t action_t(const Ctx& c, const double* Xe, const double* pe, double* out, cudaStream_t s)
{
    action_kernel<Model, R><<<reduce_grid(c.M), kBlock, 0, s>>>(c, Xe, pe, out);
    return cudaGetLastError();
}
template <class Model, class R>
static cudaError_t grad_t(const Ctx& c, const double* Xe, const double* pe, double beta, double* gX, double* gp,
                          cudaStream_t s)
{
    // sites a tile: spread over every SM while that leaves at most kBlock - 1 a tile
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t T = (c.M + 1 + sms - 1) / (sms > 0 ? sms : 1);
    T = T < 1 ? 1 : (T > kBlock - 1 ? kBlock - 1 : T);
    const int64_t ntile = (c.M + 1 + T - 1) / T;
    const unsigned grid = (unsigned)(ntile < kMaxGrid ? ntile : kMaxGrid);
    grad_kernel<Model, R><<<grid, kBlock, 0, s>>>(c, Xe, pe, beta, gX, gp, (int)T);
    return cudaGetLastError();
}



cudaError_t launch_init_path(int model, int prec, const Ctx& c, cudaStream_t s) { PIMC_DISPATCH(init_t, c, s); }
cudaError_t launch_refresh_cache(int model, int prec, const Ctx& c, cudaStream_t s)
{
    PIMC_DISPATCH(refresh_t, c, s);
}
cudaError_t launch_load_refresh(int model, int prec, const Ctx& c, const double* y64, const double* I64, int refresh,
                                cudaStream_t s)
{
    PIMC_DISPATCH(load_refresh_t, c, y64, I64, refresh, s);
}
cudaError_t launch_action(int model, int prec, const Ctx& c, const double* X_ext, const double* p_ext, double* out,
                          cudaStream_t s)
{
    PIMC_DISPATCH(action_t, c, X_ext, p_ext, out, s);
}
cudaError_t launch_grad(int model, int prec, const Ctx& c, const double* X_ext, const double* p_ext, double beta,
                        double* gX, double* gp, cudaStream_t s)
{
    PIMC_DISPATCH(grad_t, c, X_ext, p_ext, beta, gX, gp, s);
}
cudaError_t launch_forecast(int model, int prec, const Ctx& c, int64_t n_steps, const double* I, int n_ens,
                            int noise, uint64_t seed, double* out, cudaStream_t s)
{
    PIMC_DISPATCH(forecast_t, c, n_steps, I, n_ens, noise, seed, out, s);
}

cudaError_t launch_convert(int prec, const double* src, void* dst, int64_t n, cudaStream_t s)
{
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (grid == 0) return cudaSuccess;
    if (prec == 0) convert_kernel<double><<<grid, 256, 0, s>>>(src, (double*)dst, n);
    else convert_kernel<float><<<grid, 256, 0, s>>>(src, (float*)dst, n);
    return cudaGetLastError();
}

cudaError_t launch_path_io(int prec, const Ctx& c, int D, double* dense, int to_state, cudaStream_t s)
{
    const int64_t tot = (int64_t)D * (c.M + 1);
    const unsigned grid = (unsigned)((tot + 255) / 256);
    if (prec == 0) path_io_kernel<double><<<grid, 256, 0, s>>>(c, D, dense, to_state);
    else path_io_kernel<float><<<grid, 256, 0, s>>>(c, D, dense, to_state);
    return cudaGetLastError();
}

// Throughput probe of the FP32 HH map alone: every thread iterates x <- f(x)
// `iters` times from registers (no memory traffic, no synchronisation), one
// state (T = float) or two (T = float2, the packed lane form) a thread; the
// sum of the final states goes to out[thread] so nothing is optimised away.
// The rate it reaches is the ceiling of a sweep's map arithmetic.
template <class T, int MINB>
__global__ void __launch_bounds__(256, MINB) map_rate_kernel(int64_t iters, float* out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const float v0 = -65.0f + 0.001f * (float)(t & 1023), v1 = -60.0f + 0.001f * (float)(t & 511);
    T x[4];
    if constexpr (std::is_same<T, float2>::value) {
        x[0] = make_float2(v0, v1);
        x[1] = make_float2(0.05f, 0.06f);
        x[2] = make_float2(0.6f, 0.58f);
        x[3] = make_float2(0.32f, 0.33f);
    } else {
        x[0] = v0;
        x[1] = 0.05f;
        x[2] = 0.6f;
        x[3] = 0.32f;
    }
    const float qs[kMaxP] = {120.f, 36.f, 0.3f, 50.f, -77.f, -54.4f, 1.f, 1.f};
    T q[kMaxP];
#pragma unroll
    for (int j = 0; j < kMaxP; ++j) q[j] = splat<T>(qs[j]);
    const float dt = 0.02f;
    const T I = splat<T>(10.0f), dtv = splat<T>(dt), hdt = splat<T>(__fmul_rn(0.5f, dt)),
            sdt = splat<T>(__fdiv_rn(dt, 6.0f));
    for (int64_t it = 0; it < iters; ++it) {
        T f[4];
        hh_rk4_lanes<T>(x, q, I, dtv, hdt, sdt, f);
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = f[a];
    }
    float acc = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        if constexpr (std::is_same<T, float2>::value) acc += x[a].x + x[a].y;
        else acc += x[a];
    }
    out[t] = acc;
}

template <class T, int MINB>
static cudaError_t map_rate_t(int n_sm, int64_t iters, float* out, cudaStream_t s)
{
    map_rate_kernel<T, MINB><<<n_sm * MINB, 256, 0, s>>>(iters, out);
    return cudaGetLastError();
}

// The FP64 form of the same probe: the FP64 HH map (rk4_map<HH<double>>, the
// map of the plain FP64 sweep) iterated from registers, one state a thread.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) map_rate_fp64_kernel(int64_t iters, float* out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[4] = {-65.0 + 0.001 * (double)(t & 1023), 0.05, 0.6, 0.32};
    const double ps[kMaxP] = {120.0, 36.0, 0.3, 50.0, -77.0, -54.4, 1.0, 0.0};
    double q[kMaxP];
    HH<double>::prep(ps, q);
    for (int64_t it = 0; it < iters; ++it) {
        double f[4];
        rk4_map<HH<double>, double>(x, q, 10.0, 0.02, f);
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = f[a];
    }
    out[t] = (float)(x[0] + x[1] + x[2] + x[3]);
}

cudaError_t launch_map_rate(int packed, int ctas_per_sm, int n_sm, int64_t iters, float* out, cudaStream_t s)
{
    if (packed == 2) {  // FP64
        if (ctas_per_sm == 1) map_rate_fp64_kernel<1><<<n_sm, 256, 0, s>>>(iters, out);
        else if (ctas_per_sm == 2) map_rate_fp64_kernel<2><<<n_sm * 2, 256, 0, s>>>(iters, out);
        else map_rate_fp64_kernel<4><<<n_sm * 4, 256, 0, s>>>(iters, out);
        return cudaGetLastError();
    }
    if (packed) {
        if (ctas_per_sm == 1) return map_rate_t<float2, 1>(n_sm, iters, out, s);
        if (ctas_per_sm == 2) return map_rate_t<float2, 2>(n_sm, iters, out, s);
        return map_rate_t<float2, 4>(n_sm, iters, out, s);
    }
    if (ctas_per_sm == 1) return map_rate_t<float, 1>(n_sm, iters, out, s);
    if (ctas_per_sm == 2) return map_rate_t<float, 2>(n_sm, iters, out, s);
    return map_rate_t<float, 4>(n_sm, iters, out, s);
}

}  // namespace pimc
