// Whole-path Hybrid Monte Carlo (X and the free parameters move together),
// driven by the reverse-mode gradient of the action through the RK4 map.  The
// paper points to gradient-using proposals (Sec. 3.1; Hybrid Monte Carlo is
// named among the methods that sample exp(-A)); this is that form.
//
// One trajectory is a fixed sequence of launches on the handle's stream:
// begin (state -> positions Q_0, momenta P drawn, kinetic energy K0, step
// jitter and accept uniform), then n_leap + 1 leapfrog kernels -- step
// k evaluates the gradient at Q_k and applies P -= c_k eps g (c = 1/2 at both
// ends, 1 between) and Q_{k+1} = Q_k + eps invm P, with the action at Q_0 and
// at Q_L and the final kinetic energy and accept test folded into the end
// steps -- then commit (accepted Q_L -> state, f cache refreshed), statistics
// and the counter tick.  The host captures it once in a CUDA graph and
// replays the graph per trajectory; every decision stays on the device.
#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "scheme.cuh"
#include "stats.cuh"

namespace pimc {

// Programmatic dependent launch between the kernels of a trajectory: each
// kernel lets the next one start at once (its CTAs become resident and run
// up to pdl_wait while this one finishes), and pdl_wait returns when the
// previous kernel has completed and its writes are visible.  Without the
// launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Site positions, momenta and step scales eps invm of the HMC state.  FP64
// form: doubles.  FP32-mixed form: an unevaluated sum hi + lo of two floats
// (about 48 significant bits) in the same 8 bytes, so the per-site leapfrog
// arithmetic runs on the FP32 pipe -- Knuth's two-sum, Dekker's fast
// two-sum and an FMA-exact product (the FP64 pipe issues a warp instruction
// in about 64 cycles on this part).  x() is the value in the arithmetic
// type (hi, the float nearest hi + lo); parameter slots stay FP64.
template <class R> struct HmcVal;
template <> struct HmcVal<double> {
    using S = double;
    static __device__ __forceinline__ S load(const double* b, int64_t j) { return b[j]; }
    static __device__ __forceinline__ void store(double* b, int64_t j, S v) { b[j] = v; }
    static __device__ __forceinline__ double x(S v) { return v; }
    static __device__ __forceinline__ double dbl(S v) { return v; }
    static __device__ __forceinline__ S of(double v) { return v; }
    static __device__ __forceinline__ S kick(S p, S c, double g) { return p - c * g; }  // p - c g
    static __device__ __forceinline__ S drift(S q, S e, S p) { return q + e * p; }      // q + e p
};
template <> struct HmcVal<float> {
    using S = float2;
    static __device__ __forceinline__ S load(const double* b, int64_t j)
    {
        return reinterpret_cast<const float2*>(b)[j];
    }
    static __device__ __forceinline__ void store(double* b, int64_t j, S v) { reinterpret_cast<float2*>(b)[j] = v; }
    static __device__ __forceinline__ float x(S v) { return v.x; }
    static __device__ __forceinline__ double dbl(S v) { return (double)v.x + (double)v.y; }
    static __device__ __forceinline__ S of(double v)
    {
        const float h = (float)v;
        return make_float2(h, (float)(v - (double)h));  // v - h is exact in FP64
    }
    // s + e = a + b exactly (Knuth)
    static __device__ __forceinline__ S two_sum(float a, float b)
    {
        const float s = a + b, bb = s - a;
        return make_float2(s, (a - (s - bb)) + (b - bb));
    }
    // s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
    static __device__ __forceinline__ S fast_two_sum(float a, float b)
    {
        const float s = a + b;
        return make_float2(s, b - (s - a));
    }
    static __device__ __forceinline__ S add(S a, S b)
    {
        const S s = two_sum(a.x, b.x);
        return fast_two_sum(s.x, s.y + (a.y + b.y));
    }
    static __device__ __forceinline__ S mul(S a, float b)
    {
        const float p = a.x * b;
        return fast_two_sum(p, fmaf(a.y, b, fmaf(a.x, b, -p)));
    }
    static __device__ __forceinline__ S mul(S a, S b)
    {
        const float p = a.x * b.x;
        return fast_two_sum(p, fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p))));
    }
    static __device__ __forceinline__ S kick(S p, S c, float g)
    {
        const S t = mul(c, g);
        return add(p, make_float2(-t.x, -t.y));
    }
    static __device__ __forceinline__ S drift(S q, S e, S p) { return add(q, mul(e, p)); }
};

// Q = current state (FP64), P_j = z_j / sqrt(invm_j) (fixed parameters: 0),
// K0 = 1/2 sum P^2 invm; step jitter eps (0.8 + 0.4 u') and -log u of the
// accept uniform from the trajectory's accept block.  Components 2q and
// 2q + 1 take the two normals of Philox block q (one thread a pair).
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_begin_kernel(Ctx c, HmcScalars* hs, double* Q, double* P, double* EM,
                                                           const double* invm, double eps, uint64_t seed)
{
    using V = HmcVal<R>;
    constexpr int D = Model::D, NP = Model::NP;
    __shared__ double wsum[1][kBlock / 32];
    __shared__ int last;
    const int64_t nx = (int64_t)D * (c.M + 1), nq = nx + NP, npair = (nq + 1) / 2;
    pdl_trigger();
    const uint64_t traj = (uint64_t)c.st->sweep;
    const uint4 wacc = draw_block(seed, c.chain, traj, 0u, kKindHmcAcc, 0u);
    const double eps_t = eps * (0.8 + 0.4 * u01d(wacc.z, wacc.w));  // this trajectory's step
    double v[1] = {0.0};
    for (int64_t q = (int64_t)blockIdx.x * kBlock + threadIdx.x; q < npair; q += (int64_t)gridDim.x * kBlock) {
        double z[2];
        Num<double>::box_muller(draw_block(seed, c.chain, traj, (uint32_t)q, kKindHmcMom, 0u), z[0], z[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t j = 2 * q + h;
            if (j >= nq) break;
            if (j < nx) {
                const int64_t a = j / (c.M + 1), n = j - a * (c.M + 1);
                V::store(Q, j, V::of((double)((const R*)c.X)[a * c.ldx + n]));
                const typename V::S pj = V::of(z[h] / sqrt(invm[j]));
                V::store(P, j, pj);
                V::store(EM, j, V::of(eps_t * invm[j]));
                const double pd = V::dbl(pj);
                v[0] += 0.5 * pd * pd * invm[j];
            } else {
                const int l = (int)(j - nx);
                Q[j] = c.st->p[l];
                const double pj = ((c.st->free_mask >> l) & 1u) ? z[h] / sqrt(invm[j]) : 0.0;
                P[j] = pj;
                hs->pp[0][l] = pj;  // P_p(0), read by the leapfrog steps
                v[0] += 0.5 * pj * pj * invm[j];
            }
        }
    }
    double k0[1];
    grid_sums_last_block<1>(c, v, k0, wsum, &last);
    if (last && threadIdx.x == 0) {
        hs->K0 = k0[0];
        hs->E = -log(u01d(wacc.x, wacc.y));
        hs->eps = eps_t;
        hs->oob = 0;
        hs->accept = 0;  // set by the last leapfrog step
    }
}

// Leapfrog step k (0..L) fused with the adjoint, in gather form: a CTA owns
// T <= kBlock - 1 sites n0..n0+T-1 a tile and thread i <= T evaluates model
// term n0 - 1 + i (thread 0 recomputes the term of the tile before, whose
// cotangent reaches x_{n0}), so every gradient element is one sum
// g_n = Rm (x_{n,0} - y_n) + own_n + nxt_{n-1} formed by its owner (no atomics
// and no zeroing pass).  Then P_n -= c_k eps g_n (c = 1/2 at k = 0 and k = L,
// else 1) and, for k < L, Q_{k+1,n} = Q_{k,n} + eps invm_n P_n into the other
// position buffer.  The parameter gradient dA/dp at Q_k is left as fixed-order
// CTA sums in the arithmetic type; step k + 1 finishes step k's parameter
// move: warp 0 of every CTA adds the CTA sums in the same fixed order, forms
// P_p(k + 1/2) and Q_p(k + 1) -- identical in every CTA -- and prepares them
// for its own terms (CTA 0 stores them; a parameter leaving its box marks the
// trajectory).  So only the last step needs a grid-wide ticket: its last CTA
// forms P_p at Q_L, the energies (A_o and A_f at Q_0 and Q_L, summed from
// the end steps' CTA sums, and K1 = 1/2 P^2 invm) and the accept test
// dH = (A1 + K1) - (A0 + K0) < -log u.  Every global load a tile needs is
// issued before its first barrier (the kernel is latency-bound at one warp
// per scheduler); loads of data no kernel of the trajectory writes (drive,
// observations, inverse masses, bounds) precede the wait on the step before.
//
// Buffers by step parity: Qk = Q_(k&1) (sites of Q_k; CTA 0 writes Q_p(k) into
// its parameter slots), Qn = Q_((k+1)&1) (sites of Q_{k+1} written here; its
// parameter slots hold Q_p(k-1)); CTA sums of step k in c.red set k & 1,
// quantity-major so a warp reads 32 CTAs' sums of one quantity coalesced:
// rows 0..NP-1 dA/dp (in R); 8..10 A_o, A_f, kinetic energy of the last
// step; 11..12 A_o, A_f of step 0, in set 0 (FP64); a row is kMaxGrid long.
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_leap_kernel(Ctx c, HmcScalars* hs, double* Qk, double* Qn, double* P,
                                                          const double* EM, const double* invm, int k, int n_leap,
                                                          int T)
{
    using V = HmcVal<R>;
    using S = typename V::S;
    constexpr int D = Model::D, NP = Model::NP, NW = kBlock / 32;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ R xs[D][kBlock + 1];
    __shared__ R nxs[D][kBlock];
    __shared__ R wp[NP][NW];
    __shared__ double we[3][NW];
    __shared__ R prs[kMaxP];
    __shared__ double tot[5], kin[NP];
    __shared__ int last;
    const bool first = k == 0, fin = k == n_leap, ends = first || fin;
    const double fa = ends ? 0.5 : 1.0;
    const bool rk4 = c.scheme == kSchemeRK4;
    const int i = threadIdx.x, lane = i & 31, wid = i >> 5;
    const int64_t ld = c.M + 1, nx = (int64_t)D * ld;
    const R* y = (const R*)c.y;
    const R* I = (const R*)c.I;
    double* red_own = c.red + (int64_t)(k & 1) * kMaxGrid * kRedStride;
    const double* red_prev = c.red + (int64_t)((k + 1) & 1) * kMaxGrid * kRedStride;
    pdl_trigger();
    const Coef<R> kc(c);
    // lane l < NP of warp 0 carries parameter l
    double p_im = 0.0, p_lo = 0.0, p_hi = 0.0;
    bool p_moving = false;
    if (i < NP) {
        p_im = invm[nx + i];
        p_lo = c.st->lo[i];
        p_hi = c.st->hi[i];
        p_moving = (c.st->free_mask >> i) & 1u;
    }
    const int64_t ntile = (ld + T - 1) / T;
    // per-site data no kernel of the trajectory writes
    auto load_fixed = [&](int64_t tile, double* im, R& yk, R& In, R& In1) {
        const int64_t kk = tile * T - 1 + i;
        const bool term = i <= T && kk >= 0 && kk < c.M, owner = i >= 1 && i <= T && kk <= c.M;
#pragma unroll
        for (int a = 0; a < D; ++a) im[a] = (owner && fin) ? invm[a * ld + kk] : 0.0;  // K1 of the last step
        yk = (owner && kk >= 1) ? y[kk] : R(0);
        In = term ? I[kk] : R(0);
        In1 = (term && !rk4) ? I[kk + 1 < c.M ? kk + 1 : c.M - 1] : R(0);
    };
    double im0[D];
    R yk0, In0, In10;
    load_fixed(blockIdx.x, im0, yk0, In0, In10);
    pdl_wait();  // the previous step's positions, momenta and CTA sums
    const double eps = hs->eps;
    const S c_kick = V::of(fa * eps);

    double p_pj = 0.0;  // lane l < NP of warp 0: P_p(k - 1/2) (P_p(0) at k = 0)
    R pr[kMaxP];
    R vp[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) vp[l] = R(0);
    double ve[3] = {0.0, 0.0, 0.0};  // A_o, A_f, kinetic energy of the sites
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const bool head = tile == blockIdx.x;
        const int64_t n0 = tile * T, kk = n0 - 1 + i;
        const bool has_x = i <= T && kk >= 0 && kk <= c.M, term = i <= T && kk >= 0 && kk < c.M;
        const bool owner = i >= 1 && i <= T && kk <= c.M;
        const bool halo = i == 0 && n0 + T <= c.M;
        S q[D], pv[D], em[D], qh[D];
        double im[D];
        R yk = yk0, In = In0, In1 = In10;
#pragma unroll
        for (int a = 0; a < D; ++a) im[a] = im0[a];
        if (!head) load_fixed(tile, im, yk, In, In1);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            q[a] = has_x ? V::load(Qk, a * ld + kk) : S{};
            qh[a] = halo ? V::load(Qk, a * ld + n0 + T) : S{};
            pv[a] = owner ? V::load(P, a * ld + kk) : S{};
            em[a] = (owner && !fin) ? V::load(EM, a * ld + kk) : S{};
        }
        if (head && wid == 0) {
            // the parameters at Q_k: finish step k - 1's parameter move
            double q_l = 0.0;
            if (first) {
                if (lane < NP) {
                    q_l = Qk[nx + lane];
                    p_pj = hs->pp[0][lane];
                }
            } else {
                double pj = 0.0, qp = 0.0;
                if (lane < NP) {
                    pj = hs->pp[(k + 1) & 1][lane];  // P_p(k - 3/2)
                    qp = Qn[nx + lane];              // Q_p(k - 1)
                }
                // lane t adds the sums of CTAs t, t + 32, ... in that order; the
                // loads of up to kSumUnroll CTAs a lane are in flight together
                constexpr int kSumUnroll = 8;
                R tg[NP];
#pragma unroll
                for (int l = 0; l < NP; ++l) tg[l] = R(0);
                for (int b0 = 0; b0 < (int)gridDim.x; b0 += 32 * kSumUnroll) {
                    R part[kSumUnroll][NP];
#pragma unroll
                    for (int u = 0; u < kSumUnroll; ++u) {
                        const int b = b0 + 32 * u + lane;
#pragma unroll
                        for (int l = 0; l < NP; ++l)
                            part[u][l] = b < (int)gridDim.x ? __ldcg((const R*)red_prev + l * kMaxGrid + b) : R(0);
                    }
#pragma unroll
                    for (int u = 0; u < kSumUnroll; ++u) {
#pragma unroll
                        for (int l = 0; l < NP; ++l) tg[l] += part[u][l];
                    }
                }
                R gl = R(0);
#pragma unroll
                for (int l = 0; l < NP; ++l) {
                    const R t = __shfl_sync(kFull, warp_sum<R>(tg[l]), 0);
                    if (lane == l) gl = t;
                }
                if (lane < NP) {
                    const double fprev = (k == 1) ? 0.5 : 1.0;
                    if (p_moving) {
                        pj = pj - fprev * eps * (double)gl;
                        qp = qp + eps * p_im * pj;
                    }
                    q_l = qp;
                    p_pj = pj;
                    if (blockIdx.x == 0) {
                        hs->pp[k & 1][lane] = pj;
                        Qk[nx + lane] = qp;
                        if (p_moving && !(qp >= p_lo && qp <= p_hi)) hs->oob = 1;
                    }
                }
            }
            double qv[kMaxP];
#pragma unroll
            for (int l = 0; l < kMaxP; ++l) qv[l] = __shfl_sync(kFull, q_l, l);
            if (lane == 0) Model::prep(qv, prs);
        }
        if (has_x) {
#pragma unroll
            for (int a = 0; a < D; ++a) xs[a][i] = V::x(q[a]);
        }
        if (halo) {
#pragma unroll
            for (int a = 0; a < D; ++a) xs[a][T + 1] = V::x(qh[a]);
        }
        __syncthreads();
        if (head) {
#pragma unroll
            for (int l = 0; l < kMaxP; ++l) pr[l] = prs[l];
        }
        R own[D];
#pragma unroll
        for (int a = 0; a < D; ++a) own[a] = R(0);
        if (term) {
            R x[D], x1[D], e[D], nxt[D], gpl[kMaxP];
#pragma unroll
            for (int a = 0; a < D; ++a) {
                x[a] = xs[a][i];
                x1[a] = xs[a][i + 1];
            }
            term_adjoint<Model, R>(c, kc, kc.Rf, x, x1, pr, In, In1, e, own, nxt, gpl);
#pragma unroll
            for (int a = 0; a < D; ++a) nxs[a][i] = nxt[a];
            if (i >= 1) {
#pragma unroll
                for (int l = 0; l < NP; ++l) vp[l] += gpl[l];
                if (ends) {
#pragma unroll
                    for (int a = 0; a < D; ++a) ve[1] += 0.5 * c.Rf[a] * (double)e[a] * (double)e[a];
                }
            }
        }
        __syncthreads();
        if (owner) {
            R g[D];
#pragma unroll
            for (int a = 0; a < D; ++a) g[a] = own[a];
            if (kk >= 1) {
                const R d = xs[0][i] - yk;
                g[0] = kc.Rm * d + g[0];
                if (ends) ve[0] += 0.5 * c.Rm * (double)d * (double)d;
#pragma unroll
                for (int a = 0; a < D; ++a) g[a] += nxs[a][i - 1];
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const int64_t j = a * ld + kk;
                const S pj = V::kick(pv[a], c_kick, g[a]);
                V::store(P, j, pj);
                if (fin) {
                    const double pd = V::dbl(pj);
                    ve[2] += 0.5 * pd * pd * im[a];
                } else {
                    V::store(Qn, j, V::drift(q[a], em[a], pj));
                }
            }
        }
        if (tile + gridDim.x < ntile) __syncthreads();  // xs and nxs are reused by the next tile
    }

    // CTA sums: parameter gradient in R, energies in FP64 (end steps only)
#pragma unroll
    for (int l = 0; l < NP; ++l) {
        const R w = warp_sum<R>(vp[l]);
        if (lane == 0) wp[l][wid] = w;
    }
    if (ends) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double w = warp_sum<double>(ve[q]);
            if (lane == 0) we[q][wid] = w;
        }
    }
    __syncthreads();
    if (i < NP) {
        R t = R(0);
        for (int w = 0; w < NW; ++w) t += wp[i][w];
        ((R*)red_own)[i * kMaxGrid + blockIdx.x] = t;
    } else if (ends && i >= 32 && i < 35) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += we[i - 32][w];
        if (fin) red_own[(8 + (i - 32)) * kMaxGrid + blockIdx.x] = t;
        if (first && i < 34) red_own[(11 + (i - 32)) * kMaxGrid + blockIdx.x] = t;  // A_o, A_f at Q_0
    }
    if (!fin) return;

    __syncthreads();
    if (i == 0) {
        __threadfence();  // the CTA's slot writes (ordered by the barrier) before the ticket
        last = (atomicAdd(c.ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();

    // grid totals: each thread a fixed stride of CTAs, then the warp tree, then the warps
    R tg[NP];
    double te[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int l = 0; l < NP; ++l) tg[l] = R(0);
    for (unsigned b = i; b < gridDim.x; b += kBlock) {
#pragma unroll
        for (int l = 0; l < NP; ++l) tg[l] += __ldcg((const R*)red_own + l * kMaxGrid + b);
#pragma unroll
        for (int q = 0; q < 3; ++q) te[q] += __ldcg(red_own + (8 + q) * kMaxGrid + b);
        te[3] += __ldcg(c.red + 11 * kMaxGrid + b);  // set 0: step 0's action
        te[4] += __ldcg(c.red + 12 * kMaxGrid + b);
    }
#pragma unroll
    for (int l = 0; l < NP; ++l) {
        const R w = warp_sum<R>(tg[l]);
        if (lane == 0) wp[l][wid] = w;
    }
    __shared__ double wt[5][NW];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double w = warp_sum<double>(te[q]);
        if (lane == 0) wt[q][wid] = w;
    }
    __syncthreads();
    if (i < NP) {
        R gsum = R(0);
        for (int w = 0; w < NW; ++w) gsum += wp[i][w];
        const double pj = p_moving ? p_pj - fa * eps * (double)gsum : p_pj;  // P_p(L)
        kin[i] = 0.5 * pj * pj * p_im;
    } else if (i >= 32 && i < 37) {
        double t = 0.0;
        for (int w = 0; w < NW; ++w) t += wt[i - 32][w];
        tot[i - 32] = t;
    }
    __syncthreads();
    if (i == 0) {
        hs->A0[0] = tot[3] + tot[4];
        hs->A0[1] = tot[3];
        hs->A0[2] = tot[4];
        hs->A1[0] = tot[0] + tot[1];
        hs->A1[1] = tot[0];
        hs->A1[2] = tot[1];
        double k1 = tot[2];
        for (int l = 0; l < NP; ++l) k1 += kin[l];
        hs->K1 = k1;
        const double dH = (hs->A1[0] + k1) - (hs->A0[0] + hs->K0);
        hs->dH = dH;
        const int acc = (!hs->oob && dH < hs->E) ? 1 : 0;
        hs->accept = acc;
        hs->n_acc += (unsigned long long)acc;
        hs->n_traj += 1ull;
        *c.ticket = 0u;
    }
}

// Accepted trajectory: Q_L -> state (positions in the storage precision).
// Then the f cache of every site from the state as it now stands (the new
// parameters are read from Q_L, so no thread waits for another's write).
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_commit_kernel(Ctx c, const HmcScalars* hs, const double* Q)
{
    constexpr int D = Model::D;
    pdl_trigger();
    pdl_wait();
    const int64_t n = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (n > c.M) return;
    const bool acc = hs->accept != 0;
    const int64_t ld = c.M + 1, nx = (int64_t)D * ld;
    const double* pnew = acc ? Q + nx : c.st->p;
    if (acc && n == 0)
        for (int l = 0; l < Model::NP; ++l) c.st->p[l] = Q[nx + l];
    R x[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (acc) {
            x[a] = HmcVal<R>::x(HmcVal<R>::load(Q, a * ld + n));
            ((R*)c.X)[a * c.ldx + n] = x[a];
        } else {
            x[a] = ((const R*)c.X)[a * c.ldx + n];
        }
    }
    if (n >= cache_len(c)) return;
    R pr[kMaxP], f[D];
    Model::prep(pnew, pr);
    const Coef<R> kc(c);
    cache_value<Model, R>(c, kc, x, pr, n, f);
    R* F = (R*)c.F[c.st->fidx];
#pragma unroll
    for (int a = 0; a < D; ++a) F[a * c.ldf + n] = f[a];
}

// Statistics of the trajectory's end state when due (same schedule as a sweep).
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_record_kernel(Ctx c)
{
    pdl_trigger();
    pdl_wait();
    const long long s = c.st->sweep;
    if (!(s >= c.n_init && (s - c.n_init) % c.n_skip == 0)) return;
    const int64_t n0 = (int64_t)blockIdx.x * kBlock;
    const int64_t n1 = min(n0 + (int64_t)kBlock, c.M + 1);
    record_sample<Model, R>(c, n0, n1, blockIdx.x == 0, c.st->p, c.st->J == 0, threadIdx.x, kBlock,
                            (const R*)c.F[c.st->fidx]);
}

// Counters after a trajectory; the parameter trace gets the end state.
template <int NP>
__global__ void hmc_tick_kernel(Ctx c)
{
    pdl_wait();
    DevState* g = c.st;
    const long long s = g->sweep;
    if (s >= c.n_init && (s - c.n_init) % c.n_skip == 0) g->J += 1;
    g->sweep = s + 1;
    if (c.trace) {
        for (int l = 0; l < NP; ++l) c.trace[(g->tr_n % c.trace_cap) * NP + l] = g->p[l];
        g->tr_n += 1;
    }
}

// Launch on s; with pdl, the kernel may start while the previous one on s
// finishes (it waits in pdl_wait for that one's results).
template <class... KArgs, class... Args>
static cudaError_t launch_after(void (*kern)(KArgs...), unsigned grid, int block, cudaStream_t s, bool pdl,
                                Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <class Model, class R>
static cudaError_t hmc_traj_t(const Ctx& c, const HmcBuffers& b, int n_leap, double eps, uint64_t seed,
                              bool pdl, cudaStream_t s)
{
    constexpr int D = Model::D, NP = Model::NP;
    const int64_t nq = (int64_t)D * (c.M + 1) + NP;
    // sites a tile: spread over every SM while that leaves at most kBlock - 1 a tile
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t T = (c.M + 1 + sms - 1) / (sms > 0 ? sms : 1);
    T = T < 1 ? 1 : (T > kBlock - 1 ? kBlock - 1 : T);
    const int64_t ntile = (c.M + 1 + T - 1) / T;
    // at most two CTAs an SM (what the registers allow); beyond, CTAs stride
    // over tiles -- every CTA reads all CTAs' parameter-gradient sums
    const int64_t gmax = 2 * (int64_t)(sms > 0 ? sms : 1) < kMaxGrid ? 2 * (int64_t)(sms > 0 ? sms : 1) : kMaxGrid;
    const unsigned gl = (unsigned)(ntile < gmax ? ntile : gmax);
    // The FP64 step is bound by the FP64 pipe: a next step made resident early
    // (programmatic launch) would share SMs with the running one and leave
    // some SMs with two CTAs of it, which then take twice as long -- so only
    // the latency-bound FP32-mixed steps overlap.
    const bool pdl_leap = pdl && sizeof(R) == sizeof(float);
    int gb = (int)(((nq + 1) / 2 + kBlock - 1) / kBlock);
    if (gb > kMaxGrid) gb = kMaxGrid;
    double* Qb[2] = {b.Q, b.Q2};
    hmc_begin_kernel<Model, R><<<gb, kBlock, 0, s>>>(c, b.hs, b.Q, b.P, b.EM, b.invm, eps, seed);
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k <= n_leap && e == cudaSuccess; ++k)
        e = launch_after(hmc_leap_kernel<Model, R>, gl, kBlock, s, pdl_leap, c, b.hs, Qb[k & 1], Qb[(k + 1) & 1],
                         b.P, (const double*)b.EM, (const double*)b.invm, k, n_leap, (int)T);
    const unsigned gs = (unsigned)((c.M + 1 + kBlock - 1) / kBlock);
    if (e == cudaSuccess)
        e = launch_after(hmc_commit_kernel<Model, R>, gs, kBlock, s, pdl, c, (const HmcScalars*)b.hs,
                         (const double*)Qb[n_leap & 1]);
    if (e == cudaSuccess) e = launch_after(hmc_record_kernel<Model, R>, gs, kBlock, s, pdl, c);
    if (e == cudaSuccess) e = launch_after(hmc_tick_kernel<NP>, 1u, 1, s, pdl, c);
    return e;
}

cudaError_t launch_hmc_trajectory(int model, int prec, const Ctx& c, const HmcBuffers& b, int n_leap, double eps,
                                  uint64_t seed, bool pdl, cudaStream_t s)
{
    PIMC_DISPATCH(hmc_traj_t, c, b, n_leap, eps, seed, pdl, s);
}

}  // namespace pimc
