// Whole-path Hybrid Monte Carlo (X and the free parameters move together),
// driven by the reverse-mode gradient of the action through the RK4 map.  The
// paper points to gradient-using proposals (Sec. 3.1; Hybrid Monte Carlo is
// named among the methods that sample exp(-A)); this is that form.
//
// One trajectory is a fixed sequence of launches on the handle's stream --
// begin (copy the state to FP64 positions Q, draw momenta P, kinetic energy,
// step jitter and accept uniform), action at Q, gradient, half momentum step,
// then n_leap x (position step, gradient, momentum step), action at the end,
// end (kinetic energy, accept test), commit (accepted Q -> state), f-cache
// refresh, statistics, counter tick -- so the host captures it once in a
// CUDA graph and replays the graph per trajectory.  Every decision stays on
// the device.
#include <cstddef>

#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "stats.cuh"

namespace pimc {

// Q = current state (FP64), P_j = z_j / sqrt(invm_j) (fixed parameters: 0),
// K0 = 1/2 sum P^2 invm; step jitter eps (0.8 + 0.4 u') and -log u of the
// accept uniform from the trajectory's accept block.
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_begin_kernel(Ctx c, HmcScalars* hs, double* Q, double* P,
                                                           const double* invm, double eps, uint64_t seed)
{
    constexpr int D = Model::D, NP = Model::NP;
    __shared__ double wsum[1][kBlock / 32];
    __shared__ int last;
    const int64_t nx = (int64_t)D * (c.M + 1), nq = nx + NP;
    const uint64_t traj = (uint64_t)c.st->sweep;
    double v[1] = {0.0};
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < nq; j += (int64_t)gridDim.x * kBlock) {
        bool moving = true;
        if (j < nx) {
            const int64_t a = j / (c.M + 1), n = j - a * (c.M + 1);
            Q[j] = (double)((const R*)c.X)[a * c.ldx + n];
        } else {
            const int l = (int)(j - nx);
            Q[j] = c.st->p[l];
            moving = (c.st->free_mask >> l) & 1u;
        }
        double z0, z1;
        Num<double>::box_muller(draw_block(seed, c.chain, traj, (uint32_t)(j >> 1), kKindHmcMom, 0u), z0, z1);
        const double z = (j & 1) ? z1 : z0;
        const double pj = moving ? z / sqrt(invm[j]) : 0.0;
        P[j] = pj;
        v[0] += 0.5 * pj * pj * invm[j];
    }
    double k0[1];
    grid_sums_last_block<1>(c, v, k0, wsum, &last);
    if (last && threadIdx.x == 0) {
        hs->K0 = k0[0];
        const uint4 w = draw_block(seed, c.chain, traj, 0u, kKindHmcAcc, 0u);
        hs->E = -log(u01d(w.x, w.y));
        hs->eps = eps * (0.8 + 0.4 * u01d(w.z, w.w));
        hs->oob = 0;
    }
}

// P -= factor * eps * g (fixed parameters keep zero momentum).
template <int NP>
__global__ void hmc_momentum_kernel(Ctx c, HmcScalars* hs, double* P, const double* g, int D, double factor)
{
    const int64_t nx = (int64_t)D * (c.M + 1), nq = nx + NP;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    if (j >= nx && !((c.st->free_mask >> (int)(j - nx)) & 1u)) return;
    P[j] -= factor * hs->eps * g[j];
}

// Q += eps invm P; a free parameter leaving its box marks the trajectory.
template <int NP>
__global__ void hmc_position_kernel(Ctx c, HmcScalars* hs, double* Q, const double* P, const double* invm, int D)
{
    const int64_t nx = (int64_t)D * (c.M + 1), nq = nx + NP;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    if (j >= nx) {
        const int l = (int)(j - nx);
        if (!((c.st->free_mask >> l) & 1u)) return;
        const double q = Q[j] + hs->eps * invm[j] * P[j];
        Q[j] = q;
        if (!(q >= c.st->lo[l] && q <= c.st->hi[l])) atomicExch(&hs->oob, 1);
        return;
    }
    Q[j] += hs->eps * invm[j] * P[j];
}

// K1, dH = (A1 + K1) - (A0 + K0) and the accept test dH < -log u.
template <int NP>
__global__ void __launch_bounds__(kBlock) hmc_end_kernel(Ctx c, HmcScalars* hs, const double* P, const double* invm,
                                                         int D)
{
    __shared__ double wsum[1][kBlock / 32];
    __shared__ int last;
    const int64_t nq = (int64_t)D * (c.M + 1) + NP;
    double v[1] = {0.0};
    for (int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x; j < nq; j += (int64_t)gridDim.x * kBlock)
        v[0] += 0.5 * P[j] * P[j] * invm[j];
    double k1[1];
    grid_sums_last_block<1>(c, v, k1, wsum, &last);
    if (last && threadIdx.x == 0) {
        hs->K1 = k1[0];
        const double dH = (hs->A1[0] + k1[0]) - (hs->A0[0] + hs->K0);
        hs->dH = dH;
        const int acc = (!hs->oob && dH < hs->E) ? 1 : 0;
        hs->accept = acc;
        hs->n_acc += (unsigned long long)acc;
        hs->n_traj += 1ull;
    }
}

// Accepted trajectory: Q -> state (positions in the storage precision).
template <class Model, class R>
__global__ void hmc_commit_kernel(Ctx c, const HmcScalars* hs, const double* Q)
{
    constexpr int D = Model::D, NP = Model::NP;
    if (!hs->accept) return;
    const int64_t nx = (int64_t)D * (c.M + 1);
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nx) {
        const int64_t a = j / (c.M + 1), n = j - a * (c.M + 1);
        ((R*)c.X)[a * c.ldx + n] = R(Q[j]);
    } else if (j < nx + NP) {
        c.st->p[j - nx] = Q[j];
    }
}

// Statistics of the trajectory's end state when due (same schedule as a sweep).
template <class Model, class R>
__global__ void __launch_bounds__(kBlock) hmc_record_kernel(Ctx c)
{
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
    DevState* g = c.st;
    const long long s = g->sweep;
    if (s >= c.n_init && (s - c.n_init) % c.n_skip == 0) g->J += 1;
    g->sweep = s + 1;
    if (c.trace) {
        for (int l = 0; l < NP; ++l) c.trace[(g->tr_n % c.trace_cap) * NP + l] = g->p[l];
        g->tr_n += 1;
    }
}

template <class Model, class R>
static cudaError_t hmc_traj_t(const Ctx& c, const HmcBuffers& b, int n_leap, double eps, uint64_t seed,
                              cudaStream_t s)
{
    constexpr int D = Model::D, NP = Model::NP;
    const int64_t nx = (int64_t)D * (c.M + 1), nq = nx + NP;
    const unsigned ge = (unsigned)((nq + 255) / 256);
    // device addresses of the action slots (no host dereference of b.hs)
    double* a0 = (double*)((char*)b.hs + offsetof(HmcScalars, A0));
    double* a1 = (double*)((char*)b.hs + offsetof(HmcScalars, A1));
    int gr = (int)((nq + kBlock - 1) / kBlock);
    if (gr > kMaxGrid) gr = kMaxGrid;
    cudaError_t e;
    hmc_begin_kernel<Model, R><<<gr, kBlock, 0, s>>>(c, b.hs, b.Q, b.P, b.invm, eps, seed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_action(ModelId<Model>::value, prec_of<R>(), c, b.Q, b.Q + nx, a0, s)) != cudaSuccess)
        return e;
    if ((e = launch_grad(ModelId<Model>::value, prec_of<R>(), c, b.Q, b.Q + nx, 1.0, b.g, b.g + nx, s)) != cudaSuccess)
        return e;
    hmc_momentum_kernel<NP><<<ge, 256, 0, s>>>(c, b.hs, b.P, b.g, D, 0.5);
    for (int i = 1; i <= n_leap; ++i) {
        hmc_position_kernel<NP><<<ge, 256, 0, s>>>(c, b.hs, b.Q, b.P, b.invm, D);
        if ((e = launch_grad(ModelId<Model>::value, prec_of<R>(), c, b.Q, b.Q + nx, 1.0, b.g, b.g + nx, s)) != cudaSuccess)
            return e;
        hmc_momentum_kernel<NP><<<ge, 256, 0, s>>>(c, b.hs, b.P, b.g, D, i < n_leap ? 1.0 : 0.5);
    }
    if ((e = launch_action(ModelId<Model>::value, prec_of<R>(), c, b.Q, b.Q + nx, a1, s)) != cudaSuccess) return e;
    hmc_end_kernel<NP><<<gr, kBlock, 0, s>>>(c, b.hs, b.P, b.invm, D);
    hmc_commit_kernel<Model, R><<<ge, 256, 0, s>>>(c, b.hs, b.Q);
    if ((e = launch_refresh_cache(ModelId<Model>::value, prec_of<R>(), c, s)) != cudaSuccess) return e;
    hmc_record_kernel<Model, R><<<(unsigned)((c.M + 1 + kBlock - 1) / kBlock), kBlock, 0, s>>>(c);
    hmc_tick_kernel<NP><<<1, 1, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_hmc_trajectory(int model, int prec, const Ctx& c, const HmcBuffers& b, int n_leap, double eps,
                                  uint64_t seed, cudaStream_t s)
{
    PIMC_DISPATCH(hmc_traj_t, c, b, n_leap, eps, seed, s);
}

}  // namespace pimc
